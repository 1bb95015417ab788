// Executor for many independent snapshots (map_batch).
//
// Front stages per snapshot -- tree, tree-walk and node h, Voronoi grid,
// pairs -- on a pool of host threads that each drive their own context on
// their own non-blocking stream: small snapshots are bound by launch latency
// and by the few host reads of output sizes, and with several streams in
// flight those gaps of one snapshot are filled by the kernels of others.
// Snapshots are handed out largest first (by particles + sites), the
// longest-processing-time rule, so that the last ones to start are the short
// ones.
//
// The mapping then runs once for all snapshots: their pseudo-particles, cells
// (with face and vertex offsets shifted) and pair lists (particle and cell
// indices shifted) are gathered into one concatenated set on a stream of its
// own, and a single map_exact maps every pair of the batch -- one launch of
// the FP32 pass and one of the FP64 recompute, or one FP64 launch.  A pair's
// weight does not depend on the other pairs of its warp, so the results are
// bit for bit those of one map_exact per snapshot.  The inverse mapping runs
// per snapshot on its slice of the weights.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

// dst[t] = src_s[t - pre[s]] + add[s] for t in [pre[s], pre[s + 1]): the
// segments of several device arrays gathered into one, each shifted.
template <class T>
__global__ void k_gather_add(int nseg, const int64_t *__restrict__ pre, const T *const *__restrict__ src,
                             const T *__restrict__ add, T *__restrict__ dst)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= pre[nseg]) return;
    int lo = 0, hi = nseg;   // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid;
        else hi = mid;
    }
    dst[t] = src[lo][t - pre[lo]] + (add ? add[lo] : T(0));
}

// Flagged pairs (global pair ids, ~id for the full form) counted per
// snapshot, from the snapshots' pair offsets.
__global__ void k_count_flagged(const int *__restrict__ nflag, const int32_t *__restrict__ flagged, int nseg,
                                const int64_t *__restrict__ kpre, unsigned long long *__restrict__ counts)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *nflag) return;
    const int32_t c = flagged[t];
    const int64_t k = c >= 0 ? c : ~c;
    int lo = 0, hi = nseg;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (kpre[mid] <= k) lo = mid;
        else hi = mid;
    }
    atomicAdd(counts + lo, 1ull);
}

struct Front {
    em_tree *t = nullptr;
    em_pseudo *ps = nullptr;
    em_voronoi *v = nullptr;
    em_pairs *pr = nullptr;
    int64_t npairs = 0;
};

int run_front(em_ctx *ctx, em_snapshot &s, const em_params *p, Front &f)
{
    int rc = build_tree(ctx, s.n, s.d_x, s.d_y, s.d_z, s.d_m, s.box, p->leaf_max, &f.t);
    if (rc == EM_OK) {
        rc = make_pseudo_particles(ctx, f.t, s.d_h, s.nsrc, s.h_src, p, &f.ps);
        if (rc == EM_ENOTCONV) rc = EM_OK;   // some node kept h_0; the outputs are valid
    }
    if (rc == EM_OK) rc = build_voronoi(ctx, s.ngen, s.d_gx, s.d_gy, s.d_gz, s.box, p, &f.v);
    if (rc == EM_OK) rc = find_pairs(ctx, f.ps->n, f.ps->x, f.ps->y, f.ps->z, f.ps->h, f.v, &f.pr, &f.npairs);
    // the handles are used on the mapping stream next
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (rc == EM_OK && e != cudaSuccess) {
        em_set_error("map_batch: %s", cudaGetErrorString(e));
        rc = EM_ECUDA;
    }
    return rc;
}

void release_front(Front &f)
{
    if (f.pr) pairs_destroy(f.pr);
    if (f.v) voronoi_destroy(f.v);
    if (f.ps) pseudo_destroy(f.ps);
    if (f.t) tree_destroy(f.t);
    f = Front{};
}

// One gather: the segments' sources and shifts to the device, then the kernel.
template <class T>
int gather(em_ctx *ctx, DevArena &tmp, const std::vector<const T *> &src, const std::vector<int64_t> &count,
           const std::vector<T> *add, T *dst)
{
    const int nseg = (int)src.size();
    std::vector<int64_t> pre(nseg + 1, 0);
    for (int k = 0; k < nseg; ++k) pre[k + 1] = pre[k] + count[k];
    if (pre[nseg] == 0) return EM_OK;
    int64_t *d_pre;
    const T **d_src;
    T *d_add = nullptr;
    EM_TRY(tmp.alloc(&d_pre, nseg + 1));
    EM_TRY(tmp.alloc(&d_src, nseg));
    EM_CUDA(cudaMemcpyAsync(d_pre, pre.data(), (nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    EM_CUDA(cudaMemcpyAsync(d_src, src.data(), nseg * sizeof(T *), cudaMemcpyHostToDevice, ctx->stream));
    if (add) {
        EM_TRY(tmp.alloc(&d_add, nseg));
        EM_CUDA(cudaMemcpyAsync(d_add, add->data(), nseg * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    }
    // copies from pageable host memory return once the data is staged, so
    // the host vectors may go
    k_gather_add<T><<<em_grid(pre[nseg], 256), 256, 0, ctx->stream>>>(nseg, d_pre, d_src, d_add, dst);
    EM_LAUNCHED(ctx);
    return EM_OK;
}

// Records (planes, edges) gathered as 32-bit words, unshifted.
template <class R>
int gather_records(em_ctx *ctx, DevArena &tmp, const std::vector<const R *> &src, const std::vector<int64_t> &count,
                   R *dst)
{
    static_assert(sizeof(R) % 4 == 0, "records of whole words");
    std::vector<const uint32_t *> s(src.size());
    std::vector<int64_t> c(count.size());
    for (size_t k = 0; k < src.size(); ++k) {
        s[k] = reinterpret_cast<const uint32_t *>(src[k]);
        c[k] = count[k] * (int64_t)(sizeof(R) / 4);
    }
    return gather<uint32_t>(ctx, tmp, s, c, nullptr, reinterpret_cast<uint32_t *>(dst));
}

// The concatenated mapping of the snapshots in `idx` (see the file comment).
int map_all(em_ctx *ctx, const std::vector<int> &idx, em_snapshot *all_snaps, std::vector<Front> &all_fr,
            const em_params *p, int tune, int *h_variant, double *h_map_ms)
{
    const int nsnap = (int)idx.size();
    std::vector<Front> fr(nsnap);
    std::vector<em_snapshot *> sp(nsnap);
    for (int k = 0; k < nsnap; ++k) {
        fr[k] = all_fr[idx[k]];
        sp[k] = &all_snaps[idx[k]];
    }
    auto snaps = [&](int k) -> em_snapshot & { return *sp[k]; };
    int64_t P = 0, Cn = 0, F = 0, V = 0, K = 0;
    std::vector<int64_t> Pk(nsnap), Ck(nsnap), Fk(nsnap), Vk(nsnap), Kk(nsnap + 1);
    for (int k = 0; k < nsnap; ++k) {
        Pk[k] = P;
        Ck[k] = Cn;
        Fk[k] = F;
        Vk[k] = V;
        Kk[k] = K;
        P += fr[k].ps->n;
        Cn += fr[k].v->ncell;
        F += fr[k].v->nface;
        V += fr[k].v->nfv;
        K += fr[k].npairs;
    }
    Kk[nsnap] = K;
    if (P >= INT32_MAX || Cn >= INT32_MAX || K >= INT32_MAX) {
        em_set_error("map_batch: the batch's %lld particles, %lld cells or %lld pairs exceed 2^31 - 1", (long long)P,
                     (long long)Cn, (long long)K);
        return EM_ECAPACITY;
    }
    DevArena tmp(ctx->stream, true);
    em_voronoi cv(ctx->stream);
    em_pairs cp(ctx->stream);
    cv.mem.scoped = cp.mem.scoped = true;
    cv.device = cp.device = ctx->device;
    cv.ncell = Cn;
    cv.nface = F;
    cv.nfv = V;
    cp.npairs = K;
    cp.np = P;
    cp.ncell = Cn;
    double *x, *y, *z, *h, *m, *w, *rho, *fq = nullptr;
    int32_t *flagged;
    int *nflag;
    unsigned long long *counts;
    EM_TRY(tmp.alloc(&x, P));
    EM_TRY(tmp.alloc(&y, P));
    EM_TRY(tmp.alloc(&z, P));
    EM_TRY(tmp.alloc(&h, P));
    EM_TRY(tmp.alloc(&m, P));
    EM_TRY(tmp.alloc(&w, K));
    EM_TRY(tmp.alloc(&rho, Cn));
    EM_TRY(tmp.alloc(&flagged, K));
    EM_TRY(tmp.alloc(&nflag, 1));
    EM_TRY(tmp.alloc(&counts, nsnap));
    EM_TRY(cv.mem.alloc(&cv.gen, 3 * Cn));
    EM_TRY(cv.mem.alloc(&cv.radius, Cn));
    EM_TRY(cv.mem.alloc(&cv.volume, Cn));
    EM_TRY(cv.mem.alloc(&cv.cell_face_off, Cn + 1));
    EM_TRY(cv.mem.alloc(&cv.face_vert_off, F + 1));
    EM_TRY(cv.mem.alloc(&cv.plane, F));
    EM_TRY(cv.mem.alloc(&cv.plane_f, F));
    EM_TRY(cv.mem.alloc(&cv.plane_fl, F));
    EM_TRY(cv.mem.alloc(&cv.edge, V));
    EM_TRY(cv.mem.alloc(&cv.edge_f, V));
    EM_TRY(cv.mem.alloc(&cv.edge_fl, V));
    EM_TRY(cp.mem.alloc(&cp.pair_i, K));
    EM_TRY(cp.mem.alloc(&cp.pair_j, K));
    EM_TRY(cp.mem.alloc(&cp.cell_pair_off, Cn + 1));

    // particles, sites, per-cell and per-face data: plain copies in order
    {
        std::vector<int64_t> np(nsnap), nc(nsnap), nc3(nsnap), nf(nsnap), nv(nsnap), npr(nsnap);
        for (int k = 0; k < nsnap; ++k) {
            np[k] = fr[k].ps->n;
            nc[k] = fr[k].v->ncell;
            nc3[k] = 3 * nc[k];
            nf[k] = fr[k].v->nface;
            nv[k] = fr[k].v->nfv;
            npr[k] = fr[k].npairs;
        }
        auto dsrc = [&](auto get) {
            std::vector<const double *> s(nsnap);
            for (int k = 0; k < nsnap; ++k) s[k] = get(fr[k]);
            return s;
        };
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.ps->x; }), np, nullptr, x));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.ps->y; }), np, nullptr, y));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.ps->z; }), np, nullptr, z));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.ps->h; }), np, nullptr, h));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.ps->m; }), np, nullptr, m));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.v->gen; }), nc3, nullptr, cv.gen));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.v->radius; }), nc, nullptr,
                              cv.radius));
        EM_TRY(gather<double>(ctx, tmp, dsrc([](Front &f) { return (const double *)f.v->volume; }), nc, nullptr,
                              cv.volume));
        std::vector<const PlaneD *> pd(nsnap);
        std::vector<const PlaneF *> pf(nsnap), pfl(nsnap);
        std::vector<const EdgeD *> ed(nsnap);
        std::vector<const EdgeF *> ef(nsnap), efl(nsnap);
        for (int k = 0; k < nsnap; ++k) {
            pd[k] = fr[k].v->plane;
            pf[k] = fr[k].v->plane_f;
            pfl[k] = fr[k].v->plane_fl;
            ed[k] = fr[k].v->edge;
            ef[k] = fr[k].v->edge_f;
            efl[k] = fr[k].v->edge_fl;
        }
        EM_TRY(gather_records(ctx, tmp, pd, nf, cv.plane));
        EM_TRY(gather_records(ctx, tmp, pf, nf, cv.plane_f));
        EM_TRY(gather_records(ctx, tmp, pfl, nf, cv.plane_fl));
        EM_TRY(gather_records(ctx, tmp, ed, nv, cv.edge));
        EM_TRY(gather_records(ctx, tmp, ef, nv, cv.edge_f));
        EM_TRY(gather_records(ctx, tmp, efl, nv, cv.edge_fl));
        // offsets shifted by the earlier snapshots' counts; the closing entry
        // of each offset array comes from the last snapshot's
        std::vector<const int64_t *> so(nsnap + 1);
        std::vector<int64_t> co(nsnap + 1), ao(nsnap + 1);
        for (int k = 0; k < nsnap; ++k) {
            so[k] = fr[k].v->cell_face_off;
            co[k] = nc[k];
            ao[k] = Fk[k];
        }
        so[nsnap] = fr[nsnap - 1].v->cell_face_off + nc[nsnap - 1];
        co[nsnap] = 1;
        ao[nsnap] = Fk[nsnap - 1];
        EM_TRY(gather<int64_t>(ctx, tmp, so, co, &ao, cv.cell_face_off));
        for (int k = 0; k < nsnap; ++k) {
            so[k] = fr[k].v->face_vert_off;
            co[k] = nf[k];
            ao[k] = Vk[k];
        }
        so[nsnap] = fr[nsnap - 1].v->face_vert_off + nf[nsnap - 1];
        ao[nsnap] = Vk[nsnap - 1];
        EM_TRY(gather<int64_t>(ctx, tmp, so, co, &ao, cv.face_vert_off));
        for (int k = 0; k < nsnap; ++k) {
            so[k] = fr[k].pr->cell_pair_off;
            co[k] = nc[k];
            ao[k] = Kk[k];
        }
        so[nsnap] = fr[nsnap - 1].pr->cell_pair_off + nc[nsnap - 1];
        ao[nsnap] = Kk[nsnap - 1];
        EM_TRY(gather<int64_t>(ctx, tmp, so, co, &ao, cp.cell_pair_off));
        std::vector<const int32_t *> si(nsnap);
        std::vector<int32_t> ai(nsnap);
        for (int k = 0; k < nsnap; ++k) {
            si[k] = fr[k].pr->pair_i;
            ai[k] = (int32_t)Pk[k];
        }
        EM_TRY(gather<int32_t>(ctx, tmp, si, npr, &ai, cp.pair_i));
        for (int k = 0; k < nsnap; ++k) {
            si[k] = fr[k].pr->pair_j;
            ai[k] = (int32_t)Ck[k];
        }
        EM_TRY(gather<int32_t>(ctx, tmp, si, npr, &ai, cp.pair_j));
    }

    em_params q = *p;
    if (tune && p->precision == 1) {
        int best = 0;
        EM_TRY(map_autotune(ctx, &cp, x, y, z, h, &cv, p, &best, nullptr));
        q.fp32_variant = best;
    }
    if (h_variant) *h_variant = q.fp32_variant;
    EM_TRY(em_ctx_set_timing(ctx, 1));   // the mapping context is the executor's own
    int rc = em_map_exact_impl(ctx, &cp, x, y, z, h, m, &cv, &q, w, rho, nullptr, nullptr, false, flagged, nflag);
    if (rc != EM_OK) return rc;
    // per-snapshot densities and FP64 counts
    for (int k = 0; k < nsnap; ++k)
        EM_CUDA(cudaMemcpyAsync(snaps(k).d_rho, rho + Ck[k], fr[k].v->ncell * sizeof(double), cudaMemcpyDeviceToDevice,
                                ctx->stream));
    std::vector<unsigned long long> hc(nsnap, 0);
    if (q.precision == 1 && K) {
        int64_t *d_kpre;
        EM_TRY(tmp.alloc(&d_kpre, nsnap + 1));
        EM_CUDA(cudaMemcpyAsync(d_kpre, Kk.data(), (nsnap + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
        EM_CUDA(cudaMemsetAsync(counts, 0, nsnap * sizeof(unsigned long long), ctx->stream));
        k_count_flagged<<<em_grid(K, 256), 256, 0, ctx->stream>>>(nflag, flagged, nsnap, d_kpre, counts);
        EM_LAUNCHED(ctx);
        EM_CUDA(cudaMemcpyAsync(hc.data(), counts, nsnap * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                ctx->stream));
    }
    // inverse mapping per snapshot, on its slice of the weights
    bool any_f = false;
    for (int k = 0; k < nsnap; ++k) any_f = any_f || snaps(k).d_f_cell;
    if (any_f) EM_TRY(tmp.alloc(&fq, P));
    for (int k = 0; k < nsnap && rc == EM_OK; ++k)
        if (snaps(k).d_f_cell)
            rc = map_back(ctx, fr[k].pr, w + Kk[k], snaps(k).d_f_cell, fq + Pk[k], fr[k].ps, fr[k].t, snaps(k).d_f);
    if (rc != EM_OK) return rc;
    EM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h_map_ms) EM_TRY(em_ctx_map_times(ctx, h_map_ms, h_map_ms + 1));
    for (int k = 0; k < nsnap; ++k) {
        snaps(k).npseudo = fr[k].ps->n;
        snaps(k).npairs = fr[k].npairs;
        snaps(k).nfp64 = (int64_t)hc[k];
    }
    return EM_OK;
}

}  // namespace

EM_EXPORT int map_batch(int device, int nsnap, em_snapshot *snaps, const em_params *p, int nworkers, int tune,
                        int *h_variant, double *h_map_ms, int64_t *h_launches)
{
    EM_CHECK_ARG(p && nsnap >= 0 && (nsnap == 0 || snaps));
    EM_CHECK_ARG(nworkers >= 1 && nworkers <= 64);
    EM_CHECK_ARG(p->precision == 0 || p->precision == 1);
    for (int k = 0; k < nsnap; ++k) {
        const em_snapshot &s = snaps[k];
        EM_CHECK_ARG(s.n >= 1 && s.ngen >= 1 && s.d_x && s.d_y && s.d_z && s.d_m && s.d_h && s.d_gx && s.d_gy &&
                     s.d_gz && s.d_rho && s.h_src && s.nsrc >= 1);
        EM_CHECK_ARG((s.d_f_cell == nullptr) == (s.d_f == nullptr));
    }
    if (h_launches) *h_launches = 0;
    if (h_variant) *h_variant = p->fp32_variant;
    if (h_map_ms) h_map_ms[0] = h_map_ms[1] = 0.0;
    for (int k = 0; k < nsnap; ++k) {
        snaps[k].status = -1;
        snaps[k].npseudo = snaps[k].npairs = snaps[k].nfp64 = 0;
    }
    if (nsnap == 0) return EM_OK;
    std::vector<int> order(nsnap);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return snaps[a].n + snaps[a].ngen > snaps[b].n + snaps[b].ngen;
    });
    // one context and stream per worker, and one for the mapping; all kept
    // until the handles made on them are freed
    const int nw = std::min(nworkers, nsnap);
    std::vector<cudaStream_t> streams(nw + 1, nullptr);
    std::vector<em_ctx *> ctxs(nw + 1, nullptr);
    int rc = cudaSetDevice(device) == cudaSuccess ? EM_OK : EM_ECUDA;
    for (int id = 0; id <= nw && rc == EM_OK; ++id) {
        if (cudaStreamCreateWithFlags(&streams[id], cudaStreamNonBlocking) != cudaSuccess) rc = EM_ECUDA;
        if (rc == EM_OK) rc = em_ctx_create(&ctxs[id], device, streams[id]);
    }
    if (rc == EM_ECUDA) em_set_error("map_batch: no stream on device %d", device);
    std::vector<Front> fr(nsnap);
    std::vector<int> wrc(nw, EM_OK);
    std::vector<std::string> wmsg(nw);
    if (rc == EM_OK) {
        std::atomic<int> next{0};
        auto worker = [&](int id) {
            if (cudaSetDevice(device) != cudaSuccess) {
                wrc[id] = EM_ECUDA;
                wmsg[id] = "cudaSetDevice failed";
                return;
            }
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= nsnap) break;
                em_snapshot &s = snaps[order[i]];
                s.status = run_front(ctxs[id], s, p, fr[order[i]]);
                if (s.status != EM_OK && wrc[id] == EM_OK) {
                    wrc[id] = s.status;
                    wmsg[id] = std::string("snapshot ") + std::to_string(order[i]) + ": " + em_last_error();
                }
            }
        };
        std::vector<std::thread> pool;
        for (int id = 0; id < nw; ++id) pool.emplace_back(worker, id);
        for (auto &th : pool) th.join();
        for (int id = 0; id < nw && rc == EM_OK; ++id)
            if (wrc[id] != EM_OK) {
                em_set_error("%s", wmsg[id].c_str());
                rc = wrc[id];
            }
    }
    // map the snapshots whose front stages succeeded; a failure is reported
    // with its snapshot's index after the others have finished
    if (ctxs[nw]) {
        std::vector<int> ok;
        for (int k = 0; k < nsnap; ++k)
            if (snaps[k].status == EM_OK && fr[k].pr) ok.push_back(k);
        const std::string front_msg = rc == EM_OK ? std::string() : std::string(em_last_error());
        if (!ok.empty()) {
            const int mrc = map_all(ctxs[nw], ok, snaps, fr, p, tune, h_variant, h_map_ms);
            if (mrc != EM_OK) {
                const std::string msg = em_last_error();
                for (int k : ok) snaps[k].status = mrc;
                if (rc == EM_OK) {
                    rc = mrc;
                    em_set_error("map_batch: mapping: %s", msg.c_str());
                }
            }
        }
        if (!front_msg.empty()) em_set_error("%s", front_msg.c_str());
    }
    // handles free in their own streams' order; wait for everything before
    // the streams go
    for (auto &f : fr) release_front(f);
    int64_t launches = 0;
    for (int id = 0; id <= nw; ++id) {
        if (streams[id]) cudaStreamSynchronize(streams[id]);
        if (ctxs[id]) {
            launches += ctxs[id]->launches;
            em_ctx_destroy(ctxs[id]);
        }
        if (streams[id]) cudaStreamDestroy(streams[id]);
    }
    if (h_launches) *h_launches = launches;
    return rc;
}

// The batch as a handle: the snapshots' records collected by map_batch_add,
// mapped together by map_batch_run.
struct em_batch {
    int device;
    em_params p;
    int nworkers;
    std::vector<em_snapshot> snaps;
};

EM_EXPORT int map_batch_create(int device, const em_params *p, int nworkers, em_batch **out)
{
    EM_CHECK_ARG(p && out && device >= 0 && nworkers >= 1 && nworkers <= 64);
    EM_CHECK_ARG(p->precision == 0 || p->precision == 1);
    *out = new em_batch{device, *p, nworkers, {}};
    return EM_OK;
}

EM_EXPORT int map_batch_add(em_batch *b, const em_snapshot *s, int *h_index)
{
    EM_CHECK_ARG(b && s && b->snaps.size() < (size_t)INT32_MAX);
    EM_CHECK_ARG(s->n >= 1 && s->ngen >= 1 && s->d_x && s->d_y && s->d_z && s->d_m && s->d_h && s->d_gx &&
                 s->d_gy && s->d_gz && s->d_rho && s->h_src && s->nsrc >= 1);
    EM_CHECK_ARG((s->d_f_cell == nullptr) == (s->d_f == nullptr));
    b->snaps.push_back(*s);
    em_snapshot &r = b->snaps.back();
    r.status = -1;
    r.npseudo = r.npairs = r.nfp64 = 0;
    if (h_index) *h_index = (int)b->snaps.size() - 1;
    return EM_OK;
}

EM_EXPORT int map_batch_run(em_batch *b, int tune, int *h_variant, double *h_map_ms, int64_t *h_launches)
{
    EM_CHECK_ARG(b);
    return map_batch(b->device, (int)b->snaps.size(), b->snaps.data(), &b->p, b->nworkers, tune, h_variant,
                     h_map_ms, h_launches);
}

EM_EXPORT int map_batch_get(const em_batch *b, int index, em_snapshot *out)
{
    EM_CHECK_ARG(b && out && index >= 0 && (size_t)index < b->snaps.size());
    *out = b->snaps[index];
    return EM_OK;
}

EM_EXPORT int map_batch_destroy(em_batch *b)
{
    delete b;
    return EM_OK;
}
