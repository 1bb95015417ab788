// Executor for many independent snapshots: the whole path (tree, tree-walk
// and node h, Voronoi grid, pairs, Exact mapping, inverse mapping) run for
// each snapshot, the snapshots spread over a pool of host threads that each
// drive their own context on their own non-blocking stream.  Small
// snapshots are bound by launch latency and by the few host reads of output
// sizes; with several streams in flight those gaps of one snapshot are
// filled by the kernels of others.  Snapshots are handed out largest first
// (by particles + sites), the longest-processing-time rule, so that the last
// ones to start are the short ones.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

int run_snapshot(em_ctx *ctx, em_snapshot &s, const em_params *p)
{
    em_tree *t = nullptr;
    em_pseudo *ps = nullptr;
    em_voronoi *v = nullptr;
    em_pairs *pr = nullptr;
    DevArena tmp(ctx->stream, true);
    int rc = build_tree(ctx, s.n, s.d_x, s.d_y, s.d_z, s.d_m, s.box, p->leaf_max, &t);
    if (rc == EM_OK) {
        rc = make_pseudo_particles(ctx, t, s.d_h, s.nsrc, s.h_src, p, &ps);
        if (rc == EM_ENOTCONV) rc = EM_OK;   // some node kept h_0; the outputs are valid
    }
    if (rc == EM_OK) rc = build_voronoi(ctx, s.ngen, s.d_gx, s.d_gy, s.d_gz, s.box, p, &v);
    int64_t npairs = 0;
    if (rc == EM_OK) rc = find_pairs(ctx, ps->n, ps->x, ps->y, ps->z, ps->h, v, &pr, &npairs);
    double *w = nullptr, *wsum = nullptr, *fq = nullptr;
    int64_t nf = 0;
    if (rc == EM_OK) rc = tmp.alloc(&w, npairs);
    if (rc == EM_OK) rc = tmp.alloc(&wsum, ps->n);
    if (rc == EM_OK) rc = map_exact(ctx, pr, ps->x, ps->y, ps->z, ps->h, ps->m, v, p, w, s.d_rho, wsum, &nf);
    if (rc == EM_OK && s.d_f_cell && s.d_f) {
        rc = tmp.alloc(&fq, ps->n);
        if (rc == EM_OK) rc = map_back(ctx, pr, w, s.d_f_cell, fq, ps, t, s.d_f);
    }
    if (rc == EM_OK) {
        s.npseudo = ps->n;
        s.npairs = npairs;
        s.nfp64 = nf;
    }
    // handles free their memory in stream order; the wait below makes the
    // snapshot's outputs final before the worker reports it done
    if (pr) pairs_destroy(pr);
    if (v) voronoi_destroy(v);
    if (ps) pseudo_destroy(ps);
    if (t) tree_destroy(t);
    tmp.release();
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (rc == EM_OK && e != cudaSuccess) {
        em_set_error("map_batch: %s", cudaGetErrorString(e));
        rc = EM_ECUDA;
    }
    return rc;
}

}  // namespace

EM_EXPORT int map_batch(int device, int nsnap, em_snapshot *snaps, const em_params *p, int nworkers,
                        int64_t *h_launches)
{
    EM_CHECK_ARG(p && nsnap >= 0 && (nsnap == 0 || snaps));
    EM_CHECK_ARG(nworkers >= 1 && nworkers <= 64);
    for (int k = 0; k < nsnap; ++k) {
        const em_snapshot &s = snaps[k];
        EM_CHECK_ARG(s.n >= 1 && s.ngen >= 1 && s.d_x && s.d_y && s.d_z && s.d_m && s.d_h && s.d_gx && s.d_gy &&
                     s.d_gz && s.d_rho && s.h_src && s.nsrc >= 1);
        EM_CHECK_ARG((s.d_f_cell == nullptr) == (s.d_f == nullptr));
    }
    if (h_launches) *h_launches = 0;
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
    const int nw = std::min(nworkers, nsnap);
    std::atomic<int> next{0};
    std::atomic<int64_t> launches{0};
    std::vector<int> wrc(nw, EM_OK);
    std::vector<std::string> wmsg(nw);
    auto worker = [&](int id) {
        cudaStream_t st = nullptr;
        em_ctx *ctx = nullptr;
        int rc = cudaSetDevice(device) == cudaSuccess ? EM_OK : EM_ECUDA;
        if (rc == EM_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = EM_ECUDA;
        if (rc == EM_OK) rc = em_ctx_create(&ctx, device, st);
        if (rc != EM_OK) {
            if (rc == EM_ECUDA) em_set_error("map_batch: no stream on device %d", device);
            wrc[id] = rc;
            wmsg[id] = em_last_error();
        }
        while (rc == EM_OK) {
            const int i = next.fetch_add(1);
            if (i >= nsnap) break;
            em_snapshot &s = snaps[order[i]];
            s.status = run_snapshot(ctx, s, p);
            if (s.status != EM_OK && wrc[id] == EM_OK) {
                wrc[id] = s.status;
                wmsg[id] = std::string("snapshot ") + std::to_string(order[i]) + ": " + em_last_error();
            }
        }
        if (ctx) {
            launches += ctx->launches;
            em_ctx_destroy(ctx);
        }
        if (st) cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    for (int id = 0; id < nw; ++id) pool.emplace_back(worker, id);
    for (auto &th : pool) th.join();
    if (h_launches) *h_launches = launches.load();
    for (int id = 0; id < nw; ++id)
        if (wrc[id] != EM_OK) {
            em_set_error("%s", wmsg[id].c_str());
            return wrc[id];
        }
    return EM_OK;
}
