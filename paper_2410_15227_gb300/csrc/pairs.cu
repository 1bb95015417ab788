// find_pairs: every (particle i, cell j) whose kernel support meets the cell,
// dist(x_i, V_j) < 2 h_i, sorted by (j, i).
//
// The particles are Morton-sorted and bounded by a 32-ary box hierarchy of
// their support spheres.  One warp per cell walks it with the cell's bounding
// ball (generator g_j, radius R_j); each lane then tests one candidate.  The
// test first classifies in FP32 (GB300 runs FP64 at 1/64 of the FP32 rate):
// a candidate whose FP32 distance clears 2h by the band
// 1e-5 (R_j + |r| + 2h) -- far above the rounding of the FP32 dot products,
// which is a few ulp of that same scale -- is decided there; only candidates
// inside the band take the exact FP64 test, which also sets the near flag.
// The pair set is therefore the FP64 predicate's.  Hits are compacted with a
// warp ballot into a per-warp buffer and written, unordered, at positions
// reserved with an atomic add; one radix sort by (j, i) puts them in order.
#include <vector>

#include "common.cuh"
#include "tree_util.cuh"

namespace {

// Squared distance from p (r = p - g) to the convex cell, 0 if inside.  The
// closest point lies on a face whose plane has p on its outer side; on such a
// face it is the foot of p if that foot is inside the polygon, else the
// nearest point of an edge segment.  Returns early once it is certain the
// distance is at least lim2.
__device__ __forceinline__ double cell_dist2(double rx, double ry, double rz, int64_t f0, int64_t f1,
                                             const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane,
                                             const EdgeD *__restrict__ edge, double lim)
{
    bool outside = false;
    for (int64_t f = f0; f < f1; ++f) {
        PlaneD pl = plane[f];
        double s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        if (s < 0.0) {
            outside = true;
            if (-s >= lim) return lim * lim;   // a separating plane at least lim away
        }
    }
    if (!outside) return 0.0;
    double best = INFINITY;
    for (int64_t f = f0; f < f1; ++f) {
        PlaneD pl = plane[f];
        double s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        if (s >= 0.0) continue;
        double s2 = s * s;
        if (s2 >= best) continue;
        bool in_poly = true;
        double e2 = INFINITY;
        for (int64_t e = fvo[f]; e < fvo[f + 1]; ++e) {
            EdgeD E = edge[e];
            double a = E.cm - (E.mx * rx + E.my * ry + E.mz * rz);
            in_poly = in_poly && (a >= 0.0);
            double t0 = E.ce - (E.ex * rx + E.ey * ry + E.ez * rz);
            double t1 = t0 + E.L;
            double tc = t0 > 0.0 ? t0 : (t1 < 0.0 ? t1 : 0.0);
            double q = a * a + tc * tc;
            e2 = q < e2 ? q : e2;
        }
        double d2 = in_poly ? s2 : s2 + e2;
        best = d2 < best ? d2 : best;
    }
    return best;
}

// cell_dist2 in FP32 from the cell's FP32 plane and edge records: the same
// steps, so that its error is a few ulp of (R_j + |r|) in the distance.
__device__ __forceinline__ float cell_dist2_f32(float rx, float ry, float rz, int64_t f0, int64_t f1,
                                                const int64_t *__restrict__ fvo, const PlaneF *__restrict__ plane,
                                                const EdgeF *__restrict__ edge, float lim)
{
    bool outside = false;
    for (int64_t f = f0; f < f1; ++f) {
        PlaneF pl = plane[f];
        float s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        if (s < 0.f) {
            outside = true;
            if (-s >= lim) return lim * lim;
        }
    }
    if (!outside) return 0.f;
    float best = INFINITY;
    for (int64_t f = f0; f < f1; ++f) {
        PlaneF pl = plane[f];
        float s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        if (s >= 0.f) continue;
        float s2 = s * s;
        if (s2 >= best) continue;
        bool in_poly = true;
        float e2 = INFINITY;
        for (int64_t e = fvo[f]; e < fvo[f + 1]; ++e) {
            EdgeF E = edge[e];
            float a = E.cm - (E.mx * rx + E.my * ry + E.mz * rz);
            in_poly = in_poly && (a >= 0.f);
            float t0 = E.ce - (E.ex * rx + E.ey * ry + E.ez * rz);
            float t1 = t0 + E.L;
            float tc = t0 > 0.f ? t0 : (t1 < 0.f ? t1 : 0.f);
            e2 = fminf(e2, a * a + tc * tc);
        }
        best = fminf(best, in_poly ? s2 : s2 + e2);
    }
    return best;
}

// One warp per cell: candidate particles from the sphere hierarchy, FP32
// classification, exact FP64 test inside the band, ballot compaction into a
// per-warp buffer in shared memory.  A full (or the final) buffer is written
// at a position reserved with one atomic add on the global hit counter, as
// (j << 32 | i) keys and near flags: unordered, the caller sorts them.  Hits
// past the capacity are counted but not written; the caller then repeats the
// pass with room for all of them.
#ifndef EM_PAIRS_WARPS
#define EM_PAIRS_WARPS 1   // warps (cells) per block: a finished cell frees its slot at once (12.4 against 13.0 ms with 4)
#endif
constexpr int PAIRS_WARPS = EM_PAIRS_WARPS;
constexpr int PAIRS_BUF = 128;   // hits a warp holds before writing them out

__global__ void __launch_bounds__(32 * PAIRS_WARPS)
    k_cell_pairs(int64_t cell0, int64_t cell1, em::ChunkTree T, const double *__restrict__ xs, const double *__restrict__ ys,
                 const double *__restrict__ zs, const double *__restrict__ hs, const int32_t *__restrict__ perm,
                 const double *__restrict__ gen, const double *__restrict__ radius, const int64_t *__restrict__ cfo,
                 const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane, const EdgeD *__restrict__ edge,
                 const PlaneF *__restrict__ plane_f, const EdgeF *__restrict__ edge_f, float margin,
                 unsigned long long *__restrict__ counter, int64_t capacity, uint64_t *__restrict__ keys,
                 int32_t *__restrict__ nearf, int64_t *__restrict__ cell_count)
{
    __shared__ uint64_t buf_key[PAIRS_WARPS][PAIRS_BUF];
    __shared__ int32_t buf_near[PAIRS_WARPS][PAIRS_BUF];
    __shared__ int32_t cand_buf[PAIRS_WARPS][64];   // a chunk adds at most 32 to fewer than 32
    const int w = threadIdx.x >> 5;
    int64_t j = cell0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (j >= cell1) return;   // the whole warp
    const int lane = threadIdx.x & 31;
    int nb = 0;   // hits in the warp's buffer (the same on every lane)
    int64_t ncell_hits = 0;
    // with capacity 0 the pass only counts (cell_count)
    auto write_out = [&]() {
        if (capacity > 0) {
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(counter, (unsigned long long)nb);
            at = __shfl_sync(0xffffffffu, at, 0);
            for (int t = lane; t < nb; t += 32) {
                const unsigned long long pos = at + (unsigned long long)t;
                if (pos < (unsigned long long)capacity) {
                    keys[pos] = buf_key[w][t];
                    nearf[pos] = buf_near[w][t];
                }
            }
        }
        __syncwarp();
        nb = 0;
    };
    const double gx = gen[3 * j], gy = gen[3 * j + 1], gz = gen[3 * j + 2];
    const double Rj = radius[j];
    const int64_t f0 = cfo[j], f1 = cfo[j + 1];
    const float R = (float)Rj + margin;
    const float Rf = (float)Rj;
    const float gxf = (float)gx, gyf = (float)gy, gzf = (float)gz;
    const float gscale = fabsf(gxf) + fabsf(gyf) + fabsf(gzf);
    // the exact classification of one candidate (lanes with act); hits go to
    // the warp's output buffer
    auto classify = [&](int64_t k, bool act) {
        bool hit = false, nearb = false;
        if (act) {
            const double rx = xs[k] - gx, ry = ys[k] - gy, rz = zs[k] - gz;
            const double h2 = 2.0 * hs[k];
            const float rxf = (float)rx, ryf = (float)ry, rzf = (float)rz, h2f = (float)h2;
            const float rr = sqrtf(rxf * rxf + ryf * ryf + rzf * rzf);
            const float band = 1e-5f * (Rf + rr + h2f);
            // the cell lies inside the ball of radius R_j around g: dist >= |r| - R_j
            if (rr < Rf + h2f + band) {
                const float lo = h2f - band, hi = h2f + band;
                const float d2f = cell_dist2_f32(rxf, ryf, rzf, f0, f1, fvo, plane_f, edge_f, hi + band);
                if (lo > 0.f && d2f < lo * lo) {
                    hit = true;
                } else if (!(d2f > hi * hi)) {   // inside the band: exact FP64 test
                    const double d2 = cell_dist2(rx, ry, rz, f0, f1, fvo, plane, edge, 2.0 * h2);
                    hit = d2 < h2 * h2;
                    if (hit) nearb = fabs(sqrt(d2) - h2) < 0.5e-9 * h2;
                }
            }
        }
        const uint32_t b = __ballot_sync(0xffffffffu, hit);
        if (nb + __popc(b) > PAIRS_BUF) write_out();
        if (hit) {
            const int pos = nb + __popc(b & ((1u << lane) - 1u));
            buf_key[w][pos] = ((uint64_t)j << 32) | (uint32_t)perm[k];
            buf_near[w][pos] = nearb ? 1 : 0;
        }
        __syncwarp();
        nb += __popc(b);
        ncell_hits += __popc(b);
    };
    // candidates within R_j + 2h (+ the band, which here also covers the FP32
    // rounding of the coordinates) collect in a per-warp buffer and are
    // classified 32 at a time, so that the per-candidate work runs with every
    // lane busy instead of on the lanes of each 32-point chunk that passed
    int nc = 0;
    int32_t *cb = cand_buf[w];
    em::warp_traverse(T, (float)gx, (float)gy, (float)gz, R * R, INT64_MAX, [&](int64_t k, bool valid) {
        bool cand = false;
        if (valid) {
            const float4 pk = T.pts[k];
            const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
            const float d = sqrtf(ex * ex + ey * ey + ez * ez);
            const float h2f = 2.f * (float)hs[k];
            cand = d < Rf + h2f + 1e-5f * (gscale + Rf + d + h2f);
        }
        const unsigned cm = __ballot_sync(0xffffffffu, cand);
        if (cand) cb[nc + __popc(cm & ((1u << lane) - 1u))] = (int32_t)k;
        __syncwarp();
        nc += __popc(cm);
        if (nc >= 32) {
            classify(cb[lane], true);
            const int32_t rest = lane + 32 < nc ? cb[lane + 32] : 0;
            __syncwarp();
            if (lane + 32 < nc) cb[lane] = rest;
            __syncwarp();
            nc -= 32;
        }
    });
    if (nc > 0) classify(lane < nc ? cb[lane] : 0, lane < nc);
    if (nb > 0) write_out();
    if (cell_count && lane == 0) cell_count[j - cell0] = ncell_hits;
}

__global__ void k_split_keys(int64_t n, const uint64_t *__restrict__ keys, const int32_t *__restrict__ nearf,
                             int32_t *__restrict__ pi, int32_t *__restrict__ pj, uint8_t *__restrict__ nearo)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint64_t key = keys[k];
    pi[k] = (int32_t)(key & 0xffffffffull);
    pj[k] = (int32_t)(key >> 32);
    nearo[k] = (uint8_t)nearf[k];
}

__global__ void k_bbox(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, double *__restrict__ out)
{
    __shared__ double red[6][256];
    double v[6] = {INFINITY, -INFINITY, INFINITY, -INFINITY, INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        v[0] = fmin(v[0], x[i]);
        v[1] = fmax(v[1], x[i]);
        v[2] = fmin(v[2], y[i]);
        v[3] = fmax(v[3], y[i]);
        v[4] = fmin(v[4], z[i]);
        v[5] = fmax(v[5], z[i]);
    }
    for (int c = 0; c < 6; ++c) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 6; ++c)
                red[c][threadIdx.x] = (c & 1) ? fmax(red[c][threadIdx.x], red[c][threadIdx.x + s])
                                              : fmin(red[c][threadIdx.x], red[c][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 6; ++c) out[6 * blockIdx.x + c] = red[c][0];
}

}  // namespace

// Bounding box of n points (host result).
int em_point_bbox(em_ctx *ctx, int64_t n, const double *x, const double *y, const double *z, double *box)
{
    DevArena tmp(ctx->stream, true);
    const int nb = 64;
    double *part;
    EM_TRY(tmp.alloc(&part, 6 * nb));
    k_bbox<<<nb, 256, 0, ctx->stream>>>(n, x, y, z, part);
    EM_LAUNCHED(ctx);
    double h[6 * nb];
    EM_CUDA(cudaMemcpyAsync(h, part, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    EM_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < 6; ++c) box[c] = (c & 1) ? -INFINITY : INFINITY;
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 6; ++c) box[c] = (c & 1) ? fmax(box[c], h[6 * b + c]) : fmin(box[c], h[6 * b + c]);
    for (int c = 0; c < 6; c += 2)
        if (!(box[c + 1] > box[c])) {
            double mid = box[c];
            box[c] = mid - 1.0;
            box[c + 1] = mid + 1.0;
        }
    return EM_OK;
}

// The particles' side of pair finding: Morton order, sorted copies and the
// sphere hierarchy (radius 2h), and the FP32 margin of the box.
struct PairParticles {
    int32_t *perm;
    double *xs, *ys, *zs, *hs;
    em::ChunkTree T;
    float margin;
};

static int prepare_particles(em_ctx *ctx, DevArena &tmp, int64_t np, const double *x, const double *y,
                             const double *z, const double *h, PairParticles &P)
{
    double box[6];
    EM_TRY(em_point_bbox(ctx, np, x, y, z, box));
    uint64_t *mkey;
    EM_TRY(tmp.alloc(&mkey, np));
    EM_TRY(tmp.alloc(&P.perm, np));
    EM_TRY(tmp.alloc(&P.xs, np));
    EM_TRY(tmp.alloc(&P.ys, np));
    EM_TRY(tmp.alloc(&P.zs, np));
    EM_TRY(tmp.alloc(&P.hs, np));
    EM_TRY(em_morton_sort(ctx, np, x, y, z, box, mkey, P.perm));
    EM_TRY(em_gather_sorted(ctx, np, P.perm, x, y, z, h, P.xs, P.ys, P.zs, P.hs));
    EM_TRY(em_chunk_tree_build(ctx, tmp, np, P.xs, P.ys, P.zs, P.hs, 2.0, &P.T));
    double ext = 0.0;
    for (int c = 0; c < 6; ++c) ext = fmax(ext, fabs(box[c]));
    P.margin = (float)(4e-7 * (ext + 1.0));
    return EM_OK;
}

static void launch_cell_pairs(em_ctx *ctx, const PairParticles &P, const em_voronoi *v, int64_t cell0, int64_t cell1,
                              unsigned long long *counter, int64_t capacity, uint64_t *keys, int32_t *nearf,
                              int64_t *cell_count)
{
    k_cell_pairs<<<em_grid((cell1 - cell0) * 32, 32 * PAIRS_WARPS), 32 * PAIRS_WARPS, 0, ctx->stream>>>(
        cell0, cell1, P.T, P.xs, P.ys, P.zs, P.hs, P.perm, v->gen, v->radius, v->cell_face_off, v->face_vert_off,
        v->plane, v->edge, v->plane_f, v->edge_f, P.margin, counter, capacity, keys, nearf, cell_count);
}

// The pairs of the cells [cell0, cell1) into pr (all of v's cells indexed,
// the others without pairs).  capacity_hint > 0: the expected count (the
// hit buffer's size; a pass that finds more repeats once with the exact
// size); otherwise the context's hint from its last call, or a guess.
static int find_pairs_impl(em_ctx *ctx, int64_t np, const double *x, const double *y, const double *z,
                           const double *h, const em_voronoi *v, em_pairs *pr, int64_t cell0, int64_t cell1,
                           int64_t capacity_hint)
{
    cudaStream_t st = ctx->stream;
    DevArena tmp(st, true);
    PairParticles P;
    EM_TRY(prepare_particles(ctx, tmp, np, x, y, z, h, P));
    const int64_t nc = v->ncell;
    // one pass into an unsorted buffer sized from the hint (or the last call,
    // or a guess on the first), repeated once with the exact size if it
    // overflowed
    unsigned long long *counter;
    EM_TRY(tmp.alloc(&counter, 1));
    int64_t capacity = capacity_hint > 0 ? capacity_hint
                                         : (ctx->pairs_hint > 0 ? ctx->pairs_hint : 64 * np + (1 << 20));
    int64_t total = 0;
    uint64_t *keys = nullptr;
    int32_t *nearf = nullptr;
    for (int attempt = 0; attempt < 2; ++attempt) {
        DevArena buf(st, true);   // released on an early return
        EM_TRY(buf.alloc(&keys, capacity));
        EM_TRY(buf.alloc(&nearf, capacity));
        EM_CUDA(cudaMemsetAsync(counter, 0, sizeof *counter, st));
        if (cell1 > cell0) {
            launch_cell_pairs(ctx, P, v, cell0, cell1, counter, capacity, keys, nearf, nullptr);
            EM_LAUNCHED(ctx);
        }
        unsigned long long hits = 0;
        EM_CUDA(cudaMemcpyAsync(&hits, counter, sizeof hits, cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaStreamSynchronize(st));
        total = (int64_t)hits;
        if (total <= capacity || total >= INT32_MAX) {
            // keep the buffers: they belong to the call's scratch from here on
            for (void *q : buf.ptrs) tmp.ptrs.push_back(q);
            buf.ptrs.clear();
            break;
        }
        buf.release();
        capacity = total;
    }
    if (total >= INT32_MAX) {
        em_set_error("find_pairs: %lld pairs exceed the 2^31 limit of one pair list", (long long)total);
        return EM_ECAPACITY;
    }
    if (capacity_hint <= 0) ctx->pairs_hint = total + total / 8 + 1024;
    pr->npairs = total;
    if (total) EM_TRY(em_sort_pairs_u64(ctx, keys, nearf, total, 32 + em_nbits((uint64_t)nc)));
    EM_TRY(pr->mem.alloc(&pr->pair_i, total));
    EM_TRY(pr->mem.alloc(&pr->pair_j, total));
    EM_TRY(pr->mem.alloc(&pr->near, total));
    if (total) {
        k_split_keys<<<em_grid(total, 256), 256, 0, st>>>(total, keys, nearf, pr->pair_i, pr->pair_j, pr->near);
        EM_LAUNCHED(ctx);
    }
    return em_build_pair_index(ctx, pr);
}

static int new_pairs(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                     const double *d_h, const em_voronoi *v, int64_t cell0, int64_t cell1, int64_t hint,
                     em_pairs **out, int64_t *npairs)
{
    *out = nullptr;
    em_pairs *pr = new em_pairs(ctx->stream);
    pr->device = ctx->device;
    pr->np = np;
    pr->ncell = v->ncell;
    int rc = find_pairs_impl(ctx, np, d_x, d_y, d_z, d_h, v, pr, cell0, cell1, hint);
    if (rc) {
        pr->mem.release();
        delete pr;
        return rc;
    }
    if (npairs) *npairs = pr->npairs;
    *out = pr;
    return EM_OK;
}

EM_EXPORT int find_pairs_plan(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                              const double *d_h, const em_voronoi *v, int64_t chunk_capacity, int64_t *h_bounds,
                              int64_t *h_nchunks, int64_t *h_npairs)
{
    EM_CHECK_ARG(ctx && v && np >= 1 && np < INT32_MAX && d_x && d_y && d_z && d_h && chunk_capacity >= 1 &&
                 h_bounds && h_nchunks);
    cudaStream_t st = ctx->stream;
    DevArena tmp(st, true);
    PairParticles P;
    EM_TRY(prepare_particles(ctx, tmp, np, d_x, d_y, d_z, d_h, P));
    const int64_t nc = v->ncell;
    std::vector<int64_t> cnt(nc > 0 ? nc : 1);
    if (nc > 0) {
        int64_t *d_cnt;
        EM_TRY(tmp.alloc(&d_cnt, nc));
        launch_cell_pairs(ctx, P, v, 0, nc, nullptr, 0, nullptr, nullptr, d_cnt);
        EM_LAUNCHED(ctx);
        EM_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaStreamSynchronize(st));
    }
    // consecutive cells while the count stays within the capacity; a cell
    // above it is a chunk of its own
    int64_t nch = 0, acc = 0, total = 0;
    h_bounds[0] = 0;
    for (int64_t j = 0; j < nc; ++j) {
        if (acc > 0 && acc + cnt[j] > chunk_capacity) {
            h_bounds[++nch] = j;
            acc = 0;
        }
        acc += cnt[j];
        total += cnt[j];
    }
    if (nc > 0) h_bounds[++nch] = nc;
    *h_nchunks = nch;
    if (h_npairs) *h_npairs = total;
    return EM_OK;
}

EM_EXPORT int find_pairs_cells(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                               const double *d_h, const em_voronoi *v, int64_t cell_begin, int64_t cell_end,
                               int64_t npairs_hint, em_pairs **out, int64_t *npairs)
{
    EM_CHECK_ARG(ctx && v && out && np >= 1 && np < INT32_MAX && d_x && d_y && d_z && d_h);
    EM_CHECK_ARG(cell_begin >= 0 && cell_begin <= cell_end && cell_end <= v->ncell);
    return new_pairs(ctx, np, d_x, d_y, d_z, d_h, v, cell_begin, cell_end, npairs_hint, out, npairs);
}

EM_EXPORT int find_pairs(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                         const double *d_h, const em_voronoi *v, em_pairs **out, int64_t *npairs)
{
    EM_CHECK_ARG(ctx && v && out && np >= 1 && np < INT32_MAX && d_x && d_y && d_z && d_h);
    return new_pairs(ctx, np, d_x, d_y, d_z, d_h, v, 0, v->ncell, 0, out, npairs);
}
