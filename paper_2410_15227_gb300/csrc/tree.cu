// build_tree: Morton-ordered octree with node mass, centre of mass and size
// (the gravity tree of Section 2.2.1, octree form).
//
// Rounding is fixed so that the result is the same bit for bit on any
// device: products and sums that feed the centre of mass and the node size
// use explicit round-to-nearest intrinsics (no fused multiply-add), leaves
// sum their particles in Morton order and internal nodes sum their children
// in octant order.
#include "common.cuh"
#include "tree_util.cuh"

namespace {

__global__ void k_morton(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, double xlo, double xhi, double ylo, double yhi, double zlo,
                         double zhi, uint64_t *__restrict__ key, int32_t *__restrict__ idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = em::morton_key(x[i], y[i], z[i], xlo, xhi, ylo, yhi, zlo, zhi);
    idx[i] = (int32_t)i;
}

__global__ void k_gather4(int64_t n, const int32_t *__restrict__ perm, const double *__restrict__ x,
                          const double *__restrict__ y, const double *__restrict__ z, const double *__restrict__ m,
                          double *__restrict__ xs, double *__restrict__ ys, double *__restrict__ zs,
                          double *__restrict__ ms)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int32_t i = perm[k];
    xs[k] = x[i];
    ys[k] = y[i];
    zs[k] = z[i];
    if (m) ms[k] = m[i];
}

// Split nodes [lo, hi) of one level: child boundaries by binary search on the
// next 3-bit digit of the sorted keys.
__global__ void k_split_count(int64_t lo, int64_t hi, int level, int leaf_max, const uint64_t *__restrict__ key,
                              const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                              int32_t *__restrict__ nchild, int32_t *__restrict__ bounds)
{
    int64_t a = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= hi) return;
    int32_t f = first[a], c = count[a];
    int32_t *bd = bounds + 9 * (a - lo);
    if (c <= leaf_max || level >= em::kMortonBits) {
        nchild[a] = 0;
        return;
    }
    int shift = 3 * (em::kMortonBits - 1 - level);
    int nc = 0;
    bd[0] = f;
    for (int o = 1; o <= 8; ++o) {
        // first position in [f, f + c) whose digit is >= o
        int32_t l = bd[o - 1], r = f + c;
        while (l < r) {
            int32_t mid = l + (r - l) / 2;
            if ((int)((key[mid] >> shift) & 7ull) < o) l = mid + 1;
            else r = mid;
        }
        bd[o] = l;
        nc += (bd[o] > bd[o - 1]);
    }
    nchild[a] = nc;
}

__global__ void k_split_emit(int64_t lo, int64_t hi, int64_t next, const int32_t *__restrict__ nchild,
                             const int32_t *__restrict__ cofs, const int32_t *__restrict__ bounds,
                             int32_t *__restrict__ first_child, uint64_t *__restrict__ label,
                             int32_t *__restrict__ levelv, int32_t *__restrict__ parent, int32_t *__restrict__ first,
                             int32_t *__restrict__ count, int level)
{
    int64_t a = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= hi) return;
    if (nchild[a] == 0) {
        first_child[a] = -1;
        return;
    }
    int64_t c = next + cofs[a - lo];
    first_child[a] = (int32_t)c;
    const int32_t *bd = bounds + 9 * (a - lo);
    uint64_t lab = label[a];
    for (int o = 0; o < 8; ++o) {
        if (bd[o + 1] == bd[o]) continue;
        label[c] = lab * 8ull + (uint64_t)o;
        levelv[c] = level + 1;
        parent[c] = (int32_t)a;
        first[c] = bd[o];
        count[c] = bd[o + 1] - bd[o];
        ++c;
    }
}

// One level of bottom-up sums (deepest level first).
__global__ void k_node_sums(int64_t lo, int64_t hi, const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                            const int32_t *__restrict__ first_child, const int32_t *__restrict__ nchild,
                            const double *__restrict__ xs, const double *__restrict__ ys, const double *__restrict__ zs,
                            const double *__restrict__ ms, double *__restrict__ mass, double *__restrict__ mx,
                            double *__restrict__ my, double *__restrict__ mz, double *__restrict__ cx,
                            double *__restrict__ cy, double *__restrict__ cz)
{
    int64_t a = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= hi) return;
    double sm = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    if (nchild[a] == 0) {
        for (int32_t k = first[a]; k < first[a] + count[a]; ++k) {
            double mk = ms[k];
            sm = __dadd_rn(sm, mk);
            sx = __dadd_rn(sx, __dmul_rn(mk, xs[k]));
            sy = __dadd_rn(sy, __dmul_rn(mk, ys[k]));
            sz = __dadd_rn(sz, __dmul_rn(mk, zs[k]));
        }
    } else {
        for (int32_t c = first_child[a]; c < first_child[a] + nchild[a]; ++c) {
            sm = __dadd_rn(sm, mass[c]);
            sx = __dadd_rn(sx, mx[c]);
            sy = __dadd_rn(sy, my[c]);
            sz = __dadd_rn(sz, mz[c]);
        }
    }
    mass[a] = sm;
    mx[a] = sx;
    my[a] = sy;
    mz[a] = sz;
    cx[a] = __ddiv_rn(sx, sm);
    cy[a] = __ddiv_rn(sy, sm);
    cz[a] = __ddiv_rn(sz, sm);
}

// s_node = max over constituents of |x - COM|.  Nodes are cut into chunks of
// SIZE_CHUNK constituents, one warp per chunk, so that the root's million
// particles do not fall to one warp; each chunk raises its node's r^2 with an
// atomic max on the bit pattern (non-negative doubles order like their bits).
// Every term is rounded as before and max does not depend on the order, so
// the result is the same bit for bit.
constexpr int SIZE_CHUNK = 1024;

__global__ void k_size_chunks(int64_t nnode, const int32_t *__restrict__ count, int64_t *__restrict__ nchunk)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < nnode) nchunk[a] = (count[a] + SIZE_CHUNK - 1) / SIZE_CHUNK;
}

__global__ void k_node_size(int64_t nnode, int64_t ntask, const int64_t *__restrict__ task_off,
                            const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                            const double *__restrict__ xs, const double *__restrict__ ys,
                            const double *__restrict__ zs, const double *__restrict__ cx,
                            const double *__restrict__ cy, const double *__restrict__ cz,
                            unsigned long long *__restrict__ r2bits)
{
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntask) return;
    int64_t lo = 0, hi = nnode;   // task_off[lo] <= t < task_off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (task_off[mid] <= t) lo = mid;
        else hi = mid;
    }
    const int64_t a = lo;
    const int64_t c = t - task_off[a];
    const double ax = cx[a], ay = cy[a], az = cz[a];
    const int32_t k0 = first[a] + (int32_t)(c * SIZE_CHUNK);
    const int32_t k1 = min(first[a] + count[a], k0 + SIZE_CHUNK);
    double r2 = 0.0;
    for (int32_t k = k0 + lane; k < k1; k += 32) {
        double dx = __dsub_rn(xs[k], ax), dy = __dsub_rn(ys[k], ay), dz = __dsub_rn(zs[k], az);
        double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        r2 = q > r2 ? q : r2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double q = __shfl_xor_sync(0xffffffffu, r2, o);
        r2 = q > r2 ? q : r2;
    }
    if (lane == 0) atomicMax(r2bits + a, (unsigned long long)__double_as_longlong(r2));
}

__global__ void k_size_finish(int64_t nnode, double *__restrict__ size)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a < nnode) size[a] = __dsqrt_rn(size[a]);   // the bits hold r^2 as a double
}

struct TopoArrays {
    uint64_t *label = nullptr;
    int32_t *level = nullptr, *parent = nullptr, *first = nullptr, *count = nullptr, *first_child = nullptr,
            *nchild = nullptr;
};

int alloc_topo(DevArena &mem, TopoArrays &t, int64_t cap)
{
    EM_TRY(mem.alloc(&t.label, cap));
    EM_TRY(mem.alloc(&t.level, cap));
    EM_TRY(mem.alloc(&t.parent, cap));
    EM_TRY(mem.alloc(&t.first, cap));
    EM_TRY(mem.alloc(&t.count, cap));
    EM_TRY(mem.alloc(&t.first_child, cap));
    EM_TRY(mem.alloc(&t.nchild, cap));
    return EM_OK;
}

int copy_topo(cudaStream_t s, TopoArrays &dst, const TopoArrays &src, int64_t n)
{
    EM_CUDA(cudaMemcpyAsync(dst.label, src.label, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.level, src.level, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.parent, src.parent, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.first, src.first, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.count, src.count, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.first_child, src.first_child, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    EM_CUDA(cudaMemcpyAsync(dst.nchild, src.nchild, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return EM_OK;
}

__global__ void k_root(uint64_t *label, int32_t *level, int32_t *parent, int32_t *first, int32_t *count, int32_t n)
{
    label[0] = 1;
    level[0] = 0;
    parent[0] = -1;
    first[0] = 0;
    count[0] = n;
}

}  // namespace

// Morton sort of n points: keys and permutation (stable: ties by index).
int em_morton_sort(em_ctx *ctx, int64_t n, const double *x, const double *y, const double *z, const double *box,
                   uint64_t *key, int32_t *perm)
{
    k_morton<<<em_grid(n, 256), 256, 0, ctx->stream>>>(n, x, y, z, box[0], box[1], box[2], box[3], box[4], box[5],
                                                       key, perm);
    EM_LAUNCHED(ctx);
    return em_sort_pairs_u64(ctx, key, perm, n, 3 * em::kMortonBits);
}

int em_gather_sorted(em_ctx *ctx, int64_t n, const int32_t *perm, const double *x, const double *y,
                     const double *z, const double *m, double *xs, double *ys, double *zs, double *ms)
{
    k_gather4<<<em_grid(n, 256), 256, 0, ctx->stream>>>(n, perm, x, y, z, m, xs, ys, zs, ms);
    EM_LAUNCHED(ctx);
    return EM_OK;
}

static int build_tree_impl(em_ctx *ctx, em_tree *t, const double *d_x, const double *d_y, const double *d_z,
                           const double *d_m, int leaf_max)
{
    const int64_t n = t->n;
    cudaStream_t st = ctx->stream;
    DevArena &mem = t->mem;
    EM_TRY(mem.alloc(&t->key, n));
    EM_TRY(mem.alloc(&t->perm, n));
    EM_TRY(mem.alloc(&t->xs, n));
    EM_TRY(mem.alloc(&t->ys, n));
    EM_TRY(mem.alloc(&t->zs, n));
    EM_TRY(mem.alloc(&t->ms, n));
    EM_TRY(em_morton_sort(ctx, n, d_x, d_y, d_z, t->box, t->key, t->perm));
    EM_TRY(em_gather_sorted(ctx, n, t->perm, d_x, d_y, d_z, d_m, t->xs, t->ys, t->zs, t->ms));

    // topology, level by level; the node arrays grow geometrically
    DevArena topo_mem(st, false);
    TopoArrays topo;
    int64_t cap = n / 2 + 1024;
    EM_TRY(alloc_topo(topo_mem, topo, cap));
    k_root<<<1, 1, 0, st>>>(topo.label, topo.level, topo.parent, topo.first, topo.count, (int32_t)n);
    EM_LAUNCHED(ctx);
    DevArena scratch(st, true);
    int32_t *bounds = nullptr, *cofs = nullptr;
    int64_t scratch_cap = 0;
    std::vector<int64_t> loff = {0, 1};
    int level = 0;
    int rc = EM_OK;
    for (;; ++level) {
        int64_t lo = loff[level], hi = loff[level + 1], nl = hi - lo;
        if (nl > scratch_cap) {
            scratch.release();
            scratch_cap = nl * 2;
            if ((rc = scratch.alloc(&bounds, 9 * scratch_cap)) || (rc = scratch.alloc(&cofs, scratch_cap))) break;
        }
        k_split_count<<<em_grid(nl, 128), 128, 0, st>>>(lo, hi, level, leaf_max, t->key, topo.first, topo.count,
                                                         topo.nchild, bounds);
        EM_LAUNCHED(ctx);
        if ((rc = em_exclusive_scan_i32(ctx, topo.nchild + lo, cofs, nl))) break;
        int32_t last[2] = {0, 0};
        cudaMemcpyAsync(&last[0], cofs + nl - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&last[1], topo.nchild + hi - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        EM_CUDA(cudaStreamSynchronize(st));
        int64_t total = (int64_t)last[0] + last[1];
        if (hi + total > cap) {
            int64_t ncap = (hi + total) * 2;
            DevArena nm(st, false);
            TopoArrays nt;
            if ((rc = alloc_topo(nm, nt, ncap))) { nm.release(); break; }
            if ((rc = copy_topo(st, nt, topo, hi))) { nm.release(); break; }
            topo_mem.release();
            topo_mem.ptrs = nm.ptrs;
            nm.ptrs.clear();
            topo = nt;
            cap = ncap;
        }
        k_split_emit<<<em_grid(nl, 128), 128, 0, st>>>(lo, hi, hi, topo.nchild, cofs, bounds, topo.first_child,
                                                        topo.label, topo.level, topo.parent, topo.first, topo.count,
                                                        level);
        EM_LAUNCHED(ctx);
        if (total == 0) break;
        loff.push_back(hi + total);
    }
    if (rc) {
        topo_mem.release();
        return rc;
    }
    // hand the topology arrays to the tree handle
    for (void *p : topo_mem.ptrs) mem.ptrs.push_back(p);
    topo_mem.ptrs.clear();
    t->label = topo.label;
    t->level = topo.level;
    t->parent = topo.parent;
    t->first = topo.first;
    t->count = topo.count;
    t->first_child = topo.first_child;
    t->nchild = topo.nchild;
    t->depth = level;
    t->level_off = loff;
    t->nnode = loff.back();
    const int64_t nn = t->nnode;
    EM_TRY(mem.alloc(&t->mass, nn));
    EM_TRY(mem.alloc(&t->mx, nn));
    EM_TRY(mem.alloc(&t->my, nn));
    EM_TRY(mem.alloc(&t->mz, nn));
    EM_TRY(mem.alloc(&t->cx, nn));
    EM_TRY(mem.alloc(&t->cy, nn));
    EM_TRY(mem.alloc(&t->cz, nn));
    EM_TRY(mem.alloc(&t->size, nn));
    for (int L = t->depth; L >= 0; --L) {
        int64_t lo = loff[L], hi = loff[L + 1];
        k_node_sums<<<em_grid(hi - lo, 128), 128, 0, st>>>(lo, hi, t->first, t->count, t->first_child, t->nchild,
                                                            t->xs, t->ys, t->zs, t->ms, t->mass, t->mx, t->my, t->mz,
                                                            t->cx, t->cy, t->cz);
        EM_LAUNCHED(ctx);
    }
    {
        DevArena tmp(st, true);
        int64_t *nchunk, *task_off;
        EM_TRY(tmp.alloc(&nchunk, nn + 1));
        EM_TRY(tmp.alloc(&task_off, nn + 1));
        EM_CUDA(cudaMemsetAsync(nchunk + nn, 0, sizeof(int64_t), st));
        k_size_chunks<<<em_grid(nn, 256), 256, 0, st>>>(nn, t->count, nchunk);
        EM_LAUNCHED(ctx);
        EM_TRY(em_exclusive_scan_i64(ctx, nchunk, task_off, nn + 1));
        int64_t ntask = 0;
        EM_CUDA(cudaMemcpyAsync(&ntask, task_off + nn, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaStreamSynchronize(st));
        EM_CUDA(cudaMemsetAsync(t->size, 0, nn * sizeof(double), st));
        k_node_size<<<em_grid(ntask * 32, 256), 256, 0, st>>>(nn, ntask, task_off, t->first, t->count, t->xs, t->ys,
                                                                t->zs, t->cx, t->cy, t->cz,
                                                                (unsigned long long *)t->size);
        EM_LAUNCHED(ctx);
        k_size_finish<<<em_grid(nn, 256), 256, 0, st>>>(nn, t->size);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int build_tree(em_ctx *ctx, int64_t n, const double *d_x, const double *d_y, const double *d_z,
                         const double *d_m, const double *h_box, int leaf_max, em_tree **out)
{
    EM_CHECK_ARG(ctx && out && h_box && d_x && d_y && d_z && d_m);
    EM_CHECK_ARG(n >= 1 && n < INT32_MAX);
    EM_CHECK_ARG(leaf_max >= 1 && leaf_max <= 64);
    EM_CHECK_ARG(h_box[1] > h_box[0] && h_box[3] > h_box[2] && h_box[5] > h_box[4]);
    *out = nullptr;
    em_tree *t = new em_tree(ctx->stream);
    t->device = ctx->device;
    t->n = n;
    for (int k = 0; k < 6; ++k) t->box[k] = h_box[k];
    int rc = build_tree_impl(ctx, t, d_x, d_y, d_z, d_m, leaf_max);
    if (rc) {
        t->mem.release();
        delete t;
        return rc;
    }
    *out = t;
    return EM_OK;
}

// ---------------------------------------------------------------------------
// Chunk tree (32-ary boxes over Morton-ordered items)
// ---------------------------------------------------------------------------

namespace {

__global__ void k_chunk_leaf(int64_t nbox, int64_t n, const double *__restrict__ xs, const double *__restrict__ ys,
                             const double *__restrict__ zs, const double *__restrict__ r, double rscale,
                             float4 *__restrict__ lo, float4 *__restrict__ hi, float4 *__restrict__ pts)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    int64_t e = (b + 1) * 32 < n ? (b + 1) * 32 : n;
    for (int64_t k = b * 32; k < e; ++k) {
        pts[k] = make_float4((float)xs[k], (float)ys[k], (float)zs[k], 0.f);
        double rr = r ? r[k] * rscale : 0.0;
        lx = fminf(lx, __double2float_rd(xs[k] - rr));
        ly = fminf(ly, __double2float_rd(ys[k] - rr));
        lz = fminf(lz, __double2float_rd(zs[k] - rr));
        hx = fmaxf(hx, __double2float_ru(xs[k] + rr));
        hy = fmaxf(hy, __double2float_ru(ys[k] + rr));
        hz = fmaxf(hz, __double2float_ru(zs[k] + rr));
    }
    lo[b] = make_float4(lx, ly, lz, 0.f);
    hi[b] = make_float4(hx, hy, hz, 0.f);
}

__global__ void k_chunk_up(int64_t nbox, int64_t nchild, const float4 *__restrict__ clo, const float4 *__restrict__ chi,
                           float4 *__restrict__ lo, float4 *__restrict__ hi)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    float4 l = make_float4(INFINITY, INFINITY, INFINITY, 0.f), h = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    int64_t e = (b + 1) * 32 < nchild ? (b + 1) * 32 : nchild;
    for (int64_t k = b * 32; k < e; ++k) {
        float4 a = clo[k], c = chi[k];
        l.x = fminf(l.x, a.x);
        l.y = fminf(l.y, a.y);
        l.z = fminf(l.z, a.z);
        h.x = fmaxf(h.x, c.x);
        h.y = fmaxf(h.y, c.y);
        h.z = fmaxf(h.z, c.z);
    }
    lo[b] = l;
    hi[b] = h;
}

}  // namespace

int em_chunk_tree_build(em_ctx *ctx, DevArena &mem, int64_t n, const double *xs, const double *ys, const double *zs,
                        const double *r, double rscale, em::ChunkTree *out)
{
    em::ChunkTree T;
    T.count[0] = n;
    for (int l = 0; l <= em::kMaxLevels; ++l) {
        T.lo[l] = nullptr;
        T.hi[l] = nullptr;
        if (l) T.count[l] = 0;
    }
    T.nlev = 0;
    T.pts = nullptr;
    if (n == 0) {
        *out = T;
        return EM_OK;
    }
    EM_TRY(mem.alloc(&T.pts, n));
    int l = 1;
    for (;; ++l) {
        if (l > em::kMaxLevels) {
            em_set_error("chunk tree: %lld items exceed %d levels", (long long)n, em::kMaxLevels);
            return EM_ECAPACITY;
        }
        T.count[l] = (T.count[l - 1] + 31) / 32;
        EM_TRY(mem.alloc(&T.lo[l], T.count[l]));
        EM_TRY(mem.alloc(&T.hi[l], T.count[l]));
        if (l == 1)
            k_chunk_leaf<<<em_grid(T.count[1], 128), 128, 0, ctx->stream>>>(T.count[1], n, xs, ys, zs, r, rscale,
                                                                             T.lo[1], T.hi[1], T.pts);
        else
            k_chunk_up<<<em_grid(T.count[l], 128), 128, 0, ctx->stream>>>(T.count[l], T.count[l - 1], T.lo[l - 1],
                                                                           T.hi[l - 1], T.lo[l], T.hi[l]);
        EM_LAUNCHED(ctx);
        if (T.count[l] <= 32) break;
    }
    T.nlev = l;
    *out = T;
    return EM_OK;
}
