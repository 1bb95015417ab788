// Context, error reporting, parameters, handle accessors, and the
// device-wide sort / scan primitives (CUB) the other translation units use.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"

static thread_local char g_last_error[1024] = "";

void em_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

EM_EXPORT const char *em_last_error(void) { return g_last_error; }

cudaMemPool_t em_device_pool(int device)
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    static bool tried[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried[device]) {
        tried[device] = true;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t threshold = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
            pools[device] = pool;
        } else {
            cudaGetLastError();   // fall back to the default pool
        }
    }
    return pools[device];
}

EM_EXPORT void em_params_default(em_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->r_part = 0.05;
    p->r_leaf = 0.1;
    p->theta = 0.1;
    p->h_fact = 1.2;
    p->h_tol = 1e-13;
    p->max_newton = 50;
    p->precision = 0;
    p->fp64_threshold = 1e-5;
    p->knn_k = 48;
    p->leaf_max = 8;
    p->block_pairs = 0;
    p->h0_above = 0;
    p->fp32_err_ulps = 8;
}

EM_EXPORT int em_ctx_create(em_ctx **ctx, int device, void *stream)
{
    EM_CHECK_ARG(ctx);
    *ctx = nullptr;
    int ndev = 0;
    EM_CUDA(cudaGetDeviceCount(&ndev));
    EM_CHECK_ARG(device >= 0 && device < ndev);
    EM_CUDA(cudaSetDevice(device));
    int nsm = 0;
    EM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    em_ctx *c = new em_ctx;
    c->device = device;
    c->nsm = nsm > 0 ? nsm : 1;
    c->stream = (cudaStream_t)stream;
    c->launches = 0;
    c->timing = false;
    c->recorded[0] = c->recorded[1] = false;
    c->pairs_hint = 0;
    for (auto &e : c->ev) e = nullptr;
    *ctx = c;
    return EM_OK;
}

EM_EXPORT int em_ctx_destroy(em_ctx *ctx)
{
    if (ctx) {
        for (auto &e : ctx->ev)
            if (e) cudaEventDestroy(e);
    }
    delete ctx;
    return EM_OK;
}

EM_EXPORT int em_ctx_set_timing(em_ctx *ctx, int on)
{
    EM_CHECK_ARG(ctx);
    if (on && !ctx->ev[0]) {
        EM_CUDA(cudaSetDevice(ctx->device));
        for (auto &e : ctx->ev) EM_CUDA(cudaEventCreate(&e));
    }
    ctx->timing = on != 0;
    ctx->recorded[0] = ctx->recorded[1] = false;
    return EM_OK;
}

EM_EXPORT int em_ctx_map_times(em_ctx *ctx, double *ms_main, double *ms_recompute)
{
    EM_CHECK_ARG(ctx && ms_main && ms_recompute);
    *ms_main = *ms_recompute = 0.0;
    float t = 0.f;
    if (ctx->recorded[0]) {
        EM_CUDA(cudaEventSynchronize(ctx->ev[1]));
        EM_CUDA(cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]));
        *ms_main = t;
    }
    if (ctx->recorded[1]) {
        EM_CUDA(cudaEventSynchronize(ctx->ev[3]));
        EM_CUDA(cudaEventElapsedTime(&t, ctx->ev[2], ctx->ev[3]));
        *ms_recompute = t;
    }
    return EM_OK;
}

EM_EXPORT int em_ctx_sync(em_ctx *ctx)
{
    EM_CHECK_ARG(ctx);
    EM_CUDA(cudaStreamSynchronize(ctx->stream));
    return EM_OK;
}

EM_EXPORT int64_t em_ctx_launch_count(const em_ctx *ctx) { return ctx ? ctx->launches : -1; }

// ---- CUB wrappers -----------------------------------------------------------------

int em_exclusive_scan_i64(em_ctx *ctx, const int64_t *in, int64_t *out, int64_t n)
{
    DevArena tmp(ctx->stream, true);
    size_t bytes = 0;
    EM_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, ctx->stream));
    void *buf;
    EM_TRY(tmp.alloc((char **)&buf, bytes));
    EM_CUDA(cub::DeviceScan::ExclusiveSum(buf, bytes, in, out, n, ctx->stream));
    ctx->launches += 2;
    return EM_OK;
}

int em_exclusive_scan_i32(em_ctx *ctx, const int32_t *in, int32_t *out, int64_t n)
{
    DevArena tmp(ctx->stream, true);
    size_t bytes = 0;
    EM_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, ctx->stream));
    void *buf;
    EM_TRY(tmp.alloc((char **)&buf, bytes));
    EM_CUDA(cub::DeviceScan::ExclusiveSum(buf, bytes, in, out, n, ctx->stream));
    ctx->launches += 2;
    return EM_OK;
}

// Stable LSD radix sort of (key, value) pairs in place.
int em_sort_pairs_u64(em_ctx *ctx, uint64_t *keys, int32_t *vals, int64_t n, int end_bit)
{
    if (n <= 1) return EM_OK;
    DevArena tmp(ctx->stream, true);
    uint64_t *k2;
    int32_t *v2;
    EM_TRY(tmp.alloc(&k2, n));
    EM_TRY(tmp.alloc(&v2, n));
    cub::DoubleBuffer<uint64_t> kb(keys, k2);
    cub::DoubleBuffer<int32_t> vb(vals, v2);
    size_t bytes = 0;
    EM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, n, 0, end_bit, ctx->stream));
    void *buf;
    EM_TRY(tmp.alloc((char **)&buf, bytes));
    EM_CUDA(cub::DeviceRadixSort::SortPairs(buf, bytes, kb, vb, n, 0, end_bit, ctx->stream));
    if (kb.Current() != keys)
        EM_CUDA(cudaMemcpyAsync(keys, kb.Current(), n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
    if (vb.Current() != vals)
        EM_CUDA(cudaMemcpyAsync(vals, vb.Current(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->launches += (end_bit + 7) / 8 + 1;
    return EM_OK;
}

int em_sort_pairs_u32(em_ctx *ctx, uint32_t *keys, int32_t *vals, int64_t n, int end_bit)
{
    if (n <= 1) return EM_OK;
    DevArena tmp(ctx->stream, true);
    uint32_t *k2;
    int32_t *v2;
    EM_TRY(tmp.alloc(&k2, n));
    EM_TRY(tmp.alloc(&v2, n));
    cub::DoubleBuffer<uint32_t> kb(keys, k2);
    cub::DoubleBuffer<int32_t> vb(vals, v2);
    size_t bytes = 0;
    EM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, n, 0, end_bit, ctx->stream));
    void *buf;
    EM_TRY(tmp.alloc((char **)&buf, bytes));
    EM_CUDA(cub::DeviceRadixSort::SortPairs(buf, bytes, kb, vb, n, 0, end_bit, ctx->stream));
    if (kb.Current() != keys)
        EM_CUDA(cudaMemcpyAsync(keys, kb.Current(), n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    if (vb.Current() != vals)
        EM_CUDA(cudaMemcpyAsync(vals, vb.Current(), n * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->launches += (end_bit + 7) / 8 + 1;
    return EM_OK;
}

// ---- handle accessors -----------------------------------------------------------

#define COPY_OUT(dst, src, count)                                                                  \
    do {                                                                                           \
        if (dst)                                                                                   \
            EM_CUDA(cudaMemcpyAsync(dst, src, (size_t)(count) * sizeof(*(src)),                    \
                                    cudaMemcpyDeviceToDevice, ctx->stream));                       \
    } while (0)

EM_EXPORT int tree_info(const em_tree *t, int64_t *n_particles, int64_t *n_nodes, int32_t *depth)
{
    EM_CHECK_ARG(t);
    if (n_particles) *n_particles = t->n;
    if (n_nodes) *n_nodes = t->nnode;
    if (depth) *depth = t->depth;
    return EM_OK;
}

__global__ void k_interleave3(int64_t n, const double *a, const double *b, const double *c, double *out)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[3 * k] = a[k];
    out[3 * k + 1] = b[k];
    out[3 * k + 2] = c[k];
}

EM_EXPORT int tree_get(em_ctx *ctx, const em_tree *t, int32_t *d_perm, uint64_t *d_label, int32_t *d_level,
                       int32_t *d_parent, int32_t *d_first, int32_t *d_count, int32_t *d_first_child,
                       int32_t *d_nchild, double *d_mass, double *d_com, double *d_size)
{
    EM_CHECK_ARG(ctx && t);
    COPY_OUT(d_perm, t->perm, t->n);
    COPY_OUT(d_label, t->label, t->nnode);
    COPY_OUT(d_level, t->level, t->nnode);
    COPY_OUT(d_parent, t->parent, t->nnode);
    COPY_OUT(d_first, t->first, t->nnode);
    COPY_OUT(d_count, t->count, t->nnode);
    COPY_OUT(d_first_child, t->first_child, t->nnode);
    COPY_OUT(d_nchild, t->nchild, t->nnode);
    COPY_OUT(d_mass, t->mass, t->nnode);
    COPY_OUT(d_size, t->size, t->nnode);
    if (d_com && t->nnode) {
        k_interleave3<<<em_grid(t->nnode, 256), 256, 0, ctx->stream>>>(t->nnode, t->cx, t->cy, t->cz, d_com);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int tree_destroy(em_tree *t)
{
    if (!t) return EM_OK;
    t->mem.release();
    delete t;
    return EM_OK;
}

EM_EXPORT int pseudo_info(const em_pseudo *ps, int64_t *n_pseudo, int64_t *n_status)
{
    EM_CHECK_ARG(ps);
    if (n_pseudo) *n_pseudo = ps->n;
    if (n_status)
        for (int k = 0; k < 4; ++k) n_status[k] = ps->nstatus[k];
    return EM_OK;
}

EM_EXPORT int pseudo_get(em_ctx *ctx, const em_pseudo *ps, double *d_x, double *d_y, double *d_z, double *d_h,
                         double *d_m, int64_t *d_origin, int32_t *d_first, int32_t *d_count, int32_t *d_status)
{
    EM_CHECK_ARG(ctx && ps);
    COPY_OUT(d_x, ps->x, ps->n);
    COPY_OUT(d_y, ps->y, ps->n);
    COPY_OUT(d_z, ps->z, ps->n);
    COPY_OUT(d_h, ps->h, ps->n);
    COPY_OUT(d_m, ps->m, ps->n);
    COPY_OUT(d_origin, ps->origin, ps->n);
    COPY_OUT(d_first, ps->first, ps->n);
    COPY_OUT(d_count, ps->count, ps->n);
    COPY_OUT(d_status, ps->status, ps->n);
    return EM_OK;
}

EM_EXPORT int pseudo_destroy(em_pseudo *ps)
{
    if (!ps) return EM_OK;
    ps->mem.release();
    delete ps;
    return EM_OK;
}

EM_EXPORT int voronoi_info(const em_voronoi *v, int64_t *ncell, int64_t *nface, int64_t *nfv)
{
    EM_CHECK_ARG(v);
    if (ncell) *ncell = v->ncell;
    if (nface) *nface = v->nface;
    if (nfv) *nfv = v->nfv;
    return EM_OK;
}

EM_EXPORT int voronoi_get(em_ctx *ctx, const em_voronoi *v, int64_t *d_cell_face_off, int64_t *d_face_vert_off,
                          double *d_verts, double *d_normals, int64_t *d_nbr, double *d_volume)
{
    EM_CHECK_ARG(ctx && v);
    COPY_OUT(d_cell_face_off, v->cell_face_off, v->ncell + 1);
    COPY_OUT(d_face_vert_off, v->face_vert_off, v->nface + 1);
    COPY_OUT(d_verts, v->verts, 3 * v->nfv);
    COPY_OUT(d_normals, v->normals, 3 * v->nface);
    COPY_OUT(d_nbr, v->nbr, v->nface);
    COPY_OUT(d_volume, v->volume, v->ncell);
    return EM_OK;
}

EM_EXPORT int voronoi_destroy(em_voronoi *v)
{
    if (!v) return EM_OK;
    v->mem.release();
    delete v;
    return EM_OK;
}

EM_EXPORT int pairs_info(const em_pairs *pr, int64_t *npairs, int64_t *np, int64_t *ncell)
{
    EM_CHECK_ARG(pr);
    if (npairs) *npairs = pr->npairs;
    if (np) *np = pr->np;
    if (ncell) *ncell = pr->ncell;
    return EM_OK;
}

EM_EXPORT int pairs_get(em_ctx *ctx, const em_pairs *pr, int32_t *d_pair_i, int32_t *d_pair_j, uint8_t *d_near,
                        int64_t *d_cell_pair_off)
{
    EM_CHECK_ARG(ctx && pr);
    COPY_OUT(d_pair_i, pr->pair_i, pr->npairs);
    COPY_OUT(d_pair_j, pr->pair_j, pr->npairs);
    COPY_OUT(d_near, pr->near, pr->npairs);
    COPY_OUT(d_cell_pair_off, pr->cell_pair_off, pr->ncell + 1);
    return EM_OK;
}

EM_EXPORT int pairs_destroy(em_pairs *pr)
{
    if (!pr) return EM_OK;
    pr->mem.release();
    delete pr;
    return EM_OK;
}
