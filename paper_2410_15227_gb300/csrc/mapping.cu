// Exact mapping (map_exact), cell densities, inverse mapping (map_back), and
// the import paths for cells and pair lists.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "exact.cuh"
#include "quad32.cuh"
#include "split.cuh"

using namespace em;

// ---------------------------------------------------------------------------
// Derived cell geometry in each generator's frame
// ---------------------------------------------------------------------------

// Per face (one thread each): the face's cell by binary search in the cell
// offsets, the plane records, and the face and cell ids of its vertices for
// the edge pass.
__global__ void k_prepare_faces(int64_t nface, int64_t ncell, const double *__restrict__ gen,
                                const int64_t *__restrict__ cfo, const int64_t *__restrict__ fvo,
                                const double *__restrict__ verts, const double *__restrict__ normals,
                                PlaneD *__restrict__ plane, PlaneF *__restrict__ plane_f,
                                PlaneF *__restrict__ plane_fl, int32_t *__restrict__ face_of_fv,
                                int32_t *__restrict__ cell_of_face)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nface) return;
    int64_t lo = 0, hi = ncell;   // cfo[lo] <= f < cfo[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (cfo[mid] <= f) lo = mid;
        else hi = mid;
    }
    const int64_t j = lo;
    const double gx = gen[3 * j], gy = gen[3 * j + 1], gz = gen[3 * j + 2];
    const double nx = normals[3 * f], ny = normals[3 * f + 1], nz = normals[3 * f + 2];
    const int64_t v0 = fvo[f], v1 = fvo[f + 1];
    const double c = nx * (verts[3 * v0] - gx) + ny * (verts[3 * v0 + 1] - gy) + nz * (verts[3 * v0 + 2] - gz);
    plane[f] = PlaneD{nx, ny, nz, c};
    // hi and low parts: the plane = hi + lo to about 2^-48 relative (float-float)
    PlaneF F, G;
    split_df(nx, F.x, G.x);
    split_df(ny, F.y, G.y);
    split_df(nz, F.z, G.z);
    split_df(c, F.w, G.w);
    plane_f[f] = F;
    plane_fl[f] = G;
    cell_of_face[f] = (int32_t)j;
    for (int64_t k = v0; k < v1; ++k) face_of_fv[k] = (int32_t)f;
}

// Per face-vertex k (one thread each, so that the records are written by
// adjacent threads): the edge from vertex k to the next vertex of its face, in
// the generator's frame, as FP64 and FP32 hi/lo records.  The cell radius is
// the largest |V - g| over its vertices: every vertex raises its cell's r^2
// with an atomic max on the bit pattern (non-negative doubles order like their
// bits), so the result does not depend on the order.
__global__ void k_prepare_edges(int64_t nfv, const double *__restrict__ gen, const int64_t *__restrict__ fvo,
                                const double *__restrict__ verts, const double *__restrict__ normals,
                                const int32_t *__restrict__ face_of_fv, const int32_t *__restrict__ cell_of_face,
                                unsigned long long *__restrict__ r2bits, EdgeD *__restrict__ edge,
                                EdgeF *__restrict__ edge_f, EdgeF *__restrict__ edge_fl)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nfv) return;
    const int64_t f = face_of_fv[k];
    const int64_t j = cell_of_face[f];
    const double gx = gen[3 * j], gy = gen[3 * j + 1], gz = gen[3 * j + 2];
    const double nx = normals[3 * f], ny = normals[3 * f + 1], nz = normals[3 * f + 2];
    const int64_t v0 = fvo[f], v1 = fvo[f + 1];
    int64_t k1 = (k + 1 < v1) ? k + 1 : v0;
    double ax = verts[3 * k] - gx, ay = verts[3 * k + 1] - gy, az = verts[3 * k + 2] - gz;
    double bx = verts[3 * k1] - gx, by = verts[3 * k1 + 1] - gy, bz = verts[3 * k1 + 2] - gz;
    double q = ax * ax + ay * ay + az * az;
    double ex = bx - ax, ey = by - ay, ez = bz - az;
    // L and 1/L from one reciprocal square root: an FP32 seed (on the bits,
    // split.cuh) and two FP64 Newton steps, within about an ulp, for fewer
    // FP64 instructions than a square root and a division
    const double s2 = ex * ex + ey * ey + ez * ez;
    double L = 0.0;
    EdgeD E;
    if (s2 > 1e-30 && s2 < 1e30) {   // the seed in float's normal range
        double r = f64_of(rsqrtf(f32_rn(s2)));
        r = r * (1.5 - 0.5 * s2 * r * r);
        r = r * (1.5 - 0.5 * s2 * r * r);
        L = s2 * r;
        ex *= r;
        ey *= r;
        ez *= r;
    } else if (s2 > 0.0) {   // outside it: the plain operations
        L = sqrt(s2);
        ex /= L;
        ey /= L;
        ez /= L;
    }
    E.ex = ex;
    E.ey = ey;
    E.ez = ez;
    E.L = L;
    E.mx = ey * nz - ez * ny;   // e x n: in-plane outward normal
    E.my = ez * nx - ex * nz;
    E.mz = ex * ny - ey * nx;
    E.cm = E.mx * ax + E.my * ay + E.mz * az;
    E.ce = ex * ax + ey * ay + ez * az;
    E.pad = 0.0;
    edge[k] = E;
    // hi and low parts: E = hi + lo to about 2^-48 relative (float-float)
    EdgeF F, G;
    split_df(E.mx, F.mx, G.mx);
    split_df(E.my, F.my, G.my);
    split_df(E.mz, F.mz, G.mz);
    split_df(E.cm, F.cm, G.cm);
    split_df(E.ex, F.ex, G.ex);
    split_df(E.ey, F.ey, G.ey);
    split_df(E.ez, F.ez, G.ez);
    split_df(E.ce, F.ce, G.ce);
    split_df(E.L, F.L, G.L);
    F.pad0 = F.pad1 = F.pad2 = 0.f;
    G.pad0 = G.pad1 = G.pad2 = 0.f;
    edge_f[k] = F;
    edge_fl[k] = G;
    atomicMax(r2bits + j, (unsigned long long)__double_as_longlong(q));
}

__global__ void k_radius_finish(int64_t ncell, double *__restrict__ radius)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= ncell) return;
    radius[j] = sqrt(radius[j]);   // the bits hold r^2 as a double
}

int em_prepare_cells(em_ctx *ctx, em_voronoi *v)
{
    EM_TRY(v->mem.alloc(&v->radius, v->ncell));
    EM_TRY(v->mem.alloc(&v->plane, v->nface));
    EM_TRY(v->mem.alloc(&v->edge, v->nfv));
    EM_TRY(v->mem.alloc(&v->plane_f, v->nface));
    EM_TRY(v->mem.alloc(&v->plane_fl, v->nface));
    EM_TRY(v->mem.alloc(&v->edge_f, v->nfv));
    EM_TRY(v->mem.alloc(&v->edge_fl, v->nfv));
    if (v->ncell) {
        EM_CUDA(cudaMemsetAsync(v->radius, 0, v->ncell * sizeof(double), ctx->stream));
        if (v->nface) {
            DevArena tmp(ctx->stream, true);
            int32_t *face_of_fv, *cell_of_face;
            EM_TRY(tmp.alloc(&face_of_fv, v->nfv));
            EM_TRY(tmp.alloc(&cell_of_face, v->nface));
            k_prepare_faces<<<em_grid(v->nface, 128), 128, 0, ctx->stream>>>(
                v->nface, v->ncell, v->gen, v->cell_face_off, v->face_vert_off, v->verts, v->normals, v->plane,
                v->plane_f, v->plane_fl, face_of_fv, cell_of_face);
            EM_LAUNCHED(ctx);
            k_prepare_edges<<<em_grid(v->nfv, 256), 256, 0, ctx->stream>>>(
                v->nfv, v->gen, v->face_vert_off, v->verts, v->normals, face_of_fv, cell_of_face,
                (unsigned long long *)v->radius, v->edge, v->edge_f, v->edge_fl);
            EM_LAUNCHED(ctx);
        }
        k_radius_finish<<<em_grid(v->ncell, 256), 256, 0, ctx->stream>>>(v->ncell, v->radius);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int voronoi_from_cells(em_ctx *ctx, int64_t ncell, int64_t nface, int64_t nfv, const double *d_gen,
                                 const int64_t *d_cell_face_off, const int64_t *d_face_vert_off,
                                 const double *d_verts, const double *d_normals, const int64_t *d_nbr,
                                 const double *d_volume, em_voronoi **out)
{
    EM_CHECK_ARG(ctx && out && ncell >= 0 && ncell < INT32_MAX && nface >= 0 && nfv >= 0);
    EM_CHECK_ARG(d_gen && d_cell_face_off && d_face_vert_off && d_verts && d_normals && d_volume);
    *out = nullptr;
    em_voronoi *v = new em_voronoi(ctx->stream);
    v->device = ctx->device;
    v->ncell = ncell;
    v->nface = nface;
    v->nfv = nfv;
    for (int k = 0; k < 6; ++k) v->box[k] = 0.0;
    int s = EM_OK;
    auto fail = [&](int st) {
        v->mem.release();
        delete v;
        return st;
    };
    if ((s = v->mem.alloc(&v->gen, 3 * ncell)) || (s = v->mem.alloc(&v->cell_face_off, ncell + 1)) ||
        (s = v->mem.alloc(&v->face_vert_off, nface + 1)) || (s = v->mem.alloc(&v->verts, 3 * nfv)) ||
        (s = v->mem.alloc(&v->normals, 3 * nface)) || (s = v->mem.alloc(&v->nbr, nface)) ||
        (s = v->mem.alloc(&v->volume, ncell)))
        return fail(s);
    cudaStream_t st = ctx->stream;
    cudaMemcpyAsync(v->gen, d_gen, 3 * ncell * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v->cell_face_off, d_cell_face_off, (ncell + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v->face_vert_off, d_face_vert_off, (nface + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v->verts, d_verts, 3 * nfv * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(v->normals, d_normals, 3 * nface * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (d_nbr) cudaMemcpyAsync(v->nbr, d_nbr, nface * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    else cudaMemsetAsync(v->nbr, 0xff, nface * sizeof(int64_t), st);
    cudaMemcpyAsync(v->volume, d_volume, ncell * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        em_set_error("voronoi_from_cells: %s", cudaGetErrorString(e));
        return fail(EM_ECUDA);
    }
    if ((s = em_prepare_cells(ctx, v))) return fail(s);
    *out = v;
    return EM_OK;
}

// ---------------------------------------------------------------------------
// Pair index: CSR offsets by cell and the (i, j)-ordered transpose
// ---------------------------------------------------------------------------

// off[c] = first position k with key[k] >= c, for c in [0, nseg]; key sorted.
__global__ void k_segment_offsets(int64_t n, const int32_t *__restrict__ key, int64_t nseg, int64_t *__restrict__ off,
                                  int *__restrict__ bad)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k > n) return;
    int64_t prev = (k == 0) ? -1 : (int64_t)key[k - 1];
    int64_t cur = (k == n) ? nseg : (int64_t)key[k];
    if (k < n && (cur < 0 || cur >= nseg)) {
        atomicOr(bad, 1);
        return;
    }
    if (cur < prev) {
        atomicOr(bad, 2);
        return;
    }
    for (int64_t c = prev + 1; c <= cur; ++c) off[c] = k;
}

__global__ void k_iota_keys(int64_t n, const int32_t *__restrict__ src, uint32_t *__restrict__ key,
                            int32_t *__restrict__ val)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    key[k] = (uint32_t)src[k];
    val[k] = (int32_t)k;
}

__global__ void k_check_within_cell(int64_t n, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                    int64_t np, int *__restrict__ bad)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (pi[k] < 0 || pi[k] >= np) atomicOr(bad, 4);
    if (k > 0 && pj[k] == pj[k - 1] && pi[k] <= pi[k - 1]) atomicOr(bad, 8);
}

int em_build_pair_index(em_ctx *ctx, em_pairs *pr)
{
    int64_t n = pr->npairs;
    DevArena tmp(ctx->stream, true);
    int *bad;
    EM_TRY(tmp.alloc(&bad, 1));
    EM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    EM_TRY(pr->mem.alloc(&pr->cell_pair_off, pr->ncell + 1));
    EM_TRY(pr->mem.alloc(&pr->part_pair_off, pr->np + 1));
    EM_TRY(pr->mem.alloc(&pr->part_pair_idx, n));
    k_segment_offsets<<<em_grid(n + 1, 256), 256, 0, ctx->stream>>>(n, pr->pair_j, pr->ncell, pr->cell_pair_off, bad);
    EM_LAUNCHED(ctx);
    if (n) {
        k_check_within_cell<<<em_grid(n, 256), 256, 0, ctx->stream>>>(n, pr->pair_i, pr->pair_j, pr->np, bad);
        EM_LAUNCHED(ctx);
    }
    uint32_t *keys;
    EM_TRY(tmp.alloc(&keys, n));
    if (n) {
        k_iota_keys<<<em_grid(n, 256), 256, 0, ctx->stream>>>(n, pr->pair_i, keys, pr->part_pair_idx);
        EM_LAUNCHED(ctx);
        EM_TRY(em_sort_pairs_u32(ctx, keys, pr->part_pair_idx, n, em_nbits((uint64_t)pr->np)));
    }
    k_segment_offsets<<<em_grid(n + 1, 256), 256, 0, ctx->stream>>>(n, (const int32_t *)keys, pr->np,
                                                                      pr->part_pair_off, bad);
    EM_LAUNCHED(ctx);
    int hbad = 0;
    EM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    EM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hbad) {
        em_set_error("pair list invalid (code %d): indices out of range or not sorted by (j, i)", hbad);
        return EM_EINVAL;
    }
    return EM_OK;
}

EM_EXPORT int pairs_from_list(em_ctx *ctx, int64_t npairs, const int32_t *d_pair_i, const int32_t *d_pair_j,
                              int64_t np, const em_voronoi *v, em_pairs **out)
{
    EM_CHECK_ARG(ctx && v && out && npairs >= 0 && npairs < INT32_MAX && np >= 0 && np < INT32_MAX);
    EM_CHECK_ARG(npairs == 0 || (d_pair_i && d_pair_j));
    *out = nullptr;
    em_pairs *pr = new em_pairs(ctx->stream);
    pr->device = ctx->device;
    pr->npairs = npairs;
    pr->np = np;
    pr->ncell = v->ncell;
    int s;
    if ((s = pr->mem.alloc(&pr->pair_i, npairs)) || (s = pr->mem.alloc(&pr->pair_j, npairs)) ||
        (s = pr->mem.alloc(&pr->near, npairs))) {
        pr->mem.release();
        delete pr;
        return s;
    }
    if (npairs) {
        cudaMemcpyAsync(pr->pair_i, d_pair_i, npairs * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(pr->pair_j, d_pair_j, npairs * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemsetAsync(pr->near, 0, npairs, ctx->stream);
    }
    if ((s = em_build_pair_index(ctx, pr))) {
        pr->mem.release();
        delete pr;
        return s;
    }
    *out = pr;
    return EM_OK;
}

// ---------------------------------------------------------------------------
// Per-pair weight
// ---------------------------------------------------------------------------

template <class T>
struct GeomT;
template <>
struct GeomT<double> {
    using Plane = PlaneD;
    using Edge = EdgeD;
};
template <>
struct GeomT<float> {
    using Plane = PlaneF;
    using Edge = EdgeF;
};

// w for particle p (r = p - g, absolute units) and cell j; err returns the sum
// of magnitudes of the combined terms (in units of w).  ALWAYS_FULL selects
// the full form for every pair (the FP64 path).
template <class T, bool ALWAYS_FULL>
__device__ __forceinline__ T pair_weight(T rx, T ry, T rz, T h, T radius, int64_t f0, int64_t f1,
                                         const int64_t *__restrict__ fvo,
                                         const typename GeomT<T>::Plane *__restrict__ plane,
                                         const typename GeomT<T>::Edge *__restrict__ edge, T &err)
{
    const T ih = T(1) / h;
    bool inside = true;
    if (!ALWAYS_FULL) {
        for (int64_t f = f0; f < f1; ++f) {
            auto pl = plane[f];
            T s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
            inside = inside && !(s < T(0));
        }
    }
    T rr = em_sqrt(rx * rx + ry * ry + rz * rz);
    const bool full = ALWAYS_FULL || (inside && (rr + radius < T(2) * h));
    T acc = T(0), comp = T(0);   // compensated (Kahan) accumulation over faces
    err = (!full && inside) ? T(1) : T(0);
    T terr = T(0);
    for (int64_t f = f0; f < f1; ++f) {
        auto pl = plane[f];
        T s = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        T D = fabs(s) * ih;
        if (s == T(0) || (!full && D >= T(2))) continue;
        const T kd = full ? K_of<T>(D) : K_tilde<T>(D);
        T fs = T(0);
        int64_t e0 = fvo[f], e1 = fvo[f + 1];
        for (int64_t e = e0; e < e1; ++e) {
            auto E = edge[e];
            T a = E.cm - (E.mx * rx + E.my * ry + E.mz * rz);
            if (a == T(0)) continue;
            T A = fabs(a) * ih;
            T t0 = (E.ce - (E.ex * rx + E.ey * ry + E.ez * rz)) * ih;
            T t1 = t0 + E.L * ih;
            T c = full ? edge_full<T>(D, A, t0, t1, kd, terr) : edge_tilde<T>(D, A, t0, t1, kd, terr);
            fs += (a > T(0)) ? c : -c;
        }
        T term = (s > T(0)) ? fs : -fs;
        T y = term - comp;
        T t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    err += terr * Consts<T>::inv_pi;
    T w = acc * Consts<T>::inv_pi;
    return full ? w : ((inside ? T(1) : T(0)) - w);
}

// FP64 closed form, one warp per pair (both the FP64 mode and the recompute
// of the pairs the mixed pass flagged).
//
// An edge's term Phi(T1) - Phi(T0) (edge_full / edge_tilde) is linear in a
// few evaluations: the basis b(tau) at an endpoint in region 1 or 2 (a
// combination of region coefficient vectors and b0), the region-3 part at an
// endpoint beyond 2h (the two angles b0, b1 alone), and the region
// differences d1 = (c1 - c2).b(t1), d2 = (c2 - c3).b(t2), whose integer
// coefficient sums the endpoints past t1 or t2 with their signs.  So each
// lane takes an edge, lists these evaluations with their signed weights
// (face orientation, edge orientation and endpoint sign folded in; a d1 or
// d2 whose coefficient vanishes, as for both endpoints beyond t2 on one
// side, is not listed), and appends them to one of two per-warp queues, one
// of basis evaluations and one of angle evaluations.  Whenever a queue holds
// 32 entries the warp evaluates them together, one per lane, so that the
// transcendental code runs with the warp converged whatever the edges'
// regions.  Each lane adds what it evaluated; a fixed-order warp sum ends the
// pair.  The order of the evaluations depends on the pair alone, so the
// result is reproducible.  A cell with more than FW_MAXF faces (possible only
// for imported cells) is done by one lane with pair_weight.
//
// Entry t of list is k >= 0: pair k in the complement form (faces beyond 2h
// skipped; its rounding, about 1e-13, is far inside the mixed mode's
// tolerance), or ~k < 0: pair k in the full form (a particle in a face plane,
// for which such a face carries nothing).  Without a list, entry t is pair t
// in the full form (the FP64 mode).
constexpr int FW_WARPS = 4;
constexpr int FW_MAXF = 64;
constexpr int FQ = 64;   // ring capacity of each evaluation queue (a power of two, >= 63)

// Evaluations waiting for a full warp: the basis at t (code: regions rA, rB
// in bits 0-1, 2-3) weighted w0 (c_rA - c_rB).b - w1 b0, or the angles
// w0 D atan(u/A) - w1 atan(D u / (A Q)).
struct FwQueue {
    double A[FQ], B2[FQ], D[FQ], t[FQ], w0[FQ], w1[FQ];
    int code[FQ];
};

__device__ __noinline__ double fw_eval_basis(const FwQueue &q, int i)
{
    double b[6];
    basis<double>(q.A[i], q.B2[i], q.D[i], q.t[i], b);
    const int rA = q.code[i] & 3, rB = q.code[i] >> 2;
    const double p1 = dot_c1(b), p2 = dot_c2(b), p3 = dot_c3(b);
    const double dA = rA == 1 ? p1 : (rA == 2 ? p2 : p3);
    const double dB = rB == 0 ? 0.0 : (rB == 1 ? p1 : (rB == 2 ? p2 : p3));
    return q.w0[i] * (dA - dB) - q.w1[i] * b[0];
}

__device__ __noinline__ double fw_eval_angle(const FwQueue &q, int i, bool both)
{
    const double A = q.A[i], D = q.D[i], u = q.t[i];
    double v = q.w0[i] * (D * atan2(u, A));
    if (both) v -= q.w1[i] * atan2(D * u, A * sqrt(q.B2[i] + u * u));
    return v;
}

// Append this lane's entry (if has) to ring q of n entries from head.
__device__ __forceinline__ void fw_push(FwQueue &q, int head, int &n, bool has, double A, double B2, double D,
                                        double t, double w0, double w1, int code)
{
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (has) {
        const int pos = (head + n + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))) & (FQ - 1);
        q.A[pos] = A;
        q.B2[pos] = B2;
        q.D[pos] = D;
        q.t[pos] = t;
        q.w0[pos] = w0;
        q.w1[pos] = w1;
        q.code[pos] = code;
    }
    n += __popc(m);
}

// Evaluate the queues' full warps (every entry when last), lane by entry.
__device__ __forceinline__ void fw_drain(FwQueue &qb, FwQueue &qa, int &hb, int &nb, int &ha, int &na, bool both,
                                         bool last, double &acc)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    while (nb >= 32 || (last && nb > 0)) {
        if (lane < nb) acc += fw_eval_basis(qb, (hb + lane) & (FQ - 1));
        const int d = min(nb, 32);
        hb = (hb + d) & (FQ - 1);
        nb -= d;
    }
    while (na >= 32 || (last && na > 0)) {
        if (lane < na) acc += fw_eval_angle(qa, (ha + lane) & (FQ - 1), both);
        const int d = min(na, 32);
        ha = (ha + d) & (FQ - 1);
        na -= d;
    }
    __syncwarp();
}

__device__ __forceinline__ void fp64_pairs_warp(int64_t n, const int32_t *__restrict__ list,
                                                const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                const double *__restrict__ x, const double *__restrict__ y,
                                                const double *__restrict__ z, const double *__restrict__ h,
                                                const double *__restrict__ gen, const double *__restrict__ radius,
                                                const int64_t *__restrict__ cfo, const int64_t *__restrict__ fvo,
                                                const PlaneD *__restrict__ plane, const EdgeD *__restrict__ edge,
                                                double *__restrict__ w)
{
    __shared__ double fD[FW_WARPS][FW_MAXF], fK[FW_WARPS][FW_MAXF];
    __shared__ int64_t fE0[FW_WARPS][FW_MAXF];
    __shared__ int fPre[FW_WARPS][FW_MAXF + 1];
    __shared__ float fSg[FW_WARPS][FW_MAXF];
    __shared__ FwQueue fq[FW_WARPS][2];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;   // wpb <= FW_WARPS
    FwQueue &qb = fq[wi][0], &qa = fq[wi][1];
    for (int64_t t = blockIdx.x * (int64_t)wpb + wi; t < n; t += (int64_t)gridDim.x * wpb) {
        const int32_t code = list ? list[t] : ~(int32_t)t;
        const int64_t k = code >= 0 ? code : ~code;
        const int i = pi[k], j = pj[k];
        const double rx = x[i] - gen[3 * j], ry = y[i] - gen[3 * j + 1], rz = z[i] - gen[3 * j + 2];
        const double hh = h[i], ih = 1.0 / hh;
        const int64_t f0 = cfo[j];
        const int nface = (int)(cfo[j + 1] - f0);
        if (nface > FW_MAXF) {
            if (lane == 0) {
                double err;
                w[k] = code >= 0 ? pair_weight<double, false>(rx, ry, rz, hh, radius[j], f0, f0 + nface, fvo, plane,
                                                              edge, err)
                                 : pair_weight<double, true>(rx, ry, rz, hh, radius[j], f0, f0 + nface, fvo, plane,
                                                             edge, err);
            }
            continue;
        }
        // inside test over all faces, then the form
        bool ins = true;
        if (code >= 0)
            for (int f = lane; f < nface; f += 32) {
                const PlaneD pl = plane[f0 + f];
                ins = ins && !(pl.w - (pl.x * rx + pl.y * ry + pl.z * rz) < 0.0);
            }
        ins = __all_sync(0xffffffffu, ins);
        const bool full = code < 0 || (ins && sqrt(rx * rx + ry * ry + rz * rz) + radius[j] < 2.0 * hh);
        // faces: distance, constant, and how many edges each contributes
        for (int base = 0; base < nface; base += 32) {
            const int f = base + lane;
            int cnt = 0;
            if (f < nface) {
                const PlaneD pl = plane[f0 + f];
                const double sd = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
                const double D = fabs(sd) * ih;
                const bool keep = !(sd == 0.0 || (!full && D >= 2.0));
                fD[wi][f] = D;
                fK[wi][f] = full ? K_of<double>(D) : K_tilde<double>(D);
                fE0[wi][f] = fvo[f0 + f];
                fSg[wi][f] = sd > 0.0 ? 1.f : -1.f;
                if (keep) cnt = (int)(fvo[f0 + f + 1] - fvo[f0 + f]);
            }
            int xs = cnt;   // inclusive scan of the edge counts over these 32 faces
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, xs, o);
                if (lane >= o) xs += y;
            }
            const int carry = base == 0 ? 0 : fPre[wi][base];
            __syncwarp();
            if (lane == 0 && base == 0) fPre[wi][0] = 0;
            if (f < nface) fPre[wi][f + 1] = carry + xs;
            __syncwarp();
        }
        const int ne = fPre[wi][nface];
        double acc = 0.0;
        int hb = 0, nb = 0, ha = 0, na = 0;
        for (int base = 0; base < ne; base += 32) {
            const int e = base + lane;
            // this lane's edge: its evaluations (has*), weights and split points
            double A = 0.0, D = 0.0, B2 = 0.0, u0 = 0.0, u1 = 0.0, ts1 = 0.0, ts2 = 0.0;
            double bw0[2] = {0.0, 0.0}, bw1[2] = {0.0, 0.0}, aw0[2] = {0.0, 0.0}, aw1[2] = {0.0, 0.0};
            int bcode[2] = {0, 0};
            bool hasb[2] = {false, false}, hasa[2] = {false, false};
            double coef1 = 0.0, coef2 = 0.0;
            if (e < ne) {
                int lo = 0, hi = nface;   // fPre[lo] <= e < fPre[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (fPre[wi][mid] <= e) lo = mid;
                    else hi = mid;
                }
                const EdgeD E = edge[fE0[wi][lo] + (e - fPre[wi][lo])];
                const double a = E.cm - (E.mx * rx + E.my * ry + E.mz * rz);
                if (a != 0.0) {
                    A = fabs(a) * ih;
                    const double T0 = (E.ce - (E.ex * rx + E.ey * ry + E.ez * rz)) * ih;
                    const double T1 = T0 + E.L * ih;
                    D = fD[wi][lo];
                    const double kd = fK[wi][lo];
                    const double sg = (double)fSg[wi][lo] * (a > 0.0 ? 1.0 : -1.0);
                    B2 = D * D + A * A;
                    u0 = fabs(T0);
                    u1 = fabs(T1);
                    // endpoint signs: Phi(T1) - Phi(T0), Phi odd in T
                    const double cs[2] = {T0 < 0.0 ? sg : -sg, T1 < 0.0 ? -sg : sg};
                    const double uu[2] = {u0, u1};
                    const bool near = B2 < 4.0;
                    if (near) {
                        ts2 = sqrt(4.0 - B2);
                        if (B2 < 1.0) ts1 = sqrt(1.0 - B2);
                    }
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const double u = uu[s], c = cs[s];
                        if (u == 0.0) continue;
                        if (full) {
                            if (!near || u > ts2) {   // region 3: the angles alone
                                hasa[s] = true;
                                aw0[s] = c * ((near || D < 2.0) ? 7.0 / 20.0 - kd : 0.25 / D);
                                aw1[s] = c * 0.25;
                                if (near) {
                                    coef1 += c;
                                    coef2 += c;
                                }
                            } else {
                                hasb[s] = true;
                                const int r = u <= ts1 ? 1 : 2;
                                bcode[s] = r;
                                bw0[s] = c;
                                bw1[s] = c * kd;
                                if (r == 2) coef1 += c;
                            }
                        } else {
                            if (!near || u >= ts2) {   // beyond 2h: -(d1 + d2) - K~(D) b0
                                hasa[s] = true;
                                aw0[s] = -c * kd;
                                if (near) {
                                    coef1 -= c;
                                    coef2 -= c;
                                }
                            } else {
                                hasb[s] = true;
                                const bool r2 = u > ts1;
                                bcode[s] = r2 ? (3 | (2 << 2)) : (3 | (1 << 2));
                                bw0[s] = c;
                                bw1[s] = c * kd;
                                if (r2) coef1 -= c;
                            }
                        }
                    }
                    if (!(B2 < 1.0)) coef1 = 0.0;   // no region 1: d1 = 0
                }
            }
            const bool has_t1 = coef1 != 0.0, has_t2 = coef2 != 0.0;
            // six collective appends in a fixed order, draining full warps as they fill
#pragma unroll 1
            for (int step = 0; step < 6; ++step) {
                // (selects rather than indexing, so that the arrays stay in registers)
                const bool s = (step & 1) != 0;
                if (step < 4) {
                    const bool split = step >= 2;
                    const bool has = split ? (s ? has_t2 : has_t1) : (s ? hasb[1] : hasb[0]);
                    const double tt = split ? (s ? ts2 : ts1) : (s ? u1 : u0);
                    const double w0 = split ? (s ? coef2 : coef1) : (s ? bw0[1] : bw0[0]);
                    const double w1 = split ? 0.0 : (s ? bw1[1] : bw1[0]);
                    const int cd = split ? (s ? (2 | (3 << 2)) : (1 | (2 << 2))) : (s ? bcode[1] : bcode[0]);
                    fw_push(qb, hb, nb, has, A, B2, D, tt, w0, w1, cd);
                } else {
                    fw_push(qa, ha, na, s ? hasa[1] : hasa[0], A, B2, D, s ? u1 : u0, s ? aw0[1] : aw0[0],
                            s ? aw1[1] : aw1[0], 0);
                }
                if (nb >= 32 || na >= 32) fw_drain(qb, qa, hb, nb, ha, na, full, false, acc);
            }
        }
        fw_drain(qb, qa, hb, nb, ha, na, full, true, acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double s = acc * Consts<double>::inv_pi;
            w[k] = full ? s : ((ins ? 1.0 : 0.0) - s);
        }
        __syncwarp();
    }
}

// the flagged pairs of the mixed pass; the count is read on the device, so
// the launch needs no host synchronisation (grid-stride loop)
__global__ void __launch_bounds__(32 * FW_WARPS) k_map_fp64_flagged(
    const int *__restrict__ nflag, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ h, const double *__restrict__ gen, const double *__restrict__ radius,
    const int64_t *__restrict__ cfo, const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane,
    const EdgeD *__restrict__ edge, const int32_t *__restrict__ list, double *__restrict__ w)
{
    fp64_pairs_warp(*nflag, list, pi, pj, x, y, z, h, gen, radius, cfo, fvo, plane, edge, w);
}

// every pair, full form (the FP64 mode)
__global__ void __launch_bounds__(32 * FW_WARPS) k_map_fp64(
    int64_t npairs, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, const double *__restrict__ x,
    const double *__restrict__ y, const double *__restrict__ z, const double *__restrict__ h,
    const double *__restrict__ gen, const double *__restrict__ radius, const int64_t *__restrict__ cfo,
    const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane, const EdgeD *__restrict__ edge,
    double *__restrict__ w)
{
    fp64_pairs_warp(npairs, nullptr, pi, pj, x, y, z, h, gen, radius, cfo, fvo, plane, edge, w);
}

// FP32 bulk pass (quadrature form, see quad32.cuh).
//
// A warp maps 32 consecutive pairs (mostly of one cell, since pairs are
// sorted by cell), one pair per lane for the geometry: per face the plane
// distance D in float-float and an FP32 pass for the reference R = distance
// from p to the face polygon (any value used consistently for the face is
// exact when P is outside the polygon; inside, R = D), then R, 2 - R, K(R)
// and K(1) - K(R) in FP32; per edge A, T0, T1, B^2 - 1, 4 - B^2 and
// A^2 - rho^2 in float-float, each rounded once to FP32.  The FP64 pipe runs
// at 1/64 of the FP32 rate, so nothing per face, edge or quadrature segment
// touches it: the pieces are summed in float-float.
//
// Each edge yields up to four quadrature segments, which the lane appends to
// its column of a per-warp queue in shared memory; whenever a lane's column
// may overflow, the warp evaluates all queued segments together, one 4-node
// slot (a 4-point segment, or half of an 8-point sub-piece) per lane, so that
// the node loop runs with the warp converged whatever the pairs' geometry.
// Each lane then adds its own segments' results in a fixed order, which keeps
// the result bit-reproducible.  The queue is small (9.1 KB per warp) so that
// 12 two-warp blocks fit an SM: the pass is bound by instruction issue, and
// the warps hide its latencies.  The estimated error 8 eps times the sum of
// the magnitudes of the non-negative pieces flags the pair for the FP64 pass
// when it exceeds max(tol |w|, 1e-14) (relative accuracy tol for every weight
// above 1e-14 / tol, absolute 1e-14 below); so does a face plane through P.
namespace {

// factor of the FP32 pass's error estimate: fp32_err_ulps units of 2^-24
// (0 stands for the default 8)
double em_est_k(const em_params *p)
{
    return (double)(p->fp32_err_ulps > 0 ? p->fp32_err_ulps : 8) * 5.9604644775390625e-8;
}

// launch shape of the FP32 pass (build-time tuning knobs)
#ifndef EM_MQ_SLOTS
#define EM_MQ_SLOTS 6
#endif
#ifndef EM_MQ_WARPS
#define EM_MQ_WARPS 2
#endif
#ifndef EM_G8_MAXLEN_FAR
// longest 8-point sub-piece (in s) of the second kernel piece on a face
// whose plane lies beyond h (R >= 1); elsewhere 2.  On that branch the
// 8-point rule's truncation reaches ~5 ulp of the segment at length 2 and
// ~0.3 ulp at 1.5 (an FP64 model of the integrand against adaptive
// quadrature); the error estimate counts rounding only
#define EM_G8_MAXLEN_FAR 2.0
#endif
static_assert(EM_G8_MAXLEN_FAR >= 0.5 && EM_G8_MAXLEN_FAR <= 2.0, "sub-pieces per segment must stay below 256");
#ifndef EM_GL4_MAXLEN
#define EM_GL4_MAXLEN 0.125   // longest segment (in s) integrated with 4 points
#endif
#ifndef EM_MQ_MINB
// minimum resident blocks per SM asked of the compiler (0: none): 12 two-warp
// blocks, 24 warps, is what the shared memory of 12 queues allows (18.2 KB a
// block), and caps the registers at 80 without spills
#define EM_MQ_MINB 12
#endif
constexpr int MQ_SLOTS = EM_MQ_SLOTS;   // segments a lane holds between evaluations (>= 5)
constexpr int MQ_WARPS = EM_MQ_WARPS;   // warps per block
constexpr int MQ_CHUNK = 64;            // sub-piece results a warp holds between accumulations
static_assert(MQ_SLOTS >= 5, "an edge queues up to four segments");
static_assert(MQ_CHUNK % 32 == 0, "whole rounds of the warp");
// a lane holds at most MQ_SLOTS segments of at most 2 x 141 slots each (m <= 141)
constexpr int MQ_NOSLOT = 4095;
static_assert(MQ_SLOTS * 282 < MQ_NOSLOT, "slot indices fit in 12 bits");
constexpr unsigned FULL_MASK = 0xffffffffu;

struct SegQueue {
    float ts[MQ_SLOTS][32], hl[MQ_SLOTS][32], A[MQ_SLOTS][32];
    float B2[MQ_SLOTS][32], c4s[MQ_SLOTS][32], es[MQ_SLOTS][32], Rr[MQ_SLOTS][32], vv[MQ_SLOTS][32];
    float add[MQ_SLOTS][32], scale[MQ_SLOTS][32];
    // m | piece1 | tilde | gl4 (quad32.cuh) in the low 16 bits; during a
    // flush, the index of the segment's first 4-node slot among its lane's
    // in bits 16-27 (MQ_NOSLOT for an empty row)
    int meta[MQ_SLOTS][32];
    float vhi[MQ_CHUNK], vlo[MQ_CHUNK];   // scale * integral of each evaluated slot (float-float)
    int pre[33];
};

// Evaluate every queued segment of the warp and add each lane's results to
// its pair.  Called with the warp converged.  The work is spread by
// slot (4 quadrature nodes: a 4-point segment, or half of an 8-point
// sub-piece): lane L's segments hold M_L slots in queue order, the warp
// numbers all of them L by L and evaluates them 32 at a time, whoever owns
// them, so that a segment cut into many sub-pieces does not hold up the
// lanes.  Each result, times its segment's signed factor, is
// kept exactly as a float-float product; the owner then adds its own results
// in order into its float-float sum (to about 2^-44 of the magnitudes), which
// keeps the sum bit-reproducible, and their magnitudes in FP32: they only
// scale the error bound.
__device__ __forceinline__ void mq_flush(SegQueue &q, int lane, int cnt, emq::ff &acc, float &mag)
{
    int M = 0;
#pragma unroll
    for (int sl = 0; sl < MQ_SLOTS; ++sl) {
        const int mt = q.meta[sl][lane] & 0xffff;
        q.meta[sl][lane] = mt | ((sl < cnt ? M : MQ_NOSLOT) << 16);
        if (sl < cnt) M += (mt & emq::SEG_GL4) ? (mt & 255) : 2 * (mt & 255);   // 4-point: 1 slot, 8-point: 2 per sub-piece
    }
    int x = M;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    const int total = __shfl_sync(FULL_MASK, x, 31);
    q.pre[lane + 1] = x;
    if (lane == 0) q.pre[0] = 0;
    __syncwarp();
    const int mine0 = x - M;   // this lane's slots are [mine0, x)
    for (int c0 = 0; c0 < total; c0 += MQ_CHUNK) {
        const int c1 = min(total, c0 + MQ_CHUNK);
        for (int t = c0 + lane; t < c1; t += 32) {
            int lo = 0, hi = 32;   // pre[lo] <= t < pre[hi]
#pragma unroll
            for (int it = 0; it < 5; ++it) {
                const int mid = (lo + hi) >> 1;
                if (q.pre[mid] <= t) lo = mid;
                else hi = mid;
            }
            const int r = t - q.pre[lo];
            int sl = 0;
#pragma unroll
            for (int k = 1; k < MQ_SLOTS; ++k) sl += (q.meta[k][lo] >> 16) <= r ? 1 : 0;
            const int mw = q.meta[sl][lo];
            const int rr = r - (mw >> 16);
            const int mt = mw & 0xffff;
            const bool gl4 = (mt & emq::SEG_GL4) != 0;
            const int p = gl4 ? rr : rr >> 1;           // the sub-piece
            const int half = gl4 ? 2 : (rr & 1);        // which 4 nodes of its rule
            const float hl = q.hl[sl][lo];
            // sinh and cosh of s at the segment's start, ts / A and
            // sqrt(1 + (ts / A)^2) (not stored, which keeps the queue small
            // enough for more warps per SM)
            const float ts = q.ts[sl][lo], A = q.A[sl][lo];
            const float Sa = ts * __frcp_rn(A);
            const float Ca = emq::sqrt_nr(fmaf(Sa, Sa, 1.f));
            const float val = emq::slot_eval((2.f * (float)p + 1.f) * hl, hl, half, ts, Sa, Ca, A, q.B2[sl][lo],
                                             q.c4s[sl][lo], q.es[sl][lo],
                                             q.Rr[sl][lo], q.vv[sl][lo], q.add[sl][lo], mt);
            const emq::ff v = emq::ff_two_prod(q.scale[sl][lo], val);
            q.vhi[t - c0] = v.hi;
            q.vlo[t - c0] = v.lo;
        }
        __syncwarp();
        const int e1 = min(x, c1);
        for (int t = max(mine0, c0); t < e1; ++t) {
            const emq::ff v{q.vhi[t - c0], q.vlo[t - c0]};
            acc = emq::ff_add(acc, v);
            mag += fabsf(v.hi);
        }
        __syncwarp();
    }
}

// Face constants of the lane's current face.
struct FaceState {
    emq::ff dm1, d4;            // D^2 - 1, 4 - D^2 (float-float, units of h)
    float rr2;                  // rho^2 (units of h; FP32 by construction)
    float Df, R, v, KR, C1;     // v = 2 - R
    float sign;   // orientation of the face as seen from P (sign of the signed distance)
};

// Face constants from R^2 (float-float): R, v = 2 - R, K(R) (or K~(R)) and,
// for R < 1, K(1) - K(R), in FP32.  Each is written so that no sum cancels:
// 1 - R^2 and 4 - R^2 in float-float, and for R < 1 the polynomials in
// x = 1 - R with integer coefficients (times 120), where
//   K1(1) - K1(R) = (1 - R^2) P / 120,  P = 8 + 6x - 3x^3 + 3/(1 + R),
//   K1(R) = R^2 (14 + 9x - 3x^3) / 120,
//   K~1(1) - K~1(R) = (1 - R^2) N / (120 R (1 + R)),
//   N = 11 + 15x + 10x^2 - 9x^4 + 3x^5,
// sums whose terms are at most 1.6 times their value, so each constant comes
// out within a few ulp.
__device__ __forceinline__ void face_consts(emq::ff R2x, bool tilde, FaceState &fs)
{
    const float R2 = R2x.hi + R2x.lo;
    const float R = sqrtf(R2);
    const float iR = R > 0.f ? __frcp_rn(R) : 0.f;
    fs.R = R;
    if (R < 1.f) {
        const emq::ff omx = emq::ff_add(emq::ff{1.f, 0.f}, emq::ff_neg(R2x));
        const float om = (omx.hi + omx.lo) * (1.f / 120.f);
        const float x = 1.f - R;
        const float i1 = __frcp_rn(1.f + R);
        fs.v = 2.f - R;
        if (tilde) {
            const float N = fmaf(x, fmaf(x, fmaf(x * x, fmaf(3.f, x, -9.f), 10.f), 15.f), 11.f);
            const float c1 = om * (N * iR * i1);
            fs.C1 = c1;
            fs.KR = -(1.f / 60.f) - c1;
        } else {
            const float P = fmaf(x, fmaf(-3.f * x, x, 6.f), 8.f) + 3.f * i1;
            fs.C1 = om * P;
            fs.KR = R2 * fmaf(x, fmaf(-3.f * x, x, 9.f), 14.f) * (1.f / 120.f);
        }
        return;
    }
    fs.C1 = 0.f;
    // K(R) = 7/20 - 1/(4R) - K~2(R) for R >= 1, with 7/20 - 1/(4R) = (7R - 5)/(20R)
    const float k3 = fmaf(7.f, R, -5.f) * iR * 0.05f;
    if (R >= 2.f) {
        fs.v = 0.f;
        fs.KR = tilde ? 0.f : k3;
        return;
    }
    const emq::ff fmx = emq::ff_add(emq::ff{4.f, 0.f}, emq::ff_neg(R2x));
    const float v = (fmx.hi + fmx.lo) * __frcp_rn(2.f + R);
    const float v2 = v * v;
    const float kt2 = -(v2 * v2) * v * (1.f + R) * iR * (1.f / 120.f);
    fs.v = v;
    fs.KR = tilde ? kt2 : k3 - kt2;
}

// Queue the kernel pieces of (D/pi) int over |tau| in [ua, ua + du] (one
// g-integral of an edge) with the signed factor sc; the part beyond 2h is
// added directly.  du is the range's length from an accurate difference (the
// edge length L/h, or |T| for a range starting at the foot), and every
// segment's length in s is formed from such a difference: with a = ua and
// b = ua + o,
//     asinh(b/A) - asinh(a/A) = asinh(o (a + b) / (b sqrt(A^2 + a^2) + a sqrt(A^2 + b^2))),
// an identity whose right side keeps the relative precision of o.  The
// difference of two asinh values, each rounded to FP32, would carry an
// absolute error of about 2^-24 |s|, which on a short segment (a small face
// seen from afar: |T| ~ 1, L/h ~ 0.05) is tens of ulps of the segment, and
// the error estimate, which counts rounding relative to the segments' sizes,
// would not see it.  Where a segment starts (sa) needs no such care: shifting
// a short segment moves its integral only by the integrand's change across it.
__device__ __forceinline__ void mq_push_g(SegQueue &q, int lane, int &cnt, float ua, float du, float A, float B2,
                                          emq::ff c1x, emq::ff c4x, emq::ff ccx, float sc, const FaceState &fs,
                                          bool tilde, emq::ff &acc, float &mag)
{
    const float c1 = c1x.hi + c1x.lo, c4 = c4x.hi + c4x.lo;
    const float t1 = c1 < 0.f ? emq::sqrt_nr(-c1) : 0.f;
    const float t2 = c4 > 0.f ? emq::sqrt_nr(c4) : 0.f;
    const int tflag = tilde ? emq::SEG_TILDE : 0;
    // a segment of kernel piece `piece` from tau = ts (s-length len)
    auto push = [&](int piece, float ts, float len) {
        // 4 points for a short segment, else 8 on sub-pieces of length <= 2
        const bool gl4 = len <= (float)EM_GL4_MAXLEN;
        const float g8 = (piece == 2 && fs.R >= 1.f) ? (float)EM_G8_MAXLEN_FAR : 2.f;
        // m <= ceil(70.5 / g8) <= 141: A >= 1e-30, |tau| <= 2
        const int m = len > g8 ? (int)ceilf(len * (1.f / g8)) : 1;
        const int sl = cnt++;
        const bool ref1 = piece == 2 && fs.R < 1.f;   // difference split at Q = 1
        // Q^2 - Rr^2 and 4 - Q^2 at ts, from the edge's float-float
        // differences and ts^2 as an exact product
        const emq::ff ts2 = emq::ff_two_prod(ts, ts);
        const emq::ff es = emq::ff_add(ref1 ? c1x : ccx, ts2);
        const emq::ff c4s = emq::ff_add(c4x, emq::ff_neg(ts2));
        q.ts[sl][lane] = ts;
        q.hl[sl][lane] = 0.5f * len / (float)m;
        q.A[sl][lane] = A;
        q.B2[sl][lane] = B2;
        q.c4s[sl][lane] = c4s.hi + c4s.lo;
        q.es[sl][lane] = es.hi + es.lo;
        q.Rr[sl][lane] = ref1 ? 1.f : fs.R;
        q.vv[sl][lane] = ref1 ? 1.f : fs.v;
        q.add[sl][lane] = ref1 ? fs.C1 : 0.f;
        q.scale[sl][lane] = sc;
        q.meta[sl][lane] = m | (piece == 1 ? emq::SEG_PIECE1 : 0) | tflag | (gl4 ? emq::SEG_GL4 : 0);
    };
    // piece 1 is |tau| in [ua, b1], piece 2 in [a2, b2]; when both are present
    // they meet at t1
    const float ub = ua + du;
    const float b1 = fminf(ub, t1), a2 = fmaxf(ua, t1), b2 = fminf(ub, t2);
    const bool has1 = b1 > ua, has2 = b2 > a2;
    if (has1 || has2) {
        const float ra = emq::sqrt_nr(fmaf(ua, ua, A * A));
        // s at ua + o minus s at ua, from the offset o
        auto ds = [&](float o) {
            const float b = ua + o;
            const float rb = emq::sqrt_nr(fmaf(b, b, A * A));
            return asinhf(__fdividef(o * (ua + b), fmaf(b, ra, ua * rb)));
        };
        // offset in s of the end of the quadrature (ub, or Q = 2), and of Q = 1
        const float d_end = ds(has2 && ub > t2 ? t2 - ua : du);
        const float d_mid = (has1 && has2) ? ds(t1 - ua) : 0.f;
        if (has1) push(1, ua, has2 ? d_mid : d_end);
        if (has2) push(2, a2, d_end - d_mid);
    }
    if (tilde) {   // beyond 2h: K~(Q) = 0, the integrand is -K~(R) >= 0
        const float a = fmaxf(ua, t2), b = ub;
        if (b > a) {
            const float ba = ua >= t2 ? du : du - (t2 - ua);   // b - a from the offsets
            const emq::ff v = emq::ff_two_prod(sc, -fs.KR * atan2f(ba * A, A * A + a * b));
            acc = emq::ff_add(acc, v);
            mag += fabsf(v.hi);
        }
    }
}

}  // namespace

// Launch shapes of the FP32 pass (em_params.fp32_variant, map_autotune):
// warps per block and the minimum resident blocks per SM asked of the
// compiler (0: none).  Variant 0 is the default shape; the others trade
// registers (no minimum: 92-94) against warps per SM.
constexpr int MQ_NVARIANT = 4;
constexpr int MQ_VARIANT_WARPS[MQ_NVARIANT] = {MQ_WARPS, 1, 4, 2};
constexpr int MQ_VARIANT_MINB[MQ_NVARIANT] = {EM_MQ_MINB, 0, 6, 0};

template <int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_map_fp32(int64_t npairs, const int32_t *__restrict__ pi,
                                                        const int32_t *__restrict__ pj, const double *__restrict__ x,
                                                        const double *__restrict__ y, const double *__restrict__ z,
                                                        const double *__restrict__ h, const double *__restrict__ gen,
                                                        const double *__restrict__ radius,
                                                        const int64_t *__restrict__ cfo, const int64_t *__restrict__ fvo,
                                                        const PlaneF *__restrict__ plane_f,
                                                        const PlaneF *__restrict__ plane_fl,
                                                        const EdgeF *__restrict__ edge_f,
                                                        const EdgeF *__restrict__ edge_fl, float tol, double est_k,
                                                        double *__restrict__ w, int32_t *__restrict__ flagged,
                                                        int *__restrict__ nflag)
{
    __shared__ SegQueue queues[WARPS];
    SegQueue &q = queues[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t k0 = (blockIdx.x * (int64_t)WARPS + (threadIdx.x >> 5)) * 32;
    if (k0 >= npairs) return;   // the whole warp
    const int64_t k = k0 + lane;
    const bool valid = k < npairs;

    double rx = 0.0, ry = 0.0, rz = 0.0, hh = 1.0, rad = 0.0;
    int64_t f = 0, f1 = 0;
    if (valid) {
        const int i = pi[k], j = pj[k];
        rx = x[i] - gen[3 * j];
        ry = y[i] - gen[3 * j + 1];
        rz = z[i] - gen[3 * j + 2];
        hh = h[i];
        f = cfo[j];
        f1 = cfo[j + 1];
        rad = radius[j];
    }
    const double ih = 1.0 / hh;
    // float-float copies of r = p - g and 1/h for the plane and edge geometry,
    // and their FP32 roundings
    const emq::ff rxx = emq::ff_from_double(rx), ryy = emq::ff_from_double(ry), rzz = emq::ff_from_double(rz);
    const emq::ff ihh = emq::ff_from_double(ih);
    const float rxf = rxx.hi, ryf = ryy.hi, rzf = rzz.hi, ihf = ihh.hi;
    // signed distance c - n.r of P from face g's plane (positive inside), in
    // float-float; the inside test and the faces' orientations below both
    // take their signs from this one value
    auto plane_dist = [&](int64_t g) {
        const PlaneF H = plane_f[g], Lo = plane_fl[g];
        return emq::ff_offset_dot(H.w, Lo.w, H.x, Lo.x, H.y, Lo.y, H.z, Lo.z, rxx, ryy, rzz);
    };
    // the full kernel applies when P is inside a cell that lies entirely
    // within 2h of it; otherwise the complement form, and whether P is inside
    // is read off the face loop's own plane distances
    bool inside = valid, full = false;
    if (valid && sqrt(rx * rx + ry * ry + rz * rz) + rad < 2.0 * hh) {
        for (int64_t g = f; g < f1; ++g) inside = inside && !(plane_dist(g).hi < 0.f);
        full = inside;
    }
    const bool tilde = !full;

    // the quadrature's results are added in the order of the lane's own
    // segments (mq_flush), the angles beyond 2h in the order of its edges, each
    // into its own sum: neither order depends on when the warp flushes, so a
    // pair's weight does not depend on the other pairs of its warp
    emq::ff acc{0.f, 0.f}, acc_far{0.f, 0.f};
    float mag = 0.f, mag_far = 0.f;
    bool force = false;   // the FP32 form does not apply: recompute in FP64
    int cnt = 0;   // segments queued by this lane
    const int nface = valid ? (int)(f1 - f) : 0;
    // faces and edges in lockstep across the warp: consecutive pairs mostly
    // share their cell, so the per-face geometry runs with the lanes converged
    // One pass more than the warp has faces, with one empty edge, evaluates
    // what is left: the flush has a single call site, so that a slot's result
    // cannot depend on which copy of the code (the compiler may round two
    // copies differently) evaluated it, that is on the other pairs of the warp.
    for (int fi = 0;; ++fi) {
        const bool last = !__any_sync(FULL_MASK, fi < nface);
        int64_t e0 = 0;
        int ne = 0;
        FaceState fs{};
        if (fi < nface) {
            const int64_t g = f + fi;
            const emq::ff sd = plane_dist(g);
            inside = inside && !(sd.hi < 0.f);
            const emq::ff D = emq::ff_mul(sd.hi < 0.f ? emq::ff_neg(sd) : sd, ihh);
            // P in (or within underflow of) the face plane: in the complement
            // form such a face would carry half of the kernel
            if (tilde && D.hi < 1e-30f) force = true;
            const bool beyond = D.hi > 2.f || (D.hi == 2.f && D.lo >= 0.f);
            if (!(sd.hi == 0.f || (tilde && beyond))) {
                // reference distance to the polygon (FP32)
                const int64_t g0 = fvo[g], g1 = fvo[g + 1];
                bool inpoly = true;
                float rho2 = INFINITY;
                for (int64_t q1 = g0; q1 < g1; ++q1) {
                    EdgeF E = edge_f[q1];
                    float a = (E.cm - (E.mx * rxf + E.my * ryf + E.mz * rzf)) * ihf;
                    float t0 = (E.ce - (E.ex * rxf + E.ey * ryf + E.ez * rzf)) * ihf;
                    float t1 = t0 + E.L * ihf;
                    inpoly = inpoly && a > 0.f;
                    float tc = t0 > 0.f ? t0 : (t1 < 0.f ? t1 : 0.f);
                    rho2 = fminf(rho2, a * a + tc * tc);
                }
                const float rr2 = inpoly ? 0.f : rho2;
                const emq::ff D2 = emq::ff_mul(D, D);
                const emq::ff R2 = emq::ff_add(D2, emq::ff{rr2, 0.f});
                const bool far = R2.hi > 4.f || (R2.hi == 4.f && R2.lo >= 0.f);
                if (!(tilde && far)) {   // else the polygon lies entirely beyond 2h
                    fs.rr2 = rr2;
                    fs.dm1 = emq::ff_add(D2, emq::ff{-1.f, 0.f});
                    fs.d4 = emq::ff_add(emq::ff{4.f, 0.f}, emq::ff_neg(D2));
                    fs.Df = D.hi + D.lo;
                    face_consts(R2, tilde, fs);
                    fs.sign = sd.hi > 0.f ? 1.f : -1.f;
                    e0 = g0;
                    ne = (int)(g1 - g0);
                }
            }
        }
        for (int ei = 0; last ? ei == 0 : __any_sync(FULL_MASK, ei < ne); ++ei) {
            if (ei < ne) {
                // edge geometry in float-float (see quad32.cuh): A, T0, T1 and
                // B^2 - 1, 4 - B^2, A^2 - rho^2 each rounded once to FP32
                const EdgeF H = edge_f[e0 + ei], Lo = edge_fl[e0 + ei];
                const emq::ff ah = emq::ff_offset_dot(H.cm, Lo.cm, H.mx, Lo.mx, H.my, Lo.my, H.mz, Lo.mz, rxx, ryy, rzz);
                const emq::ff a = emq::ff_mul(ah, ihh);
                if (a.hi != 0.f) {
                    const emq::ff th = emq::ff_offset_dot(H.ce, Lo.ce, H.ex, Lo.ex, H.ey, Lo.ey, H.ez, Lo.ez, rxx, ryy, rzz);
                    const emq::ff t0 = emq::ff_mul(th, ihh);
                    const emq::ff lh = emq::ff_mul(emq::ff{H.L, Lo.L}, ihh);   // L/h
                    const emq::ff t1 = emq::ff_add(t0, lh);
                    const emq::ff a2 = emq::ff_mul(a, a);
                    // A below 1e-30 h changes the integral by ~1e-30 relative and would
                    // make the s-range of the sinh substitution unbounded
                    const float A = fmaxf(fabsf(a.hi + a.lo), 1e-30f), T0 = t0.hi + t0.lo, T1 = t1.hi + t1.lo;
                    const float dT = lh.hi + lh.lo;   // T1 - T0 = L/h, from the edge length itself
                    const float B2f = fs.Df * fs.Df + A * A;
                    const emq::ff c1x = emq::ff_add(fs.dm1, a2), c4x = emq::ff_add(fs.d4, emq::ff_neg(a2));
                    const emq::ff ccx = emq::ff_add(a2, emq::ff{-fs.rr2, 0.f});

                    // signed factor: D/pi, face orientation, side of the edge line, direction along it
                    const float base = fs.sign * (a.hi > 0.f ? 1.f : -1.f) * fs.Df * 0.31830988618379067154f;
                    // the edge's |tau| ranges: one if T0 and T1 lie on one side of
                    // the foot F, else [0, |T0|] and [0, |T1|]
                    const float u0 = fabsf(T0), u1 = fabsf(T1);
                    const bool one_side = (T0 >= 0.f && T1 >= 0.f) || (T0 <= 0.f && T1 <= 0.f);
                    const float sc = (one_side ? T1 >= T0 : T1 > T0) ? base : -base;
#pragma unroll 1
                    for (int part = 0; part < (one_side ? 1 : 2); ++part) {
                        // one side: [min |T|, min |T| + L/h]; else [0, |T0|] and [0, |T1|]
                        const float ua = one_side ? fminf(u0, u1) : 0.f;
                        const float du = one_side ? dT : (part ? u1 : u0);
                        mq_push_g(q, lane, cnt, ua, du, A, B2f, c1x, c4x, ccx, sc, fs, tilde, acc_far, mag_far);
                    }
                }
            }
            // an edge queues at most four segments
            if (__any_sync(FULL_MASK, cnt > (last ? 0 : MQ_SLOTS - 4))) {
                mq_flush(q, lane, cnt, acc, mag);
                cnt = 0;
            }
        }
        if (last) break;
    }
    bool flag = false;
    if (valid) {
        // the integrals were summed with their signs: w = sum (full kernel) or
        // [P inside] - sum (complement kernel)
        const emq::ff tot = emq::ff_add(acc, acc_far);
        const double sum = (double)tot.hi + (double)tot.lo;
        const double wk = full ? sum : ((inside ? 1.0 : 0.0) - sum);
        const double magd = (double)mag + (double)mag_far + ((inside && !full) ? 1.0 : 0.0);
        w[k] = wk;
        // error bound of the FP32 pass: est_k = (ulps) 2^-24 times the sum of
        // the non-negative pieces it summed.  With the default 8 ulps the
        // largest error/bound ratio seen against FP64 on the 1e5 and 1e6
        // clouds was 0.81; tiny cells deep inside large kernels (h / V^(1/3)
        // above ~12, as in the 8e6 cloud) need more
        const double est = est_k * magd;
        flag = force || !(est <= fmax((double)tol * fabs(wk), 1e-14));
    }
    // one append per warp: the flagged pairs of a warp (mostly of one cell)
    // stay together in the list, which keeps the FP64 pass's warps coherent
    const unsigned fm = __ballot_sync(FULL_MASK, flag);
    if (fm) {
        int base = 0;
        if (lane == 0) base = atomicAdd(nflag, __popc(fm));
        base = __shfl_sync(FULL_MASK, base, 0);
        if (flag) flagged[base + __popc(fm & ((1u << lane) - 1u))] = force ? ~(int32_t)k : (int32_t)k;
    }
}

// rho_j = sum_i m_i w_ij / V_j over the cell's pairs (ascending i), one warp per cell
__global__ void k_cell_density(int64_t ncell, const int64_t *__restrict__ off, const int32_t *__restrict__ pi,
                               const double *__restrict__ w, const double *__restrict__ m,
                               const double *__restrict__ volume, double *__restrict__ rho)
{
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= ncell) return;
    double s = 0.0;
    for (int64_t k = off[warp] + lane; k < off[warp + 1]; k += 32) s += m[pi[k]] * w[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    // a cell without pairs has density 0 (also one a range build left without volume)
    if (lane == 0) rho[warp] = off[warp + 1] > off[warp] ? s / volume[warp] : 0.0;
}

// u_i = sum_j w_ij (ascending j), one thread per particle
// Sums over a particle's pairs [k0, k1) of the (i, j)-ordered transpose, in
// ascending j, each product and each sum rounded on its own (no fused
// multiply-add): den = sum w, and with f given, num = sum w f_j.  The loads of
// PB pairs are issued before their sums, so that a thread has PB gathers in
// flight instead of one dependent chain at a time; the order of the sums is
// unchanged.
constexpr int PB = 8;
template <bool WITH_F>
__device__ __forceinline__ void pair_sums(int64_t k0, int64_t k1, const int32_t *__restrict__ idx,
                                          const int32_t *__restrict__ pj, const double *__restrict__ w,
                                          const double *__restrict__ f, double &num, double &den)
{
    int64_t k = k0;
    for (; k + PB <= k1; k += PB) {
        int32_t q[PB];
        double wq[PB], fq[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) q[u] = __ldg(idx + k + u);
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            wq[u] = __ldg(w + q[u]);
            fq[u] = WITH_F ? __ldg(f + __ldg(pj + q[u])) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < PB; ++u) {
            if (WITH_F) num = __dadd_rn(num, __dmul_rn(wq[u], fq[u]));
            den = __dadd_rn(den, wq[u]);
        }
    }
    for (; k < k1; ++k) {
        const int32_t q = idx[k];
        const double wq = w[q];
        if (WITH_F) num = __dadd_rn(num, __dmul_rn(wq, f[pj[q]]));
        den = __dadd_rn(den, wq);
    }
}

__global__ void k_particle_wsum(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                const double *__restrict__ w, double *__restrict__ u)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    double num = 0.0, s = 0.0;
    pair_sums<false>(off[i], off[i + 1], idx, nullptr, w, nullptr, num, s);
    u[i] = s;
}

// The FP32 pass in launch shape `variant` (see MQ_VARIANT_*).
template <int V>
static void launch_variant(cudaStream_t st, int64_t n, const int32_t *pi, const int32_t *pj, const double *x,
                           const double *y, const double *z, const double *h, const double *gen, const double *radius,
                           const int64_t *cfo, const int64_t *fvo, const PlaneF *pf, const PlaneF *pfl,
                           const EdgeF *ef, const EdgeF *efl, float tol, double est_k, double *w, int32_t *flagged,
                           int *nflag)
{
    constexpr int W = MQ_VARIANT_WARPS[V], B = MQ_VARIANT_MINB[V];
    k_map_fp32<W, B><<<em_grid((n + 31) / 32, W), 32 * W, 0, st>>>(n, pi, pj, x, y, z, h, gen, radius, cfo, fvo, pf,
                                                                 pfl, ef, efl, tol, est_k, w, flagged, nflag);
}

static void launch_map_fp32(int variant, cudaStream_t st, int64_t n, const int32_t *pi, const int32_t *pj,
                            const double *x, const double *y, const double *z, const double *h, const double *gen,
                            const double *radius, const int64_t *cfo, const int64_t *fvo, const PlaneF *pf,
                            const PlaneF *pfl, const EdgeF *ef, const EdgeF *efl, float tol, double est_k, double *w,
                            int32_t *flagged, int *nflag)
{
    switch (variant) {
    case 1: launch_variant<1>(st, n, pi, pj, x, y, z, h, gen, radius, cfo, fvo, pf, pfl, ef, efl, tol, est_k, w, flagged, nflag); break;
    case 2: launch_variant<2>(st, n, pi, pj, x, y, z, h, gen, radius, cfo, fvo, pf, pfl, ef, efl, tol, est_k, w, flagged, nflag); break;
    case 3: launch_variant<3>(st, n, pi, pj, x, y, z, h, gen, radius, cfo, fvo, pf, pfl, ef, efl, tol, est_k, w, flagged, nflag); break;
    default: launch_variant<0>(st, n, pi, pj, x, y, z, h, gen, radius, cfo, fvo, pf, pfl, ef, efl, tol, est_k, w, flagged, nflag); break;
    }
}

// map_exact, map_exact_noalloc and map_batch: the mixed pass's flagged-pair
// list and counter are stream-ordered scratch, the caller's scratch
// (d_flag_buf, d_flag_count: map_batch), or the library's fixed device array
// (fixed == true, at most EM_NOALLOC_MAX_PAIRS pairs).
static int noalloc_buffers(em_ctx *ctx, int32_t **flagged, int **count);

int em_map_exact_impl(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                      const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p, double *d_w_out,
                      double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64, bool fixed, int32_t *d_flag_buf,
                      int *d_flag_count)
{
    EM_CHECK_ARG(ctx && pr && v && p && pr->ncell == v->ncell);
    EM_CHECK_ARG(pr->npairs == 0 || (d_x && d_y && d_z && d_h && d_w_out));
    EM_CHECK_ARG(d_rho_out == nullptr || d_m != nullptr);
    EM_CHECK_ARG(p->precision == 0 || p->precision == 1);
    const int64_t n = pr->npairs;
    if (fixed && n > EM_NOALLOC_MAX_PAIRS) {
        em_set_error("map_exact_noalloc: %lld pairs exceed the fixed capacity of %d pairs", (long long)n,
                     EM_NOALLOC_MAX_PAIRS);
        return EM_ECAPACITY;
    }
    const int block = p->block_pairs > 0 ? p->block_pairs : 128;
    EM_CHECK_ARG(block % 32 == 0 && block <= 128);
    EM_CHECK_ARG(p->fp32_variant >= 0 && p->fp32_variant < MQ_NVARIANT);
    if (h_nfp64) *h_nfp64 = 0;
    if (ctx->timing) ctx->recorded[0] = ctx->recorded[1] = false;
    if (n) {
        const int fgrid = (int)std::min<int64_t>((n + block / 32 - 1) / (block / 32), (int64_t)ctx->nsm * 64);
        if (ctx->timing) EM_CUDA(cudaEventRecord(ctx->ev[0], ctx->stream));
        if (p->precision == 0) {
            k_map_fp64<<<fgrid, block, 0, ctx->stream>>>(n, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h, v->gen,
                                                         v->radius, v->cell_face_off, v->face_vert_off, v->plane,
                                                         v->edge, d_w_out);
            EM_LAUNCHED(ctx);
            if (ctx->timing) {
                EM_CUDA(cudaEventRecord(ctx->ev[1], ctx->stream));
                ctx->recorded[0] = true;
            }
        } else {
            DevArena tmp(ctx->stream, true);
            int32_t *flagged;
            int *nflag;
            if (fixed) {
                EM_TRY(noalloc_buffers(ctx, &flagged, &nflag));
            } else if (d_flag_buf && d_flag_count) {   // the caller's scratch (map_batch), n entries
                flagged = d_flag_buf;
                nflag = d_flag_count;
            } else {
                EM_TRY(tmp.alloc(&flagged, n));
                EM_TRY(tmp.alloc(&nflag, 1));
            }
            EM_CUDA(cudaMemsetAsync(nflag, 0, sizeof(int), ctx->stream));
            launch_map_fp32(p->fp32_variant, ctx->stream, n, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h, v->gen,
                            v->radius, v->cell_face_off, v->face_vert_off, v->plane_f, v->plane_fl, v->edge_f,
                            v->edge_fl, (float)p->fp64_threshold, em_est_k(p), d_w_out, flagged, nflag);
            EM_LAUNCHED(ctx);
            if (ctx->timing) {
                EM_CUDA(cudaEventRecord(ctx->ev[1], ctx->stream));
                EM_CUDA(cudaEventRecord(ctx->ev[2], ctx->stream));
            }
            // FP64 recompute of the flagged pairs; the count stays on the device
            k_map_fp64_flagged<<<fgrid, block, 0, ctx->stream>>>(nflag, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h,
                                                                 v->gen, v->radius, v->cell_face_off,
                                                                 v->face_vert_off, v->plane, v->edge, flagged,
                                                                 d_w_out);
            EM_LAUNCHED(ctx);
            if (ctx->timing) {
                EM_CUDA(cudaEventRecord(ctx->ev[3], ctx->stream));
                ctx->recorded[0] = ctx->recorded[1] = true;
            }
            if (h_nfp64) {
                int hflag = 0;
                EM_CUDA(cudaMemcpyAsync(&hflag, nflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
                EM_CUDA(cudaStreamSynchronize(ctx->stream));
                *h_nfp64 = hflag;
            }
        }
    }
    if (d_rho_out && v->ncell) {
        k_cell_density<<<em_grid(v->ncell * 32, 256), 256, 0, ctx->stream>>>(v->ncell, pr->cell_pair_off, pr->pair_i,
                                                                               d_w_out, d_m, v->volume, d_rho_out);
        EM_LAUNCHED(ctx);
    }
    if (d_wsum_out && pr->np) {
        k_particle_wsum<<<em_grid(pr->np, 256), 256, 0, ctx->stream>>>(pr->np, pr->part_pair_off, pr->part_pair_idx,
                                                                        d_w_out, d_wsum_out);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int map_exact(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                        const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p,
                        double *d_w_out, double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64)
{
    return em_map_exact_impl(ctx, pr, d_x, d_y, d_z, d_h, d_m, v, p, d_w_out, d_rho_out, d_wsum_out, h_nfp64, false,
                             nullptr, nullptr);
}

// Time the FP32 pass in every launch shape on the given pairs (a warm-up
// launch, then the median of three CUDA-event-timed launches each) and return
// the fastest.  Scratch only; the caller's arrays are read, never written.
EM_EXPORT int map_autotune(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                           const double *d_h, const em_voronoi *v, const em_params *p, int *h_best, double *h_ms)
{
    EM_CHECK_ARG(ctx && pr && v && p && h_best && pr->ncell == v->ncell);
    EM_CHECK_ARG(pr->npairs == 0 || (d_x && d_y && d_z && d_h));
    *h_best = 0;
    const int64_t n = pr->npairs;
    if (n == 0) {
        if (h_ms)
            for (int k = 0; k < MQ_NVARIANT; ++k) h_ms[k] = 0.0;
        return EM_OK;
    }
    DevArena tmp(ctx->stream, true);
    double *w;
    int32_t *flagged;
    int *nflag;
    EM_TRY(tmp.alloc(&w, n));
    EM_TRY(tmp.alloc(&flagged, n));
    EM_TRY(tmp.alloc(&nflag, 1));
    cudaEvent_t e0, e1;
    EM_CUDA(cudaEventCreate(&e0));
    EM_CUDA(cudaEventCreate(&e1));
    int rc = EM_OK;
    double best = 1e300;
    for (int k = 0; k < MQ_NVARIANT && rc == EM_OK; ++k) {
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        for (int r = 0; r < 4 && rc == EM_OK; ++r) {
            cudaMemsetAsync(nflag, 0, sizeof(int), ctx->stream);
            cudaEventRecord(e0, ctx->stream);
            launch_map_fp32(k, ctx->stream, n, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h, v->gen, v->radius,
                            v->cell_face_off, v->face_vert_off, v->plane_f, v->plane_fl, v->edge_f, v->edge_fl,
                            (float)p->fp64_threshold, em_est_k(p), w, flagged, nflag);
            ctx->launches++;
            cudaEventRecord(e1, ctx->stream);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], e0, e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                em_set_error("map_autotune: variant %d: %s", k, cudaGetErrorString(e));
                rc = EM_ECUDA;
            }
        }
        const float a = t[1], b = t[2], c = t[3];   // t[0] is the warm-up
        const double med = fmax(fmin(a, b), fmin(fmax(a, b), c));
        if (h_ms) h_ms[k] = med;
        if (rc == EM_OK && med < best) {
            best = med;
            *h_best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// ---------------------------------------------------------------------------
// map_exact without allocation, for callers that cannot allocate device
// memory during the call (their own pool holds all free memory, or they cannot
// take an allocation's synchronisation every step): the mixed pass's
// flagged-pair list and its counter live in a fixed device array instead of
// stream-ordered scratch.
// ---------------------------------------------------------------------------

namespace {

// Zeroed at the start of every call (the counter); the list needs no reset,
// the FP32 pass writes entries [0, count) before the FP64 pass reads them.
static __device__ __align__(256) int32_t g_noalloc_flagged[EM_NOALLOC_MAX_PAIRS];
static __device__ __align__(256) int g_noalloc_count[1];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
int32_t *g_noalloc_flagged_addr[NOALLOC_MAX_DEVICES];
int *g_noalloc_count_addr[NOALLOC_MAX_DEVICES];

}  // namespace

// Device addresses of the two arrays on ctx's device, looked up once per
// device with that device current.
static int noalloc_buffers(em_ctx *ctx, int32_t **flagged, int **count)
{
    EM_CHECK_ARG(ctx->device >= 0 && ctx->device < NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_flagged_addr[ctx->device]) {
        int cur = -1;
        EM_CUDA(cudaGetDevice(&cur));
        if (cur != ctx->device) EM_CUDA(cudaSetDevice(ctx->device));
        void *a = nullptr, *b = nullptr;
        cudaError_t e1 = cudaGetSymbolAddress(&a, g_noalloc_flagged);
        cudaError_t e2 = e1 == cudaSuccess ? cudaGetSymbolAddress(&b, g_noalloc_count) : e1;
        if (cur != ctx->device && cur >= 0) cudaSetDevice(cur);
        if (e2 != cudaSuccess) {
            em_set_error("map_exact_noalloc: cudaGetSymbolAddress failed on device %d: %s", ctx->device,
                         cudaGetErrorString(e2));
            return EM_ECUDA;
        }
        g_noalloc_count_addr[ctx->device] = (int *)b;
        g_noalloc_flagged_addr[ctx->device] = (int32_t *)a;
    }
    *flagged = g_noalloc_flagged_addr[ctx->device];
    *count = g_noalloc_count_addr[ctx->device];
    return EM_OK;
}

EM_EXPORT int map_exact_noalloc(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y,
                                const double *d_z, const double *d_h, const double *d_m, const em_voronoi *v,
                                const em_params *p, double *d_w_out, double *d_rho_out, double *d_wsum_out,
                                int64_t *h_nfp64)
{
    return em_map_exact_impl(ctx, pr, d_x, d_y, d_z, d_h, d_m, v, p, d_w_out, d_rho_out, d_wsum_out, h_nfp64, true,
                             nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// Inverse mapping
// ---------------------------------------------------------------------------

__global__ void k_map_back(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                           const int32_t *__restrict__ pj, const double *__restrict__ w,
                           const double *__restrict__ f_cell, double *__restrict__ f_out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    // ascending j, each product and each sum rounded on its own (pair_sums),
    // so that equal weights give bit-identical results on any implementation
    // that sums in the same order
    double num = 0.0, den = 0.0;
    pair_sums<true>(off[i], off[i + 1], idx, pj, w, f_cell, num, den);
    f_out[i] = num / den;
}

// every SPH particle takes the value of the pseudo-particle it belongs to
__global__ void k_inherit(int64_t npseudo, const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                          const int32_t *__restrict__ perm, const double *__restrict__ f_pseudo,
                          double *__restrict__ f_particle)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= npseudo) return;
    double f = f_pseudo[a];
    for (int32_t k = first[a]; k < first[a] + count[a]; ++k) f_particle[perm[k]] = f;
}

// The two sums of map_back per particle, added into num and den (ascending
// j, every product and sum rounded on its own, as k_map_back).
__global__ void k_map_back_sums(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                const int32_t *__restrict__ pj, const double *__restrict__ w,
                                const double *__restrict__ f_cell, double *__restrict__ num, double *__restrict__ den)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    double a = 0.0, b = 0.0;
    pair_sums<true>(off[i], off[i + 1], idx, pj, w, f_cell, a, b);
    num[i] = __dadd_rn(num[i], a);
    den[i] = __dadd_rn(den[i], b);
}

EM_EXPORT int map_back_sums(em_ctx *ctx, const em_pairs *pr, const double *d_w, const double *d_f_cell,
                            double *d_num, double *d_den)
{
    EM_CHECK_ARG(ctx && pr && d_num && d_den && (pr->npairs == 0 || d_w) && (pr->ncell == 0 || d_f_cell));
    if (pr->np) {
        k_map_back_sums<<<em_grid(pr->np, 256), 256, 0, ctx->stream>>>(pr->np, pr->part_pair_off,
                                                                        pr->part_pair_idx, pr->pair_j, d_w,
                                                                        d_f_cell, d_num, d_den);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int inherit(em_ctx *ctx, const em_pseudo *ps, const em_tree *t, const double *d_f_pseudo,
                      double *d_f_particle_out)
{
    EM_CHECK_ARG(ctx && ps && t && d_f_particle_out && (ps->n == 0 || d_f_pseudo));
    if (ps->n) {
        k_inherit<<<em_grid(ps->n, 128), 128, 0, ctx->stream>>>(ps->n, ps->first, ps->count, t->perm, d_f_pseudo,
                                                                 d_f_particle_out);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}

EM_EXPORT int map_back(em_ctx *ctx, const em_pairs *pr, const double *d_w, const double *d_f_cell, double *d_f_out,
                       const em_pseudo *ps, const em_tree *t, double *d_f_particle_out)
{
    EM_CHECK_ARG(ctx && pr && d_f_out && (pr->npairs == 0 || d_w) && (pr->ncell == 0 || d_f_cell));
    bool inherit = ps || t || d_f_particle_out;
    EM_CHECK_ARG(!inherit || (ps && t && d_f_particle_out && ps->n == pr->np));
    if (pr->np) {
        k_map_back<<<em_grid(pr->np, 256), 256, 0, ctx->stream>>>(pr->np, pr->part_pair_off, pr->part_pair_idx,
                                                                   pr->pair_j, d_w, d_f_cell, d_f_out);
        EM_LAUNCHED(ctx);
    }
    if (inherit && ps->n) {
        k_inherit<<<em_grid(ps->n, 128), 128, 0, ctx->stream>>>(ps->n, ps->first, ps->count, t->perm, d_f_out,
                                                                 d_f_particle_out);
        EM_LAUNCHED(ctx);
    }
    return EM_OK;
}
