// Exact mapping (map_exact), cell densities, inverse mapping (map_back), and
// the import paths for cells and pair lists.
#include <cmath>

#include "common.cuh"
#include "exact.cuh"
#include "quad32.cuh"

using namespace em;

// ---------------------------------------------------------------------------
// Derived cell geometry in each generator's frame
// ---------------------------------------------------------------------------

__global__ void k_prepare_cells(int64_t ncell, const double *__restrict__ gen, const int64_t *__restrict__ cfo,
                                const int64_t *__restrict__ fvo, const double *__restrict__ verts,
                                const double *__restrict__ normals, double *__restrict__ radius,
                                PlaneD *__restrict__ plane, EdgeD *__restrict__ edge, PlaneF *__restrict__ plane_f,
                                EdgeF *__restrict__ edge_f)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= ncell) return;
    double gx = gen[3 * j], gy = gen[3 * j + 1], gz = gen[3 * j + 2];
    double r2max = 0.0;
    for (int64_t f = cfo[j]; f < cfo[j + 1]; ++f) {
        double nx = normals[3 * f], ny = normals[3 * f + 1], nz = normals[3 * f + 2];
        int64_t v0 = fvo[f], v1 = fvo[f + 1];
        double c = nx * (verts[3 * v0] - gx) + ny * (verts[3 * v0 + 1] - gy) + nz * (verts[3 * v0 + 2] - gz);
        plane[f] = PlaneD{nx, ny, nz, c};
        plane_f[f] = PlaneF{(float)nx, (float)ny, (float)nz, (float)c};
        for (int64_t k = v0; k < v1; ++k) {
            int64_t k1 = (k + 1 < v1) ? k + 1 : v0;
            double ax = verts[3 * k] - gx, ay = verts[3 * k + 1] - gy, az = verts[3 * k + 2] - gz;
            double bx = verts[3 * k1] - gx, by = verts[3 * k1 + 1] - gy, bz = verts[3 * k1 + 2] - gz;
            double q = ax * ax + ay * ay + az * az;
            r2max = q > r2max ? q : r2max;
            double ex = bx - ax, ey = by - ay, ez = bz - az;
            double L = sqrt(ex * ex + ey * ey + ez * ez);
            EdgeD E;
            if (L > 0.0) {
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
            EdgeF F;
            F.mx = (float)E.mx;
            F.my = (float)E.my;
            F.mz = (float)E.mz;
            F.cm = (float)E.cm;
            F.ex = (float)E.ex;
            F.ey = (float)E.ey;
            F.ez = (float)E.ez;
            F.ce = (float)E.ce;
            F.L = (float)E.L;
            F.pad0 = F.pad1 = F.pad2 = 0.f;
            edge_f[k] = F;
        }
    }
    radius[j] = sqrt(r2max);
}

int em_prepare_cells(em_ctx *ctx, em_voronoi *v)
{
    EM_TRY(v->mem.alloc(&v->radius, v->ncell));
    EM_TRY(v->mem.alloc(&v->plane, v->nface));
    EM_TRY(v->mem.alloc(&v->edge, v->nfv));
    EM_TRY(v->mem.alloc(&v->plane_f, v->nface));
    EM_TRY(v->mem.alloc(&v->edge_f, v->nfv));
    if (v->ncell) {
        k_prepare_cells<<<em_grid(v->ncell, 128), 128, 0, ctx->stream>>>(
            v->ncell, v->gen, v->cell_face_off, v->face_vert_off, v->verts, v->normals, v->radius, v->plane,
            v->edge, v->plane_f, v->edge_f);
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

__global__ void __launch_bounds__(128) k_map_fp64(int64_t npairs, const int32_t *__restrict__ pi,
                                                  const int32_t *__restrict__ pj, const double *__restrict__ x,
                                                  const double *__restrict__ y, const double *__restrict__ z,
                                                  const double *__restrict__ h, const double *__restrict__ gen,
                                                  const double *__restrict__ radius, const int64_t *__restrict__ cfo,
                                                  const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane,
                                                  const EdgeD *__restrict__ edge, const int32_t *__restrict__ list,
                                                  double *__restrict__ w)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= npairs) return;
    int64_t k = list ? (int64_t)list[t] : t;
    int i = pi[k], j = pj[k];
    double err;
    w[k] = pair_weight<double, true>(x[i] - gen[3 * j], y[i] - gen[3 * j + 1], z[i] - gen[3 * j + 2], h[i], radius[j],
                               cfo[j], cfo[j + 1], fvo, plane, edge, err);
}

// FP32 bulk pass (quadrature form, see quad32.cuh).  Per face: the reference
// R = distance from p to the face polygon (FP32 is enough: any value used
// consistently for the face is exact when P is outside the polygon; inside,
// R = D), then R, 2 - R, K(R) and K(1) - K(R) from FP64.  Per edge: D, A,
// T0, T1, B^2, B^2 - 1, 4 - B^2 and A^2 - rho^2 in FP64 (one rounding each),
// the quadrature nodes in FP32.  The estimated error 12 eps times the sum of
// the magnitudes of the non-negative pieces flags the pair for the FP64 pass
// when it exceeds tol |w| + 1e-14; so does a face plane through P.
__global__ void __launch_bounds__(128) k_map_fp32(int64_t npairs, const int32_t *__restrict__ pi,
                                                  const int32_t *__restrict__ pj, const double *__restrict__ x,
                                                  const double *__restrict__ y, const double *__restrict__ z,
                                                  const double *__restrict__ h, const double *__restrict__ gen,
                                                  const double *__restrict__ radius, const int64_t *__restrict__ cfo,
                                                  const int64_t *__restrict__ fvo, const PlaneD *__restrict__ plane,
                                                  const EdgeD *__restrict__ edge, const PlaneF *__restrict__ plane_f,
                                                  const EdgeF *__restrict__ edge_f, float tol, double *__restrict__ w,
                                                  int32_t *__restrict__ flagged, int *__restrict__ nflag)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const int i = pi[k], j = pj[k];
    const double rx = x[i] - gen[3 * j], ry = y[i] - gen[3 * j + 1], rz = z[i] - gen[3 * j + 2];
    const double hh = h[i], ih = 1.0 / hh;
    const float rxf = (float)rx, ryf = (float)ry, rzf = (float)rz, ihf = (float)ih;
    const int64_t f0 = cfo[j], f1 = cfo[j + 1];
    bool inside = true;
    for (int64_t f = f0; f < f1; ++f) {
        PlaneD pl = plane[f];
        inside = inside && !(pl.w - (pl.x * rx + pl.y * ry + pl.z * rz) < 0.0);
    }
    const bool full = inside && (sqrt(rx * rx + ry * ry + rz * rz) + radius[j] < 2.0 * hh);
    double acc = 0.0, mag = 0.0;
    bool force = false;   // the FP32 form does not apply: recompute in FP64
    for (int64_t f = f0; f < f1; ++f) {
        PlaneD pl = plane[f];
        const double sd = pl.w - (pl.x * rx + pl.y * ry + pl.z * rz);
        const double D64 = fabs(sd) * ih;
        // P in (or within underflow of) the face plane: in the complement
        // form such a face would carry half of the kernel, so leave it to FP64
        if (!full && D64 < 1e-30) force = true;
        if (sd == 0.0 || (!full && D64 >= 2.0)) continue;
        const int64_t e0 = fvo[f], e1 = fvo[f + 1];
        // reference distance to the polygon (FP32)
        bool inpoly = true;
        float rho2 = INFINITY;
        for (int64_t e = e0; e < e1; ++e) {
            EdgeF E = edge_f[e];
            float a = (E.cm - (E.mx * rxf + E.my * ryf + E.mz * rzf)) * ihf;
            float t0 = (E.ce - (E.ex * rxf + E.ey * ryf + E.ez * rzf)) * ihf;
            float t1 = t0 + E.L * ihf;
            inpoly = inpoly && a > 0.f;
            float tc = t0 > 0.f ? t0 : (t1 < 0.f ? t1 : 0.f);
            rho2 = fminf(rho2, a * a + tc * tc);
        }
        const float Df = (float)D64;
        const double rr2 = inpoly ? 0.0 : (double)rho2;
        const double R2 = D64 * D64 + rr2;
        if (!full && R2 >= 4.0) continue;   // the polygon lies entirely beyond 2h
        const double R64 = sqrt(R2);
        emq::FaceRef fr;
        fr.tilde = !full;
        fr.R = (float)R64;
        fr.R2 = fr.R * fr.R;
        fr.R3 = fr.R2 * fr.R;
        fr.R4 = fr.R2 * fr.R2;
        fr.v = (float)(2.0 - R64);
        fr.v2 = fr.v * fr.v;
        fr.v3 = fr.v2 * fr.v;
        fr.v4 = fr.v2 * fr.v2;
        fr.KR = (float)(full ? em::K_of(R64) : em::K_tilde(R64));
        fr.C1 = R64 < 1.0 ? (float)(full ? em::K_of(1.0) - em::K_of(R64) : em::K_tilde(1.0) - em::K_tilde(R64)) : 0.f;
        float fs = 0.f, fm = 0.f;
        for (int64_t e = e0; e < e1; ++e) {
            EdgeD E = edge[e];
            const double a = (E.cm - (E.mx * rx + E.my * ry + E.mz * rz)) * ih;
            if (a == 0.0) continue;
            const double t0 = (E.ce - (E.ex * rx + E.ey * ry + E.ez * rz)) * ih;
            const double t1 = t0 + E.L * ih;
            const double B2 = D64 * D64 + a * a;
            emq::EdgeRef er;
            er.cc = (float)(a * a - rr2);
            er.c1 = (float)(B2 - 1.0);
            er.c4 = (float)(4.0 - B2);
            float mg;
            const float v = emq::edge_q(Df, (float)fabs(a), (float)t0, (float)t1, (float)B2, fr, er, mg);
            fs += a > 0.0 ? v : -v;
            fm += mg;
        }
        acc += sd > 0.0 ? (double)fs : -(double)fs;
        mag += (double)fm;
    }
    const double wk = full ? acc : ((inside ? 1.0 : 0.0) - acc);
    if (inside && !full) mag += 1.0;
    w[k] = wk;
    // error bound of the FP32 pass: 12 ulp of every non-negative piece it
    // summed (pieces are relative-accurate to a few ulp; the factor carries a
    // 1.5x margin over the largest error/bound ratio seen against FP64)
    const double est = 12.0 * 5.9604644775390625e-8 * mag;
    if (force || !(est <= (double)tol * fabs(wk) + 1e-14)) {
        int slot = atomicAdd(nflag, 1);
        flagged[slot] = (int32_t)k;
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
    if (lane == 0) rho[warp] = s / volume[warp];
}

// u_i = sum_j w_ij (ascending j), one thread per particle
__global__ void k_particle_wsum(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                const double *__restrict__ w, double *__restrict__ u)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    double s = 0.0;
    for (int64_t k = off[i]; k < off[i + 1]; ++k) s += w[idx[k]];
    u[i] = s;
}

EM_EXPORT int map_exact(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                        const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p,
                        double *d_w_out, double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64)
{
    EM_CHECK_ARG(ctx && pr && v && p && pr->ncell == v->ncell);
    EM_CHECK_ARG(pr->npairs == 0 || (d_x && d_y && d_z && d_h && d_w_out));
    EM_CHECK_ARG(d_rho_out == nullptr || d_m != nullptr);
    EM_CHECK_ARG(p->precision == 0 || p->precision == 1);
    int64_t n = pr->npairs;
    int block = p->block_pairs > 0 ? p->block_pairs : 128;
    EM_CHECK_ARG(block % 32 == 0 && block <= 128);
    if (h_nfp64) *h_nfp64 = 0;
    if (n) {
        if (p->precision == 0) {
            k_map_fp64<<<em_grid(n, block), block, 0, ctx->stream>>>(n, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h,
                                                                     v->gen, v->radius, v->cell_face_off,
                                                                     v->face_vert_off, v->plane, v->edge, nullptr,
                                                                     d_w_out);
            EM_LAUNCHED(ctx);
        } else {
            DevArena tmp(ctx->stream, true);
            int32_t *flagged;
            int *nflag;
            EM_TRY(tmp.alloc(&flagged, n));
            EM_TRY(tmp.alloc(&nflag, 1));
            EM_CUDA(cudaMemsetAsync(nflag, 0, sizeof(int), ctx->stream));
            k_map_fp32<<<em_grid(n, block), block, 0, ctx->stream>>>(
                n, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h, v->gen, v->radius, v->cell_face_off,
                v->face_vert_off, v->plane, v->edge, v->plane_f, v->edge_f, (float)p->fp64_threshold, d_w_out,
                flagged, nflag);
            EM_LAUNCHED(ctx);
            int hflag = 0;
            EM_CUDA(cudaMemcpyAsync(&hflag, nflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            EM_CUDA(cudaStreamSynchronize(ctx->stream));
            if (hflag) {
                k_map_fp64<<<em_grid(hflag, block), block, 0, ctx->stream>>>(
                    hflag, pr->pair_i, pr->pair_j, d_x, d_y, d_z, d_h, v->gen, v->radius, v->cell_face_off,
                    v->face_vert_off, v->plane, v->edge, flagged, d_w_out);
                EM_LAUNCHED(ctx);
            }
            if (h_nfp64) *h_nfp64 = hflag;
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

// ---------------------------------------------------------------------------
// Inverse mapping
// ---------------------------------------------------------------------------

__global__ void k_map_back(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                           const int32_t *__restrict__ pj, const double *__restrict__ w,
                           const double *__restrict__ f_cell, double *__restrict__ f_out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    double num = 0.0, den = 0.0;
    for (int64_t k = off[i]; k < off[i + 1]; ++k) {
        int32_t q = idx[k];
        num += w[q] * f_cell[pj[q]];
        den += w[q];
    }
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
