// make_pseudo_particles: adaptive tree-walk selection (Section 2.4.1, Eq. 4),
// node neighbour search and the node smoothing-length solver (Section 2.4.2,
// Eqs. 6-11).
//
// Selection is evaluated per node instead of by a sequential walk: a node is
// reached when every ancestor is opened; a reached internal node that is not
// opened, or a reached leaf outside r_part, becomes a pseudo-particle; a
// reached leaf inside r_part is replaced by its particles.  The predicates use
// explicit round-to-nearest products, so the selected set is bit-identical to
// a sequential walk with the same arithmetic.
//
// The neighbour search runs inside every solver iteration: a warp walks a
// 32-ary box hierarchy over the solver population (selected nodes plus the
// leaves of extracted particles, Morton order) with radius 2h, so the sum
// n(h) = sum_b W(r_ab, h) always covers every neighbour of the current h.
#include <cmath>

#include "common.cuh"
#include "split.cuh"
#include "tree_util.cuh"

namespace {

enum : uint8_t { F_LEAF = 1, F_EXTRACT = 2, F_OPEN = 4, F_REACHED = 8 };

__global__ void k_node_flags(int64_t nnode, const int32_t *__restrict__ nchild, const double *__restrict__ cx,
                             const double *__restrict__ cy, const double *__restrict__ cz,
                             const double *__restrict__ size, int nsrc, const double *__restrict__ src, double rp2,
                             double rl2, double th2, const uint8_t *__restrict__ force, uint8_t *__restrict__ flags)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nnode) return;
    double r2 = INFINITY;
    for (int s = 0; s < nsrc; ++s) {
        double dx = __dsub_rn(cx[a], src[3 * s]), dy = __dsub_rn(cy[a], src[3 * s + 1]),
               dz = __dsub_rn(cz[a], src[3 * s + 2]);
        double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        r2 = q < r2 ? q : r2;
    }
    uint8_t f = 0;
    // a node the refinement check found under-resolved (Eq. 5) is opened, or
    // if a leaf has its particles extracted
    const bool forced = force != nullptr && force[a] != 0;
    if (nchild[a] == 0) {
        f |= F_LEAF;
        if (r2 < rp2 || forced) f |= F_EXTRACT;
    } else {
        // open inside r_leaf, or when theta^2 < (s/r)^2 (Eq. 4)
        if (forced || r2 < rl2 || __dmul_rn(size[a], size[a]) > __dmul_rn(th2, r2)) f |= F_OPEN;
    }
    flags[a] = f;
}

__global__ void k_reached(int64_t nnode, const int32_t *__restrict__ parent, uint8_t *__restrict__ flags)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nnode) return;
    bool r = true;
    for (int32_t p = parent[a]; p >= 0 && r; p = parent[p]) r = (flags[p] & F_OPEN) != 0;
    if (r) flags[a] |= F_REACHED;
}

// Mark Morton positions that start a pseudo-particle / a population entry.
__global__ void k_mark(int64_t nnode, const uint8_t *__restrict__ flags, const int32_t *__restrict__ first,
                       const int32_t *__restrict__ count, int32_t *__restrict__ start, int32_t *__restrict__ owner,
                       int32_t *__restrict__ popstart)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= nnode) return;
    uint8_t f = flags[a];
    if (!(f & F_REACHED)) return;
    bool leaf = f & F_LEAF;
    if (leaf && (f & F_EXTRACT)) {
        for (int32_t k = first[a]; k < first[a] + count[a]; ++k) {
            start[k] = 1;
            owner[k] = -1 - (int32_t)a;
        }
        popstart[first[a]] = 1;
    } else if (leaf || !(f & F_OPEN)) {
        start[first[a]] = 1;
        owner[first[a]] = (int32_t)a;
        popstart[first[a]] = 1;
    }
}

__global__ void k_emit(int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ pidx,
                       const int32_t *__restrict__ owner, const int32_t *__restrict__ popstart,
                       const int32_t *__restrict__ popidx, const uint64_t *__restrict__ label,
                       const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                       const double *__restrict__ mass, const double *__restrict__ cx, const double *__restrict__ cy,
                       const double *__restrict__ cz, const double *__restrict__ size, const double *__restrict__ xs,
                       const double *__restrict__ ys, const double *__restrict__ zs, const double *__restrict__ ms,
                       const int32_t *__restrict__ perm, const double *__restrict__ hpart, double h_fact,
                       double *__restrict__ px, double *__restrict__ py, double *__restrict__ pz,
                       double *__restrict__ ph, double *__restrict__ pm, int64_t *__restrict__ origin,
                       int32_t *__restrict__ pfirst, int32_t *__restrict__ pcount, int32_t *__restrict__ status,
                       int32_t *__restrict__ pnode, int32_t node_status, double *__restrict__ popx,
                       double *__restrict__ popy, double *__restrict__ popz)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (start[k]) {
        int32_t q = pidx[k];
        int32_t a = owner[k];
        if (a >= 0) {
            px[q] = cx[a];
            py[q] = cy[a];
            pz[q] = cz[a];
            pm[q] = mass[a];
            origin[q] = (int64_t)label[a];
            pfirst[q] = first[a];
            pcount[q] = count[a];
            pnode[q] = a;
            status[q] = node_status;   // -1: to be solved; 2: takes h_0 without a solve
            // h_0 = h_fact (2 s_node) (Eq. 11); a one-particle node starts from its particle's h
            ph[q] = (count[a] == 1 || size[a] == 0.0) ? hpart[perm[first[a]]] : (2.0 * h_fact) * size[a];
        } else {
            px[q] = xs[k];
            py[q] = ys[k];
            pz[q] = zs[k];
            pm[q] = ms[k];
            origin[q] = -(int64_t)perm[k] - 1;
            pfirst[q] = (int32_t)k;
            pcount[q] = 1;
            pnode[q] = -1;
            status[q] = 3;
            ph[q] = hpart[perm[k]];
        }
    }
    if (popstart[k]) {
        // the population entry at this position is the node whose range starts here
        int32_t a = owner[k];
        if (a < 0) a = -1 - a;
        int32_t q = popidx[k];
        popx[q] = cx[a];
        popy[q] = cy[a];
        popz[q] = cz[a];
    }
}

struct Density {
    double n, dn;
};

// Neighbour candidates that pass the FP32 prefilter are collected in a
// per-warp buffer and summed in FP64 32 at a time, one per lane, so that the
// FP64 work (the costly part on GB300, whose FP64 rate is 1/64 of FP32) runs
// with every lane busy instead of on the few lanes of each 32-point chunk
// that hold a neighbour.
constexpr int HS_WARPS = 4;
constexpr int HS_BUF = 64;   // two batches: a chunk adds at most 32 to fewer than 32

// The FP32 prefilter: candidates clearly beyond 2h skip the FP64 work.  The
// band, 1e-5 of the coordinates' scale plus 2h, is far above the FP32 rounding
// of the positions, so no neighbour is dropped.  Appends the warp's passing
// candidates to buf (nb entries, the same on every lane).
__device__ __forceinline__ void collect(const em::ChunkTree &T, int64_t k, bool valid, float xaf, float yaf,
                                        float zaf, float lim2, int32_t *buf, int &nb)
{
    const int lane = threadIdx.x & 31;
    bool cand = false;
    if (valid) {
        const float4 pk = T.pts[k];
        const float ex = pk.x - xaf, ey = pk.y - yaf, ez = pk.z - zaf;
        cand = ex * ex + ey * ey + ez * ez < lim2;
    }
    const unsigned b = __ballot_sync(0xffffffffu, cand);
    if (cand) buf[nb + __popc(b & ((1u << lane) - 1u))] = (int32_t)k;
    __syncwarp();
    nb += __popc(b);
}

// Drop the first 32 entries of buf (already summed).
__device__ __forceinline__ void shift32(int32_t *buf, int &nb)
{
    const int lane = threadIdx.x & 31;
    const int32_t v = lane + 32 < nb ? buf[lane + 32] : 0;
    __syncwarp();
    if (lane + 32 < nb) buf[lane] = v;
    __syncwarp();
    nb -= 32;
}

// q = sqrt(q2) from an FP32 reciprocal square root (within 2^-22 relative)
// and one FP64 Newton step, which squares that error: within about 1e-13
// relative, far below the solver's tolerance on h and the 1e-12 to which h is
// held, at four FP64 instructions fewer than a second step; below 1e-30 q is 0
// (W then differs from W(0) by about 1e-30).  The conversions to and from
// float are done on the bits (split.cuh), which gives the same values off the
// FP64 pipe; q2 < 4 here.
__device__ __forceinline__ double q_of(double q2)
{
    if (!(q2 > 1e-30)) return 0.0;
    double r = em::f64_of(rsqrtf(em::f32_of(q2)));
    r = r * (1.5 - 0.5 * q2 * r * r);
    return q2 * r;
}

// 1/x for 2^-100 <= |x| < 2^100 (h and f' here): an FP32 reciprocal (its
// conversions on the bits, split.cuh) and two FP64 Newton steps, within about
// an ulp.  The solver's divisions have the same operands on every lane, so
// each FP64 instruction costs the pipe a full warp; this takes about half the
// FP64 instructions of a division.
__device__ __forceinline__ double rcp64(double x)
{
    // outside that range (zero, infinities, NaN included) the plain division;
    // the test reads the exponent's bits, off the FP64 pipe
    const int e = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
    if (e < 923 || e >= 1123) return 1.0 / x;
    double r = em::f64_of(__frcp_rn(em::f32_of(x)));
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
}

// The M4 spline w(q) and g(q) = 3 w(q) + q w'(q), the two sums of the
// solver, for q < 2 (q2 = q^2).
__device__ __forceinline__ void m4_wg(double q, double q2, double &w, double &g)
{
    if (q < 1.0) {
        w = 1.0 + q2 * (-1.5 + 0.75 * q);
        g = 3.0 + q2 * (-7.5 + 4.5 * q);
    } else {
        const double t = 2.0 - q, t2 = t * t;
        w = 0.25 * t2 * t;
        g = 0.75 * t2 * (t - q);
    }
}

// n(h) and dn/dh for the pseudo-particle at (xa, ya, za), summed over the
// population inside 2h; the result is identical on all lanes.
__device__ Density warp_density(const em::ChunkTree &T, const double *__restrict__ qx,
                                const double *__restrict__ qy, const double *__restrict__ qz, double xa, double ya,
                                double za, double h, float margin, int32_t *buf)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0, ds = 0.0;
    const double ih = rcp64(h);
    const double norm = ih * ih * ih * 0.31830988618379067154;   // 1/(pi h^3)
    float R = (float)(2.0 * h) + margin;
    const float xaf = (float)xa, yaf = (float)ya, zaf = (float)za, h2f = (float)(2.0 * h);
    const float lim = h2f + 1e-5f * (fabsf(xaf) + fabsf(yaf) + fabsf(zaf) + h2f);
    const float lim2 = lim * lim;
    // sums of w and of g = 3w + q w' over the neighbours; n = norm sum w,
    // dn/dh = -norm sum g / h
    const double ih2 = ih * ih;
    auto sum_one = [&](int64_t k) {
        const double dx = qx[k] - xa, dy = qy[k] - ya, dz = qz[k] - za;
        const double q2 = (dx * dx + dy * dy + dz * dz) * ih2;
        if (q2 < 4.0) {
            double w, g;
            m4_wg(q_of(q2), q2, w, g);
            s += w;
            ds += g;
        }
    };
    int nb = 0;
    em::warp_traverse(T, xaf, yaf, zaf, R * R, INT64_MAX, [&](int64_t k, bool valid) {
        collect(T, k, valid, xaf, yaf, zaf, lim2, buf, nb);
        if (nb >= 32) {
            sum_one(buf[lane]);
            shift32(buf, nb);
        }
    });
    if (lane < nb) sum_one(buf[lane]);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
    }
    return Density{s * norm, -ds * norm * ih};
}

// Sign of f(h) = h_fact n(h)^(-1/3) - h (Eq. 8) for the bisection, which uses
// nothing else.  Every term of n is non-negative, so once the running sum
// exceeds (h_fact / h)^3 (1 + 1e-9) the sign is negative whatever the rest of
// the sum; the walk stops there (checked after each batch of 32 terms).  This
// matters for the wide first brackets (h up to 1e2 h_0), whose 2h sphere
// holds a large share of the population.  Otherwise the full sum decides, as
// in warp_density.  Returns the sign of f (+1, 0 or -1).
__device__ int warp_f_sign(const em::ChunkTree &T, const double *__restrict__ qx,
                           const double *__restrict__ qy, const double *__restrict__ qz, double xa, double ya,
                           double za, double h, double h_fact, float margin, int32_t *buf)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    const double ih = rcp64(h);
    const double norm = ih * ih * ih * 0.31830988618379067154;   // 1/(pi h^3)
    const double t = h_fact * ih;
    const double thr = t * t * t * (1.0 + 1e-9);
    float R = (float)(2.0 * h) + margin;
    const float xaf = (float)xa, yaf = (float)ya, zaf = (float)za, h2f = (float)(2.0 * h);
    const float lim = h2f + 1e-5f * (fabsf(xaf) + fabsf(yaf) + fabsf(zaf) + h2f);
    const float lim2 = lim * lim;
    // the sum of w; the walk stops once norm sum w exceeds thr
    const double ih2 = ih * ih, thrw = thr * (3.14159265358979323846 * h * h * h);   // thr / norm
    auto sum_one = [&](int64_t k) {
        const double dx = qx[k] - xa, dy = qy[k] - ya, dz = qz[k] - za;
        const double q2 = (dx * dx + dy * dy + dz * dz) * ih2;
        if (q2 < 4.0) {
            double w, g;
            m4_wg(q_of(q2), q2, w, g);
            s += w;
        }
    };
    int nb = 0;
    bool full = em::warp_traverse_until(T, xaf, yaf, zaf, R * R, [&](int64_t k, bool valid) {
        collect(T, k, valid, xaf, yaf, zaf, lim2, buf, nb);
        if (nb < 32) return true;
        sum_one(buf[lane]);
        shift32(buf, nb);
        double tot = s;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        return !(tot > thrw);
    });
    if (!full) return -1;
    if (lane < nb) sum_one(buf[lane]);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double f = h_fact * rcbrt(s * norm) - h;   // n^(-1/3) as a reciprocal cube root
    return f > 0.0 ? 1 : (f < 0.0 ? -1 : 0);
}

// One warp per pseudo-particle: Newton (Eq. 10) from h_0 (Eq. 11) until
// |dh|/h_0 < tol, bisection on [1e-2 h_0, 1e2 h_0], else h_0.
__global__ void k_h_solve(int64_t npseudo, em::ChunkTree T, const double *__restrict__ qx,
                          const double *__restrict__ qy, const double *__restrict__ qz, const double *__restrict__ px,
                          const double *__restrict__ py, const double *__restrict__ pz, double h_fact, double tol,
                          int max_newton, float margin, double *__restrict__ ph, int32_t *__restrict__ status)
{
    __shared__ int32_t bufs[HS_WARPS][HS_BUF];
    int32_t *buf = bufs[threadIdx.x >> 5];
    int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (a >= npseudo) return;
    if (status[a] != -1) return;   // extracted particles keep their own h
    const double xa = px[a], ya = py[a], za = pz[a];
    const double h0 = ph[a];
    const double ih0 = rcp64(h0), blo = 1e-2 * h0, bhi = 1e2 * h0;
    double h = h0;
    bool ok = false;
    for (int it = 0; it < max_newton; ++it) {
        Density d = warp_density(T, qx, qy, qz, xa, ya, za, h, margin, buf);
        // n^(-1/3) as a reciprocal cube root and n^(-4/3) as its fourth power:
        // the same values to an ulp or two, for a fraction of the FP64 work of
        // two general powers (every lane computes them, so each FP64
        // instruction costs the pipe a full warp)
        const double c = rcbrt(d.n);
        double f = h_fact * c - h;                                          // Eq. 8
        double fp = -h_fact * d.dn * ((c * c) * (c * c)) * (1.0 / 3.0) - 1.0;   // Eq. 9 (a product, not a division)
        double hn = h - f * rcp64(fp);                                      // Eq. 10
        if (!(hn >= blo && hn <= bhi)) break;   // left the bracket [1e-2 h0, 1e2 h0]: Newton failed
        double step = fabs(hn - h) * ih0;   // |dh| / h_0
        h = hn;
        if (step < tol) {
            ok = true;
            break;
        }
    }
    int st = 0;
    if (!ok) {
        // bisection on signs only (warp_f_sign)
        double lo = 1e-2 * h0, hi = 1e2 * h0;
        const int slo = warp_f_sign(T, qx, qy, qz, xa, ya, za, lo, h_fact, margin, buf);
        const int shi = warp_f_sign(T, qx, qy, qz, xa, ya, za, hi, h_fact, margin, buf);
        const bool plo = slo > 0;
        if (slo * shi > 0) {
            h = h0;
            st = 2;
        } else {
            for (int k = 0; k < 200 && (hi - lo) > tol * h0; ++k) {
                double mid = 0.5 * (lo + hi);
                if ((warp_f_sign(T, qx, qy, qz, xa, ya, za, mid, h_fact, margin, buf) > 0) == plo) lo = mid;
                else hi = mid;
            }
            h = 0.5 * (lo + hi);
            st = 1;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        ph[a] = h;
        status[a] = st;
    }
}

__global__ void k_status_count(int64_t n, const int32_t *__restrict__ status, unsigned long long *__restrict__ cnt)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int s = status[a];
    if (s >= 0 && s < 4) atomicAdd(&cnt[s], 1ull);
}

}  // namespace

static int pseudo_impl(em_ctx *ctx, const em_tree *t, const double *d_hp, int nsrc, const double *h_src,
                       const em_params *p, const uint8_t *d_force, em_pseudo *ps)
{
    cudaStream_t st = ctx->stream;
    const int64_t n = t->n, nn = t->nnode;
    DevArena tmp(st, true);
    double *src;
    uint8_t *flags;
    int32_t *start, *owner, *popstart, *pidx, *popidx;
    EM_TRY(tmp.alloc(&src, 3 * nsrc));
    EM_TRY(tmp.alloc(&flags, nn));
    EM_TRY(tmp.alloc(&start, n));
    EM_TRY(tmp.alloc(&owner, n));
    EM_TRY(tmp.alloc(&popstart, n));
    EM_TRY(tmp.alloc(&pidx, n));
    EM_TRY(tmp.alloc(&popidx, n));
    EM_CUDA(cudaMemcpyAsync(src, h_src, 3 * nsrc * sizeof(double), cudaMemcpyHostToDevice, st));
    EM_CUDA(cudaMemsetAsync(start, 0, n * sizeof(int32_t), st));
    EM_CUDA(cudaMemsetAsync(popstart, 0, n * sizeof(int32_t), st));
    const double rp2 = p->r_part * p->r_part, rl2 = p->r_leaf * p->r_leaf, th2 = p->theta * p->theta;
    k_node_flags<<<em_grid(nn, 256), 256, 0, st>>>(nn, t->nchild, t->cx, t->cy, t->cz, t->size, nsrc, src, rp2, rl2,
                                                   th2, d_force, flags);
    EM_LAUNCHED(ctx);
    k_reached<<<em_grid(nn, 256), 256, 0, st>>>(nn, t->parent, flags);
    EM_LAUNCHED(ctx);
    k_mark<<<em_grid(nn, 256), 256, 0, st>>>(nn, flags, t->first, t->count, start, owner, popstart);
    EM_LAUNCHED(ctx);
    EM_TRY(em_exclusive_scan_i32(ctx, start, pidx, n));
    EM_TRY(em_exclusive_scan_i32(ctx, popstart, popidx, n));
    int32_t h4[4];
    cudaMemcpyAsync(&h4[0], pidx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&h4[1], start + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&h4[2], popidx + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&h4[3], popstart + n - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    EM_CUDA(cudaStreamSynchronize(st));
    const int64_t np = (int64_t)h4[0] + h4[1], npop = (int64_t)h4[2] + h4[3];
    ps->n = np;
    ps->npop = npop;
    // more pseudo-particles than h0_above: every node keeps h_0, no neighbour
    // search and no solve (Section 2.4.2)
    const bool bypass = p->h0_above > 0 && np > (int64_t)p->h0_above;
    DevArena &m = ps->mem;
    EM_TRY(m.alloc(&ps->x, np));
    EM_TRY(m.alloc(&ps->y, np));
    EM_TRY(m.alloc(&ps->z, np));
    EM_TRY(m.alloc(&ps->h, np));
    EM_TRY(m.alloc(&ps->m, np));
    EM_TRY(m.alloc(&ps->origin, np));
    EM_TRY(m.alloc(&ps->first, np));
    EM_TRY(m.alloc(&ps->count, np));
    EM_TRY(m.alloc(&ps->status, np));
    EM_TRY(m.alloc(&ps->node, np));
    double *qx, *qy, *qz;
    EM_TRY(tmp.alloc(&qx, npop));
    EM_TRY(tmp.alloc(&qy, npop));
    EM_TRY(tmp.alloc(&qz, npop));
    k_emit<<<em_grid(n, 256), 256, 0, st>>>(n, start, pidx, owner, popstart, popidx, t->label, t->first, t->count,
                                            t->mass, t->cx, t->cy, t->cz, t->size, t->xs, t->ys, t->zs, t->ms,
                                            t->perm, d_hp, p->h_fact, ps->x, ps->y, ps->z, ps->h, ps->m, ps->origin,
                                            ps->first, ps->count, ps->status, ps->node, bypass ? 2 : -1, qx, qy,
                                            qz);
    EM_LAUNCHED(ctx);
    if (np && !bypass) {
        em::ChunkTree T;
        EM_TRY(em_chunk_tree_build(ctx, tmp, npop, qx, qy, qz, nullptr, 0.0, &T));
        double ext = 0.0;
        for (int k = 0; k < 6; ++k) ext = fmax(ext, fabs(t->box[k]));
        // float rounding of positions and boxes: widen the search radius
        const float margin = (float)(4e-7 * (ext + 1.0));
        k_h_solve<<<em_grid(np * 32, 32 * HS_WARPS), 32 * HS_WARPS, 0, st>>>(
            np, T, qx, qy, qz, ps->x, ps->y, ps->z, p->h_fact, p->h_tol, p->max_newton, margin, ps->h, ps->status);
        EM_LAUNCHED(ctx);
    }
    unsigned long long *cnt;
    EM_TRY(tmp.alloc(&cnt, 4));
    EM_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), st));
    if (np) {
        k_status_count<<<em_grid(np, 256), 256, 0, st>>>(np, ps->status, cnt);
        EM_LAUNCHED(ctx);
    }
    unsigned long long hc[4];
    EM_CUDA(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, st));
    EM_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) ps->nstatus[k] = (int64_t)hc[k];
    return EM_OK;
}

static int make_pseudo(em_ctx *ctx, const em_tree *t, const double *d_h_particle, int nsrc, const double *h_src,
                       const em_params *p, const uint8_t *d_force, em_pseudo **out)
{
    EM_CHECK_ARG(ctx && t && d_h_particle && h_src && p && out);
    EM_CHECK_ARG(nsrc >= 1 && nsrc <= 4096);
    EM_CHECK_ARG(p->theta >= 0.0 && p->r_part >= 0.0 && p->r_leaf >= 0.0 && p->h_fact > 0.0);
    EM_CHECK_ARG(p->h_tol > 0.0 && p->max_newton >= 0 && p->h0_above >= 0);
    *out = nullptr;
    em_pseudo *ps = new em_pseudo(ctx->stream);
    ps->device = ctx->device;
    int rc = pseudo_impl(ctx, t, d_h_particle, nsrc, h_src, p, d_force, ps);
    if (rc) {
        ps->mem.release();
        delete ps;
        return rc;
    }
    *out = ps;
    const bool bypass = p->h0_above > 0 && ps->n > (int64_t)p->h0_above;
    return ps->nstatus[2] && !bypass ? EM_ENOTCONV : EM_OK;
}

EM_EXPORT int make_pseudo_particles(em_ctx *ctx, const em_tree *t, const double *d_h_particle, int nsrc,
                                    const double *h_src, const em_params *p, em_pseudo **out)
{
    return make_pseudo(ctx, t, d_h_particle, nsrc, h_src, p, nullptr, out);
}

EM_EXPORT int make_pseudo_particles_forced(em_ctx *ctx, const em_tree *t, const double *d_h_particle, int nsrc,
                                           const double *h_src, const em_params *p, const uint8_t *d_force,
                                           em_pseudo **out)
{
    EM_CHECK_ARG(d_force);
    return make_pseudo(ctx, t, d_h_particle, nsrc, h_src, p, d_force, out);
}

namespace {

// Eq. 5 for every node pseudo-particle: under-resolved when its neutral
// fraction is below (K - s_root / s_node) / K (NaN, a pseudo-particle without
// pairs, does not fail; nor does a node of size 0).  cnt[1] counts the failing
// leaves.  A failing internal node not yet flagged, and a failing leaf when
// flag_leaves is set, gets its flag and is counted in cnt[0].
__global__ void k_refine_check(int64_t np, const int32_t *__restrict__ node, const int32_t *__restrict__ nchild,
                               const double *__restrict__ size, const double *__restrict__ f_neu, double K,
                               int flag_leaves, uint8_t *__restrict__ force, unsigned long long *__restrict__ cnt)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= np) return;
    const int32_t a = node[q];
    if (a < 0 || !(size[a] > 0.0)) return;
    const double lim = (K - size[0] / size[a]) / K;
    if (!(f_neu[q] < lim)) return;
    const bool leaf = nchild[a] == 0;
    if (leaf) atomicAdd(&cnt[1], 1ull);
    if ((!leaf || flag_leaves) && !force[a]) {
        force[a] = 1;
        atomicAdd(&cnt[0], 1ull);
    }
}

}  // namespace

EM_EXPORT int refine_check(em_ctx *ctx, const em_pseudo *ps, const em_tree *t, const double *d_f_neu, double K,
                           int flag_leaves, uint8_t *d_force, int64_t *h_nnew, int64_t *h_nleaf)
{
    EM_CHECK_ARG(ctx && ps && t && d_f_neu && d_force && h_nnew);
    EM_CHECK_ARG(K > 1.0);
    EM_CHECK_ARG(flag_leaves == 0 || flag_leaves == 1);
    *h_nnew = 0;
    if (h_nleaf) *h_nleaf = 0;
    if (ps->n == 0 || t->nnode == 0) return EM_OK;
    DevArena tmp(ctx->stream, true);
    unsigned long long *cnt;
    EM_TRY(tmp.alloc(&cnt, 2));
    EM_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof *cnt, ctx->stream));
    k_refine_check<<<em_grid(ps->n, 256), 256, 0, ctx->stream>>>(ps->n, ps->node, t->nchild, t->size, d_f_neu, K,
                                                                 flag_leaves, d_force, cnt);
    EM_LAUNCHED(ctx);
    unsigned long long h[2] = {0, 0};
    EM_CUDA(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    EM_CUDA(cudaStreamSynchronize(ctx->stream));
    *h_nnew = (int64_t)h[0];
    if (h_nleaf) *h_nleaf = (int64_t)h[1];
    return EM_OK;
}
