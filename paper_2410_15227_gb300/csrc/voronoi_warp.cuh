// Warp-cooperative Voronoi cell construction (one warp per cell, the cell
// in shared memory, in dual form: planes, and vertices as triangles of
// planes).  A clip removes the vertices beyond the bisector, keeps the
// others in order and appends the new vertices in the order (removed
// vertex, edge), so the vertex order is fixed by the clips alone.
// Candidates: every generator within a radius R of the site (found by a warp
// walk of the generators' box hierarchy), sorted by distance; the cell is
// exact once 2 R_max < R, otherwise the shell up to 2 R_max is clipped in as
// well.
//
// Arithmetic.  The planes are exact FP64 bisectors (g_k - g, |g_k - g|^2 / 2)
// and each vertex is the meet of its three planes.  During the construction a
// vertex is held in FP32 only, computed from the FP32 roundings of its planes
// by Cramer's rule together with a bound on its distance from the exact meet
// of the FP64 planes (meet32).  A side test in FP32 whose margin exceeds the
// bound it implies is exact; the few that do not decide take the vertex's
// FP64 meet (meet64).  The FP64 vertices of the finished cell are formed
// once, for its faces.  So the FP64 pipe, at 1/64 of the FP32 rate, carries
// the exact decisions and the output, not the construction.
#pragma once

#include <cstdint>

#include "split.cuh"
#include "tree_util.cuh"
#include "voronoi_cell.cuh"

namespace emw {

constexpr int WMAXP = emv::MAXP;
constexpr int WCAND = 256;   // candidate list (power of two for the bitonic sort)
constexpr float U32 = 5.9604645e-8f;   // 2^-24, the unit roundoff of FP32

// A cell under construction with room for NV vertices.  Plane q is the
// bisector of the site and generator sid[q] (its sorted index), or box wall
// -1 - sid[q]; its FP64 form is formed again from the generator positions
// wherever it is needed (plane64), its FP32 rounding is kept in pf[q].
template <int NV>
struct WCell {
    static constexpr int MAXV = NV;
    static_assert(NV <= 255, "vertex indices are bytes, 0xff marks a removed vertex");
    float vf[NV][4];   // FP32 vertex in the site's frame, w = |x| + |y| + |z|
    float ev[NV];      // bound on |vf - v| per coordinate, v the exact meet of its planes
    float4 pf[WMAXP];
    int sid[WMAXP];
    union {
        struct {
            float cd2[WCAND];   // sort keys of the candidates: squared distances rounded to FP32
            int cid[WCAND];
        } k;                    // while the cell is built
        double vx[NV][3];       // the FP64 vertices of the finished cell
    } u;
    // clip in progress: 1 if the vertex lies beyond the plane, then its new
    // index (0xff if removed)
    uint8_t side[NV];
    uint8_t out_list[NV];   // clip in progress: the removed vertices
    uint8_t tri[2][NV][4];
    // adj[t][e]: the vertex across edge e of vertex t, i.e. the one whose
    // triangle holds the reversed edge (tri[t][e + 1], tri[t][e])
    uint8_t adj[2][NV][4];
    int np, nt, cur;
};

// Bisector plane n.x <= d of the site g (at the origin of the cell's frame)
// and generator k: n = g_k - g, d = |n|^2 / 2.
__device__ __forceinline__ void bisector(const double *__restrict__ xs, const double *__restrict__ ys,
                                         const double *__restrict__ zs, int64_t k, double gx, double gy, double gz,
                                         double &nx, double &ny, double &nz, double &d)
{
    nx = __dsub_rn(xs[k], gx);
    ny = __dsub_rn(ys[k], gy);
    nz = __dsub_rn(zs[k], gz);
    d = __dmul_rn(0.5, __fma_rn(nz, nz, __fma_rn(ny, ny, __dmul_rn(nx, nx))));
}

// Box wall w (0..5: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) as n.x <= d in the
// site's frame.
__device__ __forceinline__ void wall_plane(const double *box, int w, double gx, double gy, double gz, double &nx,
                                           double &ny, double &nz, double &d)
{
    const int ax = w >> 1;
    const double g = ax == 0 ? gx : (ax == 1 ? gy : gz);
    nx = ax == 0 ? ((w & 1) ? 1.0 : -1.0) : 0.0;
    ny = ax == 1 ? ((w & 1) ? 1.0 : -1.0) : 0.0;
    nz = ax == 2 ? ((w & 1) ? 1.0 : -1.0) : 0.0;
    d = (w & 1) ? box[2 * ax + 1] - g : -(box[2 * ax] - g);
}

// Where the plane positions come from: the sorted generators, the box and
// the site.
struct Frame {
    const double *xs, *ys, *zs;
    const double *box;
    double gx, gy, gz;
};

__device__ __forceinline__ void plane64(const Frame &F, int sid, double &nx, double &ny, double &nz, double &d)
{
    if (sid >= 0) bisector(F.xs, F.ys, F.zs, sid, F.gx, F.gy, F.gz, nx, ny, nz, d);
    else wall_plane(F.box, -1 - sid, F.gx, F.gy, F.gz, nx, ny, nz, d);
}

// Meet of the planes A, B, C (n.x = d, FP32 roundings of FP64 planes) by
// Cramer's rule, x = (d_A (n_B x n_C) + d_B (n_C x n_A) + d_C (n_A x n_B)) / det,
// det = n_A.(n_B x n_C).  With s_P = |n_P|_1, each cross-product component is
// within 4u s s' of the exact one's over the FP64 planes (its own rounding
// and the inputs'), det within 8u S, S = s_A s_B s_C, and each numerator
// within 8u N, N = |d_A| s_B s_C + |d_B| s_C s_A + |d_C| s_A s_B; so while
// |det| >= 64u S every coordinate is within 16u (N + |x|_inf S) / |det| of the
// exact meet (10.2u by the first-order sum, the rest covering the rounding of
// the quotient and of |x|).  err = inf when |det| is below that or S leaves
// FP32's normal range.
__device__ __forceinline__ void meet32(float4 A, float4 B, float4 Cp, float &x, float &y, float &z, float &err)
{
    const float bcx = fmaf(B.y, Cp.z, -B.z * Cp.y), bcy = fmaf(B.z, Cp.x, -B.x * Cp.z),
                bcz = fmaf(B.x, Cp.y, -B.y * Cp.x);
    const float cax = fmaf(Cp.y, A.z, -Cp.z * A.y), cay = fmaf(Cp.z, A.x, -Cp.x * A.z),
                caz = fmaf(Cp.x, A.y, -Cp.y * A.x);
    const float abx = fmaf(A.y, B.z, -A.z * B.y), aby = fmaf(A.z, B.x, -A.x * B.z),
                abz = fmaf(A.x, B.y, -A.y * B.x);
    const float det = fmaf(A.x, bcx, fmaf(A.y, bcy, A.z * bcz));
    const float id = 1.f / det;
    x = fmaf(A.w, bcx, fmaf(B.w, cax, Cp.w * abx)) * id;
    y = fmaf(A.w, bcy, fmaf(B.w, cay, Cp.w * aby)) * id;
    z = fmaf(A.w, bcz, fmaf(B.w, caz, Cp.w * abz)) * id;
    const float sA = fabsf(A.x) + fabsf(A.y) + fabsf(A.z), sB = fabsf(B.x) + fabsf(B.y) + fabsf(B.z),
                sC = fabsf(Cp.x) + fabsf(Cp.y) + fabsf(Cp.z);
    const float S = sA * sB * sC;
    const float N = fabsf(A.w) * sB * sC + fabsf(B.w) * sC * sA + fabsf(Cp.w) * sA * sB;
    const float xm = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
    const float ad = fabsf(det);
    err = (ad >= 64.f * U32 * S && S >= 1e-30f) ? 16.f * U32 * (N + xm * S) / ad : INFINITY;
}

// FP64 meet of three FP64 planes (Cramer's rule, as meet32).
__device__ __forceinline__ void meet64p(const double *A, const double *B, const double *Cp, double &x, double &y,
                                        double &z)
{
    const double bcx = B[1] * Cp[2] - B[2] * Cp[1], bcy = B[2] * Cp[0] - B[0] * Cp[2], bcz = B[0] * Cp[1] - B[1] * Cp[0];
    const double cax = Cp[1] * A[2] - Cp[2] * A[1], cay = Cp[2] * A[0] - Cp[0] * A[2], caz = Cp[0] * A[1] - Cp[1] * A[0];
    const double abx = A[1] * B[2] - A[2] * B[1], aby = A[2] * B[0] - A[0] * B[2], abz = A[0] * B[1] - A[1] * B[0];
    const double id = 1.0 / (A[0] * bcx + A[1] * bcy + A[2] * bcz);
    x = (A[3] * bcx + B[3] * cax + Cp[3] * abx) * id;
    y = (A[3] * bcy + B[3] * cay + Cp[3] * aby) * id;
    z = (A[3] * bcz + B[3] * caz + Cp[3] * abz) * id;
}

// FP64 meet of vertex t's three planes.
template <class C>
__device__ void meet64(const C &c, const Frame &F, int t, double &x, double &y, double &z)
{
    double P[3][4];
#pragma unroll
    for (int e = 0; e < 3; ++e) plane64(F, c.sid[c.tri[c.cur][t][e]], P[e][0], P[e][1], P[e][2], P[e][3]);
    meet64p(P[0], P[1], P[2], x, y, z);
}

// FP32 copy of a vertex from its FP64 meet, and the bound of its rounding.
__device__ __forceinline__ void set_vf(float *vf, float &ev, double x, double y, double z)
{
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    vf[0] = xf;
    vf[1] = yf;
    vf[2] = zf;
    vf[3] = fabsf(xf) + fabsf(yf) + fabsf(zf);
    ev = U32 * fmaxf(fabsf(xf), fmaxf(fabsf(yf), fabsf(zf)));
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// The box as the starting cell: walls 0..5 (x-lo, x-hi, y-lo, y-hi, z-lo,
// z-hi), and corner i (bits x, y, z of i: 0 for lo, 1 for hi) the meet of
// walls sx, 2 + sy, 4 + sz, ordered counter-clockwise seen from outside.  The
// corner across the edge (tri[e], tri[e + 1]) shares those two walls and
// differs in the axis of the third, tri[e + 2]: i with that axis' bit flipped.
// Lane w sets wall w, lane i corner i.
template <class C>
__device__ void wcell_box(C &c, const Frame &F)
{
    const int lane = threadIdx.x & 31;
    if (lane < 6) {
        c.sid[lane] = -1 - lane;
        double nx, ny, nz, d;
        wall_plane(F.box, lane, F.gx, F.gy, F.gz, nx, ny, nz, d);
        c.pf[lane] = make_float4((float)nx, (float)ny, (float)nz, (float)d);
    }
    if (lane < 8) {
        const int i = lane;
        const int sx = i & 1, sy = (i >> 1) & 1, sz = (i >> 2) & 1;
        const uint8_t X = (uint8_t)sx, Y = (uint8_t)(2 + sy), Z = (uint8_t)(4 + sz);
        const bool pos = ((sx ? 1 : -1) * (sy ? 1 : -1) * (sz ? 1 : -1)) > 0;
        const uint8_t t[3] = {X, pos ? Y : Z, pos ? Z : Y};
        for (int e = 0; e < 3; ++e) {
            c.tri[0][i][e] = t[e];
            c.adj[0][i][e] = (uint8_t)(i ^ (1 << (t[(e + 2) % 3] >> 1)));
        }
        set_vf(c.vf[i], c.ev[i], sx ? F.box[1] - F.gx : F.box[0] - F.gx, sy ? F.box[3] - F.gy : F.box[2] - F.gy,
               sz ? F.box[5] - F.gz : F.box[4] - F.gz);
    }
    if (lane == 0) {
        c.np = 6;
        c.nt = 8;
        c.cur = 0;
    }
    __syncwarp();
}

// Drop planes no vertex refers to (one lane; rare).
template <class C>
__device__ int wcompact(C &c)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        int map[WMAXP];
        for (int q = 0; q < c.np; ++q) map[q] = -1;
        const int cur = c.cur;
        for (int t = 0; t < c.nt; ++t)
            for (int e = 0; e < 3; ++e) map[c.tri[cur][t][e]] = 0;
        int n = 0;
        for (int q = 0; q < c.np; ++q) {
            if (map[q] < 0) continue;
            map[q] = n;
            c.sid[n] = c.sid[q];
            c.pf[n] = c.pf[q];
            ++n;
        }
        for (int t = 0; t < c.nt; ++t)
            for (int e = 0; e < 3; ++e) c.tri[cur][t][e] = (uint8_t)map[c.tri[cur][t][e]];
        c.np = n;
    }
    __syncwarp();
    return c.np;
}

// Clip by the plane n.x <= d of generator sid.  Returns 1 changed, 0
// unchanged, < 0 error (all lanes).
template <class C>
__device__ int wclip(C &c, const Frame &F, double nx, double ny, double nz, double d, int sid)
{
    const int lane = threadIdx.x & 31;
    const int cur = c.cur, nxt = cur ^ 1, nt = c.nt;
    // The side of each vertex: f = n.v - d in FP32 from the FP32 vertex and
    // plane.  It differs from the exact f by at most |n|_1 ev (the vertex) +
    // 5u (|n|_1 |v|_1 + |d|) (the plane's rounding and the FP32 sum); beyond
    // the band, twice that, its sign is exact.  Inside the band the vertex's
    // FP64 meet decides, with the warp converged on the few that need it; a
    // vertex within 1e-13 of the plane's scale (above the rounding of the
    // FP64 meet and value) counts as on the plane and is kept, so that a plane
    // through existing vertices, as in degenerate (lattice) site sets, cuts
    // no sliver off.
    const float4 P = make_float4(em::f32_rn(nx), em::f32_rn(ny), em::f32_rn(nz), em::f32_rn(d));
    const float nsum = fabsf(P.x) + fabsf(P.y) + fabsf(P.z);
    bool any = false;
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        bool out = false, unsure = false;
        if (t < nt) {
            const float *vf = c.vf[t];
            const float ff = fmaf(P.x, vf[0], fmaf(P.y, vf[1], fmaf(P.z, vf[2], -P.w)));
            const float band = 2.f * (nsum * c.ev[t] + 5.f * U32 * (nsum * vf[3] + fabsf(P.w)));
            out = ff > band;
            unsure = !out && !(ff < -band);
        }
        if (__any_sync(0xffffffffu, unsure)) {
            if (unsure) {
                double x, y, z;
                meet64(c, F, t, x, y, z);
                out = nx * x + ny * y + nz * z - d > 1e-13 * (double)(nsum * c.vf[t][3] + fabsf(P.w));
            }
        }
        if (t < nt) c.side[t] = out ? 1 : 0;
        any = any || out;
    }
    if (!__any_sync(0xffffffffu, any)) return 0;
    __syncwarp();
    if (c.np >= WMAXP && wcompact(c) >= WMAXP) return -emv::VS_CAPACITY;
    const int q = c.np;
    // new index of every kept vertex (order kept), in side[]; removed ones listed
    int nk = 0, nout = 0;
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        const bool in = t < nt;
        const bool keep = in && !c.side[t];
        const bool out = in && !keep;
        const unsigned mk = __ballot_sync(0xffffffffu, keep), mo = __ballot_sync(0xffffffffu, out);
        if (in) c.side[t] = keep ? (uint8_t)(nk + __popc(mk & lanemask_lt())) : (uint8_t)0xff;
        if (out) c.out_list[nout + __popc(mo & lanemask_lt())] = (uint8_t)t;
        nk += __popc(mk);
        nout += __popc(mo);
    }
    __syncwarp();
    if (nk == 0) return -emv::VS_TOPOLOGY;
    // kept vertices into the other buffer, their neighbours renumbered (those
    // across a cut edge are set below); the FP32 copy and its bound move
    // within their buffer (a vertex never moves up, and each round reads
    // before it writes)
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        const int pos = t < nt ? c.side[t] : 0xff;
        float vfk[4], evk = 0.f;
        if (pos != 0xff) {
            for (int e = 0; e < 3; ++e) {
                c.tri[nxt][pos][e] = c.tri[cur][t][e];
                const int s_ = c.adj[cur][t][e];
                c.adj[nxt][pos][e] = s_ < nt ? c.side[s_] : (uint8_t)0xff;
            }
            for (int e = 0; e < 4; ++e) vfk[e] = c.vf[t][e];
            evk = c.ev[t];
        }
        __syncwarp();
        if (pos != 0xff) {
            for (int e = 0; e < 4; ++e) c.vf[pos][e] = vfk[e];
            c.ev[pos] = evk;
        }
        __syncwarp();
    }
    // one task per (removed vertex, edge): a new vertex where the neighbour
    // across the edge is kept, with the two linked to each other; the new
    // vertex is the meet of the edge's planes a, b and the new plane, in FP32
    // with its bound, or from the FP64 meet where the FP32 one is too
    // uncertain to be of use (planes near a common line)
    int nn = nk;
    bool bad = false;
    for (int base = 0; base < 3 * nout; base += 32) {
        const int k = base + lane;
        bool newv = false;
        uint8_t a = 0, b = 0;
        int upos = 0, ue = 0;
        float px = 0.f, py = 0.f, pz = 0.f, perr = INFINITY;
        if (k < 3 * nout) {
            const int t = c.out_list[k / 3], e = k % 3;
            a = c.tri[cur][t][e];
            b = c.tri[cur][t][(e + 1) % 3];
            const int u = c.adj[cur][t][e];
            if (u >= nt) {
                bad = true;   // inconsistent neighbours: reported, never followed
            } else if (c.side[u] != 0xff) {
                newv = true;
                upos = c.side[u];
                // the edge of u that is (b, a)
                const uint8_t *tu = c.tri[cur][u];
                ue = (tu[0] == b && tu[1] == a) ? 0 : ((tu[1] == b && tu[2] == a) ? 1 : 2);
                bad = bad || !(tu[ue] == b && tu[(ue + 1) % 3] == a);
                meet32(c.pf[a], c.pf[b], P, px, py, pz, perr);
            }
        }
        const bool poor = newv && !(perr <= 1e-4f * (fabsf(px) + fabsf(py) + fabsf(pz)));
        if (__any_sync(0xffffffffu, poor)) {
            if (poor) {
                double PL[3][4];
                plane64(F, c.sid[a], PL[0][0], PL[0][1], PL[0][2], PL[0][3]);
                plane64(F, c.sid[b], PL[1][0], PL[1][1], PL[1][2], PL[1][3]);
                PL[2][0] = nx;
                PL[2][1] = ny;
                PL[2][2] = nz;
                PL[2][3] = d;
                double x, y, z;
                meet64p(PL[0], PL[1], PL[2], x, y, z);
                px = (float)x;
                py = (float)y;
                pz = (float)z;
                // the FP64 meet's own error is far below the FP32 rounding
                // unless the planes nearly share a line, where the bound is
                // left infinite and every side test takes the FP64 meet
                perr = isfinite(x + y + z) ? 2.f * U32 * fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))) : INFINITY;
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, newv);
        if (newv) {
            int pos = nn + __popc(m & lanemask_lt());
            if (pos < C::MAXV) {
                c.tri[nxt][pos][0] = a;
                c.tri[nxt][pos][1] = b;
                c.tri[nxt][pos][2] = (uint8_t)q;
                c.adj[nxt][pos][0] = (uint8_t)upos;
                c.adj[nxt][upos][ue] = (uint8_t)pos;
                c.vf[pos][0] = px;
                c.vf[pos][1] = py;
                c.vf[pos][2] = pz;
                c.vf[pos][3] = fabsf(px) + fabsf(py) + fabsf(pz);
                c.ev[pos] = perr;
            }
        }
        nn += __popc(m);
    }
    __syncwarp();
    // the new vertices around the new face q: (a, b, q) meets the one whose
    // a is this b across (b, q), and the one whose b is this a across (q, a)
    if (nn <= C::MAXV)
        for (int n = nk + lane; n < nn; n += 32) {
            const uint8_t an = c.tri[nxt][n][0], bn = c.tri[nxt][n][1];
            int m1 = -1, m2 = -1;
            for (int o = nk; o < nn; ++o) {
                if (c.tri[nxt][o][0] == bn) m1 = o;
                if (c.tri[nxt][o][1] == an) m2 = o;
            }
            bad = bad || m1 < 0 || m2 < 0;
            c.adj[nxt][n][1] = (uint8_t)(m1 < 0 ? 0 : m1);
            c.adj[nxt][n][2] = (uint8_t)(m2 < 0 ? 0 : m2);
        }
    if (__any_sync(0xffffffffu, bad)) return -emv::VS_TOPOLOGY;
    if (nn > C::MAXV) return -emv::VS_CAPACITY;
    if (lane == 0) {
        c.sid[q] = sid;
        c.pf[q] = P;
        c.np = q + 1;
        c.nt = nn;
        c.cur = nxt;
    }
    __syncwarp();
    return 1;
}

// An upper bound of the squared distance from the site to the cell's
// farthest vertex: per vertex |vf|_2 + sqrt(3) ev (the exact vertex lies
// within ev per coordinate), squared, widened by 1e-5 for the FP32 rounding
// of the norm.  A vertex with no finite bound takes its FP64 meet.
template <class C>
__device__ double wrmax2(const C &c, const Frame &F)
{
    const int lane = threadIdx.x & 31;
    float r2 = 0.f;
    bool fp64 = false;
    for (int t = lane; t < c.nt; t += 32) {
        const float *v = c.vf[t];
        const float r = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + 1.7320509f * c.ev[t];
        if (isfinite(r)) r2 = fmaxf(r2, r * r);
        else fp64 = true;
    }
    double q2 = (double)r2 * (1.0 + 1e-5);
    if (__any_sync(0xffffffffu, fp64)) {
        for (int t = lane; t < c.nt; t += 32) {
            if (isfinite(c.ev[t])) continue;
            double x, y, z;
            meet64(c, F, t, x, y, z);
            q2 = fmax(q2, (x * x + y * y + z * z) * (1.0 + 1e-12));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q2 = fmax(q2, __shfl_xor_sync(0xffffffffu, q2, o));
    return q2;
}

// Gather every generator k != s with lo2 <= d^2 < hi2 into the candidate
// list (sorted by (d^2, k) afterwards).  Returns the count, or -1 if it
// exceeds WCAND.
template <class C>
__device__ int gather(C &c, const em::ChunkTree &T, const double *__restrict__ xs, const double *__restrict__ ys,
                      const double *__restrict__ zs, int64_t s, double gx, double gy, double gz, double lo2,
                      double hi2, float margin, int &status)
{
    int n = 0;
    float R = (float)sqrt(hi2) + margin;
    // The window test runs in FP32 on the rounded positions and keeps every
    // point whose FP32 distance lies within the window widened by a band above
    // the rounding of the coordinates: a superset of the exact window, which
    // is all the callers need (every generator in the window gets clipped).
    // The sort key is the FP32 squared distance; only near-coincident points
    // are checked in FP64.
    const float gxf = (float)gx, gyf = (float)gy, gzf = (float)gz;
    const float gabs = fabsf(gxf) + fabsf(gyf) + fabsf(gzf);
    float rhi = sqrtf((float)hi2) * (1.f + 1e-5f) + 1e-5f * gabs;
    const float rlo = lo2 > 0.0 ? sqrtf((float)lo2) * (1.f - 1e-5f) - 1e-5f * gabs : -1.f;
    const float rtiny = 1e-5f * (gabs + rhi);
    em::warp_traverse(T, gxf, gyf, gzf, R * R, INT64_MAX, [&](int64_t k, bool valid) {
        bool hit = false;
        float d2f = 0.f;
        if (valid && k != s) {
            const float4 pk = T.pts[k];
            const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
            d2f = ex * ex + ey * ey + ez * ez;
            const float rf = sqrtf(d2f);
            hit = rf <= rhi && rf >= rlo;
            if (rf < rtiny) {   // possibly the same point
                const double dx = xs[k] - gx, dy = ys[k] - gy, dz = zs[k] - gz;
                if (dx * dx + dy * dy + dz * dz == 0.0) status |= emv::VS_COINCIDENT;
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            int pos = n + __popc(m & lanemask_lt());
            if (pos < WCAND) {
                c.u.k.cd2[pos] = d2f;
                c.u.k.cid[pos] = (int)k;
            }
        }
        n += __popc(m);
    });
    status = __reduce_or_sync(0xffffffffu, status);
    __syncwarp();
    return n > WCAND ? -1 : n;
}

// Bitonic sort of the first n candidates by (d^2 in FP32, index), padded with
// (inf, max) up to the next power of two (at most WCAND).
template <class C>
__device__ void sort_cand(C &c, int n)
{
    const int lane = threadIdx.x & 31;
    float *cd2 = c.u.k.cd2;
    int *cid = c.u.k.cid;
    int len = 2;
    while (len < n) len <<= 1;
    for (int i = n + lane; i < len; i += 32) {
        cd2[i] = INFINITY;
        cid[i] = 0x7fffffff;
    }
    __syncwarp();
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < len / 2; i += 32) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                const float a = cd2[lo], b = cd2[hi];
                int ia = cid[lo], ib = cid[hi];
                bool gt = (a > b) || (a == b && ia > ib);
                if (gt == up) {
                    cd2[lo] = b;
                    cd2[hi] = a;
                    cid[lo] = ib;
                    cid[hi] = ia;
                }
            }
            __syncwarp();
        }
    }
}

// Generators k != s whose bisector may cut the current cell (some vertex v
// may have f = r_k.v - |r_k|^2/2 > 0, r_k = g_k - g), excluding those nearer
// than sqrt(skip2) (already applied), up to the window's end hi2.  Boxes are
// skipped when every vertex is at least as close to the site as to the box.
// When the list would overflow, the walk keeps the candidates whose FP32 key
// is below the median key k and goes on with hi2 narrowed to the float p just
// below k: every generator with d2 < p has a key <= p, so none is lost, and a
// kept one a little beyond p is only applied early (the half-spaces commute;
// once applied it no longer cuts).  Returns the count with hi2 the window
// actually covered, or -1 if the window cannot narrow (ties at the median).
// A listed generator that does not cut costs a clip that changes nothing.
template <class C>
__device__ int gather_cutting(C &c, const em::ChunkTree &T, const double *__restrict__ xs,
                              const double *__restrict__ ys, const double *__restrict__ zs, int64_t s, double gx,
                              double gy, double gz, double skip2, double &hi2)
{
    const int lane = threadIdx.x & 31;
    const int nt = c.nt;
    float *cd2 = c.u.k.cd2;
    int *cid = c.u.k.cid;
    // The pruning tests run in FP32 with margins above the rounding of the
    // coordinates (S below is a bound on their magnitudes) and the vertices'
    // bounds ev: a box or point is dropped only where the exact test would
    // drop it too.
    const float gxf = (float)gx, gyf = (float)gy, gzf = (float)gz;
    const float gabs = fabsf(gxf) + fabsf(gyf) + fabsf(gzf);
    float rhi = sqrtf((float)hi2) * (1.f + 1e-5f) + 1e-5f * gabs;
    const float rlo = skip2 > 0.0 ? sqrtf((float)skip2) * (1.f - 1e-5f) - 1e-5f * gabs : -1.f;
    auto box_can_cut = [&](const float4 lo, const float4 hi) -> bool {
        const float babs = fabsf(lo.x) + fabsf(lo.y) + fabsf(lo.z) + fabsf(hi.x) + fabsf(hi.y) + fabsf(hi.z);
        const float lx = lo.x - gxf, ly = lo.y - gyf, lz = lo.z - gzf;
        const float hx = hi.x - gxf, hy = hi.y - gyf, hz = hi.z - gzf;
        {   // the whole box beyond the window's outer radius
            float dx = fmaxf(fmaxf(lx, -hx), 0.f), dy = fmaxf(fmaxf(ly, -hy), 0.f), dz = fmaxf(fmaxf(lz, -hz), 0.f);
            if (sqrtf(dx * dx + dy * dy + dz * dz) > rhi + 1e-5f * babs) return false;
        }
        // some vertex nearer to the box than to the site (the exact vertex
        // lies within 1.8 ev of vf, which moves both squared distances by at
        // most 3.6 ev (|d| + |g|) + 6.5 ev^2)
        for (int t = 0; t < nt; ++t) {
            const float vx = c.vf[t][0], vy = c.vf[t][1], vz = c.vf[t][2];
            float dx = fmaxf(fmaxf(lx - vx, vx - hx), 0.f);
            float dy = fmaxf(fmaxf(ly - vy, vy - hy), 0.f);
            float dz = fmaxf(fmaxf(lz - vz, vz - hz), 0.f);
            const float db = dx * dx + dy * dy + dz * dz;
            const float dg = vx * vx + vy * vy + vz * vz;
            const float S = gabs + babs + c.vf[t][3];
            const float e = c.ev[t];
            if (!(db >= dg + 1e-5f * S * S + 7.2f * e * S + 6.5f * e * e)) return true;
        }
        return false;
    };
    uint32_t mask[em::kMaxLevels + 1];
    int64_t base[em::kMaxLevels + 1];
    const int top = T.nlev;
    int n = 0;
    {
        bool hit = lane < T.count[top] && box_can_cut(T.lo[top][lane], T.hi[top][lane]);
        mask[top] = __ballot_sync(0xffffffffu, hit);
        base[top] = 0;
    }
    int lvl = top;
    while (true) {
        if (mask[lvl] == 0) {
            if (lvl == top) break;
            ++lvl;
            continue;
        }
        int cidx = __ffs(mask[lvl]) - 1;
        mask[lvl] &= mask[lvl] - 1;
        int64_t node = base[lvl] * 32 + cidx;
        if (lvl == 1) {
            int64_t k = node * 32 + lane;
            double d2 = 0.0;
            bool hit = k < T.count[0] && k != s;
            if (hit) {
                // FP32: inside the window and some vertex possibly beyond the
                // bisector (margin above the rounding of the coordinates and
                // the vertex bounds)
                const float4 pk = T.pts[k];
                const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
                const float rf = sqrtf(ex * ex + ey * ey + ez * ez);
                hit = rf <= rhi && rf >= rlo;
                if (hit) {
                    const float df = 0.5f * rf * rf, rabs = fabsf(ex) + fabsf(ey) + fabsf(ez);
                    bool maybe = false;
                    for (int t = 0; t < nt && !maybe; ++t) {
                        const float *vf = c.vf[t];
                        const float ff = ex * vf[0] + ey * vf[1] + ez * vf[2] - df;
                        maybe = !(ff <= -(1e-5f * (gabs + rabs + vf[3]) * (vf[3] + rabs) + rabs * c.ev[t]));
                    }
                    hit = maybe;
                }
            }
            if (hit) {
                const double rx = xs[k] - gx, ry = ys[k] - gy, rz = zs[k] - gz;
                d2 = rx * rx + ry * ry + rz * rz;
                hit = d2 >= skip2 && d2 < hi2;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (n + __popc(m) > WCAND) {
                // narrow the window to the nearer half of the list (n <= WCAND here)
                sort_cand(c, n);
                const float kth = cd2[n / 2];
                const float pf = nextafterf(kth, 0.f);
                const double p2 = (double)pf;
                int keep = 0;   // the sorted prefix below the median key
                for (int b = 0; b < n; b += 32) {
                    const int i = b + lane;
                    keep += __popc(__ballot_sync(0xffffffffu, i < n && cd2[i] < kth));
                }
                if (!(kth > 0.f) || !(p2 > skip2) || !(p2 < hi2) || keep == 0) return -1;
                n = keep;
                hi2 = p2;
                rhi = sqrtf(pf) * (1.f + 1e-5f) + 1e-5f * gabs;
                hit = hit && d2 < hi2;
                m = __ballot_sync(0xffffffffu, hit);
            }
            if (hit) {
                int pos = n + __popc(m & lanemask_lt());
                if (pos < WCAND) {
                    cd2[pos] = em::f32_rn(d2);
                    cid[pos] = (int)k;
                }
            }
            n += __popc(m);
        } else {
            int64_t child = node * 32 + lane;
            bool hit = child < T.count[lvl - 1] && box_can_cut(T.lo[lvl - 1][child], T.hi[lvl - 1][child]);
            mask[lvl - 1] = __ballot_sync(0xffffffffu, hit);
            base[lvl - 1] = node;
            --lvl;
        }
    }
    __syncwarp();
    return n > WCAND ? -1 : n;
}

// Clip by the first nc (sorted) candidates.  A candidate first meets an FP32
// side test on the rounded positions (the same margin as in gather_cutting,
// above the rounding of the coordinates and the vertex bounds): one that
// every vertex clears cuts nothing and costs no FP64 work.
template <class C>
__device__ int clip_sorted(C &c, const em::ChunkTree &T, const Frame &F, int64_t n, int nc)
{
    const int lane = threadIdx.x & 31;
    const float gxf = (float)F.gx, gyf = (float)F.gy, gzf = (float)F.gz;
    const float gabs = fabsf(gxf) + fabsf(gyf) + fabsf(gzf);
    for (int i = 0; i < nc; ++i) {
        int k = c.u.k.cid[i];
        if (k < 0 || k >= n) return emv::VS_BOUNDS;
        {
            const float4 pk = T.pts[k];
            const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
            const float df = 0.5f * (ex * ex + ey * ey + ez * ez), rabs = fabsf(ex) + fabsf(ey) + fabsf(ez);
            bool maybe = false;
            for (int t = lane; t < c.nt; t += 32) {
                const float *vf = c.vf[t];
                const float ff = ex * vf[0] + ey * vf[1] + ez * vf[2] - df;
                maybe = maybe || !(ff <= -(1e-5f * (gabs + rabs + vf[3]) * (vf[3] + rabs) + rabs * c.ev[t]));
            }
            if (!__any_sync(0xffffffffu, maybe)) continue;
        }
        double nx, ny, nz, d;
        bisector(F.xs, F.ys, F.zs, k, F.gx, F.gy, F.gz, nx, ny, nz, d);
        int r = wclip(c, F, nx, ny, nz, d, k);
        if (r < 0) return -r;
    }
    return 0;
}

// Build the cell of sorted generator s.
// Stage 1: every generator within a radius R chosen from the local spacing
// (8th nearest of the site's 32-generator chunk), nearest first.  Stage 2
// (exact completion): generators whose bisector still cuts the cell, in
// distance windows [lo, hi) that shrink until they fit the candidate list,
// nearest first, until the window passes 2 R_max.  Every generator nearer
// than lo has been applied at each step.
template <class C>
__device__ int wbuild_cell(C &c, const em::ChunkTree &T, const Frame &F, int64_t s, int K, float margin)
{
    const int lane = threadIdx.x & 31;
    int status = 0;
    const double *xs = F.xs, *ys = F.ys, *zs = F.zs, *box = F.box;
    const double gx = F.gx, gy = F.gy, gz = F.gz;
    if (!(gx > box[0] && gx < box[1] && gy > box[2] && gy < box[3] && gz > box[4] && gz < box[5]))
        return emv::VS_OUTSIDE;
    wcell_box(c, F);
    const int64_t n = T.count[0];
    // local spacing: the 8th smallest distance to the other members of the
    // chunk (a starting radius only, so FP32 on the rounded positions)
    double R2;
    {
        int64_t k = (s / 32) * 32 + lane;
        float d2 = INFINITY;
        if (k < n && k != s) {
            const float4 pk = T.pts[k], ps = T.pts[s];
            const float dx = pk.x - ps.x, dy = pk.y - ps.y, dz = pk.z - ps.z;
            d2 = dx * dx + dy * dy + dz * dz;
        }
        float kthf = INFINITY;
        for (int r = 0; r < 8; ++r) {
            float m = d2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
            kthf = m;
            unsigned who = __ballot_sync(0xffffffffu, d2 == m);
            if (lane == __ffs(who) - 1) d2 = INFINITY;
        }
        double kth = kthf;
        if (!(kth > 0.0 && kth < INFINITY)) {
            const double bx = box[1] - box[0], by = box[3] - box[2], bz = box[5] - box[4];
            kth = 0.01 * (bx * bx + by * by + bz * bz);
        }
        // the chunk's own 8th nearest overestimates the local spacing (its
        // members lie mostly to one side), hence the factor 1/4
        R2 = 0.25 * kth * cbrt(1.5 * K / 8.0) * cbrt(1.5 * K / 8.0);
    }
    // round -1 is stage 1, rounds 0.. stage 2; both clip through the one call
    // site below (one inlined copy of the clip keeps the code small)
    double skip2 = -1.0;
    for (int round = -1; round < 256; ++round) {
        int m = -1;
        double hi2 = 0.0;
        if (round < 0) {
            // stage 1: shrink or grow R until the candidates fit and number at least K
            double lo_ok = 0.0, hi_bad = INFINITY;
            for (int it = 0; it < 48; ++it) {
                m = gather(c, T, xs, ys, zs, s, gx, gy, gz, -1.0, R2, margin, status);
                if (status & emv::VS_COINCIDENT) return status;
                if (m < 0) {
                    hi_bad = R2;
                    R2 = lo_ok > 0.0 ? sqrt(lo_ok * hi_bad) : 0.3 * R2;
                    continue;
                }
                if (m < K && m < n - 1 && hi_bad == INFINITY && it < 40) {
                    lo_ok = R2;
                    R2 *= 2.0;
                    continue;
                }
                break;
            }
            hi2 = m >= 0 ? R2 : -1.0;   // every generator nearer than R gets applied
        } else {
            // stage 2: windows [skip2, hi2) of generators that still cut, nearest first
            const double lim2 = 4.0 * wrmax2(c, F) * (1.0 + 1e-12);   // no generator beyond 2 R_max can cut
            if (skip2 >= lim2) return status;
            hi2 = lim2;
            for (int h = 0; h < 64; ++h) {
                m = gather_cutting(c, T, xs, ys, zs, s, gx, gy, gz, skip2, hi2);
                if (m >= 0) break;
                hi2 = (skip2 > 0.0 ? skip2 : 0.0) + 0.5 * (hi2 - (skip2 > 0.0 ? skip2 : 0.0));
            }
            if (m < 0) return status | emv::VS_CANDIDATES;
        }
        if (m > 0) {
            sort_cand(c, m);
            int st = clip_sorted(c, T, F, n, m);
            if (st) return status | st;
        }
        skip2 = hi2;
    }
    return status | emv::VS_ROUNDS;
}

// The FP64 vertices of the finished cell (each the FP64 meet of its three
// planes), into c.u.vx; the candidate list is no longer needed.
template <class C>
__device__ void finish_vertices(C &c, const Frame &F)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int t = lane; t < c.nt; t += 32) {
        double x, y, z;
        meet64(c, F, t, x, y, z);
        c.u.vx[t][0] = x;
        c.u.vx[t][1] = y;
        c.u.vx[t][2] = z;
    }
    __syncwarp();
}

// Face loop of plane q (one lane): vertex indices counter-clockwise seen from
// outside; returns the length (0 if the plane holds no vertex, -1 on error).
// From a vertex t holding q at position r, the next vertex around q is the
// one across t's edge (tri[t][r + 2], q).
template <class C>
__device__ int wface_loop(const C &c, int q, uint8_t *loop, int maxn)
{
    const int cur = c.cur, nt = c.nt;
    int t0 = -1;
    for (int t = 0; t < nt && t0 < 0; ++t)
        if (c.tri[cur][t][0] == q || c.tri[cur][t][1] == q || c.tri[cur][t][2] == q) t0 = t;
    if (t0 < 0) return 0;
    int n = 0, t = t0;
    do {
        if (n >= maxn) return -1;
        loop[n++] = (uint8_t)t;
        const uint8_t *tr = c.tri[cur][t];
        const int r = tr[0] == q ? 0 : (tr[1] == q ? 1 : 2);
        const int nx = c.adj[cur][t][(r + 2) % 3];
        if (nx >= nt) return -1;
        t = nx;
    } while (t != t0);
    return n;
}

}  // namespace emw
