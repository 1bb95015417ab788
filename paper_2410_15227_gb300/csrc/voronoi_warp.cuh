// Warp-cooperative Voronoi cell construction (one warp per cell, the cell
// in shared memory, in dual form: planes, and vertices as triangles of
// planes).  A clip removes the vertices beyond the bisector, keeps the
// others in order and appends the new vertices in the order (removed
// vertex, edge), so the vertex order is fixed by the clips alone.  Candidates: every generator within a radius R of the site (found by
// a warp walk of the generators' box hierarchy), sorted by distance; the
// cell is exact once 2 R_max < R, otherwise the shell up to 2 R_max is
// clipped in as well.
#pragma once

#include <cstdint>

#include "tree_util.cuh"
#include "voronoi_cell.cuh"

namespace emw {

constexpr int WMAXP = emv::MAXP;
constexpr int WCAND = 256;   // candidate list (power of two for the bitonic sort)

// A cell under construction with room for NV vertices.  The planes are not
// stored: plane q is the bisector of the site and generator sid[q] (its
// sorted index), or box wall -1 - sid[q], formed again from the generator
// positions wherever it is needed (bisector(), wall_plane()).
template <int NV>
struct WCell {
    static constexpr int MAXV = NV;
    static_assert(NV <= 255, "vertex indices are bytes, 0xff marks a removed vertex");
    double v[2][NV][3];
    float vf[NV][4];         // the current vertices rounded to FP32, w = |x| + |y| + |z|
    float cd2[WCAND];        // sort keys of the candidates: squared distances rounded to FP32
    int cid[WCAND];
    int sid[WMAXP];
    // clip in progress: 1 if the vertex lies beyond the plane, then its new
    // index (0xff if removed)
    uint8_t side[NV];
    uint8_t out_list[NV];    // clip in progress: the removed vertices
    uint8_t tri[2][NV][4];
    // adj[t][e]: the vertex across edge e of vertex t, i.e. the one whose
    // triangle holds the reversed edge (tri[t][e + 1], tri[t][e])
    uint8_t adj[2][NV][4];
    int np, nt, cur;
};

// Bisector plane n.x <= d of the site g (at the origin of the cell's frame)
// and generator k: n = g_k - g, d = |n|^2 / 2, every rounding explicit so that
// the builder and the face writer form the same bits.
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

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

__device__ __forceinline__ bool has_edge(const uint8_t *t, uint8_t a, uint8_t b)
{
    return (t[0] == a && t[1] == b) || (t[1] == a && t[2] == b) || (t[2] == a && t[0] == b);
}

// The FP32 copy of one vertex.
__device__ __forceinline__ void set_vf(float *vf, double x, double y, double z)
{
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    vf[0] = xf;
    vf[1] = yf;
    vf[2] = zf;
    vf[3] = fabsf(xf) + fabsf(yf) + fabsf(zf);
}

template <class C>
__device__ void wcell_box(C &c, const double *box, double gx, double gy, double gz)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        const double lo[3] = {box[0] - gx, box[2] - gy, box[4] - gz};
        const double hi[3] = {box[1] - gx, box[3] - gy, box[5] - gz};
        c.np = 6;
        for (int w = 0; w < 6; ++w) c.sid[w] = -1 - w;
        c.nt = 8;
        c.cur = 0;
        for (int i = 0; i < 8; ++i) {
            int sx = i & 1, sy = (i >> 1) & 1, sz = (i >> 2) & 1;
            uint8_t X = (uint8_t)sx, Y = (uint8_t)(2 + sy), Z = (uint8_t)(4 + sz);
            bool pos = ((sx ? 1 : -1) * (sy ? 1 : -1) * (sz ? 1 : -1)) > 0;
            c.tri[0][i][0] = X;
            c.tri[0][i][1] = pos ? Y : Z;
            c.tri[0][i][2] = pos ? Z : Y;
            c.v[0][i][0] = sx ? hi[0] : lo[0];
            c.v[0][i][1] = sy ? hi[1] : lo[1];
            c.v[0][i][2] = sz ? hi[2] : lo[2];
            set_vf(c.vf[i], c.v[0][i][0], c.v[0][i][1], c.v[0][i][2]);
        }
        for (int i = 0; i < 8; ++i)
            for (int e = 0; e < 3; ++e) {
                const uint8_t a = c.tri[0][i][e], b = c.tri[0][i][(e + 1) % 3];
                for (int s = 0; s < 8; ++s)
                    if (has_edge(c.tri[0][s], b, a)) c.adj[0][i][e] = (uint8_t)s;
            }
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
__device__ int wclip(C &c, double nx, double ny, double nz, double d, int sid)
{
    const int lane = threadIdx.x & 31;
    const int cur = c.cur, nxt = cur ^ 1, nt = c.nt;
    // the side of each vertex: from its FP32 value where that clears the band
    // (far above the FP32 rounding of n, v, d and the products; then the FP64
    // value has the same sign), else from the FP64 value, which the warp
    // evaluates only when some vertex lies in the band.  A vertex within
    // 1e-13 of the plane's scale (above the rounding of the FP64 value and of
    // the vertex) counts as on it and is kept, so that a plane through
    // existing vertices, as in degenerate (lattice) site sets, cuts no sliver
    // off; the new vertex on an edge from such a vertex is the vertex itself.
    const float nxf = (float)nx, nyf = (float)ny, nzf = (float)nz, df = (float)d;
    const float nmax = fmaxf(fmaxf(fabsf(nxf), fabsf(nyf)), fabsf(nzf));
    auto fval = [&](int t) { return nx * c.v[cur][t][0] + ny * c.v[cur][t][1] + nz * c.v[cur][t][2] - d; };
    bool any = false;
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        bool out = false, unsure = false;
        if (t < nt) {
            const float *vf = c.vf[t];
            const float ff = nxf * vf[0] + nyf * vf[1] + nzf * vf[2] - df;
            const float band = 1e-5f * (nmax * vf[3] + fabsf(df));
            out = ff > band;
            unsure = !out && !(ff < -band);
        }
        if (__any_sync(0xffffffffu, unsure)) {
            if (unsure) out = fval(t) > 1e-13 * (double)(nmax * c.vf[t][3] + fabsf(df));
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
    // across a cut edge are set below); the FP32 copy moves within its buffer
    // (a vertex never moves up, and each round reads before it writes)
    for (int base = 0; base < nt; base += 32) {
        const int t = base + lane;
        const int pos = t < nt ? c.side[t] : 0xff;
        float vfk[4];
        if (pos != 0xff) {
            for (int e = 0; e < 3; ++e) {
                c.tri[nxt][pos][e] = c.tri[cur][t][e];
                const int s_ = c.adj[cur][t][e];
                c.adj[nxt][pos][e] = s_ < nt ? c.side[s_] : (uint8_t)0xff;
                c.v[nxt][pos][e] = c.v[cur][t][e];
            }
            for (int e = 0; e < 4; ++e) vfk[e] = c.vf[t][e];
        }
        __syncwarp();
        if (pos != 0xff)
            for (int e = 0; e < 4; ++e) c.vf[pos][e] = vfk[e];
        __syncwarp();
    }
    // one task per (removed vertex, edge): a new vertex where the neighbour
    // across the edge is kept, with the two linked to each other
    int nn = nk;
    bool bad = false;
    for (int base = 0; base < 3 * nout; base += 32) {
        const int k = base + lane;
        bool newv = false;
        uint8_t a = 0, b = 0;
        int upos = 0, ue = 0;
        double px = 0, py = 0, pz = 0;
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
                // the edge's end values in FP64: ft > 0 (beyond the band or the
                // tolerance), fu taken as 0 where the kept vertex lies within the
                // tolerance on the far side
                const double fu = fmin(fval(u), 0.0), ft = fval(t);
                double s = fu / (fu - ft);
                px = c.v[cur][u][0] + s * (c.v[cur][t][0] - c.v[cur][u][0]);
                py = c.v[cur][u][1] + s * (c.v[cur][t][1] - c.v[cur][u][1]);
                pz = c.v[cur][u][2] + s * (c.v[cur][t][2] - c.v[cur][u][2]);
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
                c.v[nxt][pos][0] = px;
                c.v[nxt][pos][1] = py;
                c.v[nxt][pos][2] = pz;
                set_vf(c.vf[pos], px, py, pz);
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
        c.np = q + 1;
        c.nt = nn;
        c.cur = nxt;
    }
    __syncwarp();
    return 1;
}

// An upper bound of the squared distance from the site to the cell's
// farthest vertex: the largest squared norm of the FP32 vertex copies,
// widened by 1e-5.  Each copy is within 2^-24 of its FP64 vertex per
// coordinate and the FP32 sum of squares within 3 ulp, so the norm is
// within 3e-7 of the exact one and the widened value lies above it.  A cell
// whose squared norms fall below FP32's normal range takes the FP64 sum.
template <class C>
__device__ double wrmax2(const C &c)
{
    const int lane = threadIdx.x & 31;
    float r2 = 0.f;
    for (int t = lane; t < c.nt; t += 32) {
        const float *v = c.vf[t];
        r2 = fmaxf(r2, v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if (r2 >= 1e-30f) return (double)r2 * (1.0 + 1e-5);
    double q2 = 0.0;
    for (int t = lane; t < c.nt; t += 32) {
        const double *v = c.v[c.cur][t];
        q2 = fmax(q2, v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q2 = fmax(q2, __shfl_xor_sync(0xffffffffu, q2, o));
    return q2 * (1.0 + 1e-12);
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
                c.cd2[pos] = d2f;
                c.cid[pos] = (int)k;
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
    int len = 2;
    while (len < n) len <<= 1;
    for (int i = n + lane; i < len; i += 32) {
        c.cd2[i] = INFINITY;
        c.cid[i] = 0x7fffffff;
    }
    __syncwarp();
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < len / 2; i += 32) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                const float a = c.cd2[lo], b = c.cd2[hi];
                int ia = c.cid[lo], ib = c.cid[hi];
                bool gt = (a > b) || (a == b && ia > ib);
                if (gt == up) {
                    c.cd2[lo] = b;
                    c.cd2[hi] = a;
                    c.cid[lo] = ib;
                    c.cid[hi] = ia;
                }
            }
            __syncwarp();
        }
    }
}

// Generators k != s whose bisector cuts the current cell (some vertex v has
// f = r_k.v - |r_k|^2/2 > 0, r_k = g_k - g), excluding those nearer than
// sqrt(skip2) (already applied), up to the window's end hi2.  Boxes are
// skipped when every vertex is at least as close to the site as to the box.
// When the list would overflow, the walk keeps the candidates whose FP32 key
// is below the median key k and goes on with hi2 narrowed to the float p just
// below k: every generator with d2 < p has a key <= p, so none is lost, and a
// kept one a little beyond p is only applied early (the half-spaces commute;
// once applied it no longer cuts).  Returns the count with hi2 the window
// actually covered, or -1 if the window cannot narrow (ties at the median).
template <class C>
__device__ int gather_cutting(C &c, const em::ChunkTree &T, const double *__restrict__ xs,
                              const double *__restrict__ ys, const double *__restrict__ zs, int64_t s, double gx,
                              double gy, double gz, double skip2, double &hi2)
{
    const int lane = threadIdx.x & 31;
    const int cur = c.cur, nt = c.nt;
    // The pruning tests run in FP32 with margins above the rounding of the
    // coordinates (S below is a bound on their magnitudes): a box or point is
    // dropped only where the exact test would drop it too.
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
        // some vertex nearer to the box than to the site
        for (int t = 0; t < nt; ++t) {
            const float vx = c.vf[t][0], vy = c.vf[t][1], vz = c.vf[t][2];
            float dx = fmaxf(fmaxf(lx - vx, vx - hx), 0.f);
            float dy = fmaxf(fmaxf(ly - vy, vy - hy), 0.f);
            float dz = fmaxf(fmaxf(lz - vz, vz - hz), 0.f);
            const float db = dx * dx + dy * dy + dz * dz;
            const float dg = vx * vx + vy * vy + vz * vz;
            const float S = gabs + babs + c.vf[t][3];
            if (db < dg + 1e-5f * S * S) return true;
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
            bool hit = false;
            double d2 = 0.0;
            bool cand = k < T.count[0] && k != s;
            if (cand) {
                // FP32: inside the window and some vertex possibly beyond the bisector
                const float4 pk = T.pts[k];
                const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
                const float rf = sqrtf(ex * ex + ey * ey + ez * ez);
                cand = rf <= rhi && rf >= rlo;
                if (cand) {
                    const float df = 0.5f * rf * rf, rabs = fabsf(ex) + fabsf(ey) + fabsf(ez);
                    bool maybe = false;
                    for (int t = 0; t < nt && !maybe; ++t) {
                        const float *vf = c.vf[t];
                        const float ff = ex * vf[0] + ey * vf[1] + ez * vf[2] - df;
                        maybe = ff > -1e-5f * (gabs + rabs + vf[3]) * (vf[3] + rabs);
                    }
                    cand = maybe;
                }
            }
            double rx = 0.0, ry = 0.0, rz = 0.0;
            if (cand) {
                rx = xs[k] - gx;
                ry = ys[k] - gy;
                rz = zs[k] - gz;
                d2 = rx * rx + ry * ry + rz * rz;
                cand = d2 >= skip2 && d2 < hi2;
            }
            // FP64: a vertex beyond the bisector by more than rounding (vertices on
            // an already applied bisector sit at |f| ~ 1e-16 d and must not
            // re-qualify).  One candidate at a time, the lanes over the vertices.
            for (unsigned cm = __ballot_sync(0xffffffffu, cand); cm; cm &= cm - 1) {
                const int src = __ffs(cm) - 1;
                const double qx = __shfl_sync(0xffffffffu, rx, src), qy = __shfl_sync(0xffffffffu, ry, src),
                             qz = __shfl_sync(0xffffffffu, rz, src);
                const double d = 0.5 * (qx * qx + qy * qy + qz * qz);
                const double tol = 1e-12 * d;
                bool beyond = false;
                for (int t = lane; t < nt; t += 32) {
                    const double *v = c.v[cur][t];
                    beyond = beyond || qx * v[0] + qy * v[1] + qz * v[2] - d > tol;
                }
                if (__any_sync(0xffffffffu, beyond) && lane == src) hit = true;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (n + __popc(m) > WCAND) {
                // narrow the window to the nearer half of the list (n <= WCAND here)
                sort_cand(c, n);
                const float kth = c.cd2[n / 2];
                const float pf = nextafterf(kth, 0.f);
                const double p2 = (double)pf;
                int keep = 0;   // the sorted prefix below the median key
                for (int b = 0; b < n; b += 32) {
                    const int i = b + lane;
                    keep += __popc(__ballot_sync(0xffffffffu, i < n && c.cd2[i] < kth));
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
                    c.cd2[pos] = (float)d2;
                    c.cid[pos] = (int)k;
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
// side test on the rounded positions (the same band as in gather_cutting,
// above the rounding of the coordinates): one that every vertex clears cuts
// nothing and costs no FP64 work.
template <class C>
__device__ int clip_sorted(C &c, const em::ChunkTree &T, const double *__restrict__ xs,
                           const double *__restrict__ ys, const double *__restrict__ zs, int64_t n, double gx,
                           double gy, double gz, int nc)
{
    const int lane = threadIdx.x & 31;
    const float gxf = (float)gx, gyf = (float)gy, gzf = (float)gz;
    const float gabs = fabsf(gxf) + fabsf(gyf) + fabsf(gzf);
    for (int i = 0; i < nc; ++i) {
        int k = c.cid[i];
        if (k < 0 || k >= n) return emv::VS_BOUNDS;
        {
            const float4 pk = T.pts[k];
            const float ex = pk.x - gxf, ey = pk.y - gyf, ez = pk.z - gzf;
            const float df = 0.5f * (ex * ex + ey * ey + ez * ez), rabs = fabsf(ex) + fabsf(ey) + fabsf(ez);
            bool maybe = false;
            for (int t = lane; t < c.nt; t += 32) {
                const float *vf = c.vf[t];
                const float ff = ex * vf[0] + ey * vf[1] + ez * vf[2] - df;
                maybe = maybe || ff > -1e-5f * (gabs + rabs + vf[3]) * (vf[3] + rabs);
            }
            if (!__any_sync(0xffffffffu, maybe)) continue;
        }
        double nx, ny, nz, d;
        bisector(xs, ys, zs, k, gx, gy, gz, nx, ny, nz, d);
        int r = wclip(c, nx, ny, nz, d, k);
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
__device__ int wbuild_cell(C &c, const em::ChunkTree &T, const double *__restrict__ xs,
                           const double *__restrict__ ys, const double *__restrict__ zs,
                           int64_t s, const double *box, int K, float margin)
{
    const int lane = threadIdx.x & 31;
    int status = 0;
    const double gx = xs[s], gy = ys[s], gz = zs[s];
    if (!(gx > box[0] && gx < box[1] && gy > box[2] && gy < box[3] && gz > box[4] && gz < box[5]))
        return emv::VS_OUTSIDE;
    wcell_box(c, box, gx, gy, gz);
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
    // stage 1: shrink or grow R until the candidates fit and number at least K
    double lo_ok = 0.0, hi_bad = INFINITY;
    int nc = -1;
    for (int it = 0; it < 48; ++it) {
        nc = gather(c, T, xs, ys, zs, s, gx, gy, gz, -1.0, R2, margin, status);
        if (status & emv::VS_COINCIDENT) return status;
        if (nc < 0) {
            hi_bad = R2;
            R2 = lo_ok > 0.0 ? sqrt(lo_ok * hi_bad) : 0.3 * R2;
            continue;
        }
        if (nc < K && nc < n - 1 && hi_bad == INFINITY && it < 40) {
            lo_ok = R2;
            R2 *= 2.0;
            continue;
        }
        break;
    }
    double skip2 = -1.0;
    if (nc > 0) {
        sort_cand(c, nc);
        int st = clip_sorted(c, T, xs, ys, zs, n, gx, gy, gz, nc);
        if (st) return status | st;
    }
    if (nc >= 0) skip2 = R2;   // every generator nearer than R was applied
    // stage 2: windows [skip2, hi2) of generators that still cut, nearest first
    for (int round = 0; round < 256; ++round) {
        const double lim2 = 4.0 * wrmax2(c) * (1.0 + 1e-12);   // no generator beyond 2 R_max can cut
        if (skip2 >= lim2) return status;
        double hi2 = lim2;
        int m = -1;
        for (int h = 0; h < 64; ++h) {
            m = gather_cutting(c, T, xs, ys, zs, s, gx, gy, gz, skip2, hi2);
            if (m >= 0) break;
            hi2 = (skip2 > 0.0 ? skip2 : 0.0) + 0.5 * (hi2 - (skip2 > 0.0 ? skip2 : 0.0));
        }
        if (m < 0) return status | emv::VS_CANDIDATES;
        if (m > 0) {
            sort_cand(c, m);
            int st = clip_sorted(c, T, xs, ys, zs, n, gx, gy, gz, m);
            if (st) return status | st;
        }
        skip2 = hi2;
    }
    return status | emv::VS_ROUNDS;
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
