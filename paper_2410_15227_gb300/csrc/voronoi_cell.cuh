// Per-cell Voronoi construction shared by the build_voronoi kernels: the
// convex cell in dual form (planes + vertices as plane triangles), clipping by
// a bisector, the k-nearest candidate search over the generators' chunk tree,
// the exact completion by a radius search, and face-loop extraction.  The
// functions are __host__ __device__ so the same code can be exercised on the
// CPU.
#pragma once

#include <cmath>
#include <cstdint>

#include "tree_util.cuh"

#define EM_HD __host__ __device__

namespace emv {

constexpr int MAXP = 64;     // planes per cell (6 walls + cutting bisectors)
constexpr int MAXV = 128;    // vertices per cell
constexpr int MAXK = 64;     // nearest-neighbour list
constexpr int MAXCLIP = 192;  // recorded cutting bisectors (planes are reclaimed)
constexpr int STACK = 32 * em::kMaxLevels;

enum : int {
    VS_OK = 0, VS_CAPACITY = 1, VS_TOPOLOGY = 2, VS_COINCIDENT = 4, VS_OUTSIDE = 8, VS_BOUNDS = 16,
    VS_CLIPS = 32, VS_CANDIDATES = 64, VS_ROUNDS = 128
};

struct VCell {
    int np, nt;
    double pl[MAXP][4];
    int pid[MAXP];
    uint8_t tri[MAXV][3];
    double v[MAXV][3];
};

EM_HD void cell_box(VCell &c, const double *box, double gx, double gy, double gz)
{
    const double lo[3] = {box[0] - gx, box[2] - gy, box[4] - gz};
    const double hi[3] = {box[1] - gx, box[3] - gy, box[5] - gz};
    c.np = 6;
    for (int w = 0; w < 6; ++w) {
        int ax = w >> 1;
        c.pl[w][0] = c.pl[w][1] = c.pl[w][2] = 0.0;
        c.pl[w][ax] = (w & 1) ? 1.0 : -1.0;
        c.pl[w][3] = (w & 1) ? hi[ax] : -lo[ax];
        c.pid[w] = -1 - w;
    }
    c.nt = 8;
    for (int i = 0; i < 8; ++i) {
        int sx = i & 1, sy = (i >> 1) & 1, sz = (i >> 2) & 1;
        uint8_t X = (uint8_t)sx, Y = (uint8_t)(2 + sy), Z = (uint8_t)(4 + sz);
        bool pos = ((sx ? 1 : -1) * (sy ? 1 : -1) * (sz ? 1 : -1)) > 0;
        c.tri[i][0] = X;
        c.tri[i][1] = pos ? Y : Z;
        c.tri[i][2] = pos ? Z : Y;
        c.v[i][0] = sx ? hi[0] : lo[0];
        c.v[i][1] = sy ? hi[1] : lo[1];
        c.v[i][2] = sz ? hi[2] : lo[2];
    }
}

EM_HD __forceinline__ bool tri_has_edge(const uint8_t *t, uint8_t a, uint8_t b)
{
    return (t[0] == a && t[1] == b) || (t[1] == a && t[2] == b) || (t[2] == a && t[0] == b);
}

// Drop planes that no vertex refers to any more (renumbering the others);
// returns the new plane count.
EM_HD int compact_planes(VCell &c)
{
    int map[MAXP];
    for (int q = 0; q < c.np; ++q) map[q] = -1;
    for (int t = 0; t < c.nt; ++t)
        for (int e = 0; e < 3; ++e) map[c.tri[t][e]] = 0;
    int n = 0;
    for (int q = 0; q < c.np; ++q) {
        if (map[q] < 0) continue;
        map[q] = n;
        if (n != q) {
            for (int k = 0; k < 4; ++k) c.pl[n][k] = c.pl[q][k];
            c.pid[n] = c.pid[q];
        }
        ++n;
    }
    for (int t = 0; t < c.nt; ++t)
        for (int e = 0; e < 3; ++e) c.tri[t][e] = (uint8_t)map[c.tri[t][e]];
    c.np = n;
    return n;
}

// Clip by n.x <= d.  Returns 1 if the cell changed, 0 if not, < 0 on error.
EM_HD int cell_clip(VCell &c, double nx, double ny, double nz, double d, int id)
{
    double f[MAXV];
    bool any = false;
    for (int t = 0; t < c.nt; ++t) {
        f[t] = nx * c.v[t][0] + ny * c.v[t][1] + nz * c.v[t][2] - d;
        any = any || f[t] > 0.0;
    }
    if (!any) return 0;
    if (c.np >= MAXP && compact_planes(c) >= MAXP) return -VS_CAPACITY;
    const uint8_t q = (uint8_t)c.np;
    uint8_t ntri[MAXV][3];
    double nv[MAXV][3];
    int nn = 0;
    for (int t = 0; t < c.nt; ++t) {
        if (f[t] > 0.0) continue;
        ntri[nn][0] = c.tri[t][0];
        ntri[nn][1] = c.tri[t][1];
        ntri[nn][2] = c.tri[t][2];
        nv[nn][0] = c.v[t][0];
        nv[nn][1] = c.v[t][1];
        nv[nn][2] = c.v[t][2];
        ++nn;
    }
    if (nn == 0) return -VS_TOPOLOGY;
    for (int t = 0; t < c.nt; ++t) {
        if (!(f[t] > 0.0)) continue;
        for (int e = 0; e < 3; ++e) {
            uint8_t a = c.tri[t][e], b = c.tri[t][(e + 1) % 3];
            int u = -1;
            for (int s = 0; s < c.nt; ++s)
                if (tri_has_edge(c.tri[s], b, a)) {
                    u = s;
                    break;
                }
            if (u < 0) return -VS_TOPOLOGY;
            if (f[u] > 0.0) continue;
            if (nn >= MAXV) return -VS_CAPACITY;
            double s = f[u] / (f[u] - f[t]);
            ntri[nn][0] = a;
            ntri[nn][1] = b;
            ntri[nn][2] = q;
            nv[nn][0] = c.v[u][0] + s * (c.v[t][0] - c.v[u][0]);
            nv[nn][1] = c.v[u][1] + s * (c.v[t][1] - c.v[u][1]);
            nv[nn][2] = c.v[u][2] + s * (c.v[t][2] - c.v[u][2]);
            ++nn;
        }
    }
    c.pl[q][0] = nx;
    c.pl[q][1] = ny;
    c.pl[q][2] = nz;
    c.pl[q][3] = d;
    c.pid[q] = id;
    c.np += 1;
    c.nt = nn;
    for (int t = 0; t < nn; ++t) {
        c.tri[t][0] = ntri[t][0];
        c.tri[t][1] = ntri[t][1];
        c.tri[t][2] = ntri[t][2];
        c.v[t][0] = nv[t][0];
        c.v[t][1] = nv[t][1];
        c.v[t][2] = nv[t][2];
    }
    return 1;
}

EM_HD double cell_rmax2(const VCell &c)
{
    double r2 = 0.0;
    for (int t = 0; t < c.nt; ++t) {
        double q = c.v[t][0] * c.v[t][0] + c.v[t][1] * c.v[t][1] + c.v[t][2] * c.v[t][2];
        r2 = q > r2 ? q : r2;
    }
    return r2;
}

// bisector of g (origin) and generator at relative position (dx, dy, dz):
// n = (dx, dy, dz), d = |n|^2 / 2
EM_HD __forceinline__ int clip_by(VCell &c, double dx, double dy, double dz, int id)
{
    return cell_clip(c, dx, dy, dz, 0.5 * (dx * dx + dy * dy + dz * dz), id);
}

// Thread-level k-nearest search over the generators' chunk tree (Morton
// order).  bd2/bid sorted ascending by distance; ties keep visit order.
EM_HD int knn(const em::ChunkTree &T, const double *__restrict__ xs, const double *__restrict__ ys,
                   const double *__restrict__ zs, int64_t self, double px, double py, double pz, int K, double *bd2,
                   int32_t *bid, int &status)
{
    int64_t stack[STACK];
    int sp = 0;
    int nf = 0;
    const float fx = (float)px, fy = (float)py, fz = (float)pz;
    const int top = T.nlev;
    for (int64_t b = T.count[top] - 1; b >= 0; --b) stack[sp++] = ((int64_t)top << 56) | b;
    while (sp > 0) {
        int64_t e = stack[--sp];
        int lvl = (int)(e >> 56);
        int64_t node = e & ((1ll << 56) - 1);
        if (lvl < 1 || lvl > T.nlev || node < 0 || node >= T.count[lvl]) {
            status |= VS_BOUNDS;
            return nf;
        }
        double worst = nf < K ? INFINITY : bd2[K - 1];
        float bd = em::box_dist2(T.lo[lvl][node], T.hi[lvl][node], fx, fy, fz);
        if ((double)bd > worst * 1.00001 + 1e-300) continue;
        if (lvl == 1) {
            int64_t k1 = (node + 1) * 32 < T.count[0] ? (node + 1) * 32 : T.count[0];
            for (int64_t k = node * 32; k < k1; ++k) {
                if (k == self) continue;
                double dx = xs[k] - px, dy = ys[k] - py, dz = zs[k] - pz;
                double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0.0) status |= VS_COINCIDENT;
                double wst = nf < K ? INFINITY : bd2[K - 1];
                if (!(d2 < wst)) continue;
                int pos = nf < K ? nf : K - 1;
                while (pos > 0 && bd2[pos - 1] > d2) {
                    bd2[pos] = bd2[pos - 1];
                    bid[pos] = bid[pos - 1];
                    --pos;
                }
                bd2[pos] = d2;
                bid[pos] = (int32_t)k;
                if (nf < K) ++nf;
            }
        } else {
            int64_t c1 = (node + 1) * 32 < T.count[lvl - 1] ? (node + 1) * 32 : T.count[lvl - 1];
            for (int64_t c = c1 - 1; c >= node * 32; --c) {
                if (sp >= STACK) {
                    status |= VS_CAPACITY;
                    return nf;
                }
                stack[sp++] = ((int64_t)(lvl - 1) << 56) | c;
            }
        }
    }
    return nf;
}

// Clip by the listed candidates (ascending distance), skipping those nearer
// than skip2 (already applied) and, at exactly skip2, those in the previous
// list.  Returns a status; nclip / clip_ids record the bisectors that cut.
EM_HD int clip_list(VCell &c, const em::ChunkTree &T, const double *__restrict__ xs, const double *__restrict__ ys,
                    const double *__restrict__ zs, const int32_t *__restrict__ perm, double gx, double gy, double gz,
                    int nf, const double *bd2, const int32_t *bid, double skip2, int nprev, const int32_t *prev,
                    int32_t *clip_ids, int &nclip)
{
    for (int q = 0; q < nf; ++q) {
        int k = bid[q];
        if (k < 0 || k >= T.count[0]) return VS_BOUNDS;
        if (bd2[q] < skip2) continue;
        if (bd2[q] == skip2) {
            bool listed = false;
            for (int r = 0; r < nprev; ++r) listed = listed || prev[r] == k;
            if (listed) continue;
        }
        int r = clip_by(c, xs[k] - gx, ys[k] - gy, zs[k] - gz, perm[k]);
        if (r < 0) return -r;
        if (r > 0) {
            if (nclip >= MAXCLIP) return VS_CAPACITY;
            clip_ids[nclip++] = k;
        }
    }
    return 0;
}

// Build the cell of sorted generator s: K nearest first; if the security
// radius is not met, the MAXK nearest; if still not, every generator within
// 2 R_max.  clip_ids receives the (sorted) indices of the cutting bisectors
// in the order applied.
EM_HD int build_cell(VCell &c, const em::ChunkTree &T, const double *__restrict__ xs,
                     const double *__restrict__ ys, const double *__restrict__ zs,
                     const int32_t *__restrict__ perm, int64_t s, const double *box, int K, int32_t *clip_ids,
                     int &nclip)
{
    int status = 0;
    nclip = 0;
    const double gx = xs[s], gy = ys[s], gz = zs[s];
    if (!(gx > box[0] && gx < box[1] && gy > box[2] && gy < box[3] && gz > box[4] && gz < box[5]))
        return VS_OUTSIDE;
    cell_box(c, box, gx, gy, gz);
    double bd2[MAXK];
    int32_t bid[MAXK];
    int nf = knn(T, xs, ys, zs, s, gx, gy, gz, K, bd2, bid, status);
    if (status & VS_BOUNDS) return status;
    int st = clip_list(c, T, xs, ys, zs, perm, gx, gy, gz, nf, bd2, bid, -1.0, 0, bid, clip_ids, nclip);
    if (st) return status | st;
    double R2 = cell_rmax2(c);
    if (nf == K && K < MAXK && !(4.0 * R2 < bd2[K - 1])) {
        // second stage: the MAXK nearest, skipping the K already applied
        int32_t prev[MAXK];
        const double dK2 = bd2[K - 1];
        int np_ = 0;
        for (int q = 0; q < nf; ++q)
            if (bd2[q] == dK2) prev[np_++] = bid[q];
        K = MAXK;
        nf = knn(T, xs, ys, zs, s, gx, gy, gz, K, bd2, bid, status);
        if (status & VS_BOUNDS) return status;
        st = clip_list(c, T, xs, ys, zs, perm, gx, gy, gz, nf, bd2, bid, dK2, np_, prev, clip_ids, nclip);
        if (st) return status | st;
        R2 = cell_rmax2(c);
    }
    if (nf == K && !(4.0 * R2 < bd2[K - 1])) {
        // security radius still not met: clip by every other generator within 2 R_max
        const double dK2 = bd2[K - 1];
        int64_t stack[STACK];
        int sp = 0;
        const int top = T.nlev;
        for (int64_t b = T.count[top] - 1; b >= 0; --b) stack[sp++] = ((int64_t)top << 56) | b;
        while (sp > 0) {
            int64_t e = stack[--sp];
            int lvl = (int)(e >> 56);
            int64_t node = e & ((1ll << 56) - 1);
            if (lvl < 1 || lvl > T.nlev || node < 0 || node >= T.count[lvl]) return status | VS_BOUNDS;
            float bd = em::box_dist2(T.lo[lvl][node], T.hi[lvl][node], (float)gx, (float)gy, (float)gz);
            if ((double)bd > 4.0 * R2 * 1.00001) continue;
            if (lvl == 1) {
                int64_t k1 = (node + 1) * 32 < T.count[0] ? (node + 1) * 32 : T.count[0];
                for (int64_t k = node * 32; k < k1; ++k) {
                    if (k == s) continue;
                    double dx = xs[k] - gx, dy = ys[k] - gy, dz = zs[k] - gz;
                    double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 < dK2 || !(d2 < 4.0 * R2)) continue;
                    bool listed = false;
                    if (d2 == dK2)
                        for (int q = 0; q < nf; ++q) listed = listed || bid[q] == (int32_t)k;
                    if (listed) continue;
                    int r = clip_by(c, dx, dy, dz, perm[k]);
                    if (r < 0) return status | -r;
                    if (r > 0) {
                        if (nclip >= MAXCLIP) return status | VS_CAPACITY;
                        clip_ids[nclip++] = (int32_t)k;
                        R2 = cell_rmax2(c);
                    }
                }
            } else {
                int64_t c1 = (node + 1) * 32 < T.count[lvl - 1] ? (node + 1) * 32 : T.count[lvl - 1];
                for (int64_t cc = c1 - 1; cc >= node * 32; --cc) {
                    if (sp >= STACK) return status | VS_CAPACITY;
                    stack[sp++] = ((int64_t)(lvl - 1) << 56) | cc;
                }
            }
        }
    }
    return status;
}

// Faces of the cell: the planes still holding vertices, with their vertex
// loops (walk (q, x, y) -> (q, y, z)), counter-clockwise seen from outside.
EM_HD int face_loop(const VCell &c, int q, uint8_t *loop)
{
    if (q < 0 || q >= c.np || c.nt < 0 || c.nt > MAXV) return -1;
    int t0 = -1;
    for (int t = 0; t < c.nt && t0 < 0; ++t)
        if (c.tri[t][0] == q || c.tri[t][1] == q || c.tri[t][2] == q) t0 = t;
    if (t0 < 0) return 0;
    int n = 0, t = t0;
    do {
        if (n >= MAXV) return -1;
        loop[n++] = (uint8_t)t;
        int r = c.tri[t][0] == q ? 0 : (c.tri[t][1] == q ? 1 : 2);
        uint8_t y = c.tri[t][(r + 2) % 3];
        int nx = -1;
        for (int s = 0; s < c.nt; ++s)
            if (tri_has_edge(c.tri[s], (uint8_t)q, y)) {
                nx = s;
                break;
            }
        if (nx < 0) return -1;
        t = nx;
    } while (t != t0);
    return n;
}


}  // namespace emv
