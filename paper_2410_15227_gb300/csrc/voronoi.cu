// build_voronoi: Voronoi cells of the generation sites, clipped to the box.
//
// Each cell is built by one warp, with the cell in shared memory, in the
// generator's frame (g at the origin).  The convex cell is held in dual form:
// its planes (n.x <= d) and its vertices, each a triangle of three plane
// indices ordered counter-clockwise seen from outside, with the vertex
// position.  Clipping by a bisector removes the vertices beyond it and
// replaces each edge that crossed the plane by a new vertex (the kept
// neighbour across an edge (a, b) is the vertex holding (b, a)); the lanes
// share the vertex work (voronoi_warp.cuh).
//
// Candidates: the generators within a search radius of the site, found by a
// warp walk of the generators' box hierarchy and clipped nearest first.  The
// cell is exact once 2 R_max is below the search radius, R_max being its
// farthest vertex: no generator farther than 2 R_max can cut it.  Otherwise
// the shell up to 2 R_max is clipped in as well.  The build pass writes each
// finished cell's faces into a scratch slot of fixed capacity (64 faces, 384
// face-vertices: every vertex belongs to three faces) and its counts; after
// the scan of the counts, a copy pass moves the slots to the cells' offsets.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tree_util.cuh"

#include "voronoi_cell.cuh"
#include "voronoi_warp.cuh"

namespace {

using namespace emv;
using emw::WCell;

constexpr int VW = 2;   // warps (cells) per block
#ifndef EM_VOR_MINB
#define EM_VOR_MINB 14   // resident blocks per SM asked of the compiler in the first pass
#endif

// Capacity of a cell's scratch slot: faces (planes) and face-vertices (every
// vertex belongs to three faces).
constexpr int SLOT_F = emw::WMAXP;
constexpr int SLOT_FV = 3 * MAXV;

// Write the faces of the finished cell c of sorted site s: per face its unit
// normal, the neighbour id and the offset of its vertex loop, the loop's
// vertices (CCW seen from outside, absolute coordinates, the FP64 meets of
// emw::finish_vertices) from fvbase on; returns the counts and the volume
// (divergence theorem).  The planes are formed again from their generators
// (emw::bisector, the builder's arithmetic).  Faces beyond fcap or vertices
// beyond fvcap set bad.
template <class C>
__device__ void emit_faces(const C &c, const double *__restrict__ xs, const double *__restrict__ ys,
                           const double *__restrict__ zs, const int32_t *__restrict__ perm, const double *box,
                           double gx, double gy, double gz, int fcap, int fvcap, int32_t *__restrict__ fvo,
                           double *__restrict__ verts, double *__restrict__ normals, int64_t *__restrict__ nbr, int &nf,
                           int &nfv, double &vol, bool &bad)
{
    const int lane = threadIdx.x & 31;
    int fbase = 0, fvbase = 0;
    double v = 0.0;
    uint8_t loop[C::MAXV];
    bool err = false;
    for (int r = 0; r < c.np; r += 32) {
        int q = r + lane;
        int n = q < c.np ? emw::wface_loop(c, q, loop, C::MAXV) : 0;
        if (n < 0) err = true;
        bool face = n >= 3;
        unsigned m = __ballot_sync(0xffffffffu, face);
        int fi = fbase + __popc(m & emw::lanemask_lt());
        int len = face ? n : 0, incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int fvi = fvbase + incl - len;
        if (face) {
            if (fi >= fcap || fvi + n > fvcap) {
                err = true;
            } else {
                const int sid = c.sid[q];
                double nx, ny, nz, d;
                if (sid >= 0) emw::bisector(xs, ys, zs, sid, gx, gy, gz, nx, ny, nz, d);
                else emw::wall_plane(box, -1 - sid, gx, gy, gz, nx, ny, nz, d);
                const double ln = sqrt(nx * nx + ny * ny + nz * nz), il = 1.0 / ln;
                nx *= il;
                ny *= il;
                nz *= il;
                normals[3 * fi] = nx;
                normals[3 * fi + 1] = ny;
                normals[3 * fi + 2] = nz;
                nbr[fi] = sid >= 0 ? (int64_t)perm[sid] : (int64_t)sid;
                fvo[fi] = fvi;
                double ax = 0.0, ay = 0.0, az = 0.0;   // twice the vector area
                for (int i = 0; i < n; ++i) {
                    const double *pa = c.u.vx[loop[i]], *pb = c.u.vx[loop[(i + 1) % n]];
                    ax += pa[1] * pb[2] - pa[2] * pb[1];
                    ay += pa[2] * pb[0] - pa[0] * pb[2];
                    az += pa[0] * pb[1] - pa[1] * pb[0];
                    verts[3 * (fvi + i)] = pa[0] + gx;
                    verts[3 * (fvi + i) + 1] = pa[1] + gy;
                    verts[3 * (fvi + i) + 2] = pa[2] + gz;
                }
                double area = 0.5 * (ax * nx + ay * ny + az * nz);
                v += area * (d * il) * (1.0 / 3.0);
            }
        }
        fbase += __popc(m);
        fvbase += __shfl_sync(0xffffffffu, incl, 31);
    }
    bad = __any_sync(0xffffffffu, err);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    nf = fbase;
    nfv = fvbase;
    vol = v;
}

struct BuildArgs {
    int64_t ngen;
    em::ChunkTree T;
    const double *xs, *ys, *zs;
    const int32_t *perm;
    double box[6];
    int K;
    float margin;
    int64_t *nface, *nfv;
    int32_t *s_fvo;
    double *s_verts, *s_normals;
    int64_t *s_nbr;
    double *volume, *gen;
    int *status_or;      // [0] OR of the failing cells' status bits, [1] the first failing cell
    int *retry_n;        // cells the first pass left for the second
    int32_t *retry_list;
    int64_t cell0, cell1;   // the cells built (by generator index); the others are left without faces
};

// Build the cell of sorted site s in c and write its faces into the cell's
// scratch slot, its counts, generator and volume.  In the first pass a cell
// that outgrows c's vertex capacity is listed for the second pass instead.
template <class C>
__device__ void build_one(C &c, const BuildArgs &a, int64_t s, bool first_pass)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = a.perm[s];
    if (j < 0 || j >= a.ngen) {
        if (lane == 0) atomicOr(a.status_or, VS_BOUNDS);
        return;
    }
    const double gx = a.xs[s], gy = a.ys[s], gz = a.zs[s];
    if (j < a.cell0 || j >= a.cell1) {   // outside the range: no faces, no volume
        if (lane == 0) {
            a.nface[j] = 0;
            a.nfv[j] = 0;
            a.volume[j] = 0.0;
            a.gen[3 * j] = gx;
            a.gen[3 * j + 1] = gy;
            a.gen[3 * j + 2] = gz;
        }
        return;
    }
    const emw::Frame F{a.xs, a.ys, a.zs, a.box, gx, gy, gz};
    int st = emw::wbuild_cell(c, a.T, F, s, a.K, a.margin);
    if (first_pass && st == VS_CAPACITY) {
        if (lane == 0) a.retry_list[atomicAdd(a.retry_n, 1)] = (int32_t)s;
        return;
    }
    int nf = 0, nv = 0;
    double vol = 0.0;
    if (!st) {
        bool bad = false;
        emw::finish_vertices(c, F);
        emit_faces(c, a.xs, a.ys, a.zs, a.perm, a.box, gx, gy, gz, SLOT_F, SLOT_FV, a.s_fvo + s * SLOT_F,
                   a.s_verts + s * (3 * SLOT_FV), a.s_normals + s * (3 * SLOT_F), a.s_nbr + s * SLOT_F, nf, nv, vol,
                   bad);
        if (bad) st |= VS_TOPOLOGY;
    }
    if (lane == 0) {
        a.nface[j] = nf;
        a.nfv[j] = nv;
        a.volume[j] = vol;
        a.gen[3 * j] = gx;
        a.gen[3 * j + 1] = gy;
        a.gen[3 * j + 2] = gz;
        if (st) {
            atomicOr(a.status_or, st);
            atomicMin(a.status_or + 1, (int)s);   // first failing cell (sorted index)
        }
    }
}

// First pass: one warp per cell (sorted index s), the cell in a small
// shared-memory footprint (MAXV_FIRST vertices) so that more warps fit an SM.
__global__ void __launch_bounds__(32 * VW, EM_VOR_MINB) k_voronoi_build(BuildArgs a)
{
    __shared__ WCell<MAXV_FIRST> cells[VW];
    const int w = threadIdx.x >> 5;
    const int64_t s = blockIdx.x * (int64_t)VW + w;
    if (s < a.ngen) build_one(cells[w], a, s, true);
}

// Second pass: the cells the first pass listed, at the full capacity (MAXV
// vertices); the count is read on the device (grid-stride loop, one warp per
// cell at a time).
__global__ void __launch_bounds__(32 * VW) k_voronoi_build_large(BuildArgs a)
{
    __shared__ WCell<MAXV> cells[VW];
    const int w = threadIdx.x >> 5;
    const int64_t nr = *a.retry_n;
    for (int64_t t = blockIdx.x * (int64_t)VW + w; t < nr; t += (int64_t)gridDim.x * VW)
        build_one(cells[w], a, a.retry_list[t], false);
}

// One warp per cell: copy its scratch slot to the cell's scanned offsets.
__global__ void k_voronoi_compact(int64_t ngen, const int32_t *__restrict__ perm,
                                  const int64_t *__restrict__ cell_face_off, const int64_t *__restrict__ cell_fv_off,
                                  const int32_t *__restrict__ s_fvo, const double *__restrict__ s_verts,
                                  const double *__restrict__ s_normals, const int64_t *__restrict__ s_nbr,
                                  int64_t *__restrict__ face_vert_off, double *__restrict__ verts,
                                  double *__restrict__ normals, int64_t *__restrict__ nbr)
{
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= ngen) return;
    const int64_t j = perm[s];
    const int64_t f0 = cell_face_off[j], fv0 = cell_fv_off[j];
    const int nf = (int)(cell_face_off[j + 1] - f0), nv = (int)(cell_fv_off[j + 1] - fv0);
    for (int f = lane; f < nf; f += 32) {
        face_vert_off[f0 + f] = fv0 + s_fvo[s * SLOT_F + f];
        nbr[f0 + f] = s_nbr[s * SLOT_F + f];
    }
    for (int t = lane; t < 3 * nf; t += 32) normals[3 * f0 + t] = s_normals[s * (3 * SLOT_F) + t];
    for (int t = lane; t < 3 * nv; t += 32) verts[3 * fv0 + t] = s_verts[s * (3 * SLOT_FV) + t];
}

__global__ void k_finish_offsets(int64_t *face_vert_off, int64_t nface, int64_t nfv)
{
    face_vert_off[nface] = nfv;
}

// Centroid of every cell, the move of Lloyd's iteration (Section 2.3).  One
// warp per cell, lanes over its faces; a face is fanned into triangles
// (v_0, v_k, v_k+1), and each triangle with the generator g spans a
// tetrahedron of signed volume a.(b x c)/6 (corners relative to g) and
// centroid g + (a + b + c)/4.  The warp sums the volume-weighted centroids
// in a fixed butterfly order.
__global__ void k_cell_centroid(int64_t ncell, const double *__restrict__ gen, const int64_t *__restrict__ cfo,
                                const int64_t *__restrict__ fvo, const double *__restrict__ verts,
                                double *__restrict__ cx, double *__restrict__ cy, double *__restrict__ cz)
{
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= ncell) return;   // whole warps leave together
    const double gx = gen[3 * j], gy = gen[3 * j + 1], gz = gen[3 * j + 2];
    double v6 = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t f = cfo[j] + lane; f < cfo[j + 1]; f += 32) {
        const int64_t k0 = fvo[f], k1 = fvo[f + 1];
        const double ax = verts[3 * k0] - gx, ay = verts[3 * k0 + 1] - gy, az = verts[3 * k0 + 2] - gz;
        double bx = verts[3 * k0 + 3] - gx, by = verts[3 * k0 + 4] - gy, bz = verts[3 * k0 + 5] - gz;
        for (int64_t k = k0 + 2; k < k1; ++k) {
            const double ex = verts[3 * k] - gx, ey = verts[3 * k + 1] - gy, ez = verts[3 * k + 2] - gz;
            const double t6 = ax * (by * ez - bz * ey) + ay * (bz * ex - bx * ez) + az * (bx * ey - by * ex);
            v6 += t6;
            mx += t6 * (ax + bx + ex);
            my += t6 * (ay + by + ey);
            mz += t6 * (az + bz + ez);
            bx = ex;
            by = ey;
            bz = ez;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v6 += __shfl_xor_sync(0xffffffffu, v6, o);
        mx += __shfl_xor_sync(0xffffffffu, mx, o);
        my += __shfl_xor_sync(0xffffffffu, my, o);
        mz += __shfl_xor_sync(0xffffffffu, mz, o);
    }
    if (lane == 0) {
        const double s = 1.0 / (4.0 * v6);
        cx[j] = gx + mx * s;
        cy[j] = gy + my * s;
        cz[j] = gz + mz * s;
    }
}

}  // namespace

static int voronoi_impl(em_ctx *ctx, int64_t ngen, const double *gx, const double *gy, const double *gz,
                        const em_params *p, em_voronoi *v, bool prepare = true, int64_t cell0 = 0,
                        int64_t cell1 = -1)
{
    cudaStream_t st = ctx->stream;
    DevArena tmp(st, true);
    uint64_t *key;
    int32_t *perm;
    double *xs, *ys, *zs;
    EM_TRY(tmp.alloc(&key, ngen));
    EM_TRY(tmp.alloc(&perm, ngen));
    EM_TRY(tmp.alloc(&xs, ngen));
    EM_TRY(tmp.alloc(&ys, ngen));
    EM_TRY(tmp.alloc(&zs, ngen));
    EM_TRY(em_morton_sort(ctx, ngen, gx, gy, gz, v->box, key, perm));
    EM_TRY(em_gather_sorted(ctx, ngen, perm, gx, gy, gz, nullptr, xs, ys, zs, nullptr));
    em::ChunkTree T;
    EM_TRY(em_chunk_tree_build(ctx, tmp, ngen, xs, ys, zs, nullptr, 0.0, &T));
    int K = p->knn_k > 0 ? p->knn_k : 48;
    if (K > MAXK) K = MAXK;
    int64_t *nface, *nfv, *cfo, *cfvo;
    int *status;
    // per-cell scratch slots for the faces, written by the build pass
    int32_t *s_fvo;
    double *s_verts, *s_normals;
    int64_t *s_nbr;
    EM_TRY(tmp.alloc(&nface, ngen + 1));
    EM_TRY(tmp.alloc(&nfv, ngen + 1));
    EM_TRY(tmp.alloc(&cfvo, ngen + 1));
    EM_TRY(tmp.alloc(&s_fvo, ngen * SLOT_F));
    EM_TRY(tmp.alloc(&s_nbr, ngen * SLOT_F));
    EM_TRY(tmp.alloc(&s_normals, ngen * 3 * SLOT_F));
    EM_TRY(tmp.alloc(&s_verts, ngen * 3 * SLOT_FV));
    EM_TRY(tmp.alloc(&status, 3));
    int32_t *retry;
    EM_TRY(tmp.alloc(&retry, ngen));
    EM_TRY(v->mem.alloc(&cfo, ngen + 1));
    EM_TRY(v->mem.alloc(&v->gen, 3 * ngen));
    EM_TRY(v->mem.alloc(&v->volume, ngen));
    EM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    EM_CUDA(cudaMemsetAsync(status + 1, 0x7f, sizeof(int), st));
    EM_CUDA(cudaMemsetAsync(status + 2, 0, sizeof(int), st));
    EM_CUDA(cudaMemsetAsync(nface + ngen, 0, sizeof(int64_t), st));
    EM_CUDA(cudaMemsetAsync(nfv + ngen, 0, sizeof(int64_t), st));
    const double *b = v->box;
    double ext = 0.0;
    for (int k = 0; k < 6; ++k) ext = fmax(ext, fabs(b[k]));
    const float margin = (float)(4e-7 * (ext + 1.0));
    BuildArgs a;
    a.ngen = ngen;
    a.T = T;
    a.xs = xs;
    a.ys = ys;
    a.zs = zs;
    a.perm = perm;
    for (int k = 0; k < 6; ++k) a.box[k] = b[k];
    a.K = K;
    a.margin = margin;
    a.nface = nface;
    a.nfv = nfv;
    a.s_fvo = s_fvo;
    a.s_verts = s_verts;
    a.s_normals = s_normals;
    a.s_nbr = s_nbr;
    a.volume = v->volume;
    a.gen = v->gen;
    a.status_or = status;
    a.retry_n = status + 2;
    a.retry_list = retry;
    a.cell0 = cell0;
    a.cell1 = cell1 < 0 ? ngen : cell1;
    k_voronoi_build<<<em_grid(ngen, VW), 32 * VW, 0, st>>>(a);
    EM_LAUNCHED(ctx);
    k_voronoi_build_large<<<(unsigned)std::min<int64_t>(em_grid(ngen, VW), 8 * (int64_t)ctx->nsm), 32 * VW, 0, st>>>(a);
    EM_LAUNCHED(ctx);
    EM_TRY(em_exclusive_scan_i64(ctx, nface, cfo, ngen + 1));
    EM_TRY(em_exclusive_scan_i64(ctx, nfv, cfvo, ngen + 1));
    int64_t tot[2];
    int hstatus = 0;
    EM_CUDA(cudaMemcpyAsync(&tot[0], cfo + ngen, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    EM_CUDA(cudaMemcpyAsync(&tot[1], cfvo + ngen, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    EM_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    EM_CUDA(cudaStreamSynchronize(st));
    if (hstatus & (VS_COINCIDENT | VS_OUTSIDE)) {
        em_set_error("build_voronoi: %s", (hstatus & VS_COINCIDENT) ? "coincident generators"
                                                                      : "a generator lies outside the box");
        return EM_EINVAL;
    }
    if (hstatus & VS_BOUNDS) {
        em_set_error("build_voronoi: an index check failed (status %d)", hstatus);
        return EM_ECUDA;
    }
    if (hstatus) {
        int first[2] = {0, 0};
        EM_CUDA(cudaMemcpyAsync(first, status + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaMemcpyAsync(first + 1, perm + first[0], sizeof(int), cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaStreamSynchronize(st));
        EM_CUDA(cudaMemcpyAsync(first + 1, perm + first[0], sizeof(int), cudaMemcpyDeviceToHost, st));
        EM_CUDA(cudaStreamSynchronize(st));
        em_set_error("build_voronoi: a cell exceeded the per-cell capacity (%d planes, %d vertices) or "
                     "lost its topology (status %d, first at generator %d)", MAXP, MAXV, hstatus, first[1]);
        return EM_ECAPACITY;
    }
    v->ncell = ngen;
    v->nface = tot[0];
    v->nfv = tot[1];
    v->cell_face_off = cfo;
    EM_TRY(v->mem.alloc(&v->face_vert_off, v->nface + 1));
    EM_TRY(v->mem.alloc(&v->verts, 3 * v->nfv));
    EM_TRY(v->mem.alloc(&v->normals, 3 * v->nface));
    EM_TRY(v->mem.alloc(&v->nbr, v->nface));
    k_voronoi_compact<<<em_grid(ngen * 32, 256), 256, 0, st>>>(ngen, perm, cfo, cfvo, s_fvo, s_verts, s_normals, s_nbr,
                                                               v->face_vert_off, v->verts, v->normals, v->nbr);
    EM_LAUNCHED(ctx);
    k_finish_offsets<<<1, 1, 0, st>>>(v->face_vert_off, v->nface, v->nfv);
    EM_LAUNCHED(ctx);
    return prepare ? em_prepare_cells(ctx, v) : EM_OK;
}

static int new_voronoi(em_ctx *ctx, int64_t ngen, const double *d_gx, const double *d_gy, const double *d_gz,
                       const double *h_box, const em_params *p, int64_t cell0, int64_t cell1, em_voronoi **out)
{
    EM_CHECK_ARG(ctx && out && h_box && p && d_gx && d_gy && d_gz);
    EM_CHECK_ARG(ngen >= 1 && ngen < INT32_MAX);
    EM_CHECK_ARG(h_box[1] > h_box[0] && h_box[3] > h_box[2] && h_box[5] > h_box[4]);
    EM_CHECK_ARG(cell0 >= 0 && cell0 <= cell1 && cell1 <= ngen);
    *out = nullptr;
    em_voronoi *v = new em_voronoi(ctx->stream);
    v->device = ctx->device;
    for (int k = 0; k < 6; ++k) v->box[k] = h_box[k];
    int rc = voronoi_impl(ctx, ngen, d_gx, d_gy, d_gz, p, v, true, cell0, cell1);
    if (rc) {
        v->mem.release();
        delete v;
        return rc;
    }
    *out = v;
    return EM_OK;
}

EM_EXPORT int build_voronoi(em_ctx *ctx, int64_t ngen, const double *d_gx, const double *d_gy, const double *d_gz,
                            const double *h_box, const em_params *p, em_voronoi **out)
{
    return new_voronoi(ctx, ngen, d_gx, d_gy, d_gz, h_box, p, 0, ngen, out);
}

EM_EXPORT int build_voronoi_cells(em_ctx *ctx, int64_t ngen, const double *d_gx, const double *d_gy,
                                  const double *d_gz, const double *h_box, const em_params *p, int64_t cell_begin,
                                  int64_t cell_end, em_voronoi **out)
{
    return new_voronoi(ctx, ngen, d_gx, d_gy, d_gz, h_box, p, cell_begin, cell_end, out);
}

EM_EXPORT int voronoi_centroids(em_ctx *ctx, const em_voronoi *v, double *d_cx, double *d_cy, double *d_cz)
{
    EM_CHECK_ARG(ctx && v && d_cx && d_cy && d_cz);
    if (v->ncell == 0) return EM_OK;
    k_cell_centroid<<<em_grid(v->ncell * 32, 256), 256, 0, ctx->stream>>>(v->ncell, v->gen, v->cell_face_off,
                                                                         v->face_vert_off, v->verts, d_cx, d_cy,
                                                                         d_cz);
    EM_LAUNCHED(ctx);
    return EM_OK;
}

EM_EXPORT int lloyd(em_ctx *ctx, int64_t ngen, double *d_gx, double *d_gy, double *d_gz, const double *h_box,
                    int iters, const em_params *p)
{
    EM_CHECK_ARG(ctx && h_box && p && d_gx && d_gy && d_gz);
    EM_CHECK_ARG(ngen >= 1 && ngen < INT32_MAX && iters >= 0);
    EM_CHECK_ARG(h_box[1] > h_box[0] && h_box[3] > h_box[2] && h_box[5] > h_box[4]);
    for (int it = 0; it < iters; ++it) {
        // the cells only (no derived geometry for the mapping), then the move;
        // the cell records are freed in stream order after the move
        em_voronoi v(ctx->stream);
        v.device = ctx->device;
        for (int k = 0; k < 6; ++k) v.box[k] = h_box[k];
        int rc = voronoi_impl(ctx, ngen, d_gx, d_gy, d_gz, p, &v, false);
        if (rc == EM_OK) rc = voronoi_centroids(ctx, &v, d_gx, d_gy, d_gz);
        v.mem.release();
        if (rc) return rc;
    }
    return EM_OK;
}
