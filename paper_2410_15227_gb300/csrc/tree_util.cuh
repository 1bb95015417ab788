// Shared device utilities: Morton keys, the M4 kernel, and a 32-ary bounding
// volume hierarchy over Morton-ordered items ("chunk tree") with a
// warp-cooperative traversal.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace em {

constexpr int kMortonBits = 21;

__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// floor((x - lo) * (2^21 / (hi - lo))) clamped to [0, 2^21 - 1], each
// operation rounded to nearest separately.
__device__ __forceinline__ uint64_t quantise(double x, double lo, double hi)
{
    double scale = __ddiv_rn(2097152.0, __dsub_rn(hi, lo));
    double q = floor(__dmul_rn(__dsub_rn(x, lo), scale));
    q = q < 0.0 ? 0.0 : q;
    q = q > 2097151.0 ? 2097151.0 : q;
    return (uint64_t)q;
}

__device__ __forceinline__ uint64_t morton_key(double x, double y, double z, double xlo, double xhi, double ylo,
                                               double yhi, double zlo, double zhi)
{
    return (spread3(quantise(x, xlo, xhi)) << 2) | (spread3(quantise(y, ylo, yhi)) << 1) |
           spread3(quantise(z, zlo, zhi));
}

constexpr int kMaxLevels = 8;

// Level 0 = items (Morton order); level l >= 1 node k bounds the items
// [k 32^l, (k+1) 32^l).  The top level holds at most 32 nodes.
struct ChunkTree {
    int nlev = 0;                     // number of box levels
    int64_t count[kMaxLevels + 1];    // nodes per level (count[0] = items)
    float4 *lo[kMaxLevels + 1];       // per level l >= 1: box min (xyz)
    float4 *hi[kMaxLevels + 1];       // box max
    float4 *pts = nullptr;            // level 0: item positions rounded to FP32 (w = 0)
};

__host__ __device__ __forceinline__ float box_dist2(const float4 lo, const float4 hi, float px, float py, float pz)
{
    float dx = fmaxf(fmaxf(lo.x - px, px - hi.x), 0.f);
    float dy = fmaxf(fmaxf(lo.y - py, py - hi.y), 0.f);
    float dz = fmaxf(fmaxf(lo.z - pz, pz - hi.z), 0.f);
    return dx * dx + dy * dy + dz * dz;
}

// Warp-cooperative depth-first traversal: nodes whose box is within
// sqrt(R2) of p are opened; for each opened level-1 node every lane l calls
// visit(k, valid) with k = node*32 + l and valid = (k is an existing item),
// so visit may use warp-wide intrinsics.  All 32 lanes must call this with
// the same p and R2.  Returns false if the number of opened nodes exceeded
// max_nodes (the walk is then cut short).
template <class Visit>
__device__ __forceinline__ bool warp_traverse(const ChunkTree &T, float px, float py, float pz, float R2,
                                              int64_t max_nodes, Visit &&visit)
{
    const int lane = threadIdx.x & 31;
    uint32_t mask[kMaxLevels + 1];
    int64_t base[kMaxLevels + 1];
    const int top = T.nlev;
    if (top <= 0) return true;
    const float R2m = R2 * 1.00001f + 1e-30f;   // conservative margin for the float boxes
    {
        bool hit = lane < T.count[top] && box_dist2(T.lo[top][lane], T.hi[top][lane], px, py, pz) <= R2m;
        mask[top] = __ballot_sync(0xffffffffu, hit);
        base[top] = 0;
    }
    int lvl = top;
    int64_t opened = 0;
    while (true) {
        if (mask[lvl] == 0) {
            if (lvl == top) break;
            ++lvl;
            continue;
        }
        int c = __ffs(mask[lvl]) - 1;
        mask[lvl] &= mask[lvl] - 1;
        int64_t node = base[lvl] * 32 + c;
        if (++opened > max_nodes) return false;
        if (lvl == 1) {
            int64_t k = node * 32 + lane;
            visit(k, k < T.count[0]);
        } else {
            int64_t child = node * 32 + lane;
            bool hit = child < T.count[lvl - 1] &&
                       box_dist2(T.lo[lvl - 1][child], T.hi[lvl - 1][child], px, py, pz) <= R2m;
            mask[lvl - 1] = __ballot_sync(0xffffffffu, hit);
            base[lvl - 1] = node;
            --lvl;
        }
    }
    return true;
}

// warp_traverse whose visit returns true to go on and false to end the walk
// (a warp-uniform value).  Returns false if the walk was ended by visit.
template <class Visit>
__device__ __forceinline__ bool warp_traverse_until(const ChunkTree &T, float px, float py, float pz, float R2,
                                                    Visit &&visit)
{
    const int lane = threadIdx.x & 31;
    uint32_t mask[kMaxLevels + 1];
    int64_t base[kMaxLevels + 1];
    const int top = T.nlev;
    if (top <= 0) return true;
    const float R2m = R2 * 1.00001f + 1e-30f;   // conservative margin for the float boxes
    {
        bool hit = lane < T.count[top] && box_dist2(T.lo[top][lane], T.hi[top][lane], px, py, pz) <= R2m;
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
        int c = __ffs(mask[lvl]) - 1;
        mask[lvl] &= mask[lvl] - 1;
        int64_t node = base[lvl] * 32 + c;
        if (lvl == 1) {
            int64_t k = node * 32 + lane;
            if (!visit(k, k < T.count[0])) return false;
        } else {
            int64_t child = node * 32 + lane;
            bool hit = child < T.count[lvl - 1] &&
                       box_dist2(T.lo[lvl - 1][child], T.hi[lvl - 1][child], px, py, pz) <= R2m;
            mask[lvl - 1] = __ballot_sync(0xffffffffu, hit);
            base[lvl - 1] = node;
            --lvl;
        }
    }
    return true;
}

}  // namespace em

// Build a chunk tree over n Morton-ordered points (xs, ys, zs), each
// optionally inflated by a radius r[k] (NULL = points).  Memory from `mem`.
int em_chunk_tree_build(em_ctx *ctx, DevArena &mem, int64_t n, const double *xs, const double *ys,
                        const double *zs, const double *r, double rscale, em::ChunkTree *out);
int em_morton_sort(em_ctx *ctx, int64_t n, const double *x, const double *y, const double *z, const double *box,
                   uint64_t *key, int32_t *perm);
int em_gather_sorted(em_ctx *ctx, int64_t n, const int32_t *perm, const double *x, const double *y,
                     const double *z, const double *m, double *xs, double *ys, double *zs, double *ms);
