// Internal definitions shared by the library's translation units: context,
// handles, device-memory ownership, error reporting and launch accounting.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/exactmap.h"

#define EM_EXPORT extern "C" __attribute__((visibility("default")))

struct em_ctx {
    int device;
    int nsm;   // streaming multiprocessors of the device (grid sizes of the grid-stride kernels)
    cudaStream_t stream;
    int64_t launches;
    // optional timing of the map_exact kernels (em_ctx_set_timing):
    // ev[0..1] bracket the main pass, ev[2..3] the FP64 recompute of flagged pairs
    bool timing;
    cudaEvent_t ev[4];
    bool recorded[2];
    // size of find_pairs' unsorted hit buffer for the next call: the last
    // call's pair count plus 1/8 (0: none yet)
    int64_t pairs_hint;
};

void em_set_error(const char *fmt, ...);

#define EM_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            em_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? EM_ENOMEM : EM_ECUDA;                         \
        }                                                                                          \
    } while (0)

#define EM_TRY(expr)                                                                               \
    do {                                                                                           \
        int s_ = (expr);                                                                           \
        if (s_ != EM_OK) return s_;                                                                \
    } while (0)

#define EM_CHECK_ARG(cond)                                                                         \
    do {                                                                                           \
        if (!(cond)) {                                                                             \
            em_set_error("%s: invalid argument (%s)", __func__, #cond);                            \
            return EM_EINVAL;                                                                      \
        }                                                                                          \
    } while (0)

// Count a kernel launch on the context and surface launch errors.
#define EM_LAUNCHED(ctx)                                                                           \
    do {                                                                                           \
        (ctx)->launches++;                                                                         \
        cudaError_t e_ = cudaGetLastError();                                                       \
        if (e_ != cudaSuccess) {                                                                   \
            em_set_error("%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_));          \
            return EM_ECUDA;                                                                       \
        }                                                                                          \
    } while (0)

// The library's memory pool on a device (created on first use; null if the
// device has none): every allocation below comes from it.  Its release
// threshold is the maximum, so memory that one call frees stays reserved for
// the next call instead of going back to the system at each synchronisation
// (a step maps several GB of scratch); it is returned at process exit.  The
// device's default pool, and anyone else using it, are not touched.
cudaMemPool_t em_device_pool(int device);

// Stream-ordered device allocations released together (handle memory, or a
// call's scratch when used as a local).
struct DevArena {
    cudaStream_t stream = nullptr;
    std::vector<void *> ptrs;
    bool scoped = false;

    explicit DevArena(cudaStream_t s = nullptr, bool scoped_ = false) : stream(s), scoped(scoped_) {}
    DevArena(const DevArena &) = delete;
    DevArena &operator=(const DevArena &) = delete;
    ~DevArena()
    {
        if (scoped) release();
    }

    template <class T>
    int alloc(T **p, size_t n)
    {
        *p = nullptr;
        size_t bytes = (n ? n : 1) * sizeof(T);
        int dev = 0;
        cudaMemPool_t pool = cudaGetDevice(&dev) == cudaSuccess ? em_device_pool(dev) : nullptr;
        cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)p, bytes, pool, stream)
                             : cudaMallocAsync((void **)p, bytes, stream);
        if (e != cudaSuccess) {
            em_set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
            cudaGetLastError();
            return EM_ENOMEM;
        }
        ptrs.push_back((void *)*p);
        return EM_OK;
    }

    void release()
    {
        for (void *p : ptrs) cudaFreeAsync(p, stream);
        ptrs.clear();
    }
};

// ---- handles ------------------------------------------------------------------

struct em_tree {
    int device;
    DevArena mem;
    int64_t n = 0, nnode = 0;
    int depth = 0;
    double box[6];
    std::vector<int64_t> level_off;   // host: first node index of each level, + end
    int32_t *perm = nullptr;          // [n] original index of Morton position k
    uint64_t *key = nullptr;          // [n] sorted keys
    double *xs = nullptr, *ys = nullptr, *zs = nullptr, *ms = nullptr;   // [n] Morton order
    uint64_t *label = nullptr;
    int32_t *level = nullptr, *parent = nullptr, *first = nullptr, *count = nullptr;
    int32_t *first_child = nullptr, *nchild = nullptr;
    double *mass = nullptr, *mx = nullptr, *my = nullptr, *mz = nullptr;
    double *cx = nullptr, *cy = nullptr, *cz = nullptr, *size = nullptr;
    explicit em_tree(cudaStream_t s) : mem(s) {}
};

struct em_pseudo {
    int device;
    DevArena mem;
    int64_t n = 0, npop = 0;
    int64_t nstatus[4] = {0, 0, 0, 0};
    double *x = nullptr, *y = nullptr, *z = nullptr, *h = nullptr, *m = nullptr;
    int64_t *origin = nullptr;
    int32_t *first = nullptr, *count = nullptr, *status = nullptr;
    int32_t *node = nullptr;   // [n] tree node of a node pseudo-particle, -1 for an extracted particle
    explicit em_pseudo(cudaStream_t s) : mem(s) {}
};

// One face of a cell, in the frame of the cell's generator g.
struct __align__(32) PlaneD {
    double x, y, z, w;   // unit outward normal (x, y, z), offset w = n.(V_0 - g)
};
struct __align__(16) PlaneF {
    float x, y, z, w;
};
// One face-edge of a cell, in the frame of the cell's generator g:
// m = in-plane outward edge normal, cm = m.(V_k - g); e = unit edge
// direction, ce = e.(V_k - g); L = edge length.
struct __align__(16) EdgeD {
    double mx, my, mz, cm, ex, ey, ez, ce, L, pad;
};
struct __align__(16) EdgeF {
    float mx, my, mz, cm, ex, ey, ez, ce, L, pad0, pad1, pad2;
};

struct em_voronoi {
    int device;
    DevArena mem;
    int64_t ncell = 0, nface = 0, nfv = 0;
    double box[6];
    double *gen = nullptr;              // [3 ncell]
    int64_t *cell_face_off = nullptr;   // [ncell + 1]
    int64_t *face_vert_off = nullptr;   // [nface + 1]
    double *verts = nullptr;            // [3 nfv]
    double *normals = nullptr;          // [3 nface]
    int64_t *nbr = nullptr;             // [nface]
    double *volume = nullptr;           // [ncell]
    // derived geometry for map_exact (generator frame)
    double *radius = nullptr;           // [ncell] largest |V - g|
    PlaneD *plane = nullptr;            // [nface] (n, c = n.(V_0 - g))
    EdgeD *edge = nullptr;              // [nfv]
    PlaneF *plane_f = nullptr;
    PlaneF *plane_fl = nullptr;         // [nface] P - (double)(float)P: low parts of the plane records
    EdgeF *edge_f = nullptr;
    EdgeF *edge_fl = nullptr;           // [nfv] E - (double)(float)E: low parts of the edge records
    explicit em_voronoi(cudaStream_t s) : mem(s) {}
};

struct em_pairs {
    int device;
    DevArena mem;
    int64_t npairs = 0, np = 0, ncell = 0;
    int32_t *pair_i = nullptr, *pair_j = nullptr;   // sorted by (j, i)
    uint8_t *near = nullptr;
    int64_t *cell_pair_off = nullptr;               // [ncell + 1]
    int64_t *part_pair_off = nullptr;               // [np + 1]
    int32_t *part_pair_idx = nullptr;               // [npairs] pair ids sorted by (i, j)
    explicit em_pairs(cudaStream_t s) : mem(s) {}
};

// ---- helpers shared across translation units -------------------------------------

int em_prepare_cells(em_ctx *ctx, em_voronoi *v);                 // derived geometry
int em_build_pair_index(em_ctx *ctx, em_pairs *pr);               // CSR offsets + transpose
// map_exact's body (mapping.cu); d_flag_buf / d_flag_count: optional scratch
// for the mixed pass's flagged pairs (npairs entries), read back by map_batch
int em_map_exact_impl(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                      const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p, double *d_w_out,
                      double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64, bool fixed, int32_t *d_flag_buf,
                      int *d_flag_count);
int em_exclusive_scan_i64(em_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);
int em_exclusive_scan_i32(em_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);
int em_sort_pairs_u64(em_ctx *ctx, uint64_t *keys, int32_t *vals, int64_t n, int end_bit);
int em_sort_pairs_u32(em_ctx *ctx, uint32_t *keys, int32_t *vals, int64_t n, int end_bit);

static inline int em_grid(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : g);
}

static inline int em_nbits(uint64_t v)
{
    int b = 0;
    while (b < 64 && (v >> b)) ++b;
    return b < 1 ? 1 : b;
}
