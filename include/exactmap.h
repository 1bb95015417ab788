/*
 * exactmap.h -- C ABI of the GB300 (sm_103a) library for the pseudo-particle
 * Exact mapping of Lau, Petkova & Bonnell (2024), "Hybrid radiation
 * hydrodynamics scheme with adaptive gravity-tree-based pseudo-particles".
 *
 * The pipeline the paper describes (Section 2.3, flowchart of the code
 * overview): build the gravity tree, walk it to select pseudo-particles and
 * solve their smoothing lengths, build the Voronoi grid on the generation
 * sites, map the (pseudo-)particle density onto the grid with the Exact
 * mapping, and map per-cell results back onto the particles.  Around it:
 * the adaptive refinement of the tree-walk (Section 2.4.1, Eq. 5), Lloyd's
 * iteration on the sites (Section 2.3), and an executor that runs many
 * independent snapshots through the pipeline at once (map_batch).
 *
 * Conventions (every entry point):
 *   - returns an int status (EM_OK = 0 on success, see em_status); no call
 *     aborts, traps the device or throws; em_last_error() returns a message
 *     for the calling thread's last failure.
 *   - arrays named "d_*" are DEVICE pointers on the context's device; arrays
 *     named "h_*" are HOST pointers.  Doubles are IEEE FP64.
 *   - the caller owns every array it passes.  Opaque handles (em_tree,
 *     em_pseudo, em_voronoi, em_pairs) own the device memory the library
 *     allocates for them; release it with the matching *_destroy call.
 *   - all GPU work is enqueued on the context's stream.  Calls whose output
 *     size is data dependent (tree, pseudo-particles, cells, pairs) synchronise
 *     that stream once to read the size, and so do the calls that return a
 *     count to the host (refine_check); the others do not synchronise.
 *     map_batch takes no context: it runs on streams of its own and returns
 *     when every snapshot has finished.
 *   - results are deterministic: the same inputs give bit-identical outputs.
 *   - indices are 0-based.  Particle and cell counts must be < 2^31.
 */
#ifndef EXACTMAP_H
#define EXACTMAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EM_OK = 0,
    EM_EINVAL = 1,      /* bad argument (null pointer, size out of range) */
    EM_ENOMEM = 2,      /* device allocation failed */
    EM_ECUDA = 3,       /* a CUDA runtime call failed */
    EM_ECAPACITY = 4,   /* a fixed per-item capacity was exceeded; see message */
    EM_ENOTCONV = 5,    /* informational: some h-solves fell back (per-item status set) */
    EM_ETIMEOUT = 6     /* a bounded device loop ran out of iterations */
} em_status;

typedef struct em_ctx em_ctx;
typedef struct em_tree em_tree;
typedef struct em_pseudo em_pseudo;
typedef struct em_voronoi em_voronoi;
typedef struct em_pairs em_pairs;

/* Parameters of the method.  em_params_default() fills the values used in
 * the paper's tests where it gives them. */
typedef struct {
    double r_part;          /* radius around a source inside which leaves are replaced by their particles (Section 2.4.1) */
    double r_leaf;          /* radius inside which nodes are opened down to leaves (Section 2.4.1) */
    double theta;           /* opening angle: a node is opened if theta^2 < (s_node / r_node)^2 (Eq. 4) */
    double h_fact;          /* h = h_fact n^(-1/3) (Eq. 6); default 1.2 */
    double h_tol;           /* Newton stopping tolerance |dh| / h_0 (Section 2.4.2); paper 1e-2, parity 1e-13 */
    int max_newton;         /* Newton iterations before bisection; default 50 */
    int precision;          /* map_exact arithmetic: 0 = FP64, 1 = mixed FP32 with FP64 recompute of flagged pairs */
    double fp64_threshold;  /* mixed mode: recompute a pair in FP64 when its estimated FP32 relative error exceeds this */
    int knn_k;              /* build_voronoi: neighbours staged per generator before the exact fallback; default 48 */
    int leaf_max;           /* build_tree: particles per leaf; default 8 */
    int block_pairs;        /* map_exact: threads per block of the FP64 kernels, one pair per warp (32..128, a multiple of 32; 0 = 128) */
    int h0_above;           /* make_pseudo_particles: with more pseudo-particles than this, every node takes h_0 (Eq. 11) and
                               the neighbour search and solver are skipped (Section 2.4.2; the paper uses 10^6); 0 = never */
    int fp32_err_ulps;      /* map_exact mixed mode: a pair goes to FP64 when fp32_err_ulps 2^-24 times the sum of the
                               magnitudes of its FP32 pieces exceeds max(fp64_threshold |w|, 1e-14); 0 = the default 8 */
    int fp32_variant;       /* map_exact mixed mode: launch shape of the FP32 pass, 0..EM_FP32_VARIANTS-1 (0 = default;
                               see map_autotune); results are deterministic per shape */
    int reserved[2];
} em_params;

void em_params_default(em_params *p);

/* ---- context ------------------------------------------------------------ */

/* Create a context on `device` that enqueues all work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
int em_ctx_create(em_ctx **ctx, int device, void *stream);
int em_ctx_destroy(em_ctx *ctx);
/* Block until all work enqueued on the context's stream has finished. */
int em_ctx_sync(em_ctx *ctx);
/* Message of the calling thread's last failed call ("" if none). */
const char *em_last_error(void);
/* Number of kernels the library has launched through this context so far. */
int64_t em_ctx_launch_count(const em_ctx *ctx);
/* Turn on (on != 0) or off the recording of CUDA events around the kernels
 * of map_exact (creates the events on first use; costs two event records per
 * pass).  Library bookkeeping for measurement, not part of the method. */
int em_ctx_set_timing(em_ctx *ctx, int on);
/* Device time of the last map_exact enqueued while timing was on: ms_main =
 * the main pass (FP64 kernel, or the FP32 pass in mixed mode), ms_recompute =
 * the FP64 recompute of flagged pairs (0 in FP64 mode).  Waits for the
 * recorded events.  Both are 0 if nothing was recorded. */
int em_ctx_map_times(em_ctx *ctx, double *ms_main, double *ms_recompute);

/* ---- em_measure_peaks ---------------------------------------------------------
 * Measured arithmetic peaks of the context's device, the denominators of the
 * roofline of the ALU-bound mapping kernels (map_exact's FP32 pass is bound
 * by its FP32, integer and special-function work, its FP64 path by the FP64
 * pipe).  The paper has no counterpart: it is a measurement aid of this
 * library.  Three of the library's own kernels run independent dependency
 * chains over a grid of (SMs x resident blocks per SM) for tens of
 * milliseconds each, timed with CUDA events on the context's stream (median
 * of three launches after a warm-up); the call synchronises the stream.
 *   h_out[5] (host): [0] FP32 fused multiply-add rate, TFLOP/s (2 flops each);
 *   [1] FP64 fused multiply-add rate, TFLOP/s; [2] special-function rate
 *   (approximate reciprocal square root), Top/s; [3] the device's SM count;
 *   [4] its maximum SM clock, MHz. */
int em_measure_peaks(em_ctx *ctx, double *h_out);

/* ---- build_tree ------------------------------------------------------------
 * Morton-ordered octree of n particles (the paper's gravity tree, Section
 * 2.2.1, with an octree in place of the k-d tree; the method is independent
 * of the tree type, Section 2.4.1).
 *   d_x, d_y, d_z, d_m: n particle positions and masses (device)
 *   h_box: [xlo, xhi, ylo, yhi, zlo, zhi] (host); keys quantise 21 bits per axis
 *   leaf_max: split nodes holding more than this many particles (<= 64)
 * Node mass, centre of mass (position of the node) and size s_node =
 * largest distance from the COM to a constituent (Section 2.2.1).  Node
 * labels: root 1, child = 8 * parent + octant, so the ancestor k levels up is
 * label >> 3k (the octree form of the label arithmetic of Section 2.2.1).
 * Nodes are numbered breadth first (level, then key). */
int build_tree(em_ctx *ctx, int64_t n, const double *d_x, const double *d_y, const double *d_z,
               const double *d_m, const double *h_box, int leaf_max, em_tree **out);
int tree_info(const em_tree *t, int64_t *n_particles, int64_t *n_nodes, int32_t *depth);
/* Copy node arrays into caller device buffers (any pointer may be NULL):
 * d_perm[n]: original index of the k-th particle in Morton order;
 * per node: label (uint64), level, parent, first, count, first_child, nchild
 * (int32), mass, size (double), com (3 doubles per node, xyz interleaved). */
int tree_get(em_ctx *ctx, const em_tree *t, int32_t *d_perm, uint64_t *d_label, int32_t *d_level,
             int32_t *d_parent, int32_t *d_first, int32_t *d_count, int32_t *d_first_child,
             int32_t *d_nchild, double *d_mass, double *d_com, double *d_size);
int tree_destroy(em_tree *t);

/* ---- make_pseudo_particles ------------------------------------------------
 * Adaptive tree-walk (Section 2.4.1): leaves whose COM is within r_part of
 * the nearest source are replaced by their particles (which keep their own
 * h); nodes within r_leaf are opened down to leaves; beyond, a node is
 * opened when theta^2 < (s/r)^2 (Eq. 4).  Then node neighbour-finding
 * (Section 2.4.3) and the node smoothing-length solver (Section 2.4.2,
 * Eqs. 6-11): Newton from h_0 = 2 h_fact s_node, bisection on
 * [1e-2 h_0, 1e2 h_0], else h_0.  Particles inside r_part are represented by
 * their leaves in the solver's neighbour sums (Section 2.4.2).
 *   d_h_particle: n particle smoothing lengths (device, original order)
 *   h_src: nsrc source positions (host, xyz interleaved), nsrc >= 1
 * Pseudo-particles are ordered by their first constituent in Morton order.
 * With p->h0_above > 0 and more than p->h0_above pseudo-particles (nodes and
 * extracted particles together), no node is solved: each takes h_0 with
 * status 2 (Section 2.4.2).
 * Returns EM_ENOTCONV (with outputs valid) when some solve fell back to h_0;
 * EM_OK when every node took h_0 through h0_above. */
int make_pseudo_particles(em_ctx *ctx, const em_tree *t, const double *d_h_particle, int nsrc,
                          const double *h_src, const em_params *p, em_pseudo **out);
/* The adaptive refinement of Section 2.4.1 (Eq. 5).  make_pseudo_particles_
 * forced is make_pseudo_particles with per-node flags from refine_check:
 * d_force[n_nodes] (device, one byte per tree node, in tree_get's order); a
 * flagged internal node is opened whatever Eq. 4 says, a flagged leaf has its
 * particles extracted (what raising r_part does for it).  EM_EINVAL when
 * d_force is NULL. */
int make_pseudo_particles_forced(em_ctx *ctx, const em_tree *t, const double *d_h_particle, int nsrc,
                                 const double *h_src, const em_params *p, const uint8_t *d_force,
                                 em_pseudo **out);
/* Eq. 5: a node pseudo-particle is under-resolved when its neutral fraction
 * f_neu is below f_neu,limit = (K - s_root / s_node) / K, K > 1 (s_node the
 * node's size, s_root the root's).  ps must come from t.
 *   d_f_neu[n_pseudo] (device): the neutral fraction of each pseudo-particle
 *     (e.g. map_back of the cells' values); NaN (no pair) and nodes of size 0
 *     never fail; extracted particles are not checked.
 *   flag_leaves: 1 flags failing leaves too (their particles are extracted
 *     in the next walk); 0 leaves them unflagged, for the form of Section
 *     2.4.1 where a failing leaf makes the caller raise r_part and r_leaf.
 *   d_force[n_nodes] (device, in/out): set to 1 for every failing internal
 *     node (and leaf, with flag_leaves) not yet flagged.
 *   *h_nnew (host): the number of nodes flagged by this call.
 *   *h_nleaf (host, may be NULL): the number of failing leaves.
 * The iteration stops when *h_nnew is 0 (and, without flag_leaves, *h_nleaf
 * is 0).  Synchronises the stream to read the counts.  EM_EINVAL for K <= 1,
 * a flag_leaves other than 0 or 1, or a NULL pointer other than h_nleaf. */
int refine_check(em_ctx *ctx, const em_pseudo *ps, const em_tree *t, const double *d_f_neu, double K,
                 int flag_leaves, uint8_t *d_force, int64_t *h_nnew, int64_t *h_nleaf);
/* n_pseudo; n_status[4]: counts of solver status 0 Newton, 1 bisection,
 * 2 fallback h_0, 3 individual particle (may be NULL). */
int pseudo_info(const em_pseudo *ps, int64_t *n_pseudo, int64_t *n_status);
/* Copy out (device buffers, any may be NULL): positions (COM or particle),
 * h, mass, origin (node label > 0, or -(particle index + 1)), Morton range
 * [first, first + count) of constituents, solver status. */
int pseudo_get(em_ctx *ctx, const em_pseudo *ps, double *d_x, double *d_y, double *d_z, double *d_h,
               double *d_m, int64_t *d_origin, int32_t *d_first, int32_t *d_count, int32_t *d_status);
int pseudo_destroy(em_pseudo *ps);

/* ---- build_voronoi ---------------------------------------------------------
 * Voronoi cells of ngen generation sites clipped to the box (the grid of
 * Section 2.3).  Each cell is the box clipped by bisector half-spaces of its
 * neighbours, staged as a bounded k-nearest list, then completed exactly by a
 * tree search for any generator closer than twice the cell's radius.
 *   d_gx, d_gy, d_gz: generator positions (device); h_box as in build_tree.
 * Coincident generators are rejected with EM_EINVAL. */
int build_voronoi(em_ctx *ctx, int64_t ngen, const double *d_gx, const double *d_gy, const double *d_gz,
                  const double *h_box, const em_params *p, em_voronoi **out);
/* The cells [cell_begin, cell_end) only (by generator index; every
 * generator still bounds them), the others left without faces and with
 * volume 0: one rank's cells in a spatial split whose ranks take contiguous
 * ranges of generators sorted in Morton order.  The built cells are the
 * same, bit for bit, as build_voronoi's. */
int build_voronoi_cells(em_ctx *ctx, int64_t ngen, const double *d_gx, const double *d_gy, const double *d_gz,
                        const double *h_box, const em_params *p, int64_t cell_begin, int64_t cell_end,
                        em_voronoi **out);
/* Import cells given as faces (e.g. from another grid code):
 *   d_gen: ncell generator positions (xyz interleaved)
 *   d_cell_face_off[ncell+1], d_face_vert_off[nface+1] (int64 CSR offsets)
 *   d_verts: 3 doubles per face vertex, counter-clockwise seen from outside
 *   d_normals: 3 doubles per face (unit, outward); d_nbr: neighbour cell or < 0
 *   d_volume: ncell volumes. */
int voronoi_from_cells(em_ctx *ctx, int64_t ncell, int64_t nface, int64_t nfv, const double *d_gen,
                       const int64_t *d_cell_face_off, const int64_t *d_face_vert_off,
                       const double *d_verts, const double *d_normals, const int64_t *d_nbr,
                       const double *d_volume, em_voronoi **out);
/* Centroid of every cell, (1/V_j) times the integral of r over cell j: the
 * move of Lloyd's iteration (Section 2.3).  d_cx, d_cy, d_cz: ncell doubles
 * each (device, caller-owned), in generator order.  Enqueued, no sync. */
int voronoi_centroids(em_ctx *ctx, const em_voronoi *v, double *d_cx, double *d_cy, double *d_cz);
/* Lloyd's iteration on the sites (Section 2.3 applies five before the
 * mapping): iters times, build the cells of the sites clipped to h_box and
 * move every site to its cell's centroid.  d_gx, d_gy, d_gz (device, in/out,
 * ngen each) hold the sites; p as for build_voronoi (knn_k).  Errors as for
 * build_voronoi (EM_EINVAL for coincident sites or a site outside the box);
 * on an error the sites hold the last completed move.  iters = 0 is a no-op. */
int lloyd(em_ctx *ctx, int64_t ngen, double *d_gx, double *d_gy, double *d_gz, const double *h_box, int iters,
          const em_params *p);
int voronoi_info(const em_voronoi *v, int64_t *ncell, int64_t *nface, int64_t *nfv);
/* Copy out in the same layout as voronoi_from_cells (any may be NULL). */
int voronoi_get(em_ctx *ctx, const em_voronoi *v, int64_t *d_cell_face_off, int64_t *d_face_vert_off,
                double *d_verts, double *d_normals, int64_t *d_nbr, double *d_volume);
int voronoi_destroy(em_voronoi *v);

/* ---- find_pairs --------------------------------------------------------------
 * All particle-cell pairs whose kernel support meets the cell:
 * dist(x_i, V_j) < 2 h_i (the "particle-cell pairs" whose number sets the
 * mapping cost, Section 1).  Pairs are sorted by (cell j, particle i).
 *   d_x, d_y, d_z, d_h: np (pseudo-)particles (device).
 *   npairs (host, may be NULL): the pair count.
 * One pass writes the hits, unordered, into a buffer sized from the
 * context's previous pair count (plus 1/8; a guess on the first call) and a
 * radix sort orders them; a call that finds more pairs than the buffer holds
 * repeats the pass once with the exact size.  Synchronises the stream to
 * read the count.  EM_ECAPACITY if the pairs reach 2^31. */
int find_pairs(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
               const double *d_h, const em_voronoi *v, em_pairs **out, int64_t *npairs);
/* Streamed pair finding, for pair lists one would rather not hold at once
 * (a chunk capacity in pairs).
 *   find_pairs_plan: counts every cell's pairs (find_pairs' pass without
 *     output) and cuts the cells into consecutive ranges whose pairs number at
 *     most chunk_capacity (a cell with more is a range of its own).
 *     h_bounds (host, caller-allocated, ncell + 1 entries): the ranges are
 *     [h_bounds[c], h_bounds[c + 1]) for c < *h_nchunks; *h_npairs (may be
 *     NULL): the total.  Synchronises the stream.
 *   find_pairs_cells: the pairs of the cells [cell_begin, cell_end) only, as
 *     find_pairs returns them (sorted by (j, i); every cell of v indexed, the
 *     others without pairs).  npairs_hint: the range's count from the plan
 *     (sizes the buffer; <= 0 if unknown).
 * The chunks' pair lists together are find_pairs' list.  map_exact on a
 * chunk gives complete cell densities for its cells (0 for the others, so
 * the chunks' densities add up) and per-particle weight sums that add over
 * the chunks; map_back_sums adds the inverse mapping's sums over them. */
int find_pairs_plan(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                    const double *d_h, const em_voronoi *v, int64_t chunk_capacity, int64_t *h_bounds,
                    int64_t *h_nchunks, int64_t *h_npairs);
int find_pairs_cells(em_ctx *ctx, int64_t np, const double *d_x, const double *d_y, const double *d_z,
                     const double *d_h, const em_voronoi *v, int64_t cell_begin, int64_t cell_end,
                     int64_t npairs_hint, em_pairs **out, int64_t *npairs);
/* Import a pair list sorted by (j, i) (device int32 arrays). */
int pairs_from_list(em_ctx *ctx, int64_t npairs, const int32_t *d_pair_i, const int32_t *d_pair_j,
                    int64_t np, const em_voronoi *v, em_pairs **out);
int pairs_info(const em_pairs *pr, int64_t *npairs, int64_t *np, int64_t *ncell);
/* Copy out: pair_i, pair_j (int32, sorted by (j, i)), d_near (uint8: 1 when
 * |dist - 2h| < 1e-9 h), d_cell_pair_off[ncell + 1] (int64). */
int pairs_get(em_ctx *ctx, const em_pairs *pr, int32_t *d_pair_i, int32_t *d_pair_j, uint8_t *d_near,
              int64_t *d_cell_pair_off);
int pairs_destroy(em_pairs *pr);

/* ---- map_exact ---------------------------------------------------------------
 * Exact mapping (Section 1 and 2.3): for every pair,
 *   w_ij = int_{V_j} W(|r - x_i|, h_i) d^3r
 * with the M4 cubic spline truncated at 2h (Section 2.4.2), integrated
 * analytically by the signed decomposition of the cell into face pyramids
 * and right sub-triangles; then
 *   rho_j = sum_i m_i w_ij / V_j   (deterministic, ascending i)
 *   u_i   = sum_j w_ij             (partition-of-unity check, ascending j).
 *   d_w_out[npairs], d_rho_out[ncell] (device); d_wsum_out[np] may be NULL.
 *   p->precision: 0 = FP64 closed form for every pair.  1 = mixed: an FP32
 *   quadrature of each edge integral (float-float plane and edge geometry,
 *   per-pair sums in float-float) with a per-pair error bound; pairs whose
 *   bound exceeds max(p->fp64_threshold |w|, 1e-14), or whose particle lies
 *   in a face plane, are recomputed with the FP64 closed form on the device.
 *   h_nfp64 (host, may be NULL): number of pairs recomputed in FP64; passing
 *   it makes the call wait for the mixed pass, NULL leaves it asynchronous. */
int map_exact(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
              const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p,
              double *d_w_out, double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64);

/* ---- map_autotune ------------------------------------------------------------
 * Launch shape of map_exact's FP32 pass for a workload: times the pass in
 * each of its EM_FP32_VARIANTS launch shapes (warps per block, minimum
 * resident blocks per SM) on the given pairs and cells -- a warm-up launch,
 * then the median of three launches timed with CUDA events on the context's
 * stream -- and returns the fastest in *h_best, to be passed as
 * em_params.fp32_variant.  The paper has no counterpart (a tuning aid of this
 * library).  Each shape is deterministic; the shapes are compiled separately
 * and agree to the mixed mode's tolerance, not bit for bit (the compiler may
 * fuse a multiply and an add differently in each).  Writes nothing but its
 * outputs; synchronises the stream.
 *   arguments as for map_exact (masses are not needed); p supplies
 *   fp64_threshold and fp32_err_ulps
 *   h_best (host): the fastest variant; h_ms (host, may be NULL):
 *   [EM_FP32_VARIANTS] milliseconds per launch of each variant. */
#define EM_FP32_VARIANTS 4
int map_autotune(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                 const double *d_h, const em_voronoi *v, const em_params *p, int *h_best, double *h_ms);

/* ---- map_exact_noalloc -------------------------------------------------------
 * The same computation and results as map_exact (bit-identical w, rho, u and
 * FP64 count), for callers that cannot allocate device memory during the
 * call: a simulation code that hands all free device memory to its own pool
 * at start-up (a cudaMalloc inside the library then fails), or one that
 * calls the mapping every time step and cannot afford the device-wide
 * synchronisation an allocation may cause.  The paper has no counterpart:
 * this is a deployment variant of the library, not a step of the method.
 *   - Allocates nothing: the mixed pass's list of flagged pairs and its
 *     counter are a fixed array of EM_NOALLOC_MAX_PAIRS entries in the
 *     library's own device memory (4 MiB, held on every GPU that loads the
 *     library until the process exits); the counter is zeroed on the
 *     context's stream at the start of every call.
 *   - pr->npairs > EM_NOALLOC_MAX_PAIRS: returns EM_ECAPACITY with a message,
 *     nothing enqueued.
 *   - The first call on a device looks up the array's address (with that
 *     device made current, then restored); make it before any stream capture
 *     that is to contain the call.
 *   - The array is shared: calls that overlap in time on one device (two
 *     streams, or two host threads) race on it.  Serialise them.
 *   - Arguments, layout, ownership and h_nfp64 as for map_exact. */
#define EM_NOALLOC_MAX_PAIRS (1 << 20)
int map_exact_noalloc(em_ctx *ctx, const em_pairs *pr, const double *d_x, const double *d_y, const double *d_z,
                      const double *d_h, const double *d_m, const em_voronoi *v, const em_params *p,
                      double *d_w_out, double *d_rho_out, double *d_wsum_out, int64_t *h_nfp64);

/* ---- map_back -------------------------------------------------------------------
 * Inverse mapping of a per-cell field onto the (pseudo-)particles
 * (Section 2.3): f_i = sum_j w_ij f_j / sum_j w_ij (NaN when particle i has
 * no pair); with a pseudo-particle set and its tree, every SPH particle then
 * inherits the value of the pseudo-particle it belongs to (Section 2.5).
 *   d_f_cell[ncell], d_f_out[np] (device)
 *   ps, t, d_f_particle_out[n particles, original order]: all NULL, or all set. */
int map_back(em_ctx *ctx, const em_pairs *pr, const double *d_w, const double *d_f_cell, double *d_f_out,
             const em_pseudo *ps, const em_tree *t, double *d_f_particle_out);
/* The inverse mapping in parts (chunks of pairs, or the ranks of a spatial
 * split): map_back_sums ADDS sum_j w_ij f_j to d_num[i] and sum_j w_ij to
 * d_den[i] over the pairs of pr (ascending j, as map_back sums), so that
 * f_i = num_i / den_i once every part is in; inherit gives every SPH particle
 * the value of the pseudo-particle it belongs to (Section 2.5), as map_back
 * does with ps and t.
 *   d_num, d_den[np] (device, caller-initialised); d_f_pseudo[ps n],
 *   d_f_particle_out[n particles, original order] (device). */
int map_back_sums(em_ctx *ctx, const em_pairs *pr, const double *d_w, const double *d_f_cell, double *d_num,
                  double *d_den);
int inherit(em_ctx *ctx, const em_pseudo *ps, const em_tree *t, const double *d_f_pseudo, double *d_f_particle_out);

/* ---- map_batch ------------------------------------------------------------------
 * Many independent snapshots through the whole path (the paper's runtime
 * study runs many snapshots, Section 3): build_tree, make_pseudo_particles
 * (a node that keeps h_0 is not an error here), build_voronoi and
 * find_pairs per snapshot on nworkers host threads (1..64), each with its own
 * context on its own non-blocking stream on `device`, largest snapshot first
 * (by n + ngen); then every pair of every snapshot mapped by ONE map_exact
 * over the concatenated pseudo-particles, cells and pair lists (one launch of
 * the FP32 pass and one of the FP64 recompute in mixed mode, one FP64 launch
 * in FP64 mode), and map_back per snapshot when a cell field is given.
 * Same results, bit for bit, as those calls made one snapshot at a time with
 * the same parameters.  Returns when every snapshot has finished.
 * Per snapshot (caller-owned; device arrays on `device`):
 *   in:  n particles d_x, d_y, d_z, d_m, d_h; ngen sites d_gx, d_gy, d_gz;
 *        box (as h_box of build_tree); nsrc sources h_src (host, xyz);
 *        d_f_cell[ngen] or NULL
 *   out: d_rho[ngen] cell densities; d_f[n] (original order, set iff
 *        d_f_cell is) the cell field mapped back onto the particles;
 *        npseudo, npairs, nfp64 (pairs recomputed in FP64); status (em_status,
 *        -1 if the snapshot did not run)
 * tune != 0 (mixed mode): the FP32 pass's launch shape is chosen by
 * map_autotune on the batch's concatenated pairs before the mapping;
 * otherwise p->fp32_variant.  *h_variant (may be NULL): the shape used; the
 * results equal the per-snapshot calls made with that shape.
 * h_map_ms (host, may be NULL): [2] device milliseconds of the batch's
 * mapping: the main pass (FP32 pass, or FP64 kernel) and the FP64 recompute.
 * The batch's totals must stay below 2^31 particles, cells and pairs
 * (EM_ECAPACITY otherwise).
 * Returns EM_OK, or the first failing snapshot's status with its index in
 * em_last_error(); the snapshots whose front stages succeeded are still
 * mapped.  *h_launches (may be NULL): kernels launched in all. */
typedef struct {
    int64_t n;
    const double *d_x, *d_y, *d_z, *d_m, *d_h;
    int64_t ngen;
    const double *d_gx, *d_gy, *d_gz;
    double box[6];
    int nsrc;
    const double *h_src;
    const double *d_f_cell;
    double *d_rho;
    double *d_f;
    int64_t npseudo, npairs, nfp64;
    int status;
} em_snapshot;

int map_batch(int device, int nsnap, em_snapshot *snaps, const em_params *p, int nworkers, int tune,
              int *h_variant, double *h_map_ms, int64_t *h_launches);

/* The same batch as a handle (create, add, run), for callers that collect
 * snapshots as they come.
 *   map_batch_create: the device, parameters (copied) and host threads of
 *     the runs (as map_batch's).
 *   map_batch_add: copies the record; the arrays it points to stay the
 *     caller's and must stay valid until a run that maps it returns.
 *     *h_index (may be NULL): its index, in the order of the adds.
 *   map_batch_run: map_batch over every snapshot added so far (the same
 *     results, bit for bit); may be called again after more adds.
 *   map_batch_get: copies record `index` out, with the outputs of the last
 *     run (npseudo, npairs, nfp64, status; -1 before any run).
 *   map_batch_destroy: frees the handle (NULL is accepted).
 * EM_EINVAL for a NULL handle, a bad index or an invalid record. */
typedef struct em_batch em_batch;
int map_batch_create(int device, const em_params *p, int nworkers, em_batch **out);
int map_batch_add(em_batch *b, const em_snapshot *s, int *h_index);
int map_batch_run(em_batch *b, int tune, int *h_variant, double *h_map_ms, int64_t *h_launches);
int map_batch_get(const em_batch *b, int index, em_snapshot *out);
int map_batch_destroy(em_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* EXACTMAP_H */
