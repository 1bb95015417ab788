/*
 * Test infrastructure -- plain FP64 CPU oracle for the gravity-tree side of the
 * pseudo-particle method.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU baseline may load it; it shares no code with the CUDA library.
 *
 *   Morton octree, <= leaf_max particles per leaf, node mass, centre of mass,
 *     size s_node = max distance COM -> constituent       (Section 2.2.1; an
 *     octree stands in for the k-d tree, which the paper says the method does
 *     not depend on, Section 2.4.1)
 *   node labels: root 1, children 8*label + octant, so the ancestor k levels up
 *     is label >> 3k -- the octree form of the labelling arithmetic of
 *     Section 2.2.1
 *   adaptive tree-walk selecting pseudo-particles: particles inside r_part,
 *     leaves inside r_leaf, opening angle criterion (Eq. 4) outside
 *                                                          (Section 2.4.1)
 *   node smoothing-length solver: h = h_fact n^(-1/3), n = sum_b W (Eqs. 6-8),
 *     Newton-Raphson (Eqs. 9-10) from h_0 = 2 h_fact s_node (Eq. 11), then
 *     bisection on [1e-2 h_0, 1e2 h_0], then h_0            (Section 2.4.2)
 *     with brute-force neighbours over the whole population (the paper's own
 *     fallback below 1e4 nodes, Section 2.4.3).
 *
 * Readings
 *   Morton keys quantise each axis to 21 bits in the given box:
 *     i = floor((x - lo) * (2^21 / (hi - lo))), clamped to [0, 2^21 - 1];
 *     ties in the key are broken by particle index.
 *   Node sums: a leaf sums its particles in sorted order, an internal node sums
 *     its children in octant order (m, and m*x, m*y, m*z); COM = (m x)/m.
 *   Distances for the walk use the node COM and the nearest source; a tie
 *     (s^2 == theta^2 r^2) does not open the node.
 *   A leaf whose COM lies inside r_part is replaced by its particles (they keep
 *     their own h); for the h-solver those particles are represented by their
 *     leaf (Section 2.4.2, last paragraph).
 *   n(h) includes the self term W(0, h).
 *   A Newton iterate outside the bisection bracket [1e-2 h_0, 1e2 h_0] counts
 *     as a Newton failure (otherwise a node without neighbours "converges" by
 *     collapsing h towards zero, where the step relative to h_0 vanishes).
 *   A node of one particle (s_node = 0) starts from that particle's own h.
 *
 * Compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define MORTON_BITS 21

double orc_W(double r, double h);
double orc_dWdh(double r, double h);

static uint64_t spread3(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < MORTON_BITS; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

static uint64_t quantise(double x, double lo, double hi)
{
    double scale = 2097152.0 / (hi - lo);
    double q = floor((x - lo) * scale);
    if (q < 0.0) q = 0.0;
    if (q > 2097151.0) q = 2097151.0;
    return (uint64_t)q;
}

void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z, const double *box,
                     uint64_t *key)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ix = quantise(x[i], box[0], box[1]);
        uint64_t iy = quantise(y[i], box[2], box[3]);
        uint64_t iz = quantise(z[i], box[4], box[5]);
        key[i] = (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
    }
}

typedef struct { uint64_t key; int64_t idx; } kv;

static int kv_cmp(const void *a, const void *b)
{
    const kv *p = (const kv *)a, *q = (const kv *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* Build the octree.  Outputs (caller allocates max_nodes entries):
 *   perm[n]       original index of the k-th particle in Morton order
 *   label, level, parent, first, count, first_child, nchild per node
 *   mass, mx, my, mz (sums), cx, cy, cz (COM), size s_node
 * Nodes are numbered breadth first: by level, then by key prefix.
 * Returns the number of nodes, or -1 if max_nodes is too small. */
int64_t orc_build_tree(int64_t n, const double *x, const double *y, const double *z, const double *m,
                       const double *box, int leaf_max, int64_t max_nodes, int64_t *perm,
                       uint64_t *label, int32_t *level, int64_t *parent, int64_t *first,
                       int64_t *count, int64_t *first_child, int32_t *nchild, double *mass,
                       double *mx, double *my, double *mz, double *cx, double *cy, double *cz,
                       double *size)
{
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    kv *s = (kv *)malloc(sizeof(kv) * (n ? n : 1));
    orc_morton_keys(n, x, y, z, box, key);
    for (int64_t i = 0; i < n; ++i) { s[i].key = key[i]; s[i].idx = i; }
    qsort(s, (size_t)n, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < n; ++i) { perm[i] = s[i].idx; key[i] = s[i].key; }
    free(s);

    int64_t nn = 1;
    label[0] = 1; level[0] = 0; parent[0] = -1; first[0] = 0; count[0] = n;
    for (int64_t a = 0; a < nn; ++a) {
        first_child[a] = -1;
        nchild[a] = 0;
        if (count[a] <= leaf_max || level[a] >= MORTON_BITS) continue;
        int shift = 3 * (MORTON_BITS - 1 - level[a]);
        int64_t b = first[a], e = first[a] + count[a];
        first_child[a] = nn;
        for (int oct = 0; oct < 8; ++oct) {
            int64_t c0 = b;
            while (b < e && (int)((key[b] >> shift) & 7ull) == oct) ++b;
            if (b == c0) continue;
            if (nn >= max_nodes) { free(key); return -1; }
            label[nn] = label[a] * 8ull + (uint64_t)oct;
            level[nn] = level[a] + 1;
            parent[nn] = a;
            first[nn] = c0;
            count[nn] = b - c0;
            nchild[a] += 1;
            ++nn;
        }
    }
    for (int64_t a = nn - 1; a >= 0; --a) {
        double sm = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        if (nchild[a] == 0) {
            for (int64_t k = first[a]; k < first[a] + count[a]; ++k) {
                int64_t i = perm[k];
                sm += m[i];
                sx += m[i] * x[i];
                sy += m[i] * y[i];
                sz += m[i] * z[i];
            }
        } else {
            for (int64_t c = first_child[a]; c < first_child[a] + nchild[a]; ++c) {
                sm += mass[c]; sx += mx[c]; sy += my[c]; sz += mz[c];
            }
        }
        mass[a] = sm; mx[a] = sx; my[a] = sy; mz[a] = sz;
        cx[a] = sx / sm; cy[a] = sy / sm; cz[a] = sz / sm;
        double r2max = 0.0;
        for (int64_t k = first[a]; k < first[a] + count[a]; ++k) {
            int64_t i = perm[k];
            double dx = x[i] - cx[a], dy = y[i] - cy[a], dz = z[i] - cz[a];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > r2max) r2max = r2;
        }
        size[a] = sqrt(r2max);
    }
    free(key);
    return nn;
}

/* Adaptive tree-walk (Section 2.4.1).  Emits pseudo-particles in walk order
 * (depth first, children in octant order = Morton order):
 *   kind[k] = 0: node pseudo-particle, ref[k] = node index
 *   kind[k] = 1: individual particle, ref[k] = its position in Morton order
 * and the h-solver population (selected nodes plus the leaves whose particles
 * were extracted), pop_node[]: node indices in the same order.
 * Returns the number of pseudo-particles (npop in *npop_out), or -1 on overflow. */
/* The adaptive tree-walk (Section 2.4.1, Eq. 4).  force (one byte per node,
 * may be NULL) marks nodes that the refinement check of Eq. 5 found
 * under-resolved: such an internal node is opened, such a leaf has its
 * particles extracted, whatever the distance criteria say. */
int64_t orc_select(int64_t nnode, const int32_t *nchild, const int64_t *first_child, const int64_t *first,
                   const int64_t *count, const double *cx, const double *cy, const double *cz,
                   const double *size, int nsrc, const double *src, double r_part, double r_leaf,
                   double theta, int64_t max_out, int32_t *kind, int64_t *ref, int64_t *pop_node,
                   int64_t *npop_out, const uint8_t *force)
{
    (void)nnode;
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * 8 * 64 + sizeof(int64_t));
    int64_t sp = 0, nout = 0, npop = 0;
    stack[sp++] = 0;
    double rp2 = r_part * r_part, rl2 = r_leaf * r_leaf, th2 = theta * theta;
    while (sp > 0) {
        int64_t a = stack[--sp];
        double r2 = INFINITY;
        for (int s = 0; s < nsrc; ++s) {
            double dx = cx[a] - src[3 * s], dy = cy[a] - src[3 * s + 1], dz = cz[a] - src[3 * s + 2];
            double q = dx * dx + dy * dy + dz * dz;
            if (q < r2) r2 = q;
        }
        int open;
        const int forced = force != NULL && force[a] != 0;
        if (nchild[a] == 0) {
            if (r2 < rp2 || forced) {
                if (nout + count[a] > max_out) { free(stack); return -1; }
                for (int64_t k = first[a]; k < first[a] + count[a]; ++k) {
                    kind[nout] = 1; ref[nout] = k; ++nout;
                }
                pop_node[npop++] = a;
                continue;
            }
            open = 0;
        } else {
            open = forced || (r2 < rl2) || (size[a] * size[a] > th2 * r2);
        }
        if (open) {
            for (int64_t c = first_child[a] + nchild[a] - 1; c >= first_child[a]; --c) stack[sp++] = c;
        } else {
            if (nout >= max_out) { free(stack); return -1; }
            kind[nout] = 0; ref[nout] = a; ++nout;
            pop_node[npop++] = a;
        }
    }
    free(stack);
    *npop_out = npop;
    return nout;
}

/* n(h) = sum over the whole population of W(|x_a - x_b|, h) and its h-derivative */
static void number_density(int64_t npop, const double *px, const double *py, const double *pz,
                           const double *xa, double h, double *n, double *dn)
{
    double s = 0.0, ds = 0.0;
    for (int64_t b = 0; b < npop; ++b) {
        double dx = px[b] - xa[0], dy = py[b] - xa[1], dz = pz[b] - xa[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        s += orc_W(r, h);
        ds += orc_dWdh(r, h);
    }
    *n = s;
    *dn = ds;
}

/* f(h) = h_fact n^(-1/3) - h  (Eq. 8) */
static double f_of_h(int64_t npop, const double *px, const double *py, const double *pz, const double *xa,
                     double h, double h_fact)
{
    double n, dn;
    number_density(npop, px, py, pz, xa, h, &n, &dn);
    return h_fact * pow(n, -1.0 / 3.0) - h;
}

/* Solve h for targets (positions tx, ty, tz; initial guesses h0).  status:
 * 0 Newton converged, 1 bisection, 2 fallback to h0.  iters: Newton steps. */
void orc_h_solve(int64_t npop, const double *px, const double *py, const double *pz, int64_t ntgt,
                 const double *tx, const double *ty, const double *tz, const double *h0, double h_fact,
                 double tol, int max_newton, double *h_out, int32_t *status, int32_t *iters,
                 int nthreads)
{
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t a = 0; a < ntgt; ++a) {
        double xa[3] = {tx[a], ty[a], tz[a]};
        double h = h0[a];
        int ok = 0, it = 0;
        for (it = 0; it < max_newton; ++it) {
            double n, dn;
            number_density(npop, px, py, pz, xa, h, &n, &dn);
            double f = h_fact * pow(n, -1.0 / 3.0) - h;
            double fp = -h_fact * dn * pow(n, -4.0 / 3.0) / 3.0 - 1.0;     /* Eq. 9 */
            double hn = h - f / fp;                                         /* Eq. 10 */
            /* an iterate outside the bisection bracket counts as a Newton failure */
            if (!(hn >= 1e-2 * h0[a] && hn <= 1e2 * h0[a])) break;
            double step = fabs(hn - h) / h0[a];
            h = hn;
            if (step < tol) { ok = 1; ++it; break; }
        }
        iters[a] = it;
        if (ok) { h_out[a] = h; status[a] = 0; continue; }
        double lo = 1e-2 * h0[a], hi = 1e2 * h0[a];
        double flo = f_of_h(npop, px, py, pz, xa, lo, h_fact);
        double fhi = f_of_h(npop, px, py, pz, xa, hi, h_fact);
        if (flo * fhi > 0.0) { h_out[a] = h0[a]; status[a] = 2; continue; }
        for (int k = 0; k < 200 && (hi - lo) > tol * h0[a]; ++k) {
            double mid = 0.5 * (lo + hi);
            double fm = f_of_h(npop, px, py, pz, xa, mid, h_fact);
            if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        h_out[a] = 0.5 * (lo + hi);
        status[a] = 1;
    }
}
