/*
 * Test infrastructure -- algorithmic work of the oracle's closed form, per
 * pair: the right sub-triangles it evaluates, its FP64 additions and
 * subtractions, multiplications, divisions, square roots and transcendental
 * calls (atan2, asinh, pow).  Only tests/ and the oracle's own scripts use it.
 *
 * exact.c is compiled a second time here, unchanged, with every `double`
 * replaced by a number type whose operators count themselves and then do the
 * same IEEE operation (one rounding per operation, nothing fused), so the
 * weights come out bit-identical to the oracle's and the counts are those of
 * the code that computed them.  Comparisons, negation and fabs are not
 * counted.  The counters are per thread; each pair resets them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

namespace {

struct Counts {
    unsigned long long tri, add, mul, div, sqrt_, trans;
};
thread_local Counts g_cnt;

struct cnum {
    double v;
    cnum() : v(0.0) {}
    cnum(double x) : v(x) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator long long() const { return (long long)v; }
    cnum operator-() const { return cnum(-v); }
    cnum &operator+=(cnum o) { ++g_cnt.add; v = v + o.v; return *this; }
    cnum &operator-=(cnum o) { ++g_cnt.add; v = v - o.v; return *this; }
    cnum &operator*=(cnum o) { ++g_cnt.mul; v = v * o.v; return *this; }
    cnum &operator/=(cnum o) { ++g_cnt.div; v = v / o.v; return *this; }
};
inline cnum operator+(cnum a, cnum b) { ++g_cnt.add; return cnum(a.v + b.v); }
inline cnum operator-(cnum a, cnum b) { ++g_cnt.add; return cnum(a.v - b.v); }
inline cnum operator*(cnum a, cnum b) { ++g_cnt.mul; return cnum(a.v * b.v); }
inline cnum operator/(cnum a, cnum b) { ++g_cnt.div; return cnum(a.v / b.v); }
inline bool operator<(cnum a, cnum b) { return a.v < b.v; }
inline bool operator>(cnum a, cnum b) { return a.v > b.v; }
inline bool operator<=(cnum a, cnum b) { return a.v <= b.v; }
inline bool operator>=(cnum a, cnum b) { return a.v >= b.v; }
inline bool operator==(cnum a, cnum b) { return a.v == b.v; }
inline bool operator!=(cnum a, cnum b) { return a.v != b.v; }
inline cnum sqrt(cnum a) { ++g_cnt.sqrt_; return cnum(std::sqrt(a.v)); }
inline cnum fabs(cnum a) { return cnum(std::fabs(a.v)); }
inline cnum floor(cnum a) { return cnum(std::floor(a.v)); }
inline cnum fmax(cnum a, cnum b) { return cnum(std::fmax(a.v, b.v)); }
inline cnum fmin(cnum a, cnum b) { return cnum(std::fmin(a.v, b.v)); }
inline cnum asinh(cnum a) { ++g_cnt.trans; return cnum(std::asinh(a.v)); }
inline cnum atan2(cnum a, cnum b) { ++g_cnt.trans; return cnum(std::atan2(a.v, b.v)); }
inline cnum pow(cnum a, cnum b) { ++g_cnt.trans; return cnum(std::pow(a.v, b.v)); }
inline cnum log(cnum a) { ++g_cnt.trans; return cnum(std::log(a.v)); }
inline cnum exp(cnum a) { ++g_cnt.trans; return cnum(std::exp(a.v)); }
inline cnum cos(cnum a) { ++g_cnt.trans; return cnum(std::cos(a.v)); }
inline cnum sin(cnum a) { ++g_cnt.trans; return cnum(std::sin(a.v)); }
inline cnum acos(cnum a) { ++g_cnt.trans; return cnum(std::acos(a.v)); }

#define ORC_COUNT_TRIANGLE() (++g_cnt.tri)
#define double cnum
#include "exact.c"
#undef double

}  // namespace

/* For each pair: w (FP64, as the oracle's orc_map_exact) and six counts:
 * right sub-triangles, add/sub, mul, div, sqrt, transcendental calls. */
extern "C" __attribute__((visibility("default"))) void orc_count_map_exact(
    int64_t npair, const int64_t *pair_i, const int64_t *pair_j, const double *x, const double *y,
    const double *z, const double *h, const int64_t *cell_face_off, const int64_t *face_vert_off,
    const double *verts, const double *normals, double *w, unsigned long long *counts, int nthreads)
{
    const cnum *cv = reinterpret_cast<const cnum *>(verts);
    const cnum *cn = reinterpret_cast<const cnum *>(normals);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int64_t k = 0; k < npair; ++k) {
        const int64_t i = pair_i[k], j = pair_j[k];
        const cnum p[3] = {x[i], y[i], z[i]};
        const int64_t f0 = cell_face_off[j], f1 = cell_face_off[j + 1];
        g_cnt = Counts{0, 0, 0, 0, 0, 0};
        w[k] = orc_cell_weight(p, cnum(h[i]), (int)(f1 - f0), face_vert_off + f0, cv, cn + 3 * f0).v;
        unsigned long long *c = counts + 6 * k;
        c[0] = g_cnt.tri;
        c[1] = g_cnt.add;
        c[2] = g_cnt.mul;
        c[3] = g_cnt.div;
        c[4] = g_cnt.sqrt_;
        c[5] = g_cnt.trans;
    }
}
