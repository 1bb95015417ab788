// FP32 evaluation of the per-edge pyramid integral for the mixed-precision
// path of map_exact.
//
// The right-triangle pyramid integral of the complement kernel G~ =
// 1/(4 pi) - G (zero beyond 2h) over the edge segment tau in [T0, T1] is
//     (D/pi) int [K~(Q(tau)) - K~(R)] A/(A^2 + tau^2) dtau,
//     Q(tau)^2 = B^2 + tau^2 = D^2 + A^2 + tau^2,
// with R the distance from the particle to the face polygon (in units of h):
// the reference K~(R) instead of K~(D) drops K~(D) - K~(R) times the
// polygon's winding angle seen from P, which is zero when P is outside the
// polygon (and R = D when it is inside).  With this reference every edge
// integrand is non-negative and no O(1) terms cancel down to small weights.
//
// Substituting tau = A sinh(s) turns A dtau/(A^2 + tau^2) into ds/cosh(s):
//     (D/pi) int [K~(Q(s)) - K~(R)] / cosh(s) ds,  Q(s)^2 = D^2 + A^2 cosh^2 s,
// an integrand that is smooth on the scale of s = 1 however small A is; it is
// integrated by Gauss-Legendre on sub-pieces of length <= 2 in s (8 points;
// 4 for a segment of length <= 1/8, see SEG_GL4), split at the kernel's
// breakpoints Q = 1 and Q = 2.  Beyond Q = 2, K~(Q) = 0
// and the piece is -K~(R) times an angle, taken analytically.
//
// Every piece of the integrand K(Q) - K(R) is formed as an exact factored
// difference, so that its FP32 value keeps a relative error of a few ulp
// even where K(Q) and K(R) nearly cancel (Q close to R over the whole face,
// which happens when the foot of the perpendicular is inside the polygon and
// the difference is integrated over the full winding angle):
//   Q, R < 1:  K1(Q) - K1(R) = d [1/6 - 3 (Q^2 + R^2)/40 + S5(Q, R)/(40 (Q + R))]
//              K~1 = -1/(4Q) + 7/20 - K1 adds d/(4 Q R (Q + R));
//   Q, R in [1, 2):  with u = 2 - Q, v = 2 - R, K~2(Q) = -u^5 (1 + Q)/(120 Q),
//              K~2(Q) - K~2(R) = d/(120 (Q + R)) [u S4(u, v) (1 + 1/Q)
//                                                  + v^4 (1 + 2/(Q R))],
//              a sum of positive terms, and K2 = K3 - K~2 with
//              K3(Q) - K3(R) = d/(4 Q R (Q + R));
//   R < 1 <= Q: the difference is split at Q = 1 (the same formula with R
//              replaced by 1), the constant K(1) - K(R) taken in FP64;
// where d = Q^2 - R^2 = c + tau^2 with c = A^2 - rho^2 per edge in float-float
// (rho the in-plane distance from the foot to the polygon), evaluated at each
// node relative to the segment's start (see the segment fields below),
// S4(u, v) = u^3 + u^2 v + u v^2 + v^3, S5(Q, R) = Q^4 + Q^3 R + ... + R^4,
// and u = 2 - Q = (4 - Q^2)/(2 + Q).  sinh and cosh of a node's offset from
// its segment's start are formed from expm1, so that they keep their relative
// precision for small offsets.
//
// The same quadrature integrates the full kernel (K instead of K~) for a
// particle inside a cell that lies entirely within 2h of it.
//
// Work is organised in segments: one segment is one kernel piece of one edge
// (an s-interval cut into m sub-pieces) with everything its integrand needs.
// A warp evaluates the segments of 32 different pairs side by side in slots
// of 4 nodes, one slot per lane, with one copy of the node loop.
#pragma once

#include <cuda_runtime.h>

#include "split.cuh"

#ifndef EM_NODE_UNROLL
#define EM_NODE_UNROLL 2   // unroll of the 8-node loop (build-time tuning knob)
#endif

namespace emq {

constexpr int kNodeUnroll = EM_NODE_UNROLL;

// e^x - 1 in FP32 for |x| <= 80, within about 1.5 ulp, at about half the
// issue slots of the library call (the pass evaluates one per quadrature
// node).  Cody and Waite's reduction x = k ln2 + r, |r| <= ln2/2, with ln2
// split into a head of 12 significant bits (so k ln2_hi is exact for
// |k| < 2^12) and the tail; e^r - 1 by its Taylor series to r^7/7!
// (truncation r^8/8! <= 5.1e-9, a quarter ulp of e^r - 1 at |r| = ln2/2),
// r + r^2 (1/2 + r (1/6 + ...)) so that the leading term stays exact; then
// e^x - 1 = 2^k (e^r - 1) + (2^k - 1), one fused multiply-add, 2^k - 1
// exact for |k| <= 24 and the sum rounded once.
__device__ __forceinline__ float ex_m1(float x)
{
    const float ln2_hi = 0.693145751953125f;           // 2839 / 4096
    const float ln2_lo = 1.4286068203094172e-06f;      // ln 2 - ln2_hi
    const float k = rintf(x * 1.4426950408889634f);   // x / ln 2, nearest integer
    float r = fmaf(-k, ln2_hi, x);
    r = fmaf(-k, ln2_lo, r);
    float p = fmaf(r, 1.f / 5040.f, 1.f / 720.f);
    p = fmaf(r, p, 1.f / 120.f);
    p = fmaf(r, p, 1.f / 24.f);
    p = fmaf(r, p, 1.f / 6.f);
    p = fmaf(r, p, 0.5f);
    p = fmaf(r * r, p, r);                              // e^r - 1
    const float s = __int_as_float(((int)k + 127) << 23);   // 2^k
    return fmaf(s, p, s - 1.f);
}

// sqrt(x) for x >= 0 within 1 ulp, at about two thirds of the issue slots
// of the correctly rounded call: x rsqrt(x) and one Newton step on y^2 = x
// with 1/(2y) taken as rsqrt(x)/2.  A subnormal x is scaled by 2^48 first
// (its root by 2^-24 after), since the reciprocal square root does not
// resolve it; 0 gives 0.
__device__ __forceinline__ float sqrt_nr(float x)
{
    const bool tiny = x < 1.17549435e-38f;                // below FP32's normal range
    const float xs = tiny ? x * 281474976710656.f : x;    // 2^48
    const float r = rsqrtf(xs);
    const float y = xs * r;
    const float s = fmaf(0.5f * r, fmaf(-y, y, xs), y);
    return x > 0.f ? (tiny ? s * 5.9604644775390625e-8f : s) : 0.f;   // 2^-24
}

// Gauss-Legendre rules on [-1, 1], by their positive abscissae and weights
// (the rules are symmetric), in two-node halves: half 0 and half 1 of the
// 8-point rule, and the 4-point rule.  A "slot" is one half: 4 nodes.
__device__ __forceinline__ void rule_half(int r, float &x0, float &w0, float &x1, float &w1)
{
    x0 = r == 0 ? 0.18343464249564978f : (r == 1 ? 0.79666647741362673f : 0.33998104358485626f);
    w0 = r == 0 ? 0.36268378337836166f : (r == 1 ? 0.22238103445337443f : 0.65214515486254614f);
    x1 = r == 0 ? 0.52553240991632899f : (r == 1 ? 0.96028985649753618f : 0.86113631159405258f);
    w1 = r == 0 ? 0.31370664587788688f : (r == 1 ? 0.10122853629037706f : 0.34785484513745386f);
}

// Segment fields (see the header comment):
//   ts      tau at the segment's start (>= 0); the segment runs from there to
//           larger |tau|, s = asinh(tau / A) from s(ts)
//   Sa, Ca  sinh and cosh of s(ts): ts / A and sqrt(1 + (ts/A)^2)
//   hl      half-length in s of every sub-piece
//   A, B2   A and B^2 of the edge
//   es      Q^2 - Rr^2 at ts (float-float sum, rounded once; >= 0)
//   c4s     4 - Q^2 at ts (piece 2)
//   Rr      reference distance of the difference (R, or 1)
//   v       2 - Rr, computed where it keeps its relative precision (piece 2)
//   add     constant added to the difference: K(1) - K(R) when Rr = 1, else 0
//   meta    m | piece1 << 8 | tilde << 9 | gl4 << 10, m the number of sub-pieces
// Each node is placed by its offset delta in s from the segment's start, and
// everything that cancels is formed from that offset: tau - ts =
// A (Sa (cosh delta - 1) + Ca sinh delta), Q^2 - Rr^2 = es + (tau - ts)(tau + ts)
// and 4 - Q^2 = c4s - (tau - ts)(tau + ts), sums whose terms do not cancel.
// Forming tau^2 itself and subtracting a constant near it instead loses
// about 2^-24 tau^2 absolutely, which for a small face seen from afar (Q ~ R
// over the whole face) is many ulps of Q^2 - R^2.
// The rule: within a piece the integrand is analytic in the strip
// |Im s| < pi/2 (its singularities are the branch points of Q(s), where
// B^2 + A^2 sinh^2 s = 0 with B >= A, and the poles of 1/cosh s; the kernel's
// breakpoints are piece boundaries), so an n-point Gauss-Legendre rule on a
// sub-piece of length L converges like rho^(-2n), rho = pi/L + sqrt(1 +
// (pi/L)^2) the Bernstein ellipse that fits in the strip.  Sub-pieces of
// length <= 2 take 8 points.  A short segment takes 4 points as one
// sub-piece; the integrand's size near the strip's edge (Q ~ D for a particle
// close to the face plane) makes the constant large, so the length limit is
// set by measurement against the FP64 closed form over every pair: 1/2 and 1/4
// leave errors of 3e-4 and 1e-4 |w|, 1/8 (the limit used, EM_GL4_MAXLEN)
// none that the 8-point rule does not also have.
constexpr int SEG_PIECE1 = 1 << 8;
constexpr int SEG_TILDE = 1 << 9;
constexpr int SEG_GL4 = 1 << 10;

// One slot: int over the 4 nodes off +- hl x0, off +- hl x1 (offsets from the
// segment's start) of half r of the rule (see rule_half) of
// [K(Q(s)) - K(R)] / cosh(s) ds.  Q and 1/Q come from one reciprocal square
// root and a Newton step (about 1 ulp); the other quotients are reciprocals of
// quantities bounded away from zero.
__device__ __forceinline__ float slot_eval(float off, float hl, int r, float ts, float Sa, float Ca, float A,
                                           float B2, float c4s, float es, float Rr, float vr, float add, int meta)
{
    const bool piece1 = (meta & SEG_PIECE1) != 0;
    const bool tilde = (meta & SEG_TILDE) != 0;
    const float R2 = Rr * Rr;
    // piece 1: powers of R; piece 2: powers of v = 2 - Rr
    const float v = piece1 ? Rr : vr;
    const float p2 = v * v, p3 = p2 * v, p4 = p2 * p2;
    const float iRr = __fdividef(1.f, Rr);   // Rr >= 1e-30 wherever it is used
    const float ts2 = 2.f * ts;
    float x0, w0, x1, w1;
    rule_half(r, x0, w0, x1, w1);
    float acc = 0.f;
#pragma unroll kNodeUnroll
    for (int i = 0; i < 4; ++i) {
        const float xi = (i >> 1) ? x1 : x0, wi = (i >> 1) ? w1 : w0;
        const float dl = fmaf((i & 1) ? -hl : hl, xi, off);   // offset from the start, > 0
        const float em = ex_m1(dl);
        const float ei = __fdividef(1.f, 1.f + em);
        const float sh = 0.5f * em * (1.f + ei);    // sinh delta
        const float cm = 0.5f * em * em * ei;       // cosh delta - 1
        const float dt = A * fmaf(Sa, cm, Ca * sh);   // tau - ts
        const float ch = fmaf(Ca, cm, fmaf(Sa, sh, Ca));   // cosh s
        const float tau = ts + dt;
        const float q2 = fmaf(tau, tau, B2);
        float iQ = rsqrtf(q2);
        iQ = iQ * fmaf(-0.5f * q2 * iQ, iQ, 1.5f);
        const float Q = q2 * iQ;
        const float dq = dt * (ts2 + dt);           // Q^2 - Q(ts)^2
        const float d = es + dq;
        const float iq = __fdividef(1.f, Q + Rr);
        float f;
        if (piece1) {
            const float s5 = (((Q + Rr) * Q + p2) * Q + p3) * Q + p4;
            const float phf = (1.f / 6.f) - 0.075f * (Q * Q + R2) + 0.025f * s5 * iq;
            f = tilde ? d * ((0.25f * iq) * iQ * iRr - phf) : d * phf;
        } else {
            const float u = __fdividef(c4s - dq, 2.f + Q);
            const float S4 = ((u + v) * u + p2) * u + p3;
            const float br = u * S4 * (1.f + iQ) + p4 * (1.f + 2.f * iQ * iRr);
            const float x = d * iq * (1.f / 120.f) * br;
            f = (tilde ? x : d * iQ * (0.25f * iRr) * iq - x) + add;
        }
        acc += wi * __fdividef(f, ch);
    }
    return acc * hl;
}

// ---------------------------------------------------------------------------
// Float-float arithmetic (a value held as hi + lo, two FP32 numbers), for the
// per-edge geometry of the FP32 pass: with the error-free transformations of
// Knuth (two-sum) and of the FMA product (two-prod), a dot product of
// float-float operands is accurate to about 2^-48 of its terms, far below
// the single FP32 rounding the quadrature's inputs need, at a fraction of the
// cost of FP64 on a part whose FP64 rate is 1/64 of its FP32 rate.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float v = s - a;
    return ff{s, (a - (s - v)) + (b - v)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    const float p = a * b;
    return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const ff p = ff_two_prod(x.hi, y.hi);
    return ff_two_sum(p.hi, p.lo + fmaf(x.hi, y.lo, x.lo * y.hi));
}
// v as hi = (float)v and lo = (float)(v - hi), formed on the bits
// (split.cuh): the conversions would issue at the FP64 rate
__device__ __forceinline__ ff ff_from_double(double v)
{
    ff r;
    em::split_df(v, r.hi, r.lo);
    return r;
}
// c - (mx rx + my ry + mz rz), every operand float-float
__device__ __forceinline__ ff ff_offset_dot(float ch, float cl, float mxh, float mxl, float myh, float myl, float mzh,
                                            float mzl, ff rx, ff ry, ff rz)
{
    const ff p0 = ff_two_prod(mxh, rx.hi), p1 = ff_two_prod(myh, ry.hi), p2 = ff_two_prod(mzh, rz.hi);
    float lo = (p0.lo + p1.lo) + p2.lo;
    lo += fmaf(mxh, rx.lo, mxl * rx.hi) + fmaf(myh, ry.lo, myl * ry.hi) + fmaf(mzh, rz.lo, mzl * rz.hi);
    const ff s1 = ff_two_sum(p0.hi, p1.hi);
    const ff s2 = ff_two_sum(s1.hi, p2.hi);
    lo += s1.lo + s2.lo;
    const ff d = ff_two_sum(ch, -s2.hi);
    return ff_two_sum(d.hi, d.lo + (cl - lo));
}

}  // namespace emq
