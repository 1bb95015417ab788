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
// integrated by 8-point Gauss-Legendre on pieces of length <= 2 in s, split
// at the kernel's breakpoints Q = 1 and Q = 2.  Beyond Q = 2, K~(Q) = 0 and
// the piece is -K~(R) times an angle, taken analytically.
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
//   R < 1 <= Q: the difference is split at Q = 1, the constant
//              K(1) - K(R) taken in FP64;
// where d = Q^2 - R^2 = c + tau^2 with c = A^2 - rho^2 per edge in FP64
// (rho the in-plane distance from the foot to the polygon),
// S4(u, v) = u^3 + u^2 v + u v^2 + v^3, S5(Q, R) = Q^4 + Q^3 R + ... + R^4,
// and u = 2 - Q = (4 - Q^2)/(2 + Q).  tau = A sinh(s) is formed from expm1
// so that it keeps its relative precision near s = 0.
//
// The same quadrature integrates the full kernel (K instead of K~) for a
// particle inside a cell that lies entirely within 2h of it.
#pragma once

#include <cuda_runtime.h>

namespace emq {

__device__ __forceinline__ float gl_x(int i)
{
    return i == 0 ? 0.18343464249564978f : i == 1 ? 0.52553240991632899f : i == 2 ? 0.79666647741362673f
                                                                                  : 0.96028985649753618f;
}
__device__ __forceinline__ float gl_w(int i)
{
    return i == 0 ? 0.36268378337836166f : i == 1 ? 0.31370664587788688f : i == 2 ? 0.22238103445337443f
                                                                                  : 0.10122853629037706f;
}

// Reference data of one face: R (distance to the polygon, units of h),
// powers of R and of v = 2 - R, K(R) (or K~(R)) and, for R < 1, the constant
// K(1) - K(R), all from FP64.
struct FaceRef {
    float R, R2, R3, R4;
    float v, v2, v3, v4;
    float KR, C1;
    bool tilde;   // complement kernel K~ (false: full kernel K)
};
// Per-edge constants from FP64: c = A^2 - rho^2, c1 = B^2 - 1, c4 = 4 - B^2.
struct EdgeRef {
    float cc, c1, c4;
};

// K~2(Q) - K~2(Rr) for Q, Rr in [1, 2); u = 2 - Q, v = 2 - Rr, d = Q^2 - Rr^2
__device__ __forceinline__ float dkt2(float Q, float iQ, float u, float d, float Rr, float v, float v2, float v3,
                                      float v4)
{
    const float S4 = ((u + v) * u + v2) * u + v3;
    const float br = u * S4 * (1.f + iQ) + v4 * (1.f + __fdividef(2.f * iQ, Rr));
    return __fdividef(d, 120.f * (Q + Rr)) * br;
}

// K(Q) - K(R) (K~ or K) at one node; piece 1: Q < 1, piece 2: 1 <= Q < 2
__device__ __forceinline__ float dk(float Q, float t2, bool piece1, const FaceRef &fr, const EdgeRef &er)
{
    if (piece1) {
        const float d = er.cc + t2;
        const float iq = __fdividef(1.f, Q + fr.R);
        const float s5 = (((Q + fr.R) * Q + fr.R2) * Q + fr.R3) * Q + fr.R4;
        const float phf = (1.f / 6.f) - 0.075f * (Q * Q + fr.R2) + 0.025f * s5 * iq;
        return fr.tilde ? d * (__fdividef(0.25f * iq, Q * fr.R) - phf) : d * phf;
    }
    const float iQ = __fdividef(1.f, Q);
    const float u = __fdividef(er.c4 - t2, 2.f + Q);
    if (fr.R >= 1.f) {
        const float d = er.cc + t2;
        const float x = dkt2(Q, iQ, u, d, fr.R, fr.v, fr.v2, fr.v3, fr.v4);
        return fr.tilde ? x : __fdividef(d * iQ, 4.f * fr.R * (Q + fr.R)) - x;
    }
    const float d1 = er.c1 + t2;
    const float x = dkt2(Q, iQ, u, d1, 1.f, 1.f, 1.f, 1.f, 1.f);
    return (fr.tilde ? x : __fdividef(d1 * iQ, 4.f * (Q + 1.f)) - x) + fr.C1;
}

// int_{sa}^{sb} [K(Q(s)) - K(R)] / cosh(s) ds on one kernel piece
__device__ __forceinline__ float seg(float sa, float sb, float A, float B2, bool piece1, const FaceRef &fr,
                                     const EdgeRef &er)
{
    const float len = sb - sa;
    const int m = len > 2.f ? (int)ceilf(0.5f * len) : 1;
    const float hl = 0.5f * len / (float)m;
    float tot = 0.f;
    for (int p = 0; p < m; ++p) {
        const float mid = sa + (2.f * p + 1.f) * hl;
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float s = mid + ((i & 1) ? -hl : hl) * gl_x(i >> 1);
            const float em = expm1f(s);
            const float e = 1.f + em;
            const float ei = __fdividef(1.f, e);
            const float ch = 0.5f * (e + ei);
            const float tau = 0.5f * A * (em * (1.f + ei));
            const float t2 = tau * tau;
            const float Q = sqrtf(B2 + t2);
            acc += gl_w(i >> 1) * __fdividef(dk(Q, t2, piece1, fr, er), ch);
        }
        tot += acc * hl;
    }
    return tot;
}

// (D/pi) int over |tau| in [ua, ub] of [K(Q) - K(R)] A/(A^2 + tau^2) dtau (>= 0)
__device__ __forceinline__ float g_int(float ua, float ub, float A, float D, float B2, const FaceRef &fr,
                                       const EdgeRef &er)
{
    const float t1 = er.c1 < 0.f ? sqrtf(-er.c1) : 0.f;
    const float t2 = er.c4 > 0.f ? sqrtf(er.c4) : 0.f;
    const float iA = 1.f / A;
    float tot = 0.f;
    {
        float a = ua, b = fminf(ub, t1);
        if (b > a) tot += seg(asinhf(a * iA), asinhf(b * iA), A, B2, true, fr, er);
    }
    {
        float a = fmaxf(ua, t1), b = fminf(ub, t2);
        if (b > a) tot += seg(asinhf(a * iA), asinhf(b * iA), A, B2, false, fr, er);
    }
    if (fr.tilde) {   // beyond 2h: K~(Q) = 0, so the integrand is -K~(R) >= 0
        float a = fmaxf(ua, t2), b = ub;
        if (b > a) tot -= fr.KR * atan2f((b - a) * A, A * A + a * b);
    }
    return tot * D * 0.31830988618379067154f;
}

// Edge from T0 to T1 along its line (signed, tau measured from the foot F).
// Returns the signed edge integral; mag receives the sum of the magnitudes
// of the non-negative pieces it is made of.
__device__ __forceinline__ float edge_q(float D, float A, float T0, float T1, float B2, const FaceRef &fr,
                                        const EdgeRef &er, float &mag)
{
    if ((T0 >= 0.f && T1 >= 0.f) || (T0 <= 0.f && T1 <= 0.f)) {
        float u0 = fabsf(T0), u1 = fabsf(T1);
        float v = g_int(fminf(u0, u1), fmaxf(u0, u1), A, D, B2, fr, er);
        mag = v;
        return T1 >= T0 ? v : -v;
    }
    float v = g_int(0.f, fabsf(T0), A, D, B2, fr, er) + g_int(0.f, fabsf(T1), A, D, B2, fr, er);
    mag = v;
    return T1 > T0 ? v : -v;
}

}  // namespace emq
