// Analytic integral of the M4 kernel over a convex cell (Exact mapping).
//
// The weight w = int_V W(|r - p|, h) d^3r is split (signed cone
// decomposition) into pyramids from p over the faces, and each face into
// triangles (P, V_k, V_k+1) from the foot P of the perpendicular, each split
// at the foot F on the edge line into two right triangles.  In units of h,
// with D = distance from p to the face plane, A = |PF|, B^2 = D^2 + A^2 and
// tau the coordinate along the edge line from F, the pyramid over the right
// triangle reaching tau = T is
//     (1/pi) int_0^T [K(Q(tau)) - K(D)] D A / (A^2 + tau^2) dtau,
//     Q(tau) = sqrt(B^2 + tau^2),
// where K(Q) = int g(Q)/Q^2 dQ and g(Q) = int_0^Q w(q) q^2 dq is the kernel's
// radial cumulative (G(R) = g(R/h)/pi).  K is a polynomial in Q and 1/Q on each
// kernel region (Q < 1, 1 <= Q < 2, Q >= 2), so the integral is a fixed
// combination of six basis functions of tau:
//   b0 = D atan(tau/A)                         b1 = atan(D tau / (A Q))
//   b2 = D J2, b3 = D J3, b4 = D J4, b5 = D J5 with
//   J2 = A tau + D^2 atan(tau/A),   J4 = A (A^2 tau + tau^3/3) + 2 D^2 A tau + D^4 atan(tau/A)
//   J1 = A asinh(tau/B) + D b1,     J3 = A U1 + D^2 J1,  J5 = A U3 + D^2 J3
//   U1 = (tau Q + B^2 asinh(tau/B))/2, U3 = tau Q^3/4 + 3 B^2 U1/4.
// Region coefficient vectors c_r (basis order b0..b5):
//   c1 = (0, 0, 1/6, 0, -3/40, 1/40)
//   c2 = (-1/20, 1/60, 1/3, -1/4, 3/40, -1/120)
//   c3 = (7/20, -1/4, 0, 0, 0, 0)
// The -K(D) atan(tau/A) part (-K(D) b0/D times D) is applied at every
// endpoint, so that it cancels against the same endpoint's terms; summing it
// per face instead (2 pi K(D)
// when P is inside the polygon) would rely on the edge angles closing to 2 pi,
// which rounded vertices break by up to ~1e-12 when P lies near an edge line.
//
// Two equivalent forms are evaluated:
//   full:       w = (1/pi) sum_f sigma_f F_f with K as above;
//   complement: w = [p in V] - (1/pi) sum_f sigma_f F~_f with K~ = K3 - K,
//               the integral of G~ = 1/(4 pi) - G, which vanishes beyond 2h,
//               so faces at D >= 2 and edges at B >= 2 contribute nothing.
// The complement form relies on the face solid angles summing to exactly
// 4 pi [p in V]; with rounded vertices this closure is off by up to ~1e-13
// near tiny faces, so FP64 uses the full form throughout.  The FP32 pass uses
// the complement form (far smaller rounding for particles outside the cell)
// unless p is inside a cell that lies entirely within 2h of it.
#pragma once

#include <cuda_runtime.h>

namespace em {

template <class T>
struct Consts;
template <>
struct Consts<double> {
    static constexpr double inv_pi = 0.31830988618379067154;
    static constexpr double two_pi = 6.28318530717958647692;
};
template <>
struct Consts<float> {
    static constexpr float inv_pi = 0.31830988618379067154f;
    static constexpr float two_pi = 6.28318530717958647692f;
};

__device__ __forceinline__ double em_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float em_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double em_atan2(double a, double b) { return atan2(a, b); }
__device__ __forceinline__ float em_atan2(float a, float b) { return atan2f(a, b); }
__device__ __forceinline__ double em_asinh(double v) { return asinh(v); }
__device__ __forceinline__ float em_asinh(float v) { return asinhf(v); }

// basis b0..b5 at tau >= 0; |b| magnitudes feed the FP32 error estimate
template <class T>
__device__ __forceinline__ void basis(T A, T B2, T D, T tau, T b[6])
{
    T tau2 = tau * tau;
    T Q2 = B2 + tau2;
    T Q = em_sqrt(Q2);
    T B = em_sqrt(B2);
    T ash = em_asinh(tau / B);
    T J0 = em_atan2(tau, A);
    T psi = em_atan2(D * tau, A * Q);
    T D2 = D * D;
    T J2 = A * tau + D2 * J0;
    T J4 = A * (A * A * tau + tau2 * tau * T(1.0 / 3.0)) + T(2) * D2 * A * tau + D2 * D2 * J0;
    T J1 = A * ash + D * psi;
    T U1 = T(0.5) * (tau * Q + B2 * ash);
    T J3 = A * U1 + D2 * J1;
    T U3 = T(0.25) * tau * Q * Q2 + T(0.75) * B2 * U1;
    T J5 = A * U3 + D2 * J3;
    b[0] = D * J0;
    b[1] = psi;
    b[2] = D * J2;
    b[3] = D * J3;
    b[4] = D * J4;
    b[5] = D * J5;
}

template <class T>
__device__ __forceinline__ T dot_c1(const T *b)
{
    return b[2] * T(1.0 / 6.0) - b[4] * T(3.0 / 40.0) + b[5] * T(1.0 / 40.0);
}
template <class T>
__device__ __forceinline__ T dot_c2(const T *b)
{
    return -b[0] * T(1.0 / 20.0) + b[1] * T(1.0 / 60.0) + b[2] * T(1.0 / 3.0) - b[3] * T(0.25) +
           b[4] * T(3.0 / 40.0) - b[5] * T(1.0 / 120.0);
}
template <class T>
__device__ __forceinline__ T dot_c3(const T *b)
{
    return b[0] * T(7.0 / 20.0) - b[1] * T(0.25);
}
// sum_n |c_n b_n| for the error estimate
template <class T>
__device__ __forceinline__ T abs_c12(const T *b)
{
    return fabs(b[0]) * T(0.05) + fabs(b[1]) * T(1.0 / 60.0) + fabs(b[2]) * T(1.0 / 3.0) +
           fabs(b[3]) * T(0.25) + fabs(b[4]) * T(3.0 / 40.0) + fabs(b[5]) * T(1.0 / 40.0);
}

// K(D) on each region (the per-endpoint in-plane-angle coefficient)
template <class T>
__device__ __forceinline__ T K_of(T D)
{
    T D2 = D * D;
    if (D < T(1)) return D2 * (T(1.0 / 6.0) - D2 * (T(3.0 / 40.0) - D * T(1.0 / 40.0)));
    if (D < T(2))
        return D2 * (T(1.0 / 3.0) - D * (T(0.25) - D * (T(3.0 / 40.0) - D * T(1.0 / 120.0)))) + T(1.0 / 60.0) / D -
               T(1.0 / 20.0);
    return T(-0.25) / D + T(7.0 / 20.0);
}
// K~(D) = K3(D) - K(D), zero for D >= 2
template <class T>
__device__ __forceinline__ T K_tilde(T D)
{
    if (D >= T(2)) return T(0);
    return T(-0.25) / D + T(7.0 / 20.0) - K_of(D);
}

// Edge term of the complement form, Phi~(T1) - Phi~(T0), with
// kt = K~(D) entering every endpoint as -kt b0(T).  err accumulates the
// magnitudes of the summed terms.
template <class T>
__device__ __forceinline__ T edge_tilde(T D, T A, T T0, T T1, T kt, T &err)
{
    T B2 = D * D + A * A;
    T b[6];
    T t1 = T(0), t2 = T(0), d1 = T(0), d2 = T(0);
    const bool near = B2 < T(4);
    if (near) {
        if (B2 < T(1)) {
            t1 = em_sqrt(T(1) - B2);
            basis(A, B2, D, t1, b);
            d1 = dot_c1(b) - dot_c2(b);
            err += abs_c12(b);
        }
        t2 = em_sqrt(T(4) - B2);
        basis(A, B2, D, t2, b);
        d2 = dot_c2(b) - dot_c3(b);
        err += abs_c12(b);
    }
    T res = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        T Tv = s ? T1 : T0;
        T u = fabs(Tv);
        if (u == T(0)) continue;
        T v;
        if (!near || u >= t2) {
            T b0 = D * em_atan2(u, A);
            v = -(d1 + d2) - kt * b0;
            err += fabs(kt * b0) + fabs(d1) + fabs(d2);
        } else {
            basis(A, B2, D, u, b);
            err += abs_c12(b) + fabs(kt * b[0]);
            v = ((u > t1) ? (dot_c3(b) - dot_c2(b) - d1) : (dot_c3(b) - dot_c1(b))) - kt * b[0];
        }
        if (Tv < T(0)) v = -v;
        res += s ? v : -v;
    }
    return res;
}

// Edge term of the full form, Phi(T1) - Phi(T0), with k = K(D) entering
// every endpoint as -k b0(T).  Beyond 2h (B >= 2) only the region-3 part
// remains: (7/20 - K(D)) b0 - b1/4, which for D >= 2 is the solid angle
// (atan(T/A) - atan(D T/(A Q)))/4 of the right triangle.
template <class T>
__device__ __forceinline__ T edge_full(T D, T A, T T0, T T1, T k, T &err)
{
    T B2 = D * D + A * A;
    if (B2 >= T(4)) {
        const T c0 = (D >= T(2)) ? T(0.25) / D : T(7.0 / 20.0) - k;
        T res = T(0);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            T Tv = s ? T1 : T0;
            T u = fabs(Tv);
            T b0 = D * em_atan2(u, A);
            T b1 = em_atan2(D * u, A * em_sqrt(B2 + u * u));
            T v = c0 * b0 - b1 * T(0.25);
            err += fabs(c0 * b0) + fabs(b1) * T(0.25);
            if (Tv < T(0)) v = -v;
            res += s ? v : -v;
        }
        return res;
    }
    T b[6];
    T t1 = T(0), t2 = em_sqrt(T(4) - B2), d1 = T(0), d2;
    if (B2 < T(1)) {
        t1 = em_sqrt(T(1) - B2);
        basis(A, B2, D, t1, b);
        d1 = dot_c1(b) - dot_c2(b);
        err += abs_c12(b);
    }
    basis(A, B2, D, t2, b);
    d2 = dot_c2(b) - dot_c3(b);
    err += abs_c12(b);
    T res = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        T Tv = s ? T1 : T0;
        T u = fabs(Tv);
        if (u == T(0)) continue;
        basis(A, B2, D, u, b);
        err += abs_c12(b) + fabs(k * b[0]);
        T v;
        if (u <= t1) v = dot_c1(b);
        else if (u <= t2) v = dot_c2(b) + d1;
        else v = dot_c3(b) + d1 + d2;
        v -= k * b[0];
        if (Tv < T(0)) v = -v;
        res += s ? v : -v;
    }
    return res;
}

}  // namespace em
