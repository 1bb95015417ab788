// A double as the float-float pair hi = (float)x, lo = (float)(x - (double)hi)
// (rounded to nearest even, as those conversions are), formed with integer
// operations.  On this part the conversions between double and float issue
// at the FP64 rate, 1/64 of the FP32 rate, and the derived-geometry pass
// splits nine values per face-vertex.
#pragma once

#include <cuda_runtime.h>

namespace em {

// The significand M (53 bits) of x = +-M 2^k, k = e - 1075, is cut after its
// top 24 bits; hi keeps them, rounded to nearest even (a carry to 2^24 moves
// hi to the next binade), and x - hi = +-R 2^k exactly with |R| <= 2^28.
// (float)R rounds R to 24 bits as (float)(x - hi) would, and the power of two
// scales it exactly, since |R 2^k| >= 2^-112 stays a normal float for
// |x| >= 2^-60.  Smaller values, and those beyond float's range (with 0,
// infinities and NaN), take the conversions.
__device__ __forceinline__ void split_df(double x, float &hi, float &lo)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ff);
    if (e < 963 || e > 1149) {
        hi = __double2float_rn(x);
        lo = __double2float_rn(x - (double)hi);
        return;
    }
    const unsigned long long M = (u & 0xfffffffffffffull) | 0x10000000000000ull;
    unsigned long long Mh = M >> 29;
    const unsigned long long r = M & 0x1fffffffull;
    if (r > 0x10000000ull || (r == 0x10000000ull && (Mh & 1ull))) ++Mh;
    const int R = (int)((long long)M - (long long)(Mh << 29));
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const unsigned eh = (unsigned)(e - 1023 + 127);
    const unsigned hb = (Mh >> 24) ? (eh + 1u) << 23 : (eh << 23) | (unsigned)(Mh & 0x7fffffull);
    hi = __uint_as_float(hb | sign);
    const float l = (float)R * __int_as_float((e - 1075 + 127) << 23);
    lo = R == 0 ? 0.f : (sign ? -l : l);
}

// (float)x, rounded to nearest even, for 2^-100 <= |x| < 2^100 (the caller's
// range), by the same integer rounding as split_df.
__device__ __forceinline__ float f32_of(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ff);
    const unsigned long long M = (u & 0xfffffffffffffull) | 0x10000000000000ull;
    unsigned long long Mh = M >> 29;
    const unsigned long long r = M & 0x1fffffffull;
    if (r > 0x10000000ull || (r == 0x10000000ull && (Mh & 1ull))) ++Mh;
    const unsigned eh = (unsigned)(e - 1023 + 127);
    const unsigned hb = (Mh >> 24) ? (eh + 1u) << 23 : (eh << 23) | (unsigned)(Mh & 0x7fffffull);
    return __uint_as_float(hb | ((unsigned)(u >> 63) << 31));
}

// (float)x for any x: f32_of inside its range, the conversion outside it
// (zero, tiny or huge values, infinities, NaN).
__device__ __forceinline__ float f32_rn(double x)
{
    const int e = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
    if (e < 923 || e > 1149) return __double2float_rn(x);
    return f32_of(x);
}

// (double)x for a normal float x, exactly, by moving its fields.
__device__ __forceinline__ double f64_of(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned long long e = ((b >> 23) & 0xffu) - 127u + 1023u;
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | (e << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

}  // namespace em
