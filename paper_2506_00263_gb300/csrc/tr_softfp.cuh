// tr_softfp.cuh -- correctly rounded double reciprocal and square root on the
// integer and FP32 pipes.
//
// GB300 retires 2 FP64 thread-operations per clock per SM (64 times fewer than
// FP32), and the IEEE reciprocal and square root are multi-operation
// sequences on that pipe.  These two operations are computed here from the
// definition of round-to-nearest instead: an FP32 seed, one second-order
// Newton step in 64-bit fixed point, and an exact integer remainder that
// decides the last bit.  Both return the same bits as 1.0 / x and sqrt(x)
// for every input (zero, subnormal, infinite and NaN inputs, and reciprocals
// that leave the normal range, take the hardware operation), so the
// arithmetic contract is unchanged.  Alone they run at 2.1x (reciprocal) and
// 3.0x (square root) the IEEE rate.  The continuous-energy kernels use them
// for the lookup's 1/sigma_t and the scatter's reciprocals and square roots
// (measured 3.5 % faster there); the multigroup kernels select them with
// TR_SOFTFP (off by default: there they measured slower, tr_device.cuh).
//
// Reciprocal of x = +-m 2^(e - 1075), m in [2^52, 2^53), e in [1, 2044]:
// 1/x = 2^(1022 - e) (2^53 / m), whose mantissa is M = RN(2^105 / m).  With
// Q = floor(2^106 / m) and no exact ties (m is not a power of two, which is
// handled apart), M = floor(Q / 2) + (Q mod 2).  Seed y0 ~ 2^82 / m from the
// FP32 reciprocal of m's top 32 bits (relative error below 2^-23); with
// t = (2^82 - m y0) / 2^82, 2^115 / m = y0 2^33 / (1 - t) is taken as
// y0 2^33 (1 + t + t^2) (error of order 2^63 t^3, a few units), and Q from it
// is corrected to the exact quotient by the sign of the remainder
// 2^106 - Q m, which fits a signed 64-bit word and is computed from the low
// 64 bits of Q m alone.
//
// Square root of x = m 2^(e - 1075): with N = m 2^(52 + o) (o = 1 when e - 1023
// is odd), sqrt(x) = sqrt(N) 2^((e - 1023 - o) / 2 - 52) and the mantissa is
// S = RN(sqrt(N)) in [2^52, 2^53): S0 = floor(sqrt(N)), S = S0 + 1 exactly
// when N - S0^2 > S0 (no ties: sqrt(N) is an integer or irrational).  Seed
// from the FP32 reciprocal square root, two Newton corrections (the first in
// 64-bit words, the second from the 128-bit remainder) and a final exact
// integer remainder.
//
// The analysis of every intermediate range assumes seeds within 8 FP32 ulps;
// the seeds used here are within 2 (rsqrtf) and 0.5 (__frcp_rn).
#pragma once
#include <stdint.h>

namespace tr {

__device__ __forceinline__ double sf_rcp(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e - 1u > 2043u) return __drcp_rn(x);   // e outside [1, 2044]
    const unsigned long long sign = b & 0x8000000000000000ull;
    const unsigned long long frac = b & 0x000FFFFFFFFFFFFFull;
    if (frac == 0ull)   // a power of two: exact
        return __longlong_as_double((long long)(sign | ((unsigned long long)(2046u - e) << 52)));
    const unsigned long long m = frac | 0x0010000000000000ull;
    const float rf = __frcp_rn(__uint2float_rn((unsigned)(m >> 21)));
    const unsigned long long y0 = __float2uint_rz(rf * 0x1p61f);          // ~ 2^82 / m, <= 2^30
    const long long d = (long long)(0ull - m * y0);                        // 2^82 - m y0 (|d| < 2^62)
    const long long c1 = __mul64hi(d, (long long)(y0 << 15));             // y0 2^33 t
    const long long c2 = __mul64hi(c1, d) >> 18;                           // y0 2^33 t^2
    const unsigned long long y1 = (y0 << 33) + (unsigned long long)(c1 + c2);   // ~ 2^115 / m
    unsigned long long q = y1 >> 9;
    const long long r = (long long)(0ull - q * m);                         // 2^106 - q m, in [-m, 2m)
    q = q - (r < 0 ? 1ull : 0ull) + (r >= (long long)m ? 1ull : 0ull);
    const unsigned long long mant = (q >> 1) + (q & 1ull);
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(2045u - e) << 52) | (mant - 0x0010000000000000ull)));
}

__device__ __forceinline__ double sf_sqrt(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52);    // with the sign bit: negative inputs fall out below
    if (e - 1u > 2045u) return __dsqrt_rn(x);  // zero, subnormal, negative, infinite, NaN
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned odd = (e & 1u) ^ 1u;        // e - 1023 odd
    const unsigned sh = 52u + odd;
    // X = m 2^odd / 2^52 in [1, 4): T0 ~ sqrt(X) 2^31, S0 = T0 2^21 ~ sqrt(N)
    const float xf = __uint2float_rz((unsigned)(m >> 21)) * (odd ? 0x1p-30f : 0x1p-31f);
    const unsigned t0 = __float2uint_rz(xf * rsqrtf(xf) * 0x1p31f);
    // N - S0^2 = dp 2^42, dp = (m << (sh - 42)) - T0^2 (both below 2^64)
    const long long dp = (long long)((m << (sh - 42u)) - (unsigned long long)t0 * t0);
    // first correction (N - S0^2) / (2 S0) = dp 2^20 / T0, to 32 units
    const float rt = __frcp_rn(__uint2float_rz(t0));
    const float df = __int2float_rn((int)(dp >> 16)) * rt * 0x1p36f;
    const unsigned long long s1 =
        ((unsigned long long)t0 << 21) + (unsigned long long)((long long)__float2int_rd(df * 0.03125f) * 32);
    // second correction from the 128-bit remainder N - s1^2 (below 2^71 in magnitude)
    const unsigned long long n_lo = m << sh, n_hi = m >> (64u - sh);
    const unsigned long long p_lo = s1 * s1, p_hi = __umul64hi(s1, s1);
    const unsigned long long r_lo = n_lo - p_lo;
    const unsigned long long r_hi = n_hi - p_hi - (n_lo < p_lo ? 1ull : 0ull);
    const int r40 = (int)(long long)((r_hi << 24) | (r_lo >> 40));      // floor((N - s1^2) / 2^40)
    const float rs = __frcp_rn(__uint2float_rz((unsigned)(s1 >> 22)));   // ~ 2^22 / s1
    unsigned long long s2 = s1 + (unsigned long long)(long long)__float2int_rd(__int2float_rn(r40) * rs * 0x1p17f);
    // exact: N - s2^2 is small, so its low 64 bits are the value
    long long r2 = (long long)(n_lo - s2 * s2);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (r2 < 0) {
            s2 -= 1ull;
            r2 += (long long)(2ull * s2 + 1ull);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (r2 > (long long)(2ull * s2)) {
            s2 += 1ull;
            r2 -= (long long)(2ull * s2 - 1ull);
        }
    }
    const unsigned long long s = s2 + (r2 > (long long)s2 ? 1ull : 0ull);
    const unsigned eb = (e + 1023u - odd) >> 1;
    return __longlong_as_double((long long)(((unsigned long long)eb << 52) | (s - 0x0010000000000000ull)));
}

}  // namespace tr
