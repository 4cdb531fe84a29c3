// tr_fixed.cuh -- order-independent tally accumulation.
//
// The paper leaves the reduction of the track-length tallies open and names
// tally atomics as a cost of the asynchronous scheme (Sec. 5.2).  Here every
// tally contribution c (a track length, or a track length times a cross
// section) is rounded once to the nearest multiple of 2^-FIX_F, X = round(c
// 2^FIX_F), and bins sum these integers.  Integer addition is associative, so
// a bin's sum depends only on the set of contributions, never on which thread
// or block adds them in which order: tallies are bit-identical from run to
// run, for any schedule, scheme or decomposition, and equal to the sum of
// the rounded contributions taken in any fixed order.
//
// A bin (FixBin) is two 64-bit words: lo adds the low FIX_LO bits of each X,
// hi adds X >> FIX_LO (an arithmetic shift, in two's complement), so that the
// bin's value is (hi 2^FIX_LO + lo) 2^-FIX_F exactly.  Each contribution adds
// less than 2^FIX_LO to lo, so lo cannot wrap before 2^40 contributions; hi
// holds totals up to 2^(63 + FIX_LO - FIX_F) = 2^39 in magnitude.  One
// contribution rounds by at most 2^-(FIX_F + 1) = 1.8e-15 (absolute).
//
// Per-lane accumulators (the scalar tallies) keep a single signed 64-bit sum
// of X, spilled into their bin with two integer atomics before it can reach
// 2^62 in magnitude.
#pragma once
#include <stdint.h>
#include <string.h>

namespace tr {

constexpr int FIX_F = 48;    // fractional bits of a rounded contribution
constexpr int FIX_LO = 24;   // low bits of X that go to the lo word
constexpr unsigned long long FIX_LO_MASK = (1ull << FIX_LO) - 1ull;

struct FixBin {
    unsigned long long lo, hi;
};

__host__ __device__ __forceinline__ unsigned long long fix_bits(double c)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(c);
#else
    unsigned long long b;
    memcpy(&b, &c, 8);
    return b;
#endif
}

// |c| 2^FIX_F rounded to the nearest integer (ties away from zero), for
// |c| < 2^14, from the bit pattern with integer instructions only; and the
// sign.  Zero and subnormal c give 0.
__host__ __device__ __forceinline__ unsigned long long fix_mag_small(unsigned long long b)
{
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int s = e - (1075 - FIX_F);   // |c| 2^FIX_F = m 2^s
    if (e == 0 || s < -53) return 0ull;
    if (s >= 0) return m << s;
    return (m + (1ull << (-s - 1))) >> (-s);
}

// X = round(c 2^FIX_F) as a signed integer, for |c| < 2^14 (the caller
// checks the range with fix_small).
__host__ __device__ __forceinline__ bool fix_small(double c)
{
    return ((fix_bits(c) >> 52) & 0x7FFu) < (unsigned)(1023 + 14);
}
__host__ __device__ __forceinline__ long long fix_round(double c)
{
    const unsigned long long b = fix_bits(c);
    const long long x = (long long)fix_mag_small(b);
    return (b >> 63) ? -x : x;
}

// The two words one contribution adds to a bin (any finite c with |c| below
// 2^39; larger magnitudes return false and add nothing).
__host__ __device__ __forceinline__ bool fix_split(double c, unsigned long long& lo, unsigned long long& hi)
{
    const unsigned long long b = fix_bits(c);
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int s = e - (1075 - FIX_F);
    unsigned long long xl = 0ull, xh = 0ull;   // |X| = xh 2^FIX_LO + xl
    bool ok = true;
    if (e == 0 || s < -53) {
        // zero, subnormal or below half a unit: rounds to 0
    } else if (s < 0) {
        const unsigned long long x = (m + (1ull << (-s - 1))) >> (-s);
        xl = x & FIX_LO_MASK;
        xh = x >> FIX_LO;
    } else if (s <= 34) {
        xl = (s < 64 ? (m << s) : 0ull) & FIX_LO_MASK;
        xh = s >= FIX_LO ? (m << (s - FIX_LO)) : (m >> (FIX_LO - s));
    } else {
        ok = false;   // |c| >= 2^39 (or not finite)
    }
    if ((b >> 63) && (xl | xh)) {
        // -(xh 2^FIX_LO + xl) = (-xh - 1) 2^FIX_LO + (2^FIX_LO - xl), or -xh 2^FIX_LO when xl = 0
        if (xl) {
            xl = (1ull << FIX_LO) - xl;
            xh = ~xh;
        } else {
            xh = 0ull - xh;
        }
    }
    lo = xl;
    hi = xh;
    return ok;
}

// The two words a per-lane sum of X adds to a bin (exact for any signed x).
__host__ __device__ __forceinline__ void fix_split_sum(long long x, unsigned long long& lo, unsigned long long& hi)
{
    lo = (unsigned long long)x & FIX_LO_MASK;
    hi = (unsigned long long)(x >> FIX_LO);
}

// A per-lane sum must be spilled once |x| >= 2^61 (so that adding one more
// contribution below 2^14 in magnitude cannot reach 2^63).
__host__ __device__ __forceinline__ bool fix_sum_full(long long x)
{
    return ((unsigned long long)x + (1ull << 61)) >> 62 != 0ull;
}

// The value of a bin, (hi 2^FIX_LO + lo) 2^-FIX_F: the carry of lo moved into
// hi first, so both parts convert exactly while |hi| < 2^53 (totals below
// 2^29); beyond that the single rounding of hi's conversion is deterministic.
__host__ __device__ __forceinline__ double fix_value(const FixBin& b)
{
    const unsigned long long l = b.lo & FIX_LO_MASK;
    const long long h = (long long)(b.hi + (b.lo >> FIX_LO));
    return (double)h * (1.0 / (double)(1ull << (FIX_F - FIX_LO))) + (double)l * (1.0 / (double)(1ull << 48));
}
static_assert(FIX_F == 48, "fix_value scales by 2^-48 for the lo word");

#ifdef __CUDACC__
// Atomic add of one contribution to a bin (two integer reductions; the order
// of concurrent adds does not change the result).  False if |c| >= 2^39.
__device__ __forceinline__ bool fix_add(FixBin* bin, double c)
{
    unsigned long long lo, hi;
    const bool ok = fix_split(c, lo, hi);
    atomicAdd(&bin->lo, lo);
    atomicAdd(&bin->hi, hi);
    return ok;
}

// The same for a non-negative contribution (a track length): below 2^14 the
// rounded value X fits one 64-bit word and splits with two integer
// operations; larger values take the general path.
__device__ __forceinline__ bool fix_add_nn(FixBin* bin, double c)
{
    const unsigned long long b = fix_bits(c);
    if ((b >> 52) >= (unsigned long long)(1023 + 14)) return fix_add(bin, c);
    const unsigned long long x = fix_mag_small(b);
    atomicAdd(&bin->lo, x & FIX_LO_MASK);
    atomicAdd(&bin->hi, x >> FIX_LO);
    return true;
}

__device__ __forceinline__ void fix_add_sum(FixBin* bin, long long x)
{
    unsigned long long lo, hi;
    fix_split_sum(x, lo, hi);
    atomicAdd(&bin->lo, lo);
    atomicAdd(&bin->hi, hi);
}
#endif

}  // namespace tr
