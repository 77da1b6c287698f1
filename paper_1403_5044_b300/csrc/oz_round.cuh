// The Ozaki combine's exact digit sums and their rounding to FP64, with
// integer operations only (host and device).  B300 runs FP64 arithmetic and
// int <-> double conversions on its FP64 pipe, two lanes per clock per SM;
// the combine handles every element of every block product of the set-up, so
// it forms the double's bit pattern on the integer pipes instead.
//
// oz_round_bits(hi, lo, e2) returns the bits of
//     ldexp(fma((double)hi, 2^64, (double)lo), e2)
// for the two's complement 128-bit integer hi 2^64 + lo (|hi| < 2^62): lo is
// first rounded to 53 bits (round to nearest, ties to even, as the unsigned
// conversion does), then the exact sum hi 2^64 + RN(lo) is rounded once more,
// then scaled by 2^e2.  Where the scaled value would leave the normal range
// the caller falls back to ldexp (oz_round_bits sets *fallback).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD static inline
#endif

OZ_HD int oz_clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// round the magnitude mh 2^64 + ml (nonzero, mh < 2^62) to 53 bits; returns the
// 53-bit significand q (2^52 <= q < 2^53) and the bit length *nb of the rounded
// value (value = q 2^(*nb - 53))
OZ_HD uint64_t oz_rn53(uint64_t mh, uint64_t ml, int *nb)
{
    int n = mh ? 128 - oz_clz64(mh) : 64 - oz_clz64(ml);
    if (n <= 53) {
        *nb = n;
        return ml << (53 - n);
    }
    const int k = n - 53;   // 1 <= k <= 73: bits to drop
    uint64_t q, rem, half;
    bool rem_gt = false, rem_eq = false;
    if (k < 64) {
        q = (ml >> k) | (k ? (mh << (64 - k)) : 0);
        rem = ml & ((1ull << k) - 1);
        half = 1ull << (k - 1);
        rem_gt = rem > half;
        rem_eq = rem == half;
    } else {   // k >= 64: q from mh alone, the dropped bits span all of ml
        const int kk = k - 64;
        q = mh >> kk;
        const uint64_t rh = kk ? (mh & ((1ull << kk) - 1)) : 0;
        if (kk == 0) {
            rem_gt = ml > (1ull << 63);
            rem_eq = ml == (1ull << 63);
        } else {
            const uint64_t hh = 1ull << (kk - 1);
            rem_gt = rh > hh || (rh == hh && ml != 0);
            rem_eq = rh == hh && ml == 0;
        }
    }
    if (rem_gt || (rem_eq && (q & 1))) ++q;
    if (q >> 53) {   // carried into a new leading bit
        q >>= 1;
        ++n;
    }
    *nb = n;
    return q;
}

OZ_HD uint64_t oz_round_bits(int64_t hi, uint64_t lo, int e2, bool *fallback)
{
    *fallback = false;
    // RN(lo) as an integer: lo_r = lo rounded to 53 significant bits (may be 2^64)
    uint64_t lr = lo, cy = 0;
    if (lo >> 53) {
        int nb;
        const uint64_t q = oz_rn53(0, lo, &nb);   // lo_r = q 2^(nb - 53)
        if (nb > 64) {
            cy = 1;   // q 2^(nb - 53) = 2^64
            lr = 0;
        } else {
            lr = q << (nb - 53);
        }
    }
    // the exact sum hi 2^64 + lo_r, then its magnitude and sign
    const int64_t h = hi + (int64_t)cy;
    if (h == 0 && lr == 0) return 0;   // +0.0
    const bool neg = h < 0;
    uint64_t mh = (uint64_t)h, ml = lr;
    if (neg) {   // two's complement negation of the 128-bit value
        ml = ~ml + 1;
        mh = ~mh + (ml == 0 ? 1 : 0);
    }
    int nb;
    const uint64_t q = oz_rn53(mh, ml, &nb);
    const int be = 1023 + (nb - 1) + e2;   // biased exponent of q 2^(nb - 53) 2^e2
    if (be < 1 || be > 2046) {
        *fallback = true;
        return ((uint64_t)neg << 63) | ((uint64_t)(1023 + nb - 1) << 52) | (q & ((1ull << 52) - 1));
    }
    return ((uint64_t)neg << 63) | ((uint64_t)be << 52) | (q & ((1ull << 52) - 1));
}

// S = sum_d q_d 2^(beta (s-1-d)) as 128-bit two's complement hi 2^64 + lo, for
// |q_d| < 2^25 (the digit-level products T_d, below 2^24) and s beta < 100.
OZ_HD void oz_sum_any(const int32_t *q, int s, int beta, int64_t &hi, uint64_t &lo)
{
    hi = 0;
    lo = 0;
    for (int d = 0; d < s; ++d) {
        const int64_t v = q[d];
        const int sh = beta * (s - 1 - d);
        uint64_t tl;
        int64_t th;
        if (sh == 0) {
            tl = (uint64_t)v;
            th = v >> 63;
        } else if (sh < 64) {
            tl = (uint64_t)v << sh;
            th = v >> (64 - sh);   // the high word of v 2^sh (sign-extended)
        } else {
            tl = 0;
            th = (int64_t)((uint64_t)v << (sh - 64));
        }
        lo += tl;
        hi += th + (lo < tl ? 1 : 0);
    }
}

// The same sum for fixed (S_, B_) as two int64 Horner sums: the high digits H =
// sum_{d < SH} q_d 2^(B_ (SH-1-d)) and the low digits L (the other S_ - SH),
// S = H 2^(B_ (S_ - SH)) + L.  For |q_d| < 2^25 each half stays below
// 2^(26 + B_ (SH - 1)) < 2^63, and the shifts are constants.
template <int S_, int B_>
OZ_HD void oz_horner(const int32_t *q, int64_t &hi, uint64_t &lo)
{
    constexpr int SL = S_ / 2, SH = S_ - SL, SHF = B_ * SL;
    static_assert(25 + B_ * (SH - 1) < 62 && SHF > 0 && SHF < 64, "halves must fit in int64");
    int64_t H = 0, L = 0;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int d = 0; d < SH; ++d) H = H * ((int64_t)1 << B_) + q[d];
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int d = SH; d < S_; ++d) L = L * ((int64_t)1 << B_) + q[d];
    lo = (uint64_t)H << SHF;
    hi = H >> (64 - SHF);
    const uint64_t l2 = lo + (uint64_t)L;   // + L, sign-extended to 128 bits
    hi += (L >> 63) + (l2 < lo ? 1 : 0);
    lo = l2;
}
