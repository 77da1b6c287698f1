// FP64 block products of the band LU on the bf16 tensor cores (Ozaki's
// error-free splitting; K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// B300 runs FP64 at two FMAs per clock per SM, so the set-up's Schur updates
// are bound by the FP64 pipe.  Here each n x n FP64 factor is cut into s
// digit slices of beta bits: row r of A is
//   A[r,:] = sign * 2^ea_r sum_{p<s} 2^(-beta (p+1)) a_p[r,:],  0 <= a_p < 2^beta
// (ea_r the exponent of the row's largest entry, the digits of the row's
// fixed-point magnitude truncated after s beta >= 56 bits, taken with integer
// shifts from the FP64 bit pattern); B the same by columns.  Then
//   (A B)[r,c] = 2^(ea_r + eb_c) sum_d 2^(-beta (d+2)) T_d[r,c],
//   T_d = sum_{p+q=d} a_p b_q,
// formed on the tensor cores by this library's tcgen05 kernel (umma.cu).
// Both factors' slices are stored K-major with one shape,
// [slot][row][digit][np]: row r of A's slot holds a_0[r, :] .. a_(s-1)[r, :],
// row c of B's slot holds column c of b_0 .. b_(s-1).  beta is chosen so
// that s n 2^(2 beta) <= 2^24: every partial sum of every T_d is an integer
// below 2^24, so bf16 products with FP32 accumulation compute it exactly
// whatever the summation order.  The T_d for d <= s - 1 are summed exactly in
// integer arithmetic and rounded to FP64 once; the dropped terms and the
// digit truncation are below n 2^(-56) of |A_r,:| |B_:,c|, the size of FP64's
// own rounding of the dot product, and the result does not depend on how the
// products are batched.  Matrices are padded with zeros to a multiple of 8
// (16-byte digit rows for the tensor-memory-access loads).
#include "swj_internal.h"
#include "oz_round.cuh"
#include <cuda_bf16.h>
#include <math.h>
#include <algorithm>
#include <cmath>

namespace {

// Fixed-point magnitude of |x| 2^(-e) with `bits` fractional bits (|x| < 2^e),
// truncated; from the FP64 bit pattern, integer arithmetic only.
__device__ __forceinline__ unsigned long long fixed_bits(double x, int e, int bits)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    if (ex == 0) return 0ull;   // zero (subnormals are far below the truncation)
    const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);   // |x| = m 2^(ex - 1075)
    // |x| 2^(-e) 2^bits = m 2^(ex - 1075 - e + bits) < 2^bits
    const int sh = ex - 1075 - e + bits;
    if (sh >= 0) return sh >= 11 ? 0ull : (m << sh);
    return -sh >= 64 ? 0ull : (m >> -sh);
}

// The magnitude and sign of x from its bit pattern.  B300 runs FP64
// comparisons and min/max on its FP64 pipe (two lanes per clock per SM), so the
// splits order magnitudes as integers: for finite doubles the order of
// |x|'s bit patterns is the order of |x|.
__device__ __forceinline__ unsigned long long mag_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}
// x < 0 (false for -0)
__device__ __forceinline__ bool negative(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) && (u << 1);
}

// e with |x| = f 2^e, f in [1/2, 1) (frexp's exponent) for the magnitude with
// bit pattern a; 0 for zero.  Every entry of the row is then below 2^e.
__device__ __forceinline__ int row_exponent(unsigned long long a)
{
    if (a == 0) return 0;
    const int E = (int)(a >> 52);
    if (E) return E - 1022;           // normal: [2^(E-1023), 2^(E-1022))
    return (64 - __clzll(a)) - 1074;  // subnormal: a 2^-1074
}

// Split row-major n x n FP64 matrices mats[m] by rows: slot slots[m] of sa,
// layout [slot][np rows][s][np] (row r, digit p, column j), digits with the
// entry's sign; row exponents ex[slot][np].  Block per (row, matrix).
__global__ void k_oz_split_rows(int n, int np, int s, int beta, const double *const *mats, const int *slots,
                                __nv_bfloat16 *sa, int *ex)
{
    const int r = blockIdx.x, m = blockIdx.y;
    const int slot = slots[m];
    const size_t rowlen = (size_t)s * np;
    __nv_bfloat16 *out = sa + ((size_t)slot * np + r) * rowlen;
    if (r >= n) {   // padding row
        for (size_t e = threadIdx.x; e < rowlen; e += blockDim.x) out[e] = __float2bfloat16(0.f);
        if (threadIdx.x == 0) ex[(size_t)slot * np + r] = 0;
        return;
    }
    const double *row = mats[m] + (size_t)r * n;
    __shared__ unsigned long long red[32];
    unsigned long long mx = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = umax64(mx, mag_bits(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const int e = row_exponent(red[0]);
    if (threadIdx.x == 0) ex[(size_t)slot * np + r] = e;
    const int bits = s * beta;
    const unsigned mask = (1u << beta) - 1u;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const double x = (j < n) ? row[j] : 0.0;
        const unsigned long long X = fixed_bits(x, e, bits);
        const float sg = negative(x) ? -1.f : 1.f;
        for (int p = 0; p < s; ++p) {
            const unsigned dgt = (unsigned)(X >> (beta * (s - 1 - p))) & mask;
            out[(size_t)p * np + j] = __float2bfloat16(sg * (float)dgt);   // exact: dgt < 2^8
        }
    }
}

// Split by columns: slot slots[m] of sb, layout [slot][np columns][s][np rows]
// (column c, digit q, row r: K-major, the layout of the A slices), digits
// with the entry's sign; column exponents ex[slot][np].  Block per (32-column
// strip, matrix), up to 32 warps (the launch uses 32: a set-up call splits few
// matrices, so the blocks are few): the column maxima with lanes over columns and
// warps over rows (coalesced reads), then 32 x 32 tiles through shared
// memory, written with lanes over rows (64-byte runs per column and digit).
__global__ void k_oz_split_cols(int n, int np, int s, int beta, const double *const *mats, const int *slots,
                                __nv_bfloat16 *sb, int *ex)
{
    const int c0 = blockIdx.x * 32, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = blockIdx.y;
    const double *A = mats[m];
    const int slot = slots[m];
    __shared__ double red[32][33];
    __shared__ unsigned long long mred[32][32];
    __shared__ int ec[32];
    const int c = c0 + lane;
    unsigned long long mx = 0;
    if (c < n)
        for (int r = w; r < n; r += nw) mx = umax64(mx, mag_bits(A[(size_t)r * n + c]));
    mred[w][lane] = mx;
    __syncthreads();
    if (w == 0) {
        for (int q = 1; q < nw; ++q) mx = umax64(mx, mred[q][lane]);
        const int e = (c < n) ? row_exponent(mx) : 0;
        ec[lane] = e;
        if (c < np) ex[(size_t)slot * np + c] = e;
    }
    const int bits = s * beta;
    const unsigned mask = (1u << beta) - 1u;
    const size_t rowlen = (size_t)s * np;
    __nv_bfloat16 *out = sb + (size_t)slot * np * rowlen;
    for (int r0 = 0; r0 < np; r0 += 32) {
        __syncthreads();   // ec written; the previous tile consumed
        for (int rr = w; rr < 32; rr += nw) {
            const int r = r0 + rr;
            red[rr][lane] = (r < n && c < n) ? A[(size_t)r * n + c] : 0.0;
        }
        __syncthreads();
        const int r = r0 + lane;
        for (int cc = w; cc < 32; cc += nw) {
            if (c0 + cc >= np || r >= np) continue;
            const double x = red[lane][cc];
            const unsigned long long X = fixed_bits(x, ec[cc], bits);
            const float sg = negative(x) ? -1.f : 1.f;
            __nv_bfloat16 *o = out + (size_t)(c0 + cc) * rowlen + r;
            for (int q = 0; q < s; ++q) {
                const unsigned dgt = (unsigned)(X >> (beta * (s - 1 - q))) & mask;
                o[(size_t)q * np] = __float2bfloat16(sg * (float)dgt);   // exact: dgt < 2^8
            }
        }
    }
}

// C_t = alpha 2^(ea_r + eb_c) sum_d 2^(-beta (d+2)) T_d[r, c] (+ C_t).  Every
// T_d[r, c] is an integer below 2^24 in magnitude, so the sum is the integer
// S = sum_d T_d 2^(beta (s-1-d)) (below 2^80) times 2^(-beta (s+1)): it is
// accumulated exactly in 128-bit two's complement with integer operations
// (B300's FP64 pipe, two FMAs per clock per SM, would bound it otherwise) and
// rounded to FP64 (the low word to 53 bits, then the sum; oz_round.cuh).
// Thread per element of the n x n block.
// block (32, 8) over 32 columns x 8 rows of the n x n block, grid.z = product;
// P holds T_d of levels d = 0..s-1 (the scheme's outputs) of every product.
template <int S_, int B_>
__global__ void k_oz_combine(int n, int np, int s, int beta, const OzProd *__restrict__ prods,
                             const float *__restrict__ P, const int *__restrict__ ea, const int *__restrict__ eb,
                             double alpha)
{
    const int c = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    if (r >= n || c >= n) return;
    const int t = blockIdx.z;
    const OzProd o = prods[t];
    const size_t n2 = (size_t)np * np;
    const float *Pt = P + (size_t)t * s * n2 + (size_t)r * np + c;
    int64_t hi;
    uint64_t lo;
    if constexpr (S_ > 0) {
        int32_t q[S_];
#pragma unroll
        for (int d = 0; d < S_; ++d) q[d] = __float2int_rn(Pt[(size_t)d * n2]);   // exact: |T_d| < 2^24
        oz_horner<S_, B_>(q, hi, lo);
    } else {
        int32_t q[16];
        for (int d = 0; d < s; ++d) q[d] = __float2int_rn(Pt[(size_t)d * n2]);
        oz_sum_any(q, s, beta, hi, lo);
    }
    // the double nearest to hi 2^64 + RN(lo), scaled: bit pattern from integer
    // operations (oz_round.cuh), ldexp only outside the normal range
    const int e2 = ea[(size_t)o.a * np + r] + eb[(size_t)o.b * np + c] - beta * (s + 1);
    bool fb;
    double v = __longlong_as_double((long long)oz_round_bits(hi, lo, e2, &fb));
    if (fb) v = ldexp(v, e2);
    double *C = o.C + (size_t)r * n + c;
    *C = o.accumulate ? fma(alpha, v, C[0]) : alpha * v;
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// The digit scheme for n x n products: the largest beta (digits up to
// 2^beta - 1 <= 255 are exact in bf16) with s n 2^(2 beta) <= 2^24 for s =
// ceil(56 / beta) digits, so every row (column) keeps s beta >= 56 bits of its
// fixed-point magnitude and a whole digit level sums exactly in one FP32
// accumulator: output o is level d = o (digits p = 0..d).  (Measured at n =
// 182: beta = 7 with levels split over two accumulators, 36 instead of 55
// digit products, took as long per set-up: the GEMM's CTAs are bound by
// latency, not by their MMAs, and the extra outputs cost the combine.)
void swj_ozaki_scheme(int n, OzScheme *z)
{
    int b = 8;
    for (; b > 1; --b) {
        const int sl = (56 + b - 1) / b;
        if (log2((double)sl * n) + 2.0 * b <= 24.0) break;
    }
    z->np = (n + 7) / 8 * 8;
    z->beta = b;
    z->s = (56 + b - 1) / b;
    z->nout = z->s < kOzMaxOut ? z->s : kOzMaxOut;
    for (int d = 0; d < z->nout; ++d) {
        z->d[d] = (unsigned char)d;
        z->p0[d] = 0;
        z->p1[d] = (unsigned char)d;
        z->order[d] = (unsigned char)(z->nout - 1 - d);   // the longest level first
    }
}

int swj_ozaki_split(cudaStream_t st, bool by_rows, int n, int np, int s, int beta, int count,
                    const double *const *mats, const int *slots, void *slices, int *ex)
{
    if (count <= 0) return SWJ_OK;
    __nv_bfloat16 *sl = (__nv_bfloat16 *)slices;
    SWJ_COUNT_LAUNCH();
    if (by_rows) k_oz_split_rows<<<dim3(np, count), 128, 0, st>>>(n, np, s, beta, mats, slots, sl, ex);
    else k_oz_split_cols<<<dim3(nblk(np, 32), count), 1024, 0, st>>>(n, np, s, beta, mats, slots, sl, ex);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_ozaki_products(cudaStream_t st, int n, const OzScheme &z, int count, const OzProd *prods,
                       const void *sa, size_t nsa, const int *ea, const void *sb, size_t nsb, const int *eb,
                       double alpha, float *P, int *err)
{
    if (count <= 0) return SWJ_OK;
    const int np = z.np, s = z.s, beta = z.beta;
    if (s < 1 || s > 16 || z.nout != s) return SWJ_EINVAL;
    int rc = swj_oz_gemm(st, z, count, prods, sa, nsa, sb, nsb, P, err);
    if (rc) return rc;
    SWJ_COUNT_LAUNCH();
    const dim3 grid(nblk(n, 32), nblk(n, 8), count), block(32, 8);
#define SWJ_OZ_COMBINE(S_, B_) k_oz_combine<S_, B_><<<grid, block, 0, st>>>(n, np, s, beta, prods, P, ea, eb, alpha)
    if (s == 10 && beta == 6) SWJ_OZ_COMBINE(10, 6);
    else if (s == 8 && beta == 7) SWJ_OZ_COMBINE(8, 7);
    else if (s == 12 && beta == 5) SWJ_OZ_COMBINE(12, 5);
    else if (s == 7 && beta == 8) SWJ_OZ_COMBINE(7, 8);
    else SWJ_OZ_COMBINE(0, 0);
#undef SWJ_OZ_COMBINE
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}
