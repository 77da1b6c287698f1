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
//   T_d = sum_{p+q=d} a_p b_q = [a_0 .. a_d] [b_d; ..; b_0],
// one GEMM per d, all with inner dimension s n: A's slices are stored
// interleaved by row ([a_0 .. a_(s-1)] per row) and B's in reverse order
// followed by s - 1 zero slices ([b_(s-1); ..; b_0; 0; ..; 0]), so that the s
// rows of slices starting at b_d are [b_d; ..; b_0; 0..] and every T_d is a
// plain strided product; the T_d of all products of a group are one batched
// call (the zero slices cost tensor-core flops, not launches).  beta is
// chosen so that s n 2^(2 beta) <= 2^24: every
// partial sum of every T_d is an integer below 2^24, so a bf16 GEMM with FP32
// accumulation (cuBLAS) computes it exactly whatever its summation order.
// The T_d for d <= s - 1 are summed exactly in integer arithmetic and rounded
// to FP64 once; the dropped terms and the digit truncation are below
// n 2^(-56) of |A_r,:| |B_:,c|, the size of FP64's own rounding of the dot
// product, and the result does not depend on how the products are batched.  Matrices are padded with zeros to a
// multiple of 8 (16-byte rows for the tensor-core kernels).
#include "swj_internal.h"
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <math.h>

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

__device__ __forceinline__ int row_exponent(double mx)
{
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);   // mx = f 2^e, f in [1/2, 1): every |x| < 2^e
    return e;
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
    __shared__ double red[32];
    double mx = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, fabs(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
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
        const float sg = (x < 0.0) ? -1.f : 1.f;
        for (int p = 0; p < s; ++p) {
            const unsigned dgt = (unsigned)(X >> (beta * (s - 1 - p))) & mask;
            out[(size_t)p * np + j] = __float2bfloat16(sg * (float)dgt);   // exact: dgt < 2^8
        }
    }
}

// Split by columns: slot slots[m] of sb, layout [slot][2s-1][np][np] with digit
// q at position s - 1 - q (reverse order; positions s .. 2s-2 stay zero);
// column exponents ex[slot][np].  Block per (32-column strip, matrix): lanes
// over columns, warps over rows.
__global__ void k_oz_split_cols(int n, int np, int s, int beta, const double *const *mats, const int *slots,
                                __nv_bfloat16 *sb, int *ex)
{
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = blockIdx.y;
    const double *A = mats[m];
    const int slot = slots[m];
    __shared__ double red[32][33];
    double mx = 0.0;
    if (c < n)
        for (int r = w; r < n; r += nw) mx = fmax(mx, fabs(A[(size_t)r * n + c]));
    red[w][threadIdx.x & 31] = mx;
    __syncthreads();
    if (w == 0) {
        for (int q = 1; q < nw; ++q) mx = fmax(mx, red[q][threadIdx.x & 31]);
        red[0][threadIdx.x & 31] = mx;
    }
    __syncthreads();
    if (c >= np) return;
    const int e = (c < n) ? row_exponent(red[0][threadIdx.x & 31]) : 0;
    if (w == 0) ex[(size_t)slot * np + c] = e;
    const size_t n2 = (size_t)np * np;
    __nv_bfloat16 *out = sb + (size_t)slot * (2 * s - 1) * n2 + c;
    const int bits = s * beta;
    const unsigned mask = (1u << beta) - 1u;
    for (int r = w; r < np; r += nw) {
        const double x = (c < n && r < n) ? A[(size_t)r * n + c] : 0.0;
        const unsigned long long X = fixed_bits(x, e, bits);
        const float sg = (x < 0.0) ? -1.f : 1.f;
        for (int q = 0; q < s; ++q) {
            const unsigned dgt = (unsigned)(X >> (beta * (s - 1 - q))) & mask;
            out[(size_t)(s - 1 - q) * n2 + (size_t)r * np] = __float2bfloat16(sg * (float)dgt);
        }
    }
}

// Pointer arrays of the GEMMs T_d of `count` products, d = 0..s-1: entry
// t * s + d.  Row-major T = A' B' is the column-major T^T = B'^T A'^T, so B'
// (s np rows from stored position s-1-d: b_d .. b_0 then zeros) comes first;
// A' is row-major with leading dimension s np.
__global__ void k_oz_ptrs(int count, int s, int np, const OzProd *__restrict__ prods, const __nv_bfloat16 *sa,
                          const __nv_bfloat16 *sb, float *P, const void **pA, const void **pB, void **pC)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count * s) return;
    const int t = e / s, d = e % s;
    const OzProd o = prods[t];
    const size_t n2 = (size_t)np * np;
    pA[e] = sb + ((size_t)o.b * (2 * s - 1) + (s - 1 - d)) * n2;
    pB[e] = sa + (size_t)o.a * np * s * np;
    pC[e] = P + ((size_t)t * s + d) * n2;
}

// C_t = alpha 2^(ea_r + eb_c) sum_d 2^(-beta (d+2)) T_d[r, c] (+ C_t).  Every
// T_d[r, c] is an integer below 2^24 in magnitude, so the sum is the integer
// S = sum_d T_d 2^(beta (s-1-d)) (below 2^80) times 2^(-beta (s+1)): it is
// accumulated exactly in 128-bit two's complement with integer operations
// (B300's FP64 pipe, two FMAs per clock per SM, would bound it otherwise) and
// rounded to FP64 once.  Thread per element of the n x n block.
__global__ void k_oz_combine(int n, int np, int s, int beta, const OzProd *__restrict__ prods,
                             const float *__restrict__ P, const int *__restrict__ ea, const int *__restrict__ eb,
                             double alpha)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * n) return;
    const int t = blockIdx.y;
    const OzProd o = prods[t];
    const int r = (int)(e / n), c = (int)(e % n);
    const size_t n2 = (size_t)np * np;
    const float *Pt = P + (size_t)t * s * n2 + (size_t)r * np + c;
    long long hi = 0;
    unsigned long long lo = 0;
    for (int d = 0; d < s; ++d) {
        const long long q = (long long)__float2int_rn(Pt[(size_t)d * n2]);   // exact: |T_d| < 2^24
        const int sh = beta * (s - 1 - d);                                  // 0 <= sh < 64
        const unsigned long long tl = (unsigned long long)q << sh;           // low word of q 2^sh
        const long long th = sh ? (q >> (64 - sh)) : (q >> 63);             // high word (sign-extended)
        lo += tl;
        hi += th + (lo < tl ? 1 : 0);
    }
    // |hi| < 2^16 is exact in FP64; one rounding of lo, one of the sum
    double v = fma((double)hi, 18446744073709551616.0, (double)lo);
    v = ldexp(v, ea[(size_t)o.a * np + r] + eb[(size_t)o.b * np + c] - beta * (s + 1));
    double *C = o.C + e;
    *C = o.accumulate ? fma(alpha, v, C[0]) : alpha * v;
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void swj_ozaki_params(int n, int *np, int *beta, int *s)
{
    // largest beta with s n 2^(2 beta) <= 2^24 for s = ceil(56 / beta) digits
    int b = 8;
    for (; b > 1; --b) {
        const int sl = (56 + b - 1) / b;
        if (log2((double)sl * n) + 2.0 * b <= 24.0) break;
    }
    *beta = b;
    *s = (56 + b - 1) / b;
    *np = (n + 7) / 8 * 8;
}

int swj_ozaki_split(cudaStream_t st, bool by_rows, int n, int np, int s, int beta, int count,
                    const double *const *mats, const int *slots, void *slices, int *ex)
{
    if (count <= 0) return SWJ_OK;
    __nv_bfloat16 *sl = (__nv_bfloat16 *)slices;
    SWJ_COUNT_LAUNCH();
    if (by_rows) k_oz_split_rows<<<dim3(np, count), 128, 0, st>>>(n, np, s, beta, mats, slots, sl, ex);
    else k_oz_split_cols<<<dim3(nblk(np, 32), count), 256, 0, st>>>(n, np, s, beta, mats, slots, sl, ex);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_ozaki_products(void **handle, cudaStream_t st, int n, int np, int s, int beta, int count,
                       const OzProd *prods, const void *sa_, const int *ea, const void *sb_, const int *eb,
                       double alpha, float *P, void **ptrs, int mode)
{
    if (count <= 0) return SWJ_OK;
    const __nv_bfloat16 *sa = (const __nv_bfloat16 *)sa_, *sb = (const __nv_bfloat16 *)sb_;
    const int nall = count * s;
    const void **pA = (const void **)ptrs, **pB = pA + nall;
    void **pC = ptrs + 2 * (size_t)nall;
    if (mode != SWJ_OZ_USE_PTRS) {
        SWJ_COUNT_LAUNCH();
        k_oz_ptrs<<<nblk(nall, 256), 256, 0, st>>>(count, s, np, prods, sa, sb, P, pA, pB, pC);
        SWJ_CUDA_TRY(cudaGetLastError());
        if (mode == SWJ_OZ_FILL_PTRS) return SWJ_OK;
    }
    cublasHandle_t h = (cublasHandle_t)*handle;
    if (!h) {
        if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return SWJ_ECUDA;
        *handle = h;
    }
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return SWJ_ECUDA;
    const float one = 1.0f, zero = 0.0f;
    // every T_d^T (np x np, column-major) = B'^T (np x s np) A'^T (s np x np), one call
    if (cublasGemmBatchedEx(h, CUBLAS_OP_N, CUBLAS_OP_N, np, np, s * np, &one, pA, CUDA_R_16BF, np, pB,
                            CUDA_R_16BF, s * np, &zero, pC, CUDA_R_32F, np, nall, CUBLAS_COMPUTE_32F,
                            CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS)
        return SWJ_ECUDA;
    SWJ_COUNT_LAUNCH();
    k_oz_combine<<<dim3(nblk((long)n * n, 256), count), 256, 0, st>>>(n, np, s, beta, prods, P, ea, eb, alpha);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

void swj_cublas_destroy(void *handle)
{
    if (handle) cublasDestroy((cublasHandle_t)handle);
}
