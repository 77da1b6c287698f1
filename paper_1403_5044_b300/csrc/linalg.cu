// FP64 vector and small dense linear-algebra kernels used by the JVP, GMRES
// and the preconditioner.  All reductions are two-stage with a fixed grid and
// a fixed combine order, so repeated calls give bitwise-identical results.
#include "swj_internal.h"
#include <math.h>

namespace {

constexpr int kRedBlocks = 256;   // first-stage blocks of every reduction
constexpr int kRedThreads = 256;

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b,
                        double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_axpy_dev(int n, const double *__restrict__ a, double s,
                           const double *__restrict__ x, double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += (s * a[0]) * x[i];
}

__global__ void k_scale_dev(int n, const double *__restrict__ num, double *__restrict__ x,
                            int invert)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double f = invert ? 1.0 / num[0] : num[0];
    if (i < n) x[i] *= f;
}

__global__ void k_copy(int n, const double *__restrict__ x, double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}

__global__ void k_fill(int n, double v, double *__restrict__ x)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block-wide sum of v (all threads get the result); blockDim.x multiple of 32
__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    return sh[0];
}

__device__ double block_max(double v)
{
    __shared__ double sh[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) r = warp_max(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    return sh[0];
}

// stage 1: red[b] = sum of squares, red[G + b] = max |x| or +Inf if non-finite
__global__ void k_norms1(int n, const double *__restrict__ x, double *__restrict__ red)
{
    double s = 0.0, m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = x[i];
        if (!isfinite(v)) m = INFINITY;
        s = fma(v, v, s);
        m = fmax(m, fabs(v));
    }
    s = block_sum(s);
    m = block_max(m);
    if (threadIdx.x == 0) { red[blockIdx.x] = s; red[gridDim.x + blockIdx.x] = m; }
}

__global__ void k_norms2(int G, const double *__restrict__ red, double *__restrict__ out)
{
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) { s += red[i]; m = fmax(m, red[G + i]); }
    s = block_sum(s);
    m = block_max(m);
    if (threadIdx.x == 0) { out[0] = isinf(m) ? NAN : s; out[1] = isinf(m) ? NAN : m; }
}

// stage 1 of multi-dot: red[r * G + b] = partial of row r over block b's range
__global__ void k_mdot1(int n, const double *__restrict__ V, size_t ld,
                        const double *__restrict__ w, double *__restrict__ red)
{
    int r = blockIdx.y;
    const double *v = V + (size_t)r * ld;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s = fma(v[i], w[i], s);
    s = block_sum(s);
    if (threadIdx.x == 0) red[(size_t)r * gridDim.x + blockIdx.x] = s;
}

__global__ void k_mdot2(int G, const double *__restrict__ red, double *__restrict__ out)
{
    int r = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) s += red[(size_t)r * G + i];
    s = block_sum(s);
    if (threadIdx.x == 0) out[r] = s;
}

__global__ void k_mgemv_sub(int n, int rows, const double *__restrict__ V, size_t ld,
                            const double *__restrict__ coef, double *__restrict__ w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int r = 0; r < rows; ++r) s = fma(-coef[r], V[(size_t)r * ld + i], s);
    w[i] = s;
}

__global__ void k_combine(int n, int rows, const double *__restrict__ Z, size_t ld,
                          const double *__restrict__ coef, double *__restrict__ x, int acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = acc ? x[i] : 0.0;
    for (int r = 0; r < rows; ++r) s = fma(coef[r], Z[(size_t)r * ld + i], s);
    x[i] = s;
}

// C = alpha A B + beta C (row-major), 64x64 output tile per block, 256 threads
// with 4x4 outputs each, k-tiles of 16 staged in shared memory.
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int k, double alpha, const double *const *Ap, const double *A0, int lda,
        const double *const *Bp, const double *B0, int ldb, double beta, double *const *Cp,
        double *C0, int ldc)
{
    const double *A = Ap ? Ap[blockIdx.z] : A0;
    const double *B = Bp ? Bp[blockIdx.z] : B0;
    double *C = Cp ? Cp[blockIdx.z] : C0;
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    double acc[4][4] = {};
    for (int kk = 0; kk < k; kk += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            int r = e / GK, q = e % GK;          // A tile: rows r, cols q
            int gr = row0 + r, gq = kk + q;
            As[q][r] = (gr < m && gq < k) ? A[(size_t)gr * lda + gq] : 0.0;
            int q2 = e / GT, c2 = e % GT;        // B tile: rows q2, cols c2
            int gq2 = kk + q2, gc = col0 + c2;
            Bs[q2][c2] = (gq2 < k && gc < n) ? B[(size_t)gq2 * ldb + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GK; ++q) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[q][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = row0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int cc = col0 + tx + 16 * j;
            if (cc >= n) continue;
            double *cp = C + (size_t)r * ldc + cc;
            *cp = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
        }
    }
}

// In-place inverse of one n x n row-major block per CTA by Gauss-Jordan
// elimination with partial (row) pivoting; the row interchanges are undone
// at the end as column interchanges in reverse order.  info[b] = 0 on
// success, 1 + k when column k has no non-zero pivot.
__global__ void __launch_bounds__(1024)
k_gj_inverse(int n, double *blocks, size_t stride, int *info)
{
    extern __shared__ double shm[];
    double *rowk = shm;             // n
    double *colf = shm + n;         // n
    int *piv = (int *)(shm + 2 * n);  // n
    __shared__ double bestv[32];
    __shared__ int besti[32];
    __shared__ int pivot_row;
    __shared__ int fail;
    double *a = blocks + (size_t)blockIdx.x * stride;
    const int tid = threadIdx.x, nth = blockDim.x;
    if (tid == 0) fail = 0;
    for (int k = 0; k < n; ++k) {
        // pivot search in column k, rows k..n-1 (ties: smallest row index)
        double bv = -1.0; int bi = n;
        for (int i = k + tid; i < n; i += nth) {
            double v = fabs(a[(size_t)i * n + k]);
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        __syncthreads();
        if ((tid & 31) == 0) { bestv[tid >> 5] = bv; besti[tid >> 5] = bi; }
        __syncthreads();
        if (tid < 32) {
            int nw = nth >> 5;
            double v = (tid < nw) ? bestv[tid] : -1.0;
            int ii = (tid < nw) ? besti[tid] : n;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, v, o);
                int oi = __shfl_xor_sync(0xffffffffu, ii, o);
                if (ov > v || (ov == v && oi < ii)) { v = ov; ii = oi; }
            }
            if (tid == 0) {
                pivot_row = ii;
                if (!(v > 0.0) || !isfinite(v)) fail = k + 1;
            }
        }
        __syncthreads();
        if (fail) break;
        int p = pivot_row;
        if (tid == 0) piv[k] = p;
        if (p != k) {
            for (int j = tid; j < n; j += nth) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        }
        __syncthreads();
        double pv = a[(size_t)k * n + k];
        double rp = 1.0 / pv;
        for (int j = tid; j < n; j += nth) {
            double v = (j == k) ? rp : a[(size_t)k * n + j] * rp;
            rowk[j] = v;
        }
        for (int i = tid; i < n; i += nth) colf[i] = (i == k) ? 0.0 : a[(size_t)i * n + k];
        __syncthreads();
        for (int j = tid; j < n; j += nth) a[(size_t)k * n + j] = rowk[j];
        for (size_t e = tid; e < (size_t)n * n; e += nth) {
            int i = (int)(e / n), j = (int)(e % n);
            if (i == k) continue;
            double base = (j == k) ? 0.0 : a[e];
            a[e] = fma(-colf[i], rowk[j], base);
        }
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) info[blockIdx.x] = fail;
        return;
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k) {
            for (int i = tid; i < n; i += nth) {
                double t = a[(size_t)i * n + k];
                a[(size_t)i * n + k] = a[(size_t)i * n + p];
                a[(size_t)i * n + p] = t;
            }
        }
        __syncthreads();
    }
    if (tid == 0) info[blockIdx.x] = 0;
}

}  // namespace

void swj_axpby(cudaStream_t st, int n, double a, const double *x, double b, double *y)
{
    SWJ_COUNT_LAUNCH();
    k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, a, x, b, y);
}
void swj_axpy_dev(cudaStream_t st, int n, const double *a, double s, const double *x, double *y)
{
    SWJ_COUNT_LAUNCH();
    k_axpy_dev<<<nblk(n, 256), 256, 0, st>>>(n, a, s, x, y);
}
void swj_scale_dev(cudaStream_t st, int n, const double *num, double *x, int invert)
{
    SWJ_COUNT_LAUNCH();
    k_scale_dev<<<nblk(n, 256), 256, 0, st>>>(n, num, x, invert);
}
void swj_copy(cudaStream_t st, int n, const double *x, double *y)
{
    SWJ_COUNT_LAUNCH();
    k_copy<<<nblk(n, 256), 256, 0, st>>>(n, x, y);
}
void swj_fill(cudaStream_t st, int n, double v, double *x)
{
    SWJ_COUNT_LAUNCH();
    k_fill<<<nblk(n, 256), 256, 0, st>>>(n, v, x);
}
void swj_norms(cudaStream_t st, int n, const double *x, double *red, double *out)
{
    int G = nblk(n, kRedThreads);
    if (G > kRedBlocks) G = kRedBlocks;
    if (G < 1) G = 1;
    SWJ_COUNT_LAUNCH();
    k_norms1<<<G, kRedThreads, 0, st>>>(n, x, red);
    SWJ_COUNT_LAUNCH();
    k_norms2<<<1, kRedThreads, 0, st>>>(G, red, out);
}
void swj_mdot(cudaStream_t st, int n, int rows, const double *V, size_t ld, const double *w,
              double *red, double *out)
{
    int G = nblk(n, kRedThreads);
    if (G > 64) G = 64;
    if (G < 1) G = 1;
    SWJ_COUNT_LAUNCH();
    k_mdot1<<<dim3(G, rows), kRedThreads, 0, st>>>(n, V, ld, w, red);
    SWJ_COUNT_LAUNCH();
    k_mdot2<<<rows, 64, 0, st>>>(G, red, out);
}
void swj_mgemv_sub(cudaStream_t st, int n, int rows, const double *V, size_t ld,
                   const double *coef, double *w)
{
    SWJ_COUNT_LAUNCH();
    k_mgemv_sub<<<nblk(n, 256), 256, 0, st>>>(n, rows, V, ld, coef, w);
}
void swj_combine(cudaStream_t st, int n, int rows, const double *Z, size_t ld,
                 const double *coef, double *x, int acc)
{
    SWJ_COUNT_LAUNCH();
    k_combine<<<nblk(n, 256), 256, 0, st>>>(n, rows, Z, ld, coef, x, acc);
}
void swj_dgemm_batched(cudaStream_t st, int m, int n, int k, double alpha,
                       const double *const *A, int lda, const double *const *B, int ldb,
                       double beta, double *const *C, int ldc, int batch)
{
    if (batch <= 0 || m <= 0 || n <= 0) return;
    dim3 grid(nblk(n, GT), nblk(m, GT), batch);
    SWJ_COUNT_LAUNCH();
    k_dgemm<<<grid, 256, 0, st>>>(m, n, k, alpha, A, nullptr, lda, B, nullptr, ldb, beta, C,
                                  nullptr, ldc);
}
void swj_dgemm(cudaStream_t st, int m, int n, int k, double alpha, const double *A, int lda,
               const double *B, int ldb, double beta, double *C, int ldc)
{
    if (m <= 0 || n <= 0) return;
    dim3 grid(nblk(n, GT), nblk(m, GT), 1);
    SWJ_COUNT_LAUNCH();
    k_dgemm<<<grid, 256, 0, st>>>(m, n, k, alpha, nullptr, A, lda, nullptr, B, ldb, beta,
                                  nullptr, C, ldc);
}
void swj_block_inverse(cudaStream_t st, int n, int count, double *blocks, size_t stride,
                       int *info)
{
    size_t sh = (size_t)n * (2 * sizeof(double) + sizeof(int));
    SWJ_COUNT_LAUNCH();
    k_gj_inverse<<<count, 1024, sh, st>>>(n, blocks, stride, info);
}
