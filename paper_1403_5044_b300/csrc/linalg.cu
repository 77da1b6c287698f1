// FP64 vector and small dense linear-algebra kernels used by the JVP, GMRES
// and the preconditioner.  All reductions are two-stage with a fixed grid and
// a fixed combine order, so repeated calls give bitwise-identical results.
#include "swj_internal.h"
#include <math.h>

namespace {

constexpr int kRedBlocks = 256;   // first-stage blocks of every reduction
constexpr int kRedThreads = 256;

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

__global__ void k_bcopy(int n, const double *__restrict__ x, double *__restrict__ y, size_t ld,
                        const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[inst * ld + i] = x[inst * ld + i];
}

__global__ void k_bfill(int n, double v, double *__restrict__ x, size_t ld, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[inst * ld + i] = v;
}

__global__ void k_baxpy(int n, const double *__restrict__ a_dev, size_t sstride, double a_scale,
                        const double *__restrict__ x, double *__restrict__ y, size_t ld,
                        const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double a = a_dev ? a_scale * a_dev[inst * sstride] : a_scale;
    if (i < n) y[inst * ld + i] = fma(a, x[inst * ld + i], y[inst * ld + i]);
}

__global__ void k_bscale(int n, const double *__restrict__ s_dev, size_t sstride, double s_scale,
                         int invert, const double *__restrict__ x, double *__restrict__ y, size_t ld,
                         const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double f = s_dev ? s_scale * s_dev[inst * sstride] : s_scale;
    if (invert) f = 1.0 / f;
    if (i < n) y[inst * ld + i] = f * x[inst * ld + i];
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

// stage 1 of the norms: per instance, red[b] = sum of squares of block b's
// range, red[G + b] = max |x| there (+Inf if any entry is not finite)
__global__ void k_bnorms1(int n, const double *__restrict__ x, size_t ld, double *__restrict__ red,
                          const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    x += inst * ld;
    red += (size_t)inst * SWJ_RED;
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

__global__ void k_bnorms2(int G, const double *__restrict__ red, double *__restrict__ out,
                          size_t sstride, const int *__restrict__ act)
{
    const int inst = blockIdx.x;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    red += (size_t)inst * SWJ_RED;
    double s = 0.0, m = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) { s += red[i]; m = fmax(m, red[G + i]); }
    s = block_sum(s);
    m = block_max(m);
    if (threadIdx.x == 0) {
        out[inst * sstride] = isinf(m) ? NAN : s;
        out[inst * sstride + 1] = isinf(m) ? NAN : m;
    }
}

// stage 1 of the multi-dot: red[r * G + b] = partial of row r over block b's range
__global__ void k_bmdot1(int n, const double *__restrict__ V, size_t ld, size_t vstride,
                         const double *__restrict__ w, size_t wstride, double *__restrict__ red,
                         const int *__restrict__ act)
{
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const int r = blockIdx.y;
    const double *v = V + inst * vstride + (size_t)r * ld;
    w += inst * wstride;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s = fma(v[i], w[i], s);
    s = block_sum(s);
    if (threadIdx.x == 0) red[(size_t)inst * SWJ_RED + (size_t)r * gridDim.x + blockIdx.x] = s;
}

__global__ void k_bmdot2(int G, const double *__restrict__ red, double *__restrict__ out,
                         size_t sstride, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const int r = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) s += red[(size_t)inst * SWJ_RED + (size_t)r * G + i];
    s = block_sum(s);
    if (threadIdx.x == 0) out[inst * sstride + r] = s;
}

__global__ void k_bmgemv_sub(int n, int rows, const double *__restrict__ V, size_t ld, size_t vstride,
                             const double *__restrict__ coef, size_t sstride, double *__restrict__ w,
                             size_t wstride, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *v = V + inst * vstride;
    const double *cf = coef + inst * sstride;
    double s = w[inst * wstride + i];
    for (int r = 0; r < rows; ++r) s = fma(-cf[r], v[(size_t)r * ld + i], s);
    w[inst * wstride + i] = s;
}

__global__ void k_bcombine(int n, int rows, const double *__restrict__ Z, size_t ld, size_t zstride,
                           const double *__restrict__ coef, size_t sstride, double *__restrict__ x,
                           size_t xstride, int acc, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *z = Z + inst * zstride;
    const double *cf = coef + inst * sstride;
    double s = acc ? x[inst * xstride + i] : 0.0;
    for (int r = 0; r < rows; ++r) s = fma(cf[r], z[(size_t)r * ld + i], s);
    x[inst * xstride + i] = s;
}

// C = alpha A B + beta C (row-major), TILE x TILE output tile per block, 256
// threads with (TILE/16)^2 outputs each, k-tiles of 16 staged in shared memory.
// TILE = 64 for throughput, 32 to spread one small product over more SMs
// (FP64 work on one SM is slow on this part).
constexpr int GK = 16;
template <int TILE>
__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int k, double alpha, const double *const *Ap, const double *A0, int lda,
        const double *const *Bp, const double *B0, int ldb, double beta, double *const *Cp,
        double *C0, int ldc)
{
    constexpr int R = TILE / 16;
    const double *A = Ap ? Ap[blockIdx.z] : A0;
    const double *B = Bp ? Bp[blockIdx.z] : B0;
    double *C = Cp ? Cp[blockIdx.z] : C0;
    __shared__ double As[GK][TILE + 1];
    __shared__ double Bs[GK][TILE + 1];
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    int row0 = blockIdx.y * TILE, col0 = blockIdx.x * TILE;
    double acc[R][R] = {};
    for (int kk = 0; kk < k; kk += GK) {
        for (int e = threadIdx.x; e < TILE * GK; e += 256) {
            int r = e / GK, q = e % GK;          // A tile: rows r, cols q
            int gr = row0 + r, gq = kk + q;
            As[q][r] = (gr < m && gq < k) ? A[(size_t)gr * lda + gq] : 0.0;
            int q2 = e / TILE, c2 = e % TILE;    // B tile: rows q2, cols c2
            int gq2 = kk + q2, gc = col0 + c2;
            Bs[q2][c2] = (gq2 < k && gc < n) ? B[(size_t)gq2 * ldb + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GK; ++q) {
            double a[R], b[R];
#pragma unroll
            for (int i = 0; i < R; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < R; ++j) b[j] = Bs[q][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int r = row0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int cc = col0 + tx + 16 * j;
            if (cc >= n) continue;
            double *cp = C + (size_t)r * ldc + cc;
            *cp = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *cp);
        }
    }
}

}  // namespace

void swj_bcopy(cudaStream_t st, int nb, int n, const double *x, double *y, size_t ld, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_bcopy<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, x, y, ld, act);
}
void swj_bfill(cudaStream_t st, int nb, int n, double v, double *x, size_t ld, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_bfill<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, v, x, ld, act);
}
void swj_baxpy(cudaStream_t st, int nb, int n, const double *a_dev, size_t sstride, double a_scale,
               const double *x, double *y, size_t ld, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_baxpy<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, a_dev, sstride, a_scale, x, y, ld, act);
}
void swj_bscale(cudaStream_t st, int nb, int n, const double *s_dev, size_t sstride, double s_scale,
                int invert, const double *x, double *y, size_t ld, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_bscale<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, s_dev, sstride, s_scale, invert, x, y, ld, act);
}
void swj_bnorms(cudaStream_t st, int nb, int n, const double *x, size_t ld, double *red,
                double *out, size_t sstride, const int *act)
{
    int G = nblk(n, kRedThreads);
    if (G > kRedBlocks) G = kRedBlocks;
    if (G < 1) G = 1;
    SWJ_COUNT_LAUNCH();
    k_bnorms1<<<dim3(G, nb), kRedThreads, 0, st>>>(n, x, ld, red, act);
    SWJ_COUNT_LAUNCH();
    k_bnorms2<<<nb, kRedThreads, 0, st>>>(G, red, out, sstride, act);
}
void swj_bmdot(cudaStream_t st, int nb, int n, int rows, const double *V, size_t ld, size_t vstride,
               const double *w, size_t wstride, double *red, double *out, size_t sstride, const int *act)
{
    int G = nblk(n, kRedThreads);
    if (G > 64) G = 64;
    if (G < 1) G = 1;
    SWJ_COUNT_LAUNCH();
    k_bmdot1<<<dim3(G, rows, nb), kRedThreads, 0, st>>>(n, V, ld, vstride, w, wstride, red, act);
    SWJ_COUNT_LAUNCH();
    k_bmdot2<<<dim3(rows, nb), 64, 0, st>>>(G, red, out, sstride, act);
}
void swj_bmgemv_sub(cudaStream_t st, int nb, int n, int rows, const double *V, size_t ld,
                    size_t vstride, const double *coef, size_t sstride, double *w, size_t wstride,
                    const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_bmgemv_sub<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, rows, V, ld, vstride, coef, sstride, w,
                                                        wstride, act);
}
void swj_bcombine(cudaStream_t st, int nb, int n, int rows, const double *Z, size_t ld,
                  size_t zstride, const double *coef, size_t sstride, double *x, size_t xstride,
                  int accumulate, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_bcombine<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(n, rows, Z, ld, zstride, coef, sstride, x,
                                                      xstride, accumulate, act);
}
void swj_dgemm_batched(cudaStream_t st, int m, int n, int k, double alpha,
                       const double *const *A, int lda, const double *const *B, int ldb,
                       double beta, double *const *C, int ldc, int batch, int tile)
{
    if (batch <= 0 || m <= 0 || n <= 0) return;
    SWJ_COUNT_LAUNCH();
    if (tile == 16)
        k_dgemm<16><<<dim3(nblk(n, 16), nblk(m, 16), batch), 256, 0, st>>>(
            m, n, k, alpha, A, nullptr, lda, B, nullptr, ldb, beta, C, nullptr, ldc);
    else if (tile == 32)
        k_dgemm<32><<<dim3(nblk(n, 32), nblk(m, 32), batch), 256, 0, st>>>(
            m, n, k, alpha, A, nullptr, lda, B, nullptr, ldb, beta, C, nullptr, ldc);
    else
        k_dgemm<64><<<dim3(nblk(n, 64), nblk(m, 64), batch), 256, 0, st>>>(
            m, n, k, alpha, A, nullptr, lda, B, nullptr, ldb, beta, C, nullptr, ldc);
}
void swj_dgemm(cudaStream_t st, int m, int n, int k, double alpha, const double *A, int lda,
               const double *B, int ldb, double beta, double *C, int ldc)
{
    if (m <= 0 || n <= 0) return;
    // 16 x 16 output tiles: a single product of a few hundred rows must spread
    // over the SMs (the arithmetic of an element is the same for every tile)
    dim3 grid(nblk(n, 16), nblk(m, 16), 1);
    SWJ_COUNT_LAUNCH();
    k_dgemm<16><<<grid, 256, 0, st>>>(m, n, k, alpha, nullptr, A, lda, nullptr, B, ldb, beta,
                                      nullptr, C, ldc);
}
