// Thread-block-cluster kernels of the preconditioner (FP64).
//
// B300 issues about two FP64 FMAs per clock per SM, so a dense block
// operation on one CTA is slow; these kernels spread each sequential
// factorisation / substitution over the CTAs of one cluster and exchange the
// little data that must be shared (a pivot column, the index of the pivot
// row) through distributed shared memory, with the hardware cluster barrier
// as the only synchronisation.  No kernel here spins on a flag.
#include "swj_internal.h"
#include <mutex>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int kGJThreads = 256;
constexpr int kSweepThreads = 512;

// Gauss-Jordan inverse with partial (row) pivoting of one n x n row-major
// block per cluster.  `work` holds the matrix and is overwritten; the inverse
// is written to `out` (row interchanges undone as a column permutation).
// CTA `rank` of the cluster owns columns [rank w, rank w + w).
__global__ void __launch_bounds__(kGJThreads)
k_gj_cluster(int n, double *work_base, size_t wstride, double *out_base, size_t ostride, int *info)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / ncta;
    double *a = work_base + (size_t)mat * wstride;
    double *out = out_base + (size_t)mat * ostride;
    const int w = (n + ncta - 1) / ncta;
    const int c0 = rank * w, c1 = min(n, c0 + w), nc = max(0, c1 - c0);
    extern __shared__ double sm[];
    double *colf = sm;                          // 2 x n, double buffered
    double *rowk = sm + 2 * n;                  // w
    int *piv = (int *)(rowk + w);               // n
    int *ctl = piv + n;                         // [p, fail] x 2 buffers
    int *sigma = ctl + 4;                       // n
    __shared__ double red_v[kGJThreads / 32];
    __shared__ int red_i[kGJThreads / 32];
    const int tid = threadIdx.x, nth = blockDim.x;
    int fail = 0;
    for (int k = 0; k < n; ++k) {
        const int buf = k & 1;
        const int owner = k / w;
        if (rank == owner) {
            double bv = -1.0;
            int bi = n;
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
            if ((tid & 31) == 0) { red_v[tid >> 5] = bv; red_i[tid >> 5] = bi; }
            __syncthreads();
            if (tid < 32) {
                double v = (tid < nth / 32) ? red_v[tid] : -1.0;
                int ii = (tid < nth / 32) ? red_i[tid] : n;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_xor_sync(0xffffffffu, v, o);
                    int oi = __shfl_xor_sync(0xffffffffu, ii, o);
                    if (ov > v || (ov == v && oi < ii)) { v = ov; ii = oi; }
                }
                if (tid == 0) {
                    red_i[0] = ii;
                    red_v[0] = (v > 0.0 && isfinite(v)) ? 0.0 : 1.0;
                }
            }
            __syncthreads();
            const int p = red_i[0];
            const int f = red_v[0] != 0.0 ? k + 1 : 0;
            // pivot column after the interchange of rows k and p, to every CTA
            for (int e = tid; e < n * ncta; e += nth) {
                int q = e / n, i = e % n;
                int src = (i == k) ? p : ((i == p) ? k : i);
                double v = (f || p >= n) ? 0.0 : a[(size_t)src * n + k];
                double *rc = cl.map_shared_rank(colf + buf * n, q);
                rc[i] = v;
            }
            if (tid < ncta) {
                int *rq = cl.map_shared_rank(ctl + 2 * buf, tid);
                rq[0] = p;
                rq[1] = f;
            }
        }
        cl.sync();
        const int p = ctl[2 * buf];
        fail = ctl[2 * buf + 1];
        if (fail) break;
        if (tid == 0) piv[k] = p;
        if (p != k) {
            for (int j = c0 + tid; j < c1; j += nth) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        }
        __syncthreads();
        const double *cf = colf + buf * n;
        const double rp = 1.0 / cf[k];
        for (int j = c0 + tid; j < c1; j += nth)
            rowk[j - c0] = (j == k) ? rp : a[(size_t)k * n + j] * rp;
        __syncthreads();
        for (int e = tid; e < n * nc; e += nth) {
            int i = e / nc, j = c0 + e % nc;
            size_t ij = (size_t)i * n + j;
            if (i == k) {
                a[ij] = rowk[j - c0];
            } else {
                double base = (j == k) ? 0.0 : a[ij];
                a[ij] = fma(-cf[i], rowk[j - c0], base);
            }
        }
        __syncthreads();
    }
    if (!fail) {
        // column j of the result is column idx[j] of a, idx = swaps applied in reverse
        if (tid == 0) {
            for (int j = 0; j < n; ++j) sigma[j] = j;
            for (int k = n - 1; k >= 0; --k) {
                int p = piv[k];
                int t = sigma[k]; sigma[k] = sigma[p]; sigma[p] = t;
            }
            // invert: sigma[j] = source column of output j -> dest of source column
            for (int j = 0; j < n; ++j) piv[sigma[j]] = j;
        }
        __syncthreads();
        for (int e = tid; e < n * nc; e += nth) {
            int i = e / nc, j = c0 + e % nc;
            out[(size_t)i * n + piv[j]] = a[(size_t)i * n + j];
        }
    }
    if (rank == 0 && tid == 0) info[mat] = fail;
    cl.sync();
}

// The same Gauss-Jordan inverse with each CTA's column slice held in shared
// memory (n x w doubles) for the whole elimination.  Every CTA loads its
// slice before the first cluster barrier and writes the permuted result after
// the last one, so `in` and `out` may be the same block.
__global__ void __launch_bounds__(kGJThreads)
k_gj_cluster_smem(int n, const double *in_base, size_t istride, double *out_base, size_t ostride,
                  int *info)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / ncta;
    const double *in = in_base + (size_t)mat * istride;
    double *out = out_base + (size_t)mat * ostride;
    const int w = (n + ncta - 1) / ncta;
    const int c0 = rank * w, c1 = min(n, c0 + w), nc = max(0, c1 - c0);
    extern __shared__ double sm[];
    double *colf = sm;                          // 2 x n, double buffered
    double *rowk = sm + 2 * n;                  // w
    double *A = rowk + w;                       // n x w slice (row-major, stride w)
    int *piv = (int *)(A + (size_t)n * w);      // n
    int *ctl = piv + n;                         // [p, fail] x 2 buffers
    int *sigma = ctl + 4;                       // n
    __shared__ double red_v[kGJThreads / 32];
    __shared__ int red_i[kGJThreads / 32];
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < n * nc; e += nth) {
        int i = e / nc, jj = e % nc;
        A[(size_t)i * w + jj] = in[(size_t)i * n + c0 + jj];
    }
    __syncthreads();
    int fail = 0;
    for (int k = 0; k < n; ++k) {
        const int buf = k & 1;
        const int owner = k / w;
        if (rank == owner) {
            const int kk = k - c0;
            double bv = -1.0;
            int bi = n;
            for (int i = k + tid; i < n; i += nth) {
                double v = fabs(A[(size_t)i * w + kk]);
                if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if ((tid & 31) == 0) { red_v[tid >> 5] = bv; red_i[tid >> 5] = bi; }
            __syncthreads();
            if (tid < 32) {
                double v = (tid < nth / 32) ? red_v[tid] : -1.0;
                int ii = (tid < nth / 32) ? red_i[tid] : n;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_xor_sync(0xffffffffu, v, o);
                    int oi = __shfl_xor_sync(0xffffffffu, ii, o);
                    if (ov > v || (ov == v && oi < ii)) { v = ov; ii = oi; }
                }
                if (tid == 0) {
                    red_i[0] = ii;
                    red_v[0] = (v > 0.0 && isfinite(v)) ? 0.0 : 1.0;
                }
            }
            __syncthreads();
            const int p = red_i[0];
            const int f = red_v[0] != 0.0 ? k + 1 : 0;
            for (int e = tid; e < n * ncta; e += nth) {
                int q = e / n, i = e % n;
                int src = (i == k) ? p : ((i == p) ? k : i);
                double v = (f || p >= n) ? 0.0 : A[(size_t)src * w + kk];
                double *rc = cl.map_shared_rank(colf + buf * n, q);
                rc[i] = v;
            }
            if (tid < ncta) {
                int *rq = cl.map_shared_rank(ctl + 2 * buf, tid);
                rq[0] = p;
                rq[1] = f;
            }
        }
        cl.sync();
        const int p = ctl[2 * buf];
        fail = ctl[2 * buf + 1];
        if (fail) break;
        if (tid == 0) piv[k] = p;
        if (p != k) {
            for (int jj = tid; jj < nc; jj += nth) {
                double t = A[(size_t)k * w + jj];
                A[(size_t)k * w + jj] = A[(size_t)p * w + jj];
                A[(size_t)p * w + jj] = t;
            }
        }
        __syncthreads();
        const double *cf = colf + buf * n;
        const double rp = 1.0 / cf[k];
        for (int jj = tid; jj < nc; jj += nth)
            rowk[jj] = (c0 + jj == k) ? rp : A[(size_t)k * w + jj] * rp;
        __syncthreads();
        for (int e = tid; e < n * nc; e += nth) {
            int i = e / nc, jj = e % nc;
            size_t ij = (size_t)i * w + jj;
            if (i == k) {
                A[ij] = rowk[jj];
            } else {
                double base = (c0 + jj == k) ? 0.0 : A[ij];
                A[ij] = fma(-cf[i], rowk[jj], base);
            }
        }
        __syncthreads();
    }
    if (!fail) {
        if (tid == 0) {
            for (int j = 0; j < n; ++j) sigma[j] = j;
            for (int k = n - 1; k >= 0; --k) {
                int p = piv[k];
                int t = sigma[k]; sigma[k] = sigma[p]; sigma[p] = t;
            }
            for (int j = 0; j < n; ++j) piv[sigma[j]] = j;
        }
        __syncthreads();
        for (int e = tid; e < n * nc; e += nth) {
            int i = e / nc, jj = e % nc;
            out[(size_t)i * n + piv[c0 + jj]] = A[(size_t)i * w + jj];
        }
    }
    if (rank == 0 && tid == 0) info[mat] = fail;
    cl.sync();
}

// Dot products of one row of up to `nt` n1 x n1 blocks with staged vectors,
// one warp per row.  KC = ceil(n1 / 32) column chunks per lane are loaded
// with independent, fully unrolled loads (two blocks per pass) so that the
// warp keeps 2 KC loads in flight instead of one dependent load at a time.
template <int KC>
__device__ __forceinline__ double row_dots(const double *__restrict__ base, size_t bstride,
                                           const double *__restrict__ vs, int nt, int n1, int lane)
{
    double a0 = 0.0, a1 = 0.0;
    int q = 0;
    for (; q + 1 < nt; q += 2) {
        const double *L0 = base + (size_t)q * bstride, *L1 = L0 + bstride;
        const double *v0 = vs + (size_t)q * n1, *v1 = v0 + n1;
        double x0[KC], x1[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            int c = lane + 32 * k;
            x0[k] = (c < n1) ? __ldg(L0 + c) : 0.0;
            x1[k] = (c < n1) ? __ldg(L1 + c) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            int c = lane + 32 * k;
            if (c < n1) {
                a0 = fma(x0[k], v0[c], a0);
                a1 = fma(x1[k], v1[c], a1);
            }
        }
    }
    if (q < nt) {
        const double *L0 = base + (size_t)q * bstride;
        const double *v0 = vs + (size_t)q * n1;
        double x0[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            int c = lane + 32 * k;
            x0[k] = (c < n1) ? __ldg(L0 + c) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            int c = lane + 32 * k;
            if (c < n1) a0 = fma(x0[k], v0[c], a0);
        }
    }
    double s = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// One cluster solves S x = t with the block-banded LU factors of S:
// `band` ([M][2h+1][n1][n1]) holds inv_i in slot h of row i and the blocks
// S_ij (j < i, as they were at step j) in the slots left of it; `W`
// ([M][h][n1][n1]) holds W_ik = inv_i S_ik (k > i).
//   forward   y_i = t_i - sum_{j=i-h}^{i-1} S_ij z_j  (y overwrites t),  z_i = inv_i y_i
//   backward  x_i = z_i - sum_{k=i+1}^{i+h} W_ik x_k
// Each CTA computes a slice of the rows of every block step (a warp per
// row); the vectors a step reads are staged in shared memory after the
// cluster barrier that ends the previous phase.
template <int KC>
__global__ void __launch_bounds__(kSweepThreads)
k_band_sweep(int n1, int M, int h, const double *__restrict__ band, size_t band_stride,
             const double *__restrict__ W, size_t w_stride, double *y, double *z, double *x,
             size_t vec_stride, const int *__restrict__ act)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int inst = blockIdx.x / ncta;
    if (!SWJ_INST_ACTIVE(act, inst)) return;   // the whole cluster leaves together
    band += (size_t)inst * band_stride;
    W += (size_t)inst * w_stride;
    y += (size_t)inst * vec_stride;
    z += (size_t)inst * vec_stride;
    x += (size_t)inst * vec_stride;
    const int nb = 2 * h + 1;
    const size_t n2 = (size_t)n1 * n1;
    const int rows = (n1 + ncta - 1) / ncta;
    const int r0 = rank * rows, r1 = min(n1, r0 + rows);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    extern __shared__ double vs[];   // up to max(h, 1) x n1 staged vectors
    for (int i = 0; i < M; ++i) {
        const int j0 = max(0, i - h), nt = i - j0;
        if (nt > 0) {
            for (int e = threadIdx.x; e < nt * n1; e += blockDim.x)
                vs[e] = z[(size_t)(j0 + e / n1) * n1 + e % n1];
            __syncthreads();
            for (int r = r0 + warp; r < r1; r += nw) {
                const double *L = band + ((size_t)i * nb + (j0 - i + h)) * n2 + (size_t)r * n1;
                double s = row_dots<KC>(L, n2, vs, nt, n1, lane);
                if (lane == 0) y[(size_t)i * n1 + r] -= s;
            }
            cl.sync();
        }
        for (int e = threadIdx.x; e < n1; e += blockDim.x) vs[e] = y[(size_t)i * n1 + e];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            const double *Inv = band + ((size_t)i * nb + h) * n2 + (size_t)r * n1;
            double s = row_dots<KC>(Inv, n2, vs, 1, n1, lane);
            if (lane == 0) z[(size_t)i * n1 + r] = s;
        }
        cl.sync();
    }
    for (int i = M - 1; i >= 0; --i) {
        const int k1 = min(M - 1, i + h), nt = k1 - i;
        for (int e = threadIdx.x; e < nt * n1; e += blockDim.x)
            vs[e] = x[(size_t)(i + 1 + e / n1) * n1 + e % n1];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            const double *Wm = W + ((size_t)i * h) * n2 + (size_t)r * n1;
            double s = row_dots<KC>(Wm, n2, vs, nt, n1, lane);
            if (lane == 0) x[(size_t)i * n1 + r] = z[(size_t)i * n1 + r] - s;
        }
        cl.sync();
    }
}

// 16 CTAs per cluster where the device runs such clusters (a non-portable
// size), else the portable 8.
int cluster_ctas(const void *kernel, int threads, size_t smem)
{
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 8;
    }
    return 16;
}

}  // namespace

size_t gj_smem_bytes(int n, int cs)
{
    const int w = (n + cs - 1) / cs;
    return (size_t)(2 * n + w + (size_t)n * w) * sizeof(double) + (size_t)(2 * n + 4) * sizeof(int);
}

// Lazily settled launch attributes, shared by every context and host thread.
static std::mutex g_attr_mutex;
static int g_cs_smem = 0;

// true when the shared-memory Gauss-Jordan variant applies to n x n blocks
// (then input and output may be the same block)
static int gj_smem_cluster()
{
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!g_cs_smem) g_cs_smem = cluster_ctas((const void *)k_gj_cluster_smem, kGJThreads, 64 * 1024);
    return g_cs_smem;
}

bool swj_gj_inplace(int n)
{
    return gj_smem_bytes(n, gj_smem_cluster()) <= 200 * 1024;
}

int swj_gj_inverse_cluster(cudaStream_t st, int n, int count, double *work, size_t wstride,
                           double *out, size_t ostride, int *info)
{
    static int cs_g = 0;
    static size_t set_s = 48 * 1024, set_g = 48 * 1024;
    const bool use_smem = swj_gj_inplace(n);
    const void *kern = use_smem ? (const void *)k_gj_cluster_smem : (const void *)k_gj_cluster;
    int cs;
    size_t smem;
    {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        if (!use_smem && !cs_g) cs_g = cluster_ctas((const void *)k_gj_cluster, kGJThreads, 64 * 1024);
        cs = use_smem ? g_cs_smem : cs_g;
        const int w = (n + cs - 1) / cs;
        smem = use_smem ? gj_smem_bytes(n, cs)
                        : (size_t)(2 * n + w) * sizeof(double) + (size_t)(2 * n + 4) * sizeof(int);
        size_t &set = use_smem ? set_s : set_g;
        if (smem > set) {
            SWJ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            set = smem;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * count);
    cfg.blockDim = dim3(kGJThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SWJ_COUNT_LAUNCH();
    if (use_smem)
        SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster_smem, n, (const double *)work, wstride, out,
                                        ostride, info));
    else
        SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster, n, work, wstride, out, ostride, info));
    return SWJ_OK;
}

// Cluster size and shared-memory limit of the sweep kernel are settled on the
// first call with prepare = true (from the preconditioner set-up), so that a
// launch recorded into a CUDA graph makes no attribute call.
template <int KC>
int launch_sweep(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t bs,
                 const double *W, size_t ws, double *y, double *z, double *x, size_t vs, const int *act,
                 bool prepare)
{
    static int cs_cached = 0;
    static size_t smem_set = 48 * 1024;
    const size_t smem = (size_t)(h > 0 ? h : 1) * n1 * sizeof(double);
    int cs;
    {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        if (!cs_cached) cs_cached = cluster_ctas((const void *)k_band_sweep<KC>, kSweepThreads, 64 * 1024);
        cs = cs_cached;
        if (smem > smem_set) {
            SWJ_CUDA_TRY(cudaFuncSetAttribute(k_band_sweep<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            smem_set = smem;
        }
    }
    if (prepare) return SWJ_OK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * nb);
    cfg.blockDim = dim3(kSweepThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SWJ_COUNT_LAUNCH();
    SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_sweep<KC>, n1, M, h, band, bs, W, ws, y, z, x, vs, act));
    return SWJ_OK;
}

int swj_band_sweep_cluster(cudaStream_t st, int nb, int n1, int M, int h, const double *band,
                           size_t bs, const double *W, size_t ws, double *y, double *z, double *x,
                           size_t vs, const int *act, bool prepare)
{
    const int kc = (n1 + 31) / 32;
#define SWJ_SWEEP(K) return launch_sweep<K>(st, nb, n1, M, h, band, bs, W, ws, y, z, x, vs, act, prepare)
    if (kc <= 2) SWJ_SWEEP(2);
    if (kc <= 4) SWJ_SWEEP(4);
    if (kc <= 6) SWJ_SWEEP(6);
    if (kc <= 8) SWJ_SWEEP(8);
    if (kc <= 12) SWJ_SWEEP(12);
    if (kc <= 16) SWJ_SWEEP(16);
    if (kc <= 24) SWJ_SWEEP(24);
    SWJ_SWEEP(32);
#undef SWJ_SWEEP
}
