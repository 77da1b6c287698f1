// Thread-block-cluster kernels of the preconditioner (FP64).
//
// B300 issues about two FP64 FMAs per clock per SM, so a dense block
// operation on one CTA is slow; these kernels spread each sequential
// factorisation / substitution over the CTAs of one cluster and exchange the
// little data that must be shared (a pivot column, the index of the pivot
// row) through distributed shared memory, with the hardware cluster barrier
// as the only synchronisation.  No kernel here spins on a flag.
#include "swj_internal.h"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int kGJThreads = 256;
constexpr int kSweepThreads = 256;

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

// One cluster solves S x = t with the block-banded LU factors of S stored in
// `band` ([M][2h+1][n1][n1]; slot h of row i holds inv_i, slots < h hold L_ij,
// slots > h hold W_ik = inv_i U_ik):
//   forward   y_i = t_i - sum_{j=i-h}^{i-1} L_ij y_j      (y overwrites t)
//   backward  x_i = inv_i y_i - sum_{k=i+1}^{i+h} W_ik x_k
// Each CTA computes a slice of the rows of every block step (a warp per
// row); the vectors a step reads are staged in shared memory after the
// cluster barrier that ends the previous step.
__global__ void __launch_bounds__(kSweepThreads)
k_band_sweep(int n1, int M, int h, const double *__restrict__ band, double *y, double *x)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int nb = 2 * h + 1;
    const size_t n2 = (size_t)n1 * n1;
    const int rows = (n1 + ncta - 1) / ncta;
    const int r0 = rank * rows, r1 = min(n1, r0 + rows);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    extern __shared__ double vs[];   // (h + 1) x n1 staged vectors
    for (int i = 1; i < M; ++i) {
        const int j0 = max(0, i - h), nt = i - j0;
        for (int e = threadIdx.x; e < nt * n1; e += blockDim.x)
            vs[e] = y[(size_t)(j0 + e / n1) * n1 + e % n1];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            double s = 0.0;
            for (int q = 0; q < nt; ++q) {
                const double *L = band + ((size_t)i * nb + (j0 + q - i + h)) * n2 + (size_t)r * n1;
                const double *v = vs + (size_t)q * n1;
                for (int c = lane; c < n1; c += 32) s = fma(L[c], v[c], s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[(size_t)i * n1 + r] -= s;
        }
        cl.sync();
    }
    for (int i = M - 1; i >= 0; --i) {
        const int k1 = min(M - 1, i + h), nt = k1 - i;
        for (int e = threadIdx.x; e < n1; e += blockDim.x) vs[e] = y[(size_t)i * n1 + e];
        for (int e = threadIdx.x; e < nt * n1; e += blockDim.x)
            vs[n1 + e] = x[(size_t)(i + 1 + e / n1) * n1 + e % n1];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            const double *Inv = band + ((size_t)i * nb + h) * n2 + (size_t)r * n1;
            double s = 0.0;
            for (int c = lane; c < n1; c += 32) s = fma(Inv[c], vs[c], s);
            for (int q = 0; q < nt; ++q) {
                const double *Wm = band + ((size_t)i * nb + (q + 1 + h)) * n2 + (size_t)r * n1;
                const double *v = vs + (size_t)(q + 1) * n1;
                for (int c = lane; c < n1; c += 32) s = fma(-Wm[c], v[c], s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) x[(size_t)i * n1 + r] = s;
        }
        cl.sync();
    }
}

int cluster_size_for(int n)
{
    (void)n;
    return 8;
}

}  // namespace

int swj_gj_inverse_cluster(cudaStream_t st, int n, int count, double *work, size_t wstride,
                           double *out, size_t ostride, int *info)
{
    const int cs = cluster_size_for(n);
    const int w = (n + cs - 1) / cs;
    size_t smem = (size_t)(2 * n + w) * sizeof(double) + (size_t)(2 * n + 4) * sizeof(int);
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
    SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster, n, work, wstride, out, ostride, info));
    return SWJ_OK;
}

int swj_band_sweep_cluster(cudaStream_t st, int n1, int M, int h, const double *band, double *y,
                           double *x)
{
    const int cs = 8;
    size_t smem = (size_t)(h + 1) * n1 * sizeof(double);
    if (smem > 48 * 1024) {
        static thread_local size_t set_to = 0;
        if (set_to < smem) {
            SWJ_CUDA_TRY(cudaFuncSetAttribute(k_band_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
            set_to = smem;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
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
    SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_sweep, n1, M, h, band, y, x));
    return SWJ_OK;
}
