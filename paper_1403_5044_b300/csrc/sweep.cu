// Block forward / backward substitution with the band LU factors of the
// Schur complement S (Appendix C, middle stage of the three-stage solve), FP64.
//
// The set-up leaves, for block row i of S (n1 x n1 blocks, half bandwidth h):
//   band slot h       inv_i = S_ii^-1 (after the updates of steps < i)
//   band slot h - d   L_{i,i-d} = inv_i S_{i,i-d}          (d = 1..h)
//   W[i][e - 1]       W_{i,i+e} = inv_i S_{i,i+e}          (e = 1..h)
// so that S x = t is solved by
//   p_i = inv_i t_i                                         (all i at once)
//   z_i = p_i - sum_{d=1..h} L_{i,i-d} z_{i-d}              (forward, i = 0..M-1)
//   x_i = z_i - sum_{e=1..h} W_{i,i+e} x_{i+e}              (backward, i = M-1..0)
// Only the forward and backward recurrences are sequential.  Every block
// product is a set of row dots (one warp per row, one fixed order of
// operations).  A recurrence row keeps the nearest block's dot as 32 lane
// partials, adds the farther blocks' finished dots into lanes 2, 3, ... (the
// block at distance d into lane d), sums the lanes with one butterfly and
// subtracts the sum: on B300 every FP64 instruction of a warp holds its SM
// sub-partition for ~64 cycles, so one butterfly instead of a subtraction per
// block matters on the sequential path.  The single-cluster and the
// multi-cluster sweeps below do exactly this and return identical bits.
#include "swj_internal.h"
#include <map>
#include <mutex>
#include <tuple>
#include <cooperative_groups.h>
#include <cuda_pipeline.h>

namespace cg = cooperative_groups;

namespace {

constexpr int kSweepThreads = 512;

// Bit pattern written into every value the multi-cluster sweep publishes
// before its launch: a signalling NaN, which no FP64 operation returns (a NaN
// result is always quiet), so a consumer polls a value until it differs.
constexpr unsigned long long kUnset = 0x7FF4DEAD7FF4DEADull;

// a poll that has not seen its value after poll_limit reads (a kernel
// argument; kSwjPollLimit = 2^21 by default, about a second at L2 latency)
// gives up and reports through the error word

__device__ __forceinline__ double ld_relaxed(const double *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double((long long)v);
}

__device__ __forceinline__ void st_relaxed(double *p, double x)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(x))
                 : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t map_rank(uint32_t a, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 8-byte store into the shared memory of a CTA of the cluster that completes
// `bytes` of the transaction count of that CTA's mbarrier (both addresses
// from map_rank)
__device__ __forceinline__ void st_async_f64(uint32_t dst, double v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
                 ::"r"(dst), "l"((unsigned long long)__double_as_longlong(v)), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mb, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *mb, int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *mb, int parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_addr(mb)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool unset(double x) { return (unsigned long long)__double_as_longlong(x) == kUnset; }

__device__ __forceinline__ double warp_sum(double a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Dot product of one n1-row with an n1-vector, one warp: lane l accumulates
// columns l, l + 32, ... with FMAs in that order, then a butterfly sum; every
// lane returns the result.
template <int KC>
__device__ __forceinline__ double block_dot_partial(const double *row, const double *v, int n1, int lane)
{
    double x[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        x[k] = (c < n1) ? row[c] : 0.0;
    }
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        if (c < n1) a = fma(x[k], v[c], a);
    }
    return a;
}

template <int KC>
__device__ __forceinline__ double block_dot(const double *row, const double *v, int n1, int lane)
{
    return warp_sum(block_dot_partial<KC>(row, v, n1, lane));
}

// Two dots at once (the loads of both in flight together), each with exactly
// the arithmetic of block_dot.
template <int KC>
__device__ __forceinline__ void block_dot2(const double *row0, const double *v0, const double *row1,
                                           const double *v1, int n1, int lane, double &s0, double &s1)
{
    double x0[KC], x1[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        x0[k] = (c < n1) ? row0[c] : 0.0;
        x1[k] = (c < n1) ? row1[c] : 0.0;
    }
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        if (c < n1) {
            a0 = fma(x0[k], v0[c], a0);
            a1 = fma(x1[k], v1[c], a1);
        }
    }
    s0 = warp_sum(a0);
    s1 = warp_sum(a1);
}

// v - sum_{q=0..nt-1} dot(row q, vector q) in the recurrences' order: the
// lane partials of dot 0, dot q (q >= 1, finished) added into lane q + 1, one
// butterfly, one subtraction.  Rows at base + q bstride (global memory;
// bstride may be negative), vectors at vs + q n1 (shared).
template <int KC>
__device__ __forceinline__ double sub_dots(double v, const double *base, long long bstride, const double *vs,
                                           int nt, int n1, int lane)
{
    if (nt == 0) return v - warp_sum(0.0);
    double a = block_dot_partial<KC>(base, vs, n1, lane);
    int q = 1;
    for (; q + 1 < nt; q += 2) {
        double s0, s1;
        block_dot2<KC>(base + q * bstride, vs + (size_t)q * n1, base + (q + 1) * bstride,
                       vs + (size_t)(q + 1) * n1, n1, lane, s0, s1);
        if (lane == q + 1) a += s0;
        if (lane == q + 2) a += s1;
    }
    if (q < nt) {
        const double s0 = block_dot<KC>(base + q * bstride, vs + (size_t)q * n1, n1, lane);
        if (lane == q + 1) a += s0;
    }
    return v - warp_sum(a);
}

// p_i = inv_i t_i for every block row of every active instance (one warp per
// row).  Optionally also sets fill1[0, n1f) and fill2[0, n2f) to kUnset (the
// multi-cluster sweep's published values; grid-stride over blockIdx.x of
// instance 0).
template <int KC>
__global__ void __launch_bounds__(256)
k_block_p(int n1, int M, int h, const double *__restrict__ band, size_t bs, const double *__restrict__ t,
          size_t ts, double *__restrict__ p, size_t ps, const int *__restrict__ act, double *fill1,
          size_t n1f, double *fill2, size_t n2f)
{
    const int inst = blockIdx.y;
    if (blockIdx.y == 0 && (fill1 || fill2)) {
        const double u = __longlong_as_double((long long)kUnset);
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n1f; e += stride) fill1[e] = u;
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2f; e += stride) fill2[e] = u;
    }
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n1 * M) return;
    const int l = warp / n1, r = warp % n1;
    const size_t n2 = (size_t)n1 * n1;
    const double *inv = band + (size_t)inst * bs + ((size_t)l * (2 * h + 1) + h) * n2 + (size_t)r * n1;
    const double s = block_dot<KC>(inv, t + (size_t)inst * ts + (size_t)l * n1, n1, lane);
    if (lane == 0) p[(size_t)inst * ps + (size_t)l * n1 + r] = s;
}

// One cluster per instance runs both recurrences; z holds p on entry and z
// on exit, x receives the solution.  Each CTA computes a slice of the rows of
// every block step (a warp per row); the vectors a step reads are staged in
// shared memory after the cluster barrier that ends the previous step.  The
// forward recurrence runs over block rows 1..F-1 (z_0 = p_0), the backward
// one from row Bs down to 0; rows of x above Bs are inputs (F = M and
// Bs = M - 1 for the whole band).
template <int KC>
__global__ void __launch_bounds__(kSweepThreads)
k_band_sweep(int n1, int M, int h, const double *__restrict__ band, size_t band_stride,
             const double *__restrict__ W, size_t w_stride, double *z, size_t zs, double *x, size_t xs,
             const int *__restrict__ act, int F, int Bs)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int inst = blockIdx.x / ncta;
    if (!SWJ_INST_ACTIVE(act, inst)) return;   // the whole cluster leaves together
    band += (size_t)inst * band_stride;
    W += (size_t)inst * w_stride;
    z += (size_t)inst * zs;
    x += (size_t)inst * xs;
    const int nbk = 2 * h + 1;
    const size_t n2 = (size_t)n1 * n1;
    const int rows = (n1 + ncta - 1) / ncta;
    const int r0 = min(n1, rank * rows), r1 = min(n1, r0 + rows);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    extern __shared__ double vs[];   // up to h staged vectors of n1
    for (int i = 1; i < F; ++i) {
        const int nt = min(i, h);
        // vs[d - 1] = z_{i-d}
        for (int e = threadIdx.x; e < nt * n1; e += blockDim.x) vs[e] = z[(size_t)(i - 1 - e / n1) * n1 + e % n1];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            // slots h-1, h-2, ... hold L_{i,i-1}, L_{i,i-2}, ...: stride -n2
            const double *L = band + ((size_t)i * nbk + (h - 1)) * n2 + (size_t)r * n1;
            const double v = sub_dots<KC>(z[(size_t)i * n1 + r], L, -(long long)n2, vs, nt, n1, lane);
            if (lane == 0) z[(size_t)i * n1 + r] = v;
        }
        cl.sync();
    }
    for (int i = Bs; i >= 0; --i) {
        const int nt = min(M - 1 - i, h);
        // vs[e - 1] = x_{i+e}
        for (int e = threadIdx.x; e < nt * n1; e += blockDim.x) vs[e] = x[(size_t)(i + 1 + e / n1) * n1 + e % n1];
        __syncthreads();
        for (int r = r0 + warp; r < r1; r += nw) {
            const double *Wr = W + ((size_t)i * h) * n2 + (size_t)r * n1;
            const double v = sub_dots<KC>(z[(size_t)i * n1 + r], Wr, (long long)n2, vs, nt, n1, lane);
            if (lane == 0) x[(size_t)i * n1 + r] = v;
        }
        cl.sync();
    }
}

// The same recurrences for ni instances (1 or 2) on ni + hsets (h - 1)
// clusters.  Cluster q < ni (critical for instance q) keeps only the product
// with the block next to the diagonal:
//   forward   z_i = p_i - L_{i,i-1} z_{i-1} - sum_{d>=2} c_{i,d}
//   backward  x_i = z_i - W_{i,i+1} x_{i+1} - sum_{e>=2} b_{i,e}
// and the helper clusters compute the older terms as soon as their vector
// exists: c_{j+d,d} = L_{j+d,j} z_j and b_{k-d,d} = W_{k-d,k} x_k, one helper
// per d = 2..h for every instance (hsets = 1) or for each instance (hsets =
// ni).  Nothing is signalled apart from the values
// themselves: z, x and the term slots cf, cb ([M][h+1][n1], slots 2..h used)
// are set to kUnset before the launch where it writes them, producers store
// each value once (relaxed, 8 bytes, single-copy atomic) and consumers poll it
// until it is set.  In a critical cluster each CTA owns a slice of rows (at
// least one), takes the next step's block rows into shared memory with
// cp.async while the current step runs, keeps p and then its z rows in shared
// memory, reads the helpers' terms one step ahead, and sends every new
// element of z_i / x_i into the shared memory of all CTAs of the cluster by
// st.async, whose arrival each CTA awaits on an mbarrier (no cluster barrier
// per step).  The helpers are independent CTAs.  The launch is cooperative,
// so all clusters are resident at once; a poll that runs out sets *err = 1
// (as does a barrier wait that runs out), and a launch whose clusters are not
// of cs CTAs, each with one to two rows per warp, sets *err = 2 and returns
// at once.  The forward recurrence covers rows F0..F1-1 and the backward one
// rows B1 down to B0; the rows of z below F0 and of x above B1 are inputs
// (set before the launch), and zs starts from p (pass z as p for a launch
// without forward rows).  Instance q's band, W, vectors and term slots are at
// q bst, q wst, q vst, q sst.
template <int KC>
__global__ void __launch_bounds__(kSweepThreads)
k_band_sweep_mc(int n1, int M, int h, int ni, int hsets, const double *__restrict__ band, size_t bst,
                const double *__restrict__ W, size_t wst, const double *__restrict__ p, double *z, double *x,
                size_t vst, double *cf, double *cb, size_t sst, int cs, int *err, int F0, int F1, int B1,
                int B0, int poll_limit)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    if (ncta != cs || (int)gridDim.x != cs * (ni + hsets * (h - 1)) || (cs - 1) * ((n1 + cs - 1) / cs) >= n1 ||
        (n1 + cs - 1) / cs > 2 * (kSweepThreads / 32)) {   // the same decision in every CTA
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const int rank = (int)cl.block_rank();
    const int cid = blockIdx.x / ncta;
    const int nbk = 2 * h + 1, hs = h + 1;
    const size_t n2 = (size_t)n1 * n1;
    const int rows = (n1 + ncta - 1) / ncta;
    const int r0 = min(n1, rank * rows), r1 = min(n1, r0 + rows), nr = r1 - r0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    extern __shared__ double sm[];
    double *rb = sm;                              // [2][rows][n1] block rows, by step parity
    double *vz = rb + 2 * (size_t)rows * n1;      // [2][n1]: z by parity (helpers: the staged vector)
    double *vx = vz + 2 * (size_t)n1;             // [2][n1]: x by parity
    double *zs = vx + 2 * (size_t)n1;             // [M][rows]: this CTA's rows of z
    __shared__ int bad;
    __shared__ __align__(8) uint64_t mbz[2], mbx[2];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    // rows [r0, r1) of one block into rb[buf] (16-byte copies where aligned)
    auto prefetch = [&](int buf, const double *blk) {
        double *dst = rb + (size_t)buf * rows * n1;
        const double *src = blk + (size_t)r0 * n1;
        const int ne = nr * n1;
        if ((n1 & 1) == 0) {
            for (int e = 2 * threadIdx.x; e < ne; e += 2 * blockDim.x) __pipeline_memcpy_async(dst + e, src + e, 16);
        } else {
            for (int e = threadIdx.x; e < ne; e += blockDim.x) __pipeline_memcpy_async(dst + e, src + e, 8);
        }
    };
    // finishes a poll whose first read gave v
    auto poll = [&](const double *a, double v) {
        if (unset(v) && !*(volatile int *)&bad) {
            int it = 0;
            while (unset(v = ld_relaxed(a)))
                if (++it > poll_limit || *(volatile int *)&bad) {
                    bad = 1;
                    atomicExch(err, 1);
                    break;
                }
        }
        return v;
    };
    if (cid < ni) {
        // critical cluster of instance cid
        band += (size_t)cid * bst;
        W += (size_t)cid * wst;
        p += (size_t)cid * vst;
        z += (size_t)cid * vst;
        x += (size_t)cid * vst;
        cf += (size_t)cid * sst;
        cb += (size_t)cid * sst;
        // Exchange inside the cluster: element r of z_i (x_i) goes from the CTA
        // that owns row r to vz[t & 1][r] (vx[t & 1][r]) of every CTA, t the
        // step's index in its recurrence (i - F0, B1 - i), by st.async, which
        // completes mbz[t & 1] (mbx[t & 1]) there; each CTA arms that barrier
        // for n1 * 8 bytes at the start of the step and waits on it (the use
        // count >> 1 gives the phase) before reading the vector.  A buffer is
        // rewritten two steps later, only after every CTA produced its rows of
        // the step in between, i.e. after every reader of the buffer has
        // finished with it.  An input vector next to the first step (z_{F0-1},
        // x_{B1+1}) is staged in buffer 1 directly, with the first step's
        // block rows in rb[0].
        const int rpw = (nr + nw - 1) / nw;   // rows per warp (<= 2, checked at launch)
        if (threadIdx.x == 0) {
            for (int q = 0; q < 2; ++q) {
                mbar_init(&mbz[q], 1);
                mbar_init(&mbx[q], 1);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        // this CTA's rows of p into zs (z overwrites them step by step)
        for (int e = threadIdx.x; e < M * nr; e += blockDim.x)
            zs[(size_t)(e / nr) * rows + e % nr] = p[(size_t)(e / nr) * n1 + r0 + e % nr];
        cl.sync();
        // The exchange inside the cluster goes on after a poll of another
        // cluster's value gave up (every CTA still sends its rows each step),
        // so these waits are not skipped then: a barrier is re-armed only
        // after its previous phase completed, and no CTA leaves while values
        // sent to it are in flight.  They wait on this cluster alone, so
        // their bound is the built-in one, not poll_limit.
        auto wait_bar = [&](uint64_t *mb, int parity) {
            int it = 0;
            while (!mbar_test(mb, parity))
                if (++it > kSwjPollLimit) {
                    bad = 1;
                    atomicExch(err, 1);
                    return;
                }
        };
        auto send = [&](double *vec, uint64_t *mb, int r, double v) {
            if (lane < ncta) st_async_f64(map_rank(smem_addr(vec + r), lane), v, map_rank(smem_addr(mb), lane));
        };
        // lane d (2..h) of the warp of row rr reads term d of that row (first read;
        // poll() finishes it when the value is used)
        double cur[2] = {0.0, 0.0};
        auto read_terms = [&](const double *slots, int step, int nd, double &o0, double &o1) {
            if (lane >= 2 && lane <= nd) {
                const double *a = slots + ((size_t)step * hs + lane) * n1 + r0;
                if (warp < nr) o0 = ld_relaxed(a + warp);
                if (warp + nw < nr) o1 = ld_relaxed(a + warp + nw);
            }
        };
        // ---- forward: step t = i - F0 reads L_{i,i-1} from rb[t & 1] and
        //      prefetches L_{i+1,i} into the other buffer
        const bool fpre = F0 > 0 && F1 > F0;
        if (fpre) {
            for (int e = threadIdx.x; e < n1; e += blockDim.x) vz[n1 + e] = z[(size_t)(F0 - 1) * n1 + e];
            prefetch(0, band + ((size_t)F0 * nbk + (h - 1)) * n2);
            __pipeline_commit();
        }
        if (F1 > F0) read_terms(cf, F0, min(h, F0), cur[0], cur[1]);
        for (int i = F0; i < F1; ++i) {
            const int t = i - F0;
            const int nd = min(h, i);   // terms c_{i,2..nd}
            __syncthreads();            // every warp is done with step t - 1 (rb, zs)
            if (threadIdx.x == 0) mbar_expect(&mbz[t & 1], n1 * (int)sizeof(double));
            if (i + 1 < F1) prefetch((t + 1) & 1, band + ((size_t)(i + 1) * nbk + (h - 1)) * n2);
            __pipeline_commit();
            __pipeline_wait_prior(1);
            __syncthreads();
            if (t > 0) wait_bar(&mbz[(t - 1) & 1], ((t - 1) >> 1) & 1);
            double nxt[2] = {0.0, 0.0};
            if (i + 1 < F1) read_terms(cf, i + 1, min(h, i + 1), nxt[0], nxt[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int rr = warp + q * nw;
                if (q >= rpw || rr >= nr) break;
                const int r = r0 + rr;
                double a = 0.0;
                if (t > 0 || fpre)
                    a = block_dot_partial<KC>(rb + ((size_t)(t & 1) * rows + rr) * n1, vz + (size_t)((t - 1) & 1) * n1, n1, lane);
                if (lane >= 2 && lane <= nd) a += (cur[q] = poll(cf + ((size_t)i * hs + lane) * n1 + r, cur[q]));
                const double v = zs[(size_t)i * rows + rr] - warp_sum(a);
                if (lane == 0) {
                    st_relaxed(z + (size_t)i * n1 + r, v);
                    zs[(size_t)i * rows + rr] = v;
                }
                send(vz + (size_t)(t & 1) * n1, &mbz[t & 1], r, v);
            }
            cur[0] = nxt[0];
            cur[1] = nxt[1];
        }
        // ---- backward: step t = B1 - i reads W_{i,i+1} from rb[t & 1] and
        //      prefetches W_{i-1,i} into the other buffer
        __syncthreads();
        const bool bpre = B1 >= B0 && B1 < M - 1;
        if (bpre) {
            for (int e = threadIdx.x; e < n1; e += blockDim.x) vx[n1 + e] = x[(size_t)(B1 + 1) * n1 + e];
            prefetch(0, W + ((size_t)B1 * h) * n2);
            __pipeline_commit();
        }
        if (B1 >= B0) read_terms(cb, B1, min(h, M - 1 - B1), cur[0], cur[1]);
        for (int i = B1; i >= B0; --i) {
            const int t = B1 - i;
            const int ne = min(h, M - 1 - i);   // terms b_{i,2..ne}
            __syncthreads();
            if (threadIdx.x == 0) mbar_expect(&mbx[t & 1], n1 * (int)sizeof(double));
            if (i - 1 >= B0) prefetch((t + 1) & 1, W + ((size_t)(i - 1) * h) * n2);
            __pipeline_commit();
            __pipeline_wait_prior(1);
            __syncthreads();
            if (t > 0) wait_bar(&mbx[(t - 1) & 1], ((t - 1) >> 1) & 1);
            double nxt[2] = {0.0, 0.0};
            if (i - 1 >= B0) read_terms(cb, i - 1, min(h, M - i), nxt[0], nxt[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int rr = warp + q * nw;
                if (q >= rpw || rr >= nr) break;
                const int r = r0 + rr;
                double a = 0.0;
                if (t > 0 || bpre)
                    a = block_dot_partial<KC>(rb + ((size_t)(t & 1) * rows + rr) * n1, vx + (size_t)((t - 1) & 1) * n1, n1, lane);
                if (lane >= 2 && lane <= ne) a += (cur[q] = poll(cb + ((size_t)i * hs + lane) * n1 + r, cur[q]));
                const double v = zs[(size_t)i * rows + rr] - warp_sum(a);
                if (lane == 0) st_relaxed(x + (size_t)i * n1 + r, v);
                send(vx + (size_t)(t & 1) * n1, &mbx[t & 1], r, v);
            }
            cur[0] = nxt[0];
            cur[1] = nxt[1];
        }
        __pipeline_wait_prior(0);
        // the last vectors were sent but not read: wait for them, so that no
        // store into this CTA's shared memory is in flight when it exits
        if (F1 > F0) {
            const int tl = F1 - 1 - F0;
            wait_bar(&mbz[tl & 1], (tl >> 1) & 1);
        }
        if (B1 >= B0) {
            const int tl = B1 - B0;
            wait_bar(&mbx[tl & 1], (tl >> 1) & 1);
        }
        cl.sync();
    } else {
        const int hid = cid - ni, d = hid % (h - 1) + 2;   // d = 2..h
        // the instances of this helper: all (q = q0 + 0..nq-1), or one
        const int q0 = hsets == 1 ? 0 : hid / (h - 1), nq = hsets == 1 ? ni : 1;
        // forward terms c_{j+d,d} = L_{j+d,j} z_j (slot h - d of block row j + d)
        // for the rows j + d in [F0, F1), instance by instance within a step:
        // item w = (j - j0) nq + (q - q0), the next item's block rows prefetched
        const int j0 = max(0, F0 - d), nf = max(0, F1 - d - j0) * nq;
        auto fblk = [&](int w) {
            const int j = j0 + w / nq, q = q0 + w % nq;
            return band + (size_t)q * bst + ((size_t)(j + d) * nbk + (h - d)) * n2;
        };
        if (nf > 0) prefetch(0, fblk(0));
        __pipeline_commit();
        for (int w = 0; w < nf; ++w) {
            const int j = j0 + w / nq, q = q0 + w % nq, buf = w & 1;
            if (w + 1 < nf) prefetch(buf ^ 1, fblk(w + 1));
            __pipeline_commit();
            const double *zq = z + (size_t)q * vst + (size_t)j * n1;
            for (int e = threadIdx.x; e < n1; e += blockDim.x) vz[e] = poll(zq + e, ld_relaxed(zq + e));
            __pipeline_wait_prior(1);
            __syncthreads();
            double *cq = cf + (size_t)q * sst + ((size_t)(j + d) * hs + d) * n1 + r0;
            for (int rr = warp; rr < nr; rr += nw) {
                const double s = block_dot<KC>(rb + ((size_t)buf * rows + rr) * n1, vz, n1, lane);
                if (lane == 0) st_relaxed(cq + rr, s);
            }
            __syncthreads();
        }
        __pipeline_wait_prior(0);
        __syncthreads();
        // backward terms b_{k-d,d} = W_{k-d,k} x_k for the rows k - d in [B0, B1]
        const int k0 = min(M - 1, B1 + d), nbw = max(0, k0 - d - B0 + 1) * nq;
        auto bblk = [&](int w) {
            const int k = k0 - w / nq, q = q0 + w % nq;
            return W + (size_t)q * wst + ((size_t)(k - d) * h + (d - 1)) * n2;
        };
        if (nbw > 0) prefetch(0, bblk(0));
        __pipeline_commit();
        for (int w = 0; w < nbw; ++w) {
            const int k = k0 - w / nq, q = q0 + w % nq, buf = w & 1;
            if (w + 1 < nbw) prefetch(buf ^ 1, bblk(w + 1));
            __pipeline_commit();
            const double *xq = x + (size_t)q * vst + (size_t)k * n1;
            for (int e = threadIdx.x; e < n1; e += blockDim.x) vz[e] = poll(xq + e, ld_relaxed(xq + e));
            __pipeline_wait_prior(1);
            __syncthreads();
            double *bq = cb + (size_t)q * sst + ((size_t)(k - d) * hs + d) * n1 + r0;
            for (int rr = warp; rr < nr; rr += nw) {
                const double s = block_dot<KC>(rb + ((size_t)buf * rows + rr) * n1, vz, n1, lane);
                if (lane == 0) st_relaxed(bq + rr, s);
            }
            __syncthreads();
        }
        __pipeline_wait_prior(0);
    }
}

size_t mc_smem_bytes(int n1, int M, int cs)
{
    const size_t rows = (size_t)(n1 + cs - 1) / cs;
    return (2 * rows * n1 + 4 * (size_t)n1 + (size_t)M * rows) * sizeof(double);
}

}  // namespace

// The single-cluster sweep's cluster size and shared-memory limit are settled
// on the first call with prepare = true (from the preconditioner set-up), so
// that a launch recorded into a CUDA graph makes no attribute call.
template <int KC>
static int launch_sweep(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t bs,
                        const double *W, size_t ws, double *z, size_t zs, double *x, size_t xs,
                        const int *act, bool prepare, int F, int Bs)
{
    const size_t smem = (size_t)(h > 0 ? h : 1) * n1 * sizeof(double);
    const int cs = swj_cluster_for((const void *)k_band_sweep<KC>, kSweepThreads, smem);
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
    SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_band_sweep<KC>, n1, M, h, band, bs, W, ws, z, zs, x, xs, act, F, Bs));
    return SWJ_OK;
}

// Cluster size, shared memory and helper sets of the multi-cluster sweep per
// (kernel, n1, M, h, ni): 16 CTAs, else 12, else 8, with a helper set per
// instance where ni h such clusters fit on the device at once, else one shared
// set where ni + h - 1 fit (cs = 0: the multi-cluster sweep does not apply).
struct McPick {
    int cs, hsets;
    size_t smem;
};
static std::mutex g_mc_mutex;
static std::map<std::tuple<const void *, int, int, int, int>, McPick> g_mc_cache;

template <int KC>
static int launch_sweep_mc(cudaStream_t st, int n1, int M, int h, int ni, const double *band, size_t bst,
                           const double *W, size_t wst, const double *p, double *z, double *x, size_t vst,
                           double *cf, double *cb, size_t sst, int *err, bool prepare, int F0, int F1, int B1,
                           int B0, SwjWaits waits)
{
    const void *kern = (const void *)k_band_sweep_mc<KC>;
    McPick pick = {0, 1, 0};
    {
        std::lock_guard<std::mutex> lock(g_mc_mutex);
        auto key = std::make_tuple(kern, n1, M, h, ni);
        auto it = g_mc_cache.find(key);
        if (it == g_mc_cache.end()) {
            const int hs_try[2] = {ni, 1};
            for (int hi = 0; hi < (ni > 1 ? 2 : 1) && !pick.cs; ++hi) {
                const int hs = hs_try[hi], ncl_need = ni + hs * (h - 1);
                for (int c0 : {16, 12, 8}) {
                    // as many CTAs as it takes to give each the same number of rows
                    // (every CTA owns at least one row: the exchange relies on it),
                    // at most two rows per warp
                    const int rows = (n1 + c0 - 1) / c0, c = (n1 + rows - 1) / rows;
                    if (rows > 2 * (kSweepThreads / 32)) continue;
                    const size_t sm = mc_smem_bytes(n1, M, c);
                    if (sm > 220 * 1024) continue;
                    swj_cluster_for(kern, kSweepThreads, sm);   // raises the kernel's limit to sm
                    cudaLaunchConfig_t q = {};
                    q.gridDim = dim3(c * ncl_need);
                    q.blockDim = dim3(kSweepThreads);
                    q.dynamicSmemBytes = sm;
                    cudaLaunchAttribute qa[1];
                    qa[0].id = cudaLaunchAttributeClusterDimension;
                    qa[0].val.clusterDim.x = c;
                    qa[0].val.clusterDim.y = 1;
                    qa[0].val.clusterDim.z = 1;
                    q.attrs = qa;
                    q.numAttrs = 1;
                    int ncl = 0;
                    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &q) != cudaSuccess) ncl = 0;
                    cudaGetLastError();
                    if (ncl >= ncl_need) {
                        pick = {c, hs, sm};
                        break;
                    }
                }
            }
            it = g_mc_cache.emplace(key, pick).first;
        }
        pick = it->second;
    }
    const int cs = pick.cs;
    // test hook: no helper clusters, so nobody writes the terms the critical
    // clusters poll for (every poll runs out after waits.poll_limit reads)
    const int hsets = waits.no_helpers ? 0 : pick.hsets;
    const size_t smem = pick.smem;
    if (!cs) return SWJ_EINVAL;
    if (prepare) return SWJ_OK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * (ni + hsets * (h - 1)));
    cfg.blockDim = dim3(kSweepThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    SWJ_COUNT_LAUNCH();
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_band_sweep_mc<KC>, n1, M, h, ni, hsets, band, bst, W, wst, p,
                                             z, x, vst, cf, cb, sst, cs, err, F0, F1, B1, B0,
                                             waits.poll_limit);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // a stream capture that another host thread invalidated is not a refusal
        // of this launch (SWJ_ECUDA: the caller's capture logic retries); any
        // other error, e.g. no cooperative launch with clusters: the caller falls back
        const bool capture = e == cudaErrorStreamCaptureUnsupported || e == cudaErrorStreamCaptureInvalidated ||
                             e == cudaErrorStreamCaptureMerge || e == cudaErrorStreamCaptureUnmatched ||
                             e == cudaErrorStreamCaptureUnjoined || e == cudaErrorStreamCaptureIsolation ||
                             e == cudaErrorStreamCaptureImplicit || e == cudaErrorCapturedEvent ||
                             e == cudaErrorStreamCaptureWrongThread;
        return capture ? SWJ_ECUDA : SWJ_EINVAL;
    }
    return SWJ_OK;
}

template <int KC>
static int launch_block_p(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t bs,
                          const double *t, size_t ts, double *p, size_t ps, const int *act, double *fill1,
                          size_t n1f, double *fill2, size_t n2f)
{
    SWJ_COUNT_LAUNCH();
    const long nthr = (long)n1 * M * 32;
    k_block_p<KC><<<dim3((unsigned)((nthr + 255) / 256), nb), 256, 0, st>>>(n1, M, h, band, bs, t, ts, p, ps,
                                                                             act, fill1, n1f, fill2, n2f);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

#define SWJ_KC_DISPATCH(CALL)                                                                        \
    do {                                                                                             \
        const int kc = (n1 + 31) / 32;                                                               \
        if (kc <= 2) { constexpr int K = 2; return CALL; }                                           \
        if (kc <= 4) { constexpr int K = 4; return CALL; }                                           \
        if (kc <= 6) { constexpr int K = 6; return CALL; }                                           \
        if (kc <= 8) { constexpr int K = 8; return CALL; }                                           \
        if (kc <= 12) { constexpr int K = 12; return CALL; }                                         \
        if (kc <= 16) { constexpr int K = 16; return CALL; }                                         \
        if (kc <= 24) { constexpr int K = 24; return CALL; }                                         \
        if (kc <= 32) { constexpr int K = 32; return CALL; }                                         \
        return SWJ_EINVAL;                                                                           \
    } while (0)

int swj_block_p(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t bs,
                const double *t, size_t ts, double *p, size_t ps, const int *act, double *fill1,
                size_t n1f, double *fill2, size_t n2f)
{
    SWJ_KC_DISPATCH((launch_block_p<K>(st, nb, n1, M, h, band, bs, t, ts, p, ps, act, fill1, n1f, fill2, n2f)));
}

int swj_band_sweep_cluster(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t bs,
                           const double *W, size_t ws, double *z, size_t zs, double *x, size_t xs,
                           const int *act, bool prepare, int F, int Bs)
{
    if (F < 0) F = M;
    if (Bs < -1 || Bs >= M) Bs = M - 1;
    SWJ_KC_DISPATCH((launch_sweep<K>(st, nb, n1, M, h, band, bs, W, ws, z, zs, x, xs, act, prepare, F, Bs)));
}

int swj_band_sweep_mc(cudaStream_t st, int n1, int M, int h, const double *band, const double *W,
                      const double *p, double *z, double *x, double *cf, double *cb, int *err, bool prepare,
                      SwjWaits waits)
{
    if (h < 2 || M < 2) return SWJ_EINVAL;
    SWJ_KC_DISPATCH((launch_sweep_mc<K>(st, n1, M, h, 1, band, 0, W, 0, p, z, x, 0, cf, cb, 0, err, prepare, 0, M,
                                        M - 1, 0, waits)));
}

int swj_band_sweep_mc_ranges(cudaStream_t st, int n1, int M, int h, int ni, const double *band, size_t bst,
                             const double *W, size_t wst, const double *p, double *z, double *x, size_t vst,
                             double *cf, double *cb, size_t sst, int *err, bool prepare, int F0, int F1, int B1,
                             int B0, SwjWaits waits)
{
    if (h < 2 || M < 2 || ni < 1 || ni > 2 || F0 < 0 || F1 > M || B1 >= M || B0 < 0) return SWJ_EINVAL;
    SWJ_KC_DISPATCH((launch_sweep_mc<K>(st, n1, M, h, ni, band, bst, W, wst, p, z, x, vst, cf, cb, sst, err, prepare,
                                        F0, F1, B1, B0, waits)));
}
