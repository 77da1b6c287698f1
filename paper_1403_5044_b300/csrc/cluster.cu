// Gauss-Jordan inverses of the diagonal blocks of the preconditioner (FP64),
// on thread-block clusters.
//
// B300 issues about two FP64 FMAs per clock per SM, so a dense block
// operation on one CTA is slow; these kernels spread each sequential
// elimination over the CTAs of one cluster and exchange the little data that
// must be shared (a pivot column, the index of the pivot row) through
// distributed shared memory.  The pipelined kernel also spins on per-step
// flags in shared memory, every spin with an iteration limit.
#include "swj_internal.h"
#include <map>
#include <mutex>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int kGJThreads = 256;

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

// One elimination step on a CTA's slice (rows over threads, WM >= nc columns
// per row held in registers): row k <- rowk, every other row i <- row i -
// col_k[i] rowk, with the pivot column's own entry (local index kk_own, or
// -1 if it is not in this slice) starting from zero.  Only the local columns
// lo..nc-1 other than `skip` are touched.
template <int WM>
__device__ __forceinline__ void gj_eliminate(double *A, int ws, int n, int nc, int k, int kk_own,
                                             const double *__restrict__ col_k,
                                             const double *__restrict__ rowk, int tid, int nth,
                                             int skip = -1, int lo = 0)
{
    double r[WM];
#pragma unroll
    for (int jj = 0; jj < WM; ++jj) r[jj] = (jj >= lo && jj < nc) ? rowk[jj] : 0.0;
    for (int i = tid; i < n; i += nth) {
        double *Ai = A + (size_t)i * ws;
        if (i == k) {
#pragma unroll
            for (int jj = 0; jj < WM; ++jj)
                if (jj >= lo && jj < nc && jj != skip) Ai[jj] = r[jj];
        } else {
            const double m = col_k[i];
            double v[WM];
#pragma unroll
            for (int jj = 0; jj < WM; ++jj)
                v[jj] = (jj >= lo && jj < nc && jj != kk_own && jj != skip) ? Ai[jj] : 0.0;
#pragma unroll
            for (int jj = 0; jj < WM; ++jj)
                if (jj >= lo && jj < nc && jj != skip) Ai[jj] = fma(-m, r[jj], v[jj]);
        }
    }
}

// The same step on the local columns lo..hi-1 only, with a loop over just
// those columns: each FP64 instruction of a warp occupies its SM sub-partition
// for ~64 cycles on B300, predicated off or not, so a slice's unrolled
// register loop costs WM FMAs per row however few columns are live.  Same
// arithmetic per element as gj_eliminate (no pivot column among lo..hi-1).
__device__ __forceinline__ void gj_eliminate_cols(double *A, int ws, int n, int k, int lo, int hi,
                                                  const double *__restrict__ col_k,
                                                  const double *__restrict__ rowk, int tid, int nth)
{
    if (lo >= hi) return;
    for (int i = tid; i < n; i += nth) {
        double *Ai = A + (size_t)i * ws;
        if (i == k) {
            for (int jj = lo; jj < hi; ++jj) Ai[jj] = rowk[jj];
        } else {
            const double m = col_k[i];
            int jj = lo;
            for (; jj + 1 < hi; jj += 2) {
                const double a0 = Ai[jj], a1 = Ai[jj + 1];
                Ai[jj] = fma(-m, rowk[jj], a0);
                Ai[jj + 1] = fma(-m, rowk[jj + 1], a1);
            }
            if (jj < hi) Ai[jj] = fma(-m, rowk[jj], Ai[jj]);
        }
    }
}

// One row's share of a step: the cnt columns at Ai (rowk entries at rk), W >=
// cnt held in registers; the pivot row takes rowk, the others subtract m rowk
// (the arithmetic of gj_eliminate with fewer index tests per row).
template <int W>
__device__ __forceinline__ void gj_elim_row(double *Ai, bool pivot_row, double m, const double *rk, int cnt)
{
    double r[W];
#pragma unroll
    for (int j = 0; j < W; ++j) r[j] = (j < cnt) ? rk[j] : 0.0;
    if (pivot_row) {
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (j < cnt) Ai[j] = r[j];
    } else {
        double v[W];
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = (j < cnt) ? Ai[j] : 0.0;
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (j < cnt) Ai[j] = fma(-m, r[j], v[j]);
    }
}

// Flag helpers for the pipelined Gauss-Jordan kernel: a release max-update of
// a word in another CTA's shared memory (a max, not a store: updates from two
// successive owners may land in either order, the flag must never go back)
// and an acquire load of this CTA's own word.
__device__ __forceinline__ void max_release_cluster(unsigned *local_word, int cta, unsigned v)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(local_word), ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(cta));
    asm volatile("red.release.cluster.shared::cluster.max.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_cluster(const unsigned *local_word)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(local_word), v;
    asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// (key, index) of the warp's largest 64-bit key, the smallest index among
// equal keys, in every lane: three warp reductions (high word, low word among
// the lanes with the largest high word, index among the lanes with the
// largest key) instead of a shuffle tree.  Indices are non-negative.
__device__ __forceinline__ void warp_argmax(unsigned long long &key, int &idx)
{
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const bool top = hi == mhi && lo == mlo;
    idx = (int)__reduce_min_sync(0xffffffffu, top ? (unsigned)idx : 0xffffffffu);
    key = ((unsigned long long)mhi << 32) | mlo;
}

// Status of a block from every CTA's own (read from their shared memory
// after a cluster barrier): the smallest failing pivot step (+1) any CTA saw,
// else -1 if a wait of any CTA timed out, else 0.
__device__ int gj_cluster_status(cg::cluster_group &cl, int *own, int ncta)
{
    int s = 0;
    bool timeout = false;
    for (int q = 0; q < ncta; ++q) {
        const int f = *cl.map_shared_rank(own, q);
        if (f < 0) timeout = true;
        else if (f > 0 && (s == 0 || f < s)) s = f;
    }
    return s ? s : (timeout ? -1 : 0);
}

// A flag wait gives up after spin_limit iterations (a kernel argument:
// opts.wait_limit, else kSwjSpinLimit = 2^26, far above any real wait: a step
// takes a few microseconds).

// Pipelined Gauss-Jordan inverse with partial (row) pivoting, one n x n block
// per cluster, each CTA's column slice (n x w) in shared memory.  The pivot
// steps k = 0..n-1 are owned by the CTA holding column k.  The owner searches
// the pivot in its (up to date) column, records the step (pivot row, the
// multiplier column after the interchange, the reciprocal pivot) in its own
// shared memory, raises a release flag in every other CTA and eliminates the
// columns of its slice right of the pivot; it goes on to its next step at
// once, and applies its panel's steps to the rest of its slice after the
// panel (column by column the same operations in the same order, so the
// result is that of eliminating the whole slice at every step).  Every other
// CTA waits for the
// flag of step k (acquire), reads the step from the owner's shared memory and
// applies it to its slice.  Steps are applied in order everywhere, so the
// arithmetic is that of the unblocked elimination; no CTA waits for the
// slower ones except a new panel owner, which must have applied every earlier
// step first.  A failed pivot is published as a flag above n; a flag wait that
// runs past spin_limit ends the kernel with info = -1 (every CTA's status is
// combined: a CTA that stops on a timeout while the others finish still
// fails the block).  Every CTA loads its
// slice before the first barrier and writes the (column-permuted) inverse
// after the last, so `in` and `out` may alias.
template <int WM>
__global__ void __launch_bounds__(kGJThreads)
k_gj_pipe(int n, const double *in_base, size_t istride, double *out_base, size_t ostride, int *info,
          long long spin_limit)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / ncta;
    const double *in = in_base + (size_t)mat * istride;
    double *out = out_base + (size_t)mat * ostride;
    const int w = (n + ncta - 1) / ncta;
    const int ws = w | 1;                       // odd row stride: conflict-free row-per-thread access
    const int c0 = rank * w, c1 = min(n, c0 + w), nc = max(0, c1 - c0);
    extern __shared__ double sm[];
    double *A = sm;                             // n x w slice (row-major, stride ws)
    // step records of this CTA's steps, n + 2 doubles each: the multiplier column,
    // the reciprocal pivot and the pivot row (as a double), read by the others
    const int rs = n + 2;
    double *rec = A + (size_t)n * ws;           // w x rs
    double *lrec = rec + (size_t)w * rs;        // 2 x rs: copies of other owners' records (by step parity)
    double *rowk = lrec + 2 * (size_t)rs;       // w
    int *piv = (int *)(rowk + w);               // n
    int *sigma = piv + n;                       // n
    int *ctl = sigma + n;                       // [0] step status, [2..3] prefetch counts by parity
    unsigned *flag = (unsigned *)(ctl + 4);     // published step count (written by the owners)
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < n * nc; e += nth) {
        const int i = e / nc, jj = e - i * nc;
        A[(size_t)i * ws + jj] = in[(size_t)i * n + c0 + jj];
    }
    if (tid == 0) {
        *flag = 0u;
        ctl[0] = ctl[1] = ctl[2] = ctl[3] = 0;
    }
    cl.sync();                                  // flags initialised before any remote store
    // When the rows leave the last two warps idle in the elimination (n <= nth - 64),
    // those warps fetch the next step's record from its owner meanwhile (if this CTA
    // does not own it); ctl[2 + parity] counts the threads whose copy succeeded, and
    // a step whose record was not fetched in full is fetched when it starts.
    const int npre = 64;
    const bool prefetch = n <= nth - npre;
    const bool pre_thread = prefetch && tid >= nth - npre;
    int fail = 0;
    bool ahead = false;                         // this step's pivot already searched
    for (int k = 0; k < n && !fail; ++k) {
        const int o = k / w, kk = k - o * w;
        const int nk = k + 1, no = nk / w;      // the next step and its owner
        // the prefetching warps' part of the elimination phase of step k
        auto prefetch_next = [&]() {
            if (!pre_thread || nk >= n || no == rank) return;
            long long it = 0;
            unsigned v;
            while ((v = ld_acquire_cluster(flag)) < (unsigned)(nk + 1)) {
                if (++it > spin_limit) break;
            }
            if (v < (unsigned)(nk + 1) || v > (unsigned)n) return;   // left to the next step
            const double *orec = cl.map_shared_rank(rec + (size_t)(nk - no * w) * rs, no);
            double *dst = lrec + (size_t)(nk & 1) * rs;
            for (int i = tid - (nth - npre); i < rs; i += npre) dst[i] = orec[i];
            atomicAdd(&ctl[2 + (nk & 1)], 1);
        };
        // pivot of step ks in local column kks (warp 0 of the owner): the largest
        // |a_ik|, rows ks..n-1, first index on ties (non-negative doubles order as
        // their bit patterns); a zero or non-finite pivot is told by its bit pattern
        // and the pivot row travels as the integer bits of a double: B300 takes
        // 60-400 cycles for each dependent FP64 compare, conversion or division, and
        // these steps are the kernel's critical path
        auto search = [&](int ks, int kks) {
            unsigned long long bk = 0ull;
            int bi = n;
            for (int i = ks + tid; i < n; i += 32) {
                const unsigned long long kv =
                    (unsigned long long)__double_as_longlong(A[(size_t)i * ws + kks]) & 0x7FFFFFFFFFFFFFFFull;
                if (kv > bk || (kv == bk && i < bi)) { bk = kv; bi = i; }
            }
            warp_argmax(bk, bi);
            if (tid == 0) {
                const double pv = (bi < n) ? A[(size_t)bi * ws + kks] : 0.0;
                const bool good = bi < n && bk != 0ull && (bk >> 52) < 0x7FFull;
                piv[ks] = good ? bi : ks;
                ctl[0] = good ? 0 : ks + 1;
                double *r = rec + (size_t)kks * rs;
                r[ks] = pv;
                r[n] = good ? 1.0 / pv : 0.0;        // one division per step
                r[n + 1] = __longlong_as_double((long long)(good ? bi : ks));
            }
        };
        if (rank == o) {
            // (searched at the end of the previous step when that was this panel's too)
            if (!ahead && tid < 32) search(k, kk);
            __syncthreads();
            const int f = ctl[0];
            const int p = piv[k];
            double *r = rec + (size_t)kk * rs;
            const double rp = r[n];
            if (!f) {
                // interchange rows k and p and scale the pivot row in the columns right of
                // the pivot; multipliers (pre-interchange values: row k is not written in
                // this phase, and the pivot column not at all)
                for (int jj = kk + 1 + tid; jj < nc; jj += nth) {
                    const double v = A[(size_t)p * ws + jj];
                    rowk[jj] = v * rp;
                    if (p != k) A[(size_t)p * ws + jj] = A[(size_t)k * ws + jj];
                }
                for (int i = tid; i < n; i += nth)
                    if (i != k) r[i] = (i == p) ? A[(size_t)k * ws + kk] : A[(size_t)i * ws + kk];
            }
            __syncthreads();
            // publish step k (or the failure) to every other CTA, from the last warp: its
            // remote release takes ~800 cycles, which the elimination of the other warps
            // hides (the last warp prefetches, it eliminates no rows)
            const int pl = tid - (nth - 32);
            if (pl >= 0 && pl < ncta && pl != rank) max_release_cluster(flag, pl, f ? (unsigned)(n + f) : (unsigned)(k + 1));
            if (f) { fail = f; break; }
            // Within its panel the owner eliminates only the columns right of the pivot,
            // which its next searches read; the pivot column and those left of it get
            // the panel's steps after the panel, each column still in step order.  The
            // next pivot column comes first, then warp 0 searches the next step's pivot
            // while the other warps eliminate the remaining columns (rows over them).
            if (kk + 1 < nc) {
                if (tid >= 32) gj_eliminate_cols(A, ws, n, k, kk + 1, kk + 2, r, rowk, tid - 32, nth - 32);
                __syncthreads();
                if (tid < 32) search(k + 1, kk + 1);
                else gj_eliminate_cols(A, ws, n, k, kk + 2, nc, r, rowk, tid - 32, nth - 32);
                ahead = true;
            } else {
                if (pre_thread) prefetch_next();
                ahead = false;
            }
            __syncthreads();
            if (kk == nc - 1) {
                const int k0 = k - kk;
                for (int ks = 0; ks <= kk; ++ks) {
                    // step k0 + ks on local columns 0..ks (ks: its own pivot column)
                    const int s = k0 + ks;
                    const double *rs_ = rec + (size_t)ks * rs;
                    const int ps = (int)__double_as_longlong(rs_[n + 1]);
                    const double rps = rs_[n];
                    for (int jj = tid; jj < ks; jj += nth) {
                        const double v = A[(size_t)ps * ws + jj];
                        rowk[jj] = v * rps;
                        if (ps != s) A[(size_t)ps * ws + jj] = A[(size_t)s * ws + jj];
                    }
                    __syncthreads();
                    gj_eliminate_cols(A, ws, n, s, 0, ks, rs_, rowk, tid, nth);
                    // the pivot column itself (entries from zero, as in gj_eliminate)
                    for (int i = tid; i < n; i += nth)
                        A[(size_t)i * ws + ks] = (i == s) ? rps : fma(-rs_[i], rps, 0.0);
                    __syncthreads();
                }
            }
        } else {
            double *lr = lrec + (size_t)(k & 1) * rs;
            if (!(prefetch && ctl[2 + (k & 1)] == npre)) {
                // not prefetched: every thread waits for the flag itself (acquire), then
                // copies its share of the owner's step record
                long long it = 0;
                unsigned v;
                while ((v = ld_acquire_cluster(flag)) < (unsigned)(k + 1)) {
                    if (++it > spin_limit) break;
                }
                int st = 0;
                if (v < (unsigned)(k + 1)) st = -1;                      // timed out
                else if (v > (unsigned)n) st = (int)(v - (unsigned)n);    // the owner's pivot failed
                if (!st) {
                    const double *orec = cl.map_shared_rank(rec + (size_t)kk * rs, o);
                    for (int i = tid; i < rs; i += nth) lr[i] = orec[i];
                }
                // the CTA stops if any thread timed out or saw the owner's failure
                if (__syncthreads_or(st != 0)) { fail = st ? st : -1; break; }
            }
            const int p = (int)__double_as_longlong(lr[n + 1]);
            const double rp = lr[n];
            if (tid == 0) piv[k] = p;
            for (int jj = tid; jj < nc; jj += nth) {
                const double a = A[(size_t)p * ws + jj];
                rowk[jj] = a * rp;
                if (p != k) A[(size_t)p * ws + jj] = A[(size_t)k * ws + jj];
            }
            __syncthreads();
            // every thread has read this parity's count (before the barrier above): the
            // buffer is free again for the step after next
            if (tid == 0) ctl[2 + (k & 1)] = 0;
            if (pre_thread) prefetch_next();
            else if (n <= nth - npre) {
                // one row per thread (all rows fit the non-prefetching warps)
                if (tid < n) gj_elim_row<WM>(A + (size_t)tid * ws, tid == k, tid == k ? 0.0 : lr[tid], rowk, nc);
            } else {
                gj_eliminate<WM>(A, ws, n, nc, k, -1, lr, rowk, tid, nth);
            }
            __syncthreads();
        }
    }
    // every CTA keeps its shared memory until all have read what they need;
    // ctl[1] holds this CTA's status for rank 0
    if (tid == 0) ctl[1] = fail;
    cl.sync();
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
            const int i = e / nc, jj = e - i * nc;
            out[(size_t)i * n + piv[c0 + jj]] = A[(size_t)i * ws + jj];
        }
    }
    if (rank == 0 && tid == 0) info[mat] = gj_cluster_status(cl, ctl + 1, ncta);
    cl.sync();
}

// The same inverse with the columns dealt round-robin (column j on CTA
// j mod ncta) and a one-step look-ahead: the owner of step k + 1 applies step
// k to its pivot column k + 1 first, searches the pivot of step k + 1 there,
// records and publishes it, and only then applies step k to its other
// columns.  Consecutive steps thus belong to different CTAs, and the chain of
// publications runs through one column update, one search and one
// publication per step instead of a whole slice's elimination.  Records,
// flags, failure and timeout handling are those of k_gj_pipe (a CTA's record
// for its step k sits in slot k / ncta of its record array); the elimination
// of every element is the same sequence of operations, so the result is
// that of k_gj_pipe bit for bit.
template <int WM>
__global__ void __launch_bounds__(kGJThreads)
k_gj_rr(int n, const double *in_base, size_t istride, double *out_base, size_t ostride, int *info,
        long long spin_limit)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int mat = blockIdx.x / ncta;
    const double *in = in_base + (size_t)mat * istride;
    double *out = out_base + (size_t)mat * ostride;
    const int w = (n + ncta - 1) / ncta;
    const int ws = w | 1;                       // odd row stride: conflict-free row-per-thread access
    const int nc = rank < n ? (n - 1 - rank) / ncta + 1 : 0;   // local columns j = rank + jj ncta
    extern __shared__ double sm[];
    double *A = sm;                             // n x w slice (row-major, stride ws)
    const int rs = n + 2;
    double *rec = A + (size_t)n * ws;           // w x rs: records of this CTA's steps
    double *lrec = rec + (size_t)w * rs;        // 2 x rs: copies of other owners' records (by step parity)
    double *rowk = lrec + 2 * (size_t)rs;       // w
    int *piv = (int *)(rowk + w);               // n
    int *sigma = piv + n;                       // n
    int *ctl = sigma + n;                       // [0] step status, [2..3] prefetch counts by parity
    unsigned *flag = (unsigned *)(ctl + 4);     // published step count (written by the owners)
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int e = tid; e < n * nc; e += nth) {
        const int i = e / nc, jj = e - i * nc;
        A[(size_t)i * ws + jj] = in[(size_t)i * n + rank + jj * ncta];
    }
    if (tid == 0) {
        *flag = 0u;
        ctl[0] = ctl[1] = ctl[2] = ctl[3] = 0;
    }
    cl.sync();                                  // flags initialised before any remote store
    const int npre = 64;
    const bool prefetch = n <= nth - npre;
    const bool pre_thread = prefetch && tid >= nth - npre;
    // record and publish step s of this CTA from its (up to date) local column
    // s / ncta: pivot = the largest |a_is|, rows s..n-1, first index on ties;
    // returns the failure code (0, or s + 1 for a zero or non-finite pivot)
    auto make_record = [&](int s) -> int {
        const int kk = s / ncta;
        double *r = rec + (size_t)kk * rs;
        // (one warp, one level; tests on the bit pattern and the pivot row as
        // integer bits, as in k_gj_pipe)
        if (tid < 32) {
            unsigned long long bk = 0ull;
            int bi = n;
            for (int i = s + tid; i < n; i += 32) {
                const unsigned long long kv =
                    (unsigned long long)__double_as_longlong(A[(size_t)i * ws + kk]) & 0x7FFFFFFFFFFFFFFFull;
                if (kv > bk || (kv == bk && i < bi)) { bk = kv; bi = i; }
            }
            warp_argmax(bk, bi);
            if (tid == 0) {
                const double pv = (bi < n) ? A[(size_t)bi * ws + kk] : 0.0;
                const bool good = bi < n && bk != 0ull && (bk >> 52) < 0x7FFull;
                ctl[0] = good ? 0 : s + 1;
                r[s] = pv;
                r[n] = good ? 1.0 / pv : 0.0;        // one division per step
                r[n + 1] = __longlong_as_double((long long)(good ? bi : s));
            }
        }
        __syncthreads();
        const int f = ctl[0];
        if (!f) {
            // multipliers after the interchange of rows s and p (values before it)
            const int p = (int)__double_as_longlong(r[n + 1]);
            for (int i = tid; i < n; i += nth)
                if (i != s) r[i] = (i == p) ? A[(size_t)s * ws + kk] : A[(size_t)i * ws + kk];
        }
        __syncthreads();
        if (tid < ncta && tid != rank) max_release_cluster(flag, tid, f ? (unsigned)(n + f) : (unsigned)(s + 1));
        return f;
    };
    int fail = 0;
    if (rank == 0 && n > 0) fail = make_record(0);
    for (int k = 0; k < n && !fail; ++k) {
        const int o = k % ncta, kk = k / ncta;
        const int nk = k + 1, no = nk % ncta;   // the next step and its owner
        auto prefetch_next = [&]() {
            if (!pre_thread || nk >= n || no == rank) return;
            long long it = 0;
            unsigned v;
            while ((v = ld_acquire_cluster(flag)) < (unsigned)(nk + 1)) {
                if (++it > spin_limit) break;
            }
            if (v < (unsigned)(nk + 1) || v > (unsigned)n) return;   // left to the next step
            const double *orec = cl.map_shared_rank(rec + (size_t)(nk / ncta) * rs, no);
            double *dst = lrec + (size_t)(nk & 1) * rs;
            for (int i = tid - (nth - npre); i < rs; i += npre) dst[i] = orec[i];
            atomicAdd(&ctl[2 + (nk & 1)], 1);
        };
        const double *r;
        if (rank == o) {
            r = rec + (size_t)kk * rs;
        } else {
            double *lr = lrec + (size_t)(k & 1) * rs;
            if (!(prefetch && ctl[2 + (k & 1)] == npre)) {
                long long it = 0;
                unsigned v;
                while ((v = ld_acquire_cluster(flag)) < (unsigned)(k + 1)) {
                    if (++it > spin_limit) break;
                }
                int st = 0;
                if (v < (unsigned)(k + 1)) st = -1;                      // timed out
                else if (v > (unsigned)n) st = (int)(v - (unsigned)n);    // the owner's pivot failed
                if (!st) {
                    const double *orec = cl.map_shared_rank(rec + (size_t)kk * rs, o);
                    for (int i = tid; i < rs; i += nth) lr[i] = orec[i];
                }
                if (__syncthreads_or(st != 0)) { fail = st ? st : -1; break; }
            }
            r = lr;
        }
        const int p = (int)__double_as_longlong(r[n + 1]);
        const double rp = r[n];
        const int kk_own = (rank == o) ? kk : -1;
        if (tid == 0) piv[k] = p;
        // scaled pivot row and the interchange of rows k and p, every local column
        for (int jj = tid; jj < nc; jj += nth) {
            const double a = A[(size_t)p * ws + jj];
            rowk[jj] = (jj == kk_own) ? rp : a * rp;
            if (p != k) A[(size_t)p * ws + jj] = A[(size_t)k * ws + jj];
        }
        __syncthreads();
        if (tid == 0 && rank != o) ctl[2 + (k & 1)] = 0;
        if (nk < n && no == rank) {
            // look-ahead: step k on the pivot column of step k + 1, then its record
            const int kk2 = nk / ncta;
            const double rk = rowk[kk2];
            for (int i = tid; i < n; i += nth) {
                double *a = A + (size_t)i * ws + kk2;
                *a = (i == k) ? rk : fma(-r[i], rk, *a);
            }
            __syncthreads();
            const int f = make_record(nk);
            if (f) { fail = f; break; }
            if (!pre_thread) gj_eliminate<WM>(A, ws, n, nc, k, kk_own, r, rowk, tid, nth, kk2);
        } else {
            if (pre_thread) prefetch_next();
            else gj_eliminate<WM>(A, ws, n, nc, k, kk_own, r, rowk, tid, nth);
        }
        __syncthreads();
    }
    // every CTA keeps its shared memory until all have read what they need;
    // ctl[1] holds this CTA's status for rank 0
    if (tid == 0) ctl[1] = fail;
    cl.sync();
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
            const int i = e / nc, jj = e - i * nc;
            out[(size_t)i * n + piv[rank + jj * ncta]] = A[(size_t)i * ws + jj];
        }
    }
    if (rank == 0 && tid == 0) info[mat] = gj_cluster_status(cl, ctl + 1, ncta);
    cl.sync();
}

// 16 CTAs per cluster where the device runs such clusters (a non-portable
// size), else the portable 8.  The kernel's dynamic shared-memory limit must
// already be at least `smem` (the occupancy query fails for a size above it).
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

// Cluster size (16 where the device can run such clusters of this kernel with
// `smem` bytes of dynamic shared memory per CTA, else 8) per (kernel, smem);
// also raises the kernel's shared-memory limit to `smem`.  Call with
// g_attr_mutex held.
// Lazily settled launch attributes, shared by every context and host thread.
static std::mutex g_attr_mutex;
static std::map<std::pair<const void *, size_t>, int> g_cluster_cache;
static std::map<const void *, size_t> g_smem_limit;
static int cluster_for(const void *kern, int threads, size_t smem)
{
    auto key = std::make_pair(kern, smem);
    auto it = g_cluster_cache.find(key);
    if (it != g_cluster_cache.end()) return it->second;
    // The limit only grows, and is raised before the query: other host threads
    // may be launching this kernel with a larger size meanwhile, and a launch
    // above the kernel's limit at that moment fails.
    size_t &lim = g_smem_limit[kern];
    if (smem > lim) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
            lim = smem;
        cudaGetLastError();
    }
    int cs = cluster_ctas(kern, threads, smem);
    g_cluster_cache[key] = cs;
    return cs;
}

size_t gj_smem_bytes(int n, int cs)
{
    const int w = (n + cs - 1) / cs;
    return (size_t)((size_t)n * (w | 1) + (size_t)(w + 2) * (n + 2) + w) * sizeof(double) +
           (size_t)(2 * n + 8) * sizeof(int);
}


// Instances of the blocked Gauss-Jordan kernel by maximum slice width.
// Up to 12 columns per CTA the panel kernel is faster (its owner's steps need
// no exchange; measured set-up 181x61: 20.1 ms against 21.7 with k_gj_rr), from
// 16 on the round-robin one (361x121: 149 against 162 ms: a panel owner's
// elimination of its wider slice is on the critical path every step).
static const void *gj_blocked_kernel(int w)
{
    if (w <= 8) return (const void *)k_gj_pipe<8>;
    if (w <= 12) return (const void *)k_gj_pipe<12>;
    if (w <= 16) return (const void *)k_gj_rr<16>;
    if (w <= 24) return (const void *)k_gj_rr<24>;
    return (const void *)k_gj_rr<32>;
}

// Cluster size of the blocked kernel for n x n blocks (0: it does not apply).
static int gj_blocked_cluster(int n)
{
    static std::map<int, int> cache;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    auto it = cache.find(n);
    if (it != cache.end()) return it->second;
    int cs = 0;
    for (int c : {16, 8}) {
        const int w = (n + c - 1) / c;
        const size_t smem = gj_smem_bytes(n, c);
        if (w > 32 || smem > 200 * 1024) continue;
        if (cluster_for(gj_blocked_kernel(w), kGJThreads, smem) >= c) { cs = c; break; }
    }
    cache[n] = cs;
    return cs;
}

// true when the shared-memory (blocked) Gauss-Jordan kernel applies to n x n
// blocks (then input and output may be the same block)
bool swj_gj_inplace(int n) { return gj_blocked_cluster(n) > 0; }

// The kernel, cluster size and shared memory of the Gauss-Jordan launch for
// n x n blocks; min_smem raises the shared memory (the kernel does not use the
// rest), e.g. to keep one CTA per SM.
static void gj_launch_shape(int n, size_t min_smem, const void **kern, int *cs, size_t *smem, bool *blocked)
{
    const int csb = gj_blocked_cluster(n);
    *blocked = csb > 0;
    if (*blocked) {
        *cs = csb;
        *smem = gj_smem_bytes(n, csb);
        *kern = gj_blocked_kernel((n + csb - 1) / csb);
    } else {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        *kern = (const void *)k_gj_cluster;
        *cs = cluster_for(*kern, kGJThreads, 64 * 1024);
        const int w = (n + *cs - 1) / *cs;
        *smem = (size_t)(2 * n + w) * sizeof(double) + (size_t)(2 * n + 4) * sizeof(int);
        cluster_for(*kern, kGJThreads, *smem);
    }
    if (min_smem > *smem) {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        *smem = min_smem;
        cluster_for(*kern, kGJThreads, *smem);   // raises the kernel's limit
    }
}

int swj_gj_cluster_capacity(int n, size_t min_smem)
{
    const void *kern;
    int cs;
    size_t smem;
    bool blocked;
    gj_launch_shape(n, min_smem, &kern, &cs, &smem, &blocked);
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(cs);
    q.blockDim = dim3(kGJThreads);
    q.dynamicSmemBytes = smem;
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = cs;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &q) != cudaSuccess) ncl = 0;
    cudaGetLastError();
    return ncl;
}

int swj_gj_inverse_cluster(cudaStream_t st, int n, int count, double *work, size_t wstride,
                           double *out, size_t ostride, int *info, long long spin_limit, size_t min_smem)
{
    const void *kern;
    int cs;
    size_t smem;
    bool use_smem;
    gj_launch_shape(n, min_smem, &kern, &cs, &smem, &use_smem);
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
    const double *win = work;
    void *args[] = {(void *)&n,    (void *)&win,  (void *)&wstride,   (void *)&out,
                    (void *)&ostride, (void *)&info, (void *)&spin_limit};
    if (use_smem) SWJ_CUDA_TRY(cudaLaunchKernelExC(&cfg, kern, args));
    else SWJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster, n, work, wstride, out, ostride, info));
    return SWJ_OK;
}

int swj_cluster_for(const void *kern, int threads, size_t smem)
{
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    return cluster_for(kern, threads, smem);
}
