// All-pairs boundary-integral sum of E2 (Section 3: Eq. IntegroEqn with the
// singularity of the second integral subtracted through S2, Eq. S2, and both
// integrals discretised by the trapezoidal rule).  For each half-mesh target
// t = (k + 1/2, l) and mesh node s = (i, j):
//
//   sum_s w_s [ (g_s - g*) K1 + zeta_x,s K2 - zeta_x* S2 ]
//
//   dx = x_i - x*, dy = y_j - y*, dy' = y_j + y*, dz = zeta_s - zeta*
//   r1^2 = dx^2 + dy^2 + dz^2, r2^2 = dx^2 + dy'^2 + dz^2
//   K1 = (dz - dx zeta_x,s - dy zeta_y,s) / r1^3 + (dz - dx zeta_x,s - dy' zeta_y,s) / r2^3
//   K2 = 1/r1 + 1/r2
//   S2 = (A dx^2 + B dx dy + C dy^2)^-1/2 + (A dx^2 - B dx dy' + C dy'^2)^-1/2
//
// (the image parts use y + y*; the slopes in K1 are those of the source).
// The sum is the hot loop of every residual and runs on the CUDA cores: it is
// not a contraction (four reciprocal square roots per pair).
//
// Layout: sources are staged through shared memory in tiles, every thread
// keeps R targets in registers and walks the tile, so each source record
// (read from shared memory by broadcast) serves R pairs.  The grid is
// (target tiles) x (source chunks); each block writes one partial sum per
// target and chunk, and the FP64 assembly kernel adds the chunks in a fixed
// order, so results are bitwise reproducible for a given launch plan.
//
// Lengths are in units of dy with exact index coordinates (see SrcRecS), so
// every coordinate difference is exact and nothing is rescaled per pair.
// Stated work: 7 add + 9 mul + 14 fma + 4 reciprocal square roots per pair
// (44 flop with an FMA counted as 2).
//
// FP32 (the mixed-precision path): every reciprocal square root is one
// rsqrt.approx.ftz.f32; plain FP32 within sub-tiles of 64 sources and Kahan
// compensation when a sub-tile total is added to the running sum.
// FP64 (the parity path and the refinement residual): the same FP32 seed
// refined by one Halley step; plain FP64 accumulation.
//
// Launch plan: the number of source chunks is chosen so that
// (target tiles) x (chunks) fills whole waves of resident blocks.
#include "swj_internal.h"

namespace {

// 1/sqrt(x) in FP32: one MUFU instruction (arguments are >= (dx/2)^2 in
// units of dy, never denormal).
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) in FP64: the FP32 hardware approximation y0 (relative error
// below 2^-22) refined by one step of Halley's iteration for x y^2 = 1,
//   e = 1 - x y0^2,  y1 = y0 (1 + e/2 + 3 e^2/8),
// whose error is O(e^3) ~ 2^-66 relative, below the rounding of the FP64
// arithmetic itself.  Five FP64 operations instead of a full-precision
// library reciprocal square root.
__device__ __forceinline__ double rsqrt_f64(double x)
{
    double y0 = (double)rsqrt_ftz((float)x);
    double e = fma(-x * y0, y0, 1.0);
    double p = fma(e, 0.375, 0.5);
    return fma(y0 * e, p, y0);
}

__device__ __forceinline__ float rsq(float x) { return rsqrt_ftz(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt_f64(x); }

template <typename T> struct Cfg;
template <> struct Cfg<float> { static constexpr int tile = 512; static constexpr bool kahan = true; };
template <> struct Cfg<double> { static constexpr int tile = 256; static constexpr bool kahan = false; };

constexpr int kSub = 64;   // sources per compensated sub-tile

template <typename T, int R>
__global__ void __launch_bounds__(128)
k_pairs_s(int T_, int S_, int chunk, const SrcRecS<T> *__restrict__ src, TgtArraysS<T> tg,
          double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = Cfg<T>::tile;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcRecS<T> sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    T tx[R], ty[R], tz[R], tgv[R], tzw[R], A[R], B[R], C[R], sum[R], comp[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = min(tb + r * nth, T_ - 1);
        tx[r] = tg.x[t]; ty[r] = tg.y[t]; tz[r] = tg.zeta[t]; tgv[r] = tg.g[t];
        tzw[r] = tg.zxw[t]; A[r] = tg.A[t]; B[r] = tg.B[t]; C[r] = tg.C[t];
        sum[r] = T(0); comp[r] = T(0);
    }
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) sh[i] = src[base + i];
        __syncthreads();
        for (int sb = 0; sb < nt; sb += kSub) {
            const int se = min(sb + kSub, nt);
            T loc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) loc[r] = T(0);
#pragma unroll 2
            for (int s = sb; s < se; ++s) {
                const SrcRecS<T> q = sh[s];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    T p = q.x - tx[r];
                    T qq = q.y - ty[r];
                    T qp = q.y + ty[r];
                    T dz = q.zeta - tz[r];
                    T p2 = p * p;
                    T bs = fma(dz, dz, p2);
                    T r1s = fma(qq, qq, bs);
                    T r2s = fma(qp, qp, bs);
                    T nc = fma(-p, q.zx, dz);
                    T n1 = fma(-qq, q.zy, nc);
                    T n2 = fma(-qp, q.zy, nc);
                    T i1 = rsq(r1s), i2 = rsq(r2s);
                    T i1c = i1 * i1 * i1, i2c = i2 * i2 * i2;
                    T K1 = fma(n1, i1c, n2 * i2c);
                    T K2 = i1 + i2;
                    T Ap2 = A[r] * p2;
                    T Bp = B[r] * p;
                    T Q1 = fma(fma(C[r], qq, Bp), qq, Ap2);
                    T Q2 = fma(fma(C[r], qp, -Bp), qp, Ap2);
                    T S2 = rsq(Q1) + rsq(Q2);
                    T f = q.g - tgv[r];
                    T inner = fma(q.zxw, K2, fma(f, K1, -tzw[r] * S2));
                    loc[r] = fma(q.w, inner, loc[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (Cfg<T>::kahan) {
                    T y = loc[r] - comp[r];
                    T t2 = sum[r] + y;
                    comp[r] = (t2 - sum[r]) - y;
                    sum[r] = t2;
                } else {
                    sum[r] += loc[r];
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = tb + r * nth;
        if (t < T_) partial[(size_t)blockIdx.y * T_ + t] = (double)sum[r] - (double)comp[r];
    }
}

constexpr int kTPB = 128;
constexpr int kR = 4;

// Source-chunk count P for (tiles) target tiles: (tiles x P) blocks should fill
// whole waves of `slots` resident blocks; chunks keep at least 64 sources.
PairPlan make_plan(int T, int S, int slots)
{
    PairPlan p;
    p.tpb = kTPB;
    p.R = kR;
    p.tiles = (T + kTPB * kR - 1) / (kTPB * kR);
    int maxP = S / 64 > 1 ? S / 64 : 1;
    if (maxP > 4096) maxP = 4096;
    int bestP = 1;
    double best = -1.0;
    for (int P = 1; P <= maxP; ++P) {
        long items = (long)p.tiles * P;
        long waves = (items + slots - 1) / slots;
        double eff = (double)items / (double)(waves * slots);
        // prefer a fuller last wave; among equals, fewer chunks
        if (eff > best + 0.02) { best = eff; bestP = P; }
        if (items >= 8L * slots) break;
    }
    p.chunk = (S + bestP - 1) / bestP;
    p.P = (S + p.chunk - 1) / p.chunk;
    return p;
}

int resident_blocks(const void *kernel, int threads)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

}  // namespace

PairPlan swj_pair_plan(const swj_ctx *c, int precision)
{
    const void *k = (precision == SWJ_FP64) ? (const void *)k_pairs_s<double, kR>
                                             : (const void *)k_pairs_s<float, kR>;
    int slots = c->num_sms * resident_blocks(k, kTPB);
    return make_plan(c->T, c->S, slots);
}

// One launch covers every instance (grid.z); each instance uses the chunking
// of the single-instance plan, so its result does not depend on the batch.
void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl, const int *act)
{
    dim3 grid(pl.tiles, pl.P, c->nb);
    SWJ_COUNT_LAUNCH();
    k_pairs_s<double, kR><<<grid, kTPB, 0, c->stream>>>(c->T, c->S, pl.chunk, c->src64, c->tgt64,
                                                        c->partial, act);
}

void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl, const int *act)
{
    dim3 grid(pl.tiles, pl.P, c->nb);
    SWJ_COUNT_LAUNCH();
    k_pairs_s<float, kR><<<grid, kTPB, 0, c->stream>>>(c->T, c->S, pl.chunk, c->src32, c->tgt32,
                                                       c->partial, act);
}
