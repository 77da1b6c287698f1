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
// Coordinates are exact index values: dx = (i - (k + 1/2)) dx_mesh, etc., so
// the only rounding in a coordinate difference is the one product.
//
// FP32 variant (k_pairs32): lengths in units of dy with exact index
// coordinates (see SrcRec32), the reciprocal square roots as single
// rsqrt.approx.ftz.f32 instructions (every argument is at least (dx/2)^2, so
// never denormal), plain FP32 within sub-tiles of 64 sources and Kahan
// compensation when a sub-tile total is added to the running sum.  Stated
// work: 7 FADD + 9 FMUL + 14 FFMA + 4 MUFU = 44 flop per pair.
//
// Launch plan: the number of source chunks is chosen so that
// (target tiles) x (chunks) fills whole waves of resident blocks.
#include "swj_internal.h"

namespace {

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

template <typename T> struct TileCfg;
template <> struct TileCfg<double> { static constexpr int tile = 256; };

constexpr int kSub = 32;   // sources per compensated sub-tile

template <typename T>
__device__ __forceinline__ T pair_term(const SrcRec<T> &q, T tk, T tl, T zt, T gt, T zxt,
                                       T A, T B, T C, T dX, T dY)
{
    T dx = (q.si - tk) * dX;
    T dy = (q.sj - tl) * dY;
    T dyp = (q.sj + tl) * dY;
    T dz = q.zeta - zt;
    T dx2 = dx * dx;
    T base = fma(dz, dz, dx2);
    T r1s = fma(dy, dy, base);
    T r2s = fma(dyp, dyp, base);
    T nc = fma(-dx, q.zx, dz);
    T n1 = fma(-dy, q.zy, nc);
    T n2 = fma(-dyp, q.zy, nc);
    T i1 = rsq(r1s), i2 = rsq(r2s);
    T i1c = i1 * i1 * i1, i2c = i2 * i2 * i2;
    T K1 = fma(n1, i1c, n2 * i2c);
    T K2 = i1 + i2;
    T Adx2 = A * dx2;
    T Bdx = B * dx;
    T Q1 = fma(fma(C, dy, Bdx), dy, Adx2);
    T Q2 = fma(fma(C, dyp, -Bdx), dyp, Adx2);
    T S2 = rsq(Q1) + rsq(Q2);
    T f = q.g - gt;
    T inner = fma(q.zx, K2, fma(f, K1, -zxt * S2));
    return q.w * inner;
}

template <typename T, int R, bool KAHAN>
__global__ void __launch_bounds__(128)
k_pairs(int T_, int S_, int chunk, const SrcRec<T> *__restrict__ src, TgtArrays<T> tg,
        T dX, T dY, double *__restrict__ partial)
{
    constexpr int TILE = TileCfg<T>::tile;
    __shared__ SrcRec<T> sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    T tk[R], tl[R], zt[R], gt[R], zxt[R], A[R], B[R], C[R], sum[R], comp[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = min(tb + r * nth, T_ - 1);
        tk[r] = tg.tk[t]; tl[r] = tg.tl[t]; zt[r] = tg.zeta[t]; gt[r] = tg.g[t];
        zxt[r] = tg.zx[t]; A[r] = tg.A[t]; B[r] = tg.B[t]; C[r] = tg.C[t];
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
            for (int s = sb; s < se; ++s) {
                const SrcRec<T> q = sh[s];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    loc[r] += pair_term<T>(q, tk[r], tl[r], zt[r], gt[r], zxt[r], A[r], B[r],
                                           C[r], dX, dY);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (KAHAN) {
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

__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int kTile32 = 512;
constexpr int kSub32 = 64;

template <int R>
__global__ void __launch_bounds__(128)
k_pairs32(int T_, int S_, int chunk, const SrcRec32 *__restrict__ src, TgtArrays32 tg,
          double *__restrict__ partial)
{
    __shared__ SrcRec32 sh[kTile32];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    float tx[R], ty[R], tz[R], tgv[R], tzw[R], A[R], B[R], C[R], sum[R], comp[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int t = min(tb + r * nth, T_ - 1);
        tx[r] = tg.x[t]; ty[r] = tg.y[t]; tz[r] = tg.zeta[t]; tgv[r] = tg.g[t];
        tzw[r] = tg.zxw[t]; A[r] = tg.A[t]; B[r] = tg.B[t]; C[r] = tg.C[t];
        sum[r] = 0.f; comp[r] = 0.f;
    }
    for (int base = s0; base < s1; base += kTile32) {
        const int nt = min(kTile32, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) sh[i] = src[base + i];
        __syncthreads();
        for (int sb = 0; sb < nt; sb += kSub32) {
            const int se = min(sb + kSub32, nt);
            float loc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) loc[r] = 0.f;
#pragma unroll 2
            for (int s = sb; s < se; ++s) {
                const SrcRec32 q = sh[s];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float p = q.x - tx[r];
                    float qq = q.y - ty[r];
                    float qp = q.y + ty[r];
                    float dz = q.zeta - tz[r];
                    float p2 = p * p;
                    float bs = fmaf(dz, dz, p2);
                    float r1s = fmaf(qq, qq, bs);
                    float r2s = fmaf(qp, qp, bs);
                    float nc = fmaf(-p, q.zx, dz);
                    float n1 = fmaf(-qq, q.zy, nc);
                    float n2 = fmaf(-qp, q.zy, nc);
                    float i1 = rsqrt_ftz(r1s), i2 = rsqrt_ftz(r2s);
                    float i1c = i1 * i1 * i1, i2c = i2 * i2 * i2;
                    float K1 = fmaf(n1, i1c, n2 * i2c);
                    float K2 = i1 + i2;
                    float Ap2 = A[r] * p2;
                    float Bp = B[r] * p;
                    float Q1 = fmaf(fmaf(C[r], qq, Bp), qq, Ap2);
                    float Q2 = fmaf(fmaf(C[r], qp, -Bp), qp, Ap2);
                    float S2 = rsqrt_ftz(Q1) + rsqrt_ftz(Q2);
                    float f = q.g - tgv[r];
                    float inner = fmaf(q.zxw, K2, fmaf(f, K1, -tzw[r] * S2));
                    loc[r] = fmaf(q.w, inner, loc[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float y = loc[r] - comp[r];
                float t2 = sum[r] + y;
                comp[r] = (t2 - sum[r]) - y;
                sum[r] = t2;
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
    const void *k = (precision == SWJ_FP64) ? (const void *)k_pairs<double, kR, false>
                                             : (const void *)k_pairs32<kR>;
    int slots = c->num_sms * resident_blocks(k, kTPB);
    return make_plan(c->T, c->S, slots);
}

void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    SWJ_COUNT_LAUNCH();
    k_pairs<double, kR, false><<<grid, kTPB, 0, c->stream>>>(
        c->T, c->S, pl.chunk, c->src64, c->tgt64, c->mesh.dx, c->mesh.dy, c->partial);
}

void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    SWJ_COUNT_LAUNCH();
    k_pairs32<kR><<<grid, kTPB, 0, c->stream>>>(c->T, c->S, pl.chunk, c->src32, c->tgt32,
                                                c->partial);
}

void swj_launch_pairs_generic32(cudaStream_t st, int T, int S, const SrcRec32 *src,
                                const TgtArrays32 &tgt, double *partial, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    SWJ_COUNT_LAUNCH();
    k_pairs32<kR><<<grid, kTPB, 0, st>>>(T, S, pl.chunk, src, tgt, partial);
}
