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
// FP32 variant: plain FP32 within sub-tiles of 32 sources, Kahan
// compensation when a sub-tile total is added to the running sum.
#include "swj_internal.h"

namespace {

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

template <typename T> struct TileCfg;
template <> struct TileCfg<float> { static constexpr int tile = 512; };
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

constexpr int kTPB = 128;
constexpr int kR = 4;

PairPlan make_plan(int T, int S, int num_sms)
{
    PairPlan p;
    p.tpb = kTPB;
    p.R = kR;
    p.tiles = (T + kTPB * kR - 1) / (kTPB * kR);
    int want = 4 * num_sms;
    int P = (want + p.tiles - 1) / p.tiles;
    int maxP = S / 64 > 1 ? S / 64 : 1;
    if (P > maxP) P = maxP;
    if (P < 1) P = 1;
    p.chunk = (S + P - 1) / P;
    p.P = (S + p.chunk - 1) / p.chunk;
    return p;
}

}  // namespace

PairPlan swj_pair_plan(const swj_ctx *c, int precision)
{
    (void)precision;
    return make_plan(c->T, c->S, c->num_sms);
}

void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    k_pairs<double, kR, false><<<grid, kTPB, 0, c->stream>>>(
        c->T, c->S, pl.chunk, c->src64, c->tgt64, c->mesh.dx, c->mesh.dy, c->partial);
}

void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    k_pairs<float, kR, true><<<grid, kTPB, 0, c->stream>>>(
        c->T, c->S, pl.chunk, c->src32, c->tgt32, (float)c->mesh.dx, (float)c->mesh.dy,
        c->partial);
}

void swj_launch_pairs_generic32(cudaStream_t st, int T, int S, const SrcRec<float> *src,
                                const TgtArrays<float> &tgt, float dX, float dY,
                                double *partial, const PairPlan &pl)
{
    dim3 grid(pl.tiles, pl.P);
    k_pairs<float, kR, true><<<grid, kTPB, 0, st>>>(T, S, pl.chunk, src, tgt, dX, dY, partial);
}
