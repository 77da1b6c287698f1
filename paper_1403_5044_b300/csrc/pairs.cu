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
// FP32 packed variant: Blackwell's paired FP32 instructions (FFMA2, FADD2,
// FMUL2) evaluate the same formulas for two targets per instruction, halving
// the FP32 issue slots per pair; the four reciprocal square roots stay scalar
// (MUFU), which then bounds the kernel.  Every operation and its rounding is
// the one of the scalar kernel, so both give bitwise equal sums for the same
// launch plan.
//
// Launch plan: the number of source chunks is chosen so that
// (target tiles) x (chunks) fills whole waves of resident blocks.  Several
// tile shapes (threads per block, targets per thread, packed or not) are
// compiled; the first residual of a mesh size times each one and keeps the
// fastest for every later launch in the process (the autotuner).
#include "swj_internal.h"
#include <map>
#include <mutex>
#include <tuple>

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


// Source record of the packed kernel in shared memory: each field in both
// halves of a float2 (a broadcast operand of the paired instructions), with
// the negated copies the formulas need: my = -y, nzx = -zeta_x, nzy = -zeta_y.
struct __align__(16) SrcX2 {
    float2 x, y, my, z, nzx, zy, nzy, g, w, zxw;
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsq2(float2 v) { return make_float2(rsqrt_ftz(v.x), rsqrt_ftz(v.y)); }

// RP packed pairs of targets per thread (2 RP targets): target 2m + h of the
// thread is tb + (2m + h) TPB, in lane h of pair m.  MINB = resident blocks per
// SM asked of the register allocator.
template <int RP, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB)
k_pairs_x2(int T_, int S_, int chunk, const SrcRec32 *__restrict__ src, TgtArrays32 tg,
           double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 256;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcX2 sh[TILE];
    const int tid = threadIdx.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    float2 ntx[RP], nty[RP], ntz[RP], ntg[RP], ntzw[RP], A[RP], B[RP], C[RP], sum[RP], comp[RP];
    const int tb = blockIdx.x * 2 * RP * TPB + tid;
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = min(tb + 2 * m * TPB, T_ - 1), tc = min(tb + (2 * m + 1) * TPB, T_ - 1);
        ntx[m] = make_float2(-tg.x[ta], -tg.x[tc]);
        nty[m] = make_float2(-tg.y[ta], -tg.y[tc]);
        ntz[m] = make_float2(-tg.zeta[ta], -tg.zeta[tc]);
        ntg[m] = make_float2(-tg.g[ta], -tg.g[tc]);
        ntzw[m] = make_float2(-tg.zxw[ta], -tg.zxw[tc]);
        A[m] = make_float2(tg.A[ta], tg.A[tc]);
        B[m] = make_float2(tg.B[ta], tg.B[tc]);
        C[m] = make_float2(tg.C[ta], tg.C[tc]);
        sum[m] = f2(0.f);
        comp[m] = f2(0.f);
    }
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += TPB) {
            const SrcRec32 q = src[base + i];
            SrcX2 r;
            r.x = f2(q.x); r.y = f2(q.y); r.my = f2(-q.y); r.z = f2(q.zeta);
            r.nzx = f2(-q.zx); r.zy = f2(q.zy); r.nzy = f2(-q.zy);
            r.g = f2(q.g); r.w = f2(q.w); r.zxw = f2(q.zxw);
            sh[i] = r;
        }
        __syncthreads();
        for (int sb = 0; sb < nt; sb += kSub) {
            const int se = min(sb + kSub, nt);
            float2 loc[RP];
#pragma unroll
            for (int m = 0; m < RP; ++m) loc[m] = f2(0.f);
#pragma unroll 1
            for (int s = sb; s < se; ++s) {
                const SrcX2 q = sh[s];
#pragma unroll
                for (int m = 0; m < RP; ++m) {
                    const float2 p = __fadd2_rn(q.x, ntx[m]);
                    const float2 qq = __fadd2_rn(q.y, nty[m]);
                    const float2 mqp = __fadd2_rn(q.my, nty[m]);      // -(y + y*)
                    const float2 dz = __fadd2_rn(q.z, ntz[m]);
                    const float2 p2 = __fmul2_rn(p, p);
                    const float2 bs = __ffma2_rn(dz, dz, p2);
                    const float2 r1s = __ffma2_rn(qq, qq, bs);
                    const float2 r2s = __ffma2_rn(mqp, mqp, bs);
                    const float2 nc = __ffma2_rn(p, q.nzx, dz);
                    const float2 n1 = __ffma2_rn(qq, q.nzy, nc);
                    const float2 n2 = __ffma2_rn(mqp, q.zy, nc);
                    const float2 i1 = rsq2(r1s), i2 = rsq2(r2s);
                    const float2 i1c = __fmul2_rn(__fmul2_rn(i1, i1), i1);
                    const float2 i2c = __fmul2_rn(__fmul2_rn(i2, i2), i2);
                    const float2 K1 = __ffma2_rn(n1, i1c, __fmul2_rn(n2, i2c));
                    const float2 K2 = __fadd2_rn(i1, i2);
                    const float2 Ap2 = __fmul2_rn(A[m], p2);
                    const float2 Bp = __fmul2_rn(B[m], p);
                    const float2 Q1 = __ffma2_rn(__ffma2_rn(C[m], qq, Bp), qq, Ap2);
                    const float2 Q2 = __ffma2_rn(__ffma2_rn(C[m], mqp, Bp), mqp, Ap2);
                    const float2 S2 = __fadd2_rn(rsq2(Q1), rsq2(Q2));
                    const float2 f = __fadd2_rn(q.g, ntg[m]);
                    const float2 inner = __ffma2_rn(q.zxw, K2, __ffma2_rn(f, K1, __fmul2_rn(ntzw[m], S2)));
                    loc[m] = __ffma2_rn(q.w, inner, loc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < RP; ++m) {
                float y = loc[m].x - comp[m].x, t2 = sum[m].x + y;
                comp[m].x = (t2 - sum[m].x) - y;
                sum[m].x = t2;
                y = loc[m].y - comp[m].y;
                t2 = sum[m].y + y;
                comp[m].y = (t2 - sum[m].y) - y;
                sum[m].y = t2;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = tb + 2 * m * TPB, tc = tb + (2 * m + 1) * TPB;
        if (ta < T_) partial[(size_t)blockIdx.y * T_ + ta] = (double)sum[m].x - (double)comp[m].x;
        if (tc < T_) partial[(size_t)blockIdx.y * T_ + tc] = (double)sum[m].y - (double)comp[m].y;
    }
}



// Packed kernel with the source-row terms hoisted.  Sources are ordered row
// by row (N per row, y = j exact), so within a row dy = j - y* and
// dy' = j + y* are constants of the target; with them
//   r1^2 = p^2 + (dz^2 + dy^2),   Q1 = (A p + B dy) p + C dy^2
// (and the image forms with -dy') cost 2 operations each per pair, and the
// row constants (dy, -dy', dy^2, dy'^2, B dy, -B dy', C dy^2, C dy'^2) are
// recomputed only when the source row changes: 26 FP32 operations per pair
// instead of 30 (the stated algorithmic count stays 44 flop).  The sums
// differ from the scalar kernel's in rounding only.
struct __align__(16) SrcX2R {
    float2 x, z, nzx, zy, nzy, g, w, zxw;
};

// LEAN: B, C and y* are not held in registers but reloaded (from L1) at each
// row change.  UNR: unroll factor of the source loop (more independent
// reciprocal square roots in flight per warp).
template <int RP, int TPB, int MINB, bool LEAN, int UNR>
__global__ void __launch_bounds__(TPB, MINB)
k_pairs_x2r(int T_, int S_, int chunk, int N, const SrcRec32 *__restrict__ src, TgtArrays32 tg,
            double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 256;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcX2R sh[TILE];
    const int tid = threadIdx.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    float2 ntx[RP], nty[RP], ntz[RP], ntg[RP], ntzw[RP], A[RP], B[RP], C[RP], sum[RP], comp[RP];
    float2 dy[RP], mdyp[RP], dy2[RP], dyp2[RP], Bdy[RP], mBdyp[RP], Cdy2[RP], Cdyp2[RP];
    const int tb = blockIdx.x * 2 * RP * TPB + tid;
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = min(tb + 2 * m * TPB, T_ - 1), tc = min(tb + (2 * m + 1) * TPB, T_ - 1);
        ntx[m] = make_float2(-tg.x[ta], -tg.x[tc]);
        if (!LEAN) nty[m] = make_float2(-tg.y[ta], -tg.y[tc]);
        ntz[m] = make_float2(-tg.zeta[ta], -tg.zeta[tc]);
        ntg[m] = make_float2(-tg.g[ta], -tg.g[tc]);
        ntzw[m] = make_float2(-tg.zxw[ta], -tg.zxw[tc]);
        A[m] = make_float2(tg.A[ta], tg.A[tc]);
        if (!LEAN) {
            B[m] = make_float2(tg.B[ta], tg.B[tc]);
            C[m] = make_float2(tg.C[ta], tg.C[tc]);
        }
        sum[m] = f2(0.f);
        comp[m] = f2(0.f);
    }
    int row = -1;            // source row the row constants belong to
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += TPB) {
            const SrcRec32 q = src[base + i];
            SrcX2R r;
            r.x = f2(q.x); r.z = f2(q.zeta); r.nzx = f2(-q.zx); r.zy = f2(q.zy); r.nzy = f2(-q.zy);
            r.g = f2(q.g); r.w = f2(q.w); r.zxw = f2(q.zxw);
            sh[i] = r;
        }
        __syncthreads();
        int j = base / N;                      // row of source `base`
        int row_end = (j + 1) * N - base;      // tile index where row j ends
        for (int sb = 0; sb < nt; sb += kSub) {
            const int se = min(sb + kSub, nt);
            float2 loc[RP];
#pragma unroll
            for (int m = 0; m < RP; ++m) loc[m] = f2(0.f);
            int s = sb;
            while (s < se) {
                while (s >= row_end) { ++j; row_end += N; }
                if (j != row) {
                    row = j;
                    const float2 yj = f2((float)j), myj = f2(-(float)j);
#pragma unroll
                    for (int m = 0; m < RP; ++m) {
                        float2 ny = nty[m], Bm = B[m], Cm = C[m];
                        if (LEAN) {
                            const int ta = min(tb + 2 * m * TPB, T_ - 1), tc = min(tb + (2 * m + 1) * TPB, T_ - 1);
                            ny = make_float2(-tg.y[ta], -tg.y[tc]);
                            Bm = make_float2(tg.B[ta], tg.B[tc]);
                            Cm = make_float2(tg.C[ta], tg.C[tc]);
                        }
                        dy[m] = __fadd2_rn(yj, ny);
                        mdyp[m] = __fadd2_rn(myj, ny);               // -(y_j + y*)
                        dy2[m] = __fmul2_rn(dy[m], dy[m]);
                        dyp2[m] = __fmul2_rn(mdyp[m], mdyp[m]);
                        Bdy[m] = __fmul2_rn(Bm, dy[m]);
                        mBdyp[m] = __fmul2_rn(Bm, mdyp[m]);
                        Cdy2[m] = __fmul2_rn(Cm, dy2[m]);
                        Cdyp2[m] = __fmul2_rn(Cm, dyp2[m]);
                    }
                }
                const int send = min(se, row_end);
#pragma unroll UNR
                for (; s < send; ++s) {
                    const SrcX2R q = sh[s];
#pragma unroll
                    for (int m = 0; m < RP; ++m) {
                        const float2 p = __fadd2_rn(q.x, ntx[m]);
                        const float2 dz = __fadd2_rn(q.z, ntz[m]);
                        const float2 r1s = __ffma2_rn(p, p, __ffma2_rn(dz, dz, dy2[m]));
                        const float2 r2s = __ffma2_rn(p, p, __ffma2_rn(dz, dz, dyp2[m]));
                        const float2 nc = __ffma2_rn(p, q.nzx, dz);
                        const float2 n1 = __ffma2_rn(dy[m], q.nzy, nc);
                        const float2 n2 = __ffma2_rn(mdyp[m], q.zy, nc);
                        const float2 i1 = rsq2(r1s), i2 = rsq2(r2s);
                        const float2 i1c = __fmul2_rn(__fmul2_rn(i1, i1), i1);
                        const float2 i2c = __fmul2_rn(__fmul2_rn(i2, i2), i2);
                        const float2 K1 = __ffma2_rn(n1, i1c, __fmul2_rn(n2, i2c));
                        const float2 K2 = __fadd2_rn(i1, i2);
                        const float2 Q1 = __ffma2_rn(__ffma2_rn(A[m], p, Bdy[m]), p, Cdy2[m]);
                        const float2 Q2 = __ffma2_rn(__ffma2_rn(A[m], p, mBdyp[m]), p, Cdyp2[m]);
                        const float2 S2 = __fadd2_rn(rsq2(Q1), rsq2(Q2));
                        const float2 f = __fadd2_rn(q.g, ntg[m]);
                        const float2 inner =
                            __ffma2_rn(q.zxw, K2, __ffma2_rn(f, K1, __fmul2_rn(ntzw[m], S2)));
                        loc[m] = __ffma2_rn(q.w, inner, loc[m]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < RP; ++m) {
                float y = loc[m].x - comp[m].x, t2 = sum[m].x + y;
                comp[m].x = (t2 - sum[m].x) - y;
                sum[m].x = t2;
                y = loc[m].y - comp[m].y;
                t2 = sum[m].y + y;
                comp[m].y = (t2 - sum[m].y) - y;
                sum[m].y = t2;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = tb + 2 * m * TPB, tc = tb + (2 * m + 1) * TPB;
        if (ta < T_) partial[(size_t)blockIdx.y * T_ + ta] = (double)sum[m].x - (double)comp[m].x;
        if (tc < T_) partial[(size_t)blockIdx.y * T_ + tc] = (double)sum[m].y - (double)comp[m].y;
    }
}


// FP64 kernel with the source-row terms hoisted (as k_pairs_x2r): within a
// source row dy = j - y* and dy' = j + y* are constants of the target, so r^2
// and the quadratic forms take two operations each per pair (6.6 % faster than
// k_pairs_s<double> at 181x61).  Plain FP64 accumulation.  (Seeding the
// reciprocal square root with the FP64 approximation instead of the FP32 one,
// which saves two conversions, measured 20 % slower.)
template <int R>
__global__ void __launch_bounds__(128)
k_pairs_r64(int T_, int S_, int chunk, int N, const SrcRec64 *__restrict__ src, TgtArrays64 tg,
            double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 256;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcRec64 sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    double ntx[R], ty[R], ntz[R], ntg[R], ntzw[R], A[R], B[R], C[R], sum[R];
    double dy[R], mdyp[R], dy2[R], dyp2[R], Bdy[R], mBdyp[R], Cdy2[R], Cdyp2[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = min(tb + r * nth, T_ - 1);
        ntx[r] = -tg.x[t]; ty[r] = tg.y[t]; ntz[r] = -tg.zeta[t]; ntg[r] = -tg.g[t];
        ntzw[r] = -tg.zxw[t]; A[r] = tg.A[t]; B[r] = tg.B[t]; C[r] = tg.C[t];
        sum[r] = 0.0;
    }
    int row = -1;
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) sh[i] = src[base + i];
        __syncthreads();
        int j = base / N;
        int row_end = (j + 1) * N - base;
        int s = 0;
        while (s < nt) {
            while (s >= row_end) { ++j; row_end += N; }
            if (j != row) {
                row = j;
                const double yj = (double)j;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    dy[r] = yj - ty[r];
                    mdyp[r] = -yj - ty[r];                 // -(y_j + y*)
                    dy2[r] = dy[r] * dy[r];
                    dyp2[r] = mdyp[r] * mdyp[r];
                    Bdy[r] = B[r] * dy[r];
                    mBdyp[r] = B[r] * mdyp[r];
                    Cdy2[r] = C[r] * dy2[r];
                    Cdyp2[r] = C[r] * dyp2[r];
                }
            }
            const int send = min(nt, row_end);
#pragma unroll 2
            for (; s < send; ++s) {
                const SrcRec64 q = sh[s];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double p = q.x + ntx[r];
                    const double dz = q.zeta + ntz[r];
                    const double r1s = fma(p, p, fma(dz, dz, dy2[r]));
                    const double r2s = fma(p, p, fma(dz, dz, dyp2[r]));
                    const double nc = fma(-p, q.zx, dz);
                    const double n1 = fma(-dy[r], q.zy, nc);
                    const double n2 = fma(mdyp[r], q.zy, nc);
                    const double i1 = rsqrt_f64(r1s), i2 = rsqrt_f64(r2s);
                    const double i1c = i1 * i1 * i1, i2c = i2 * i2 * i2;
                    const double K1 = fma(n1, i1c, n2 * i2c);
                    const double K2 = i1 + i2;
                    const double Q1 = fma(fma(A[r], p, Bdy[r]), p, Cdy2[r]);
                    const double Q2 = fma(fma(A[r], p, mBdyp[r]), p, Cdyp2[r]);
                    const double S2 = rsqrt_f64(Q1) + rsqrt_f64(Q2);
                    const double f = q.g + ntg[r];
                    const double inner = fma(q.zxw, K2, fma(f, K1, ntzw[r] * S2));
                    sum[r] = fma(q.w, inner, sum[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tb + r * nth;
        if (t < T_) partial[(size_t)blockIdx.y * T_ + t] = sum[r];
    }
}


// ------------------------------------------------------------ float-float
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significant bits).  The sums and products below are the classic
// error-free transformations: Knuth's two-sum, Dekker's fast two-sum (for
// |a| >= |b|) and the FMA-based exact product; every operation is an explicit
// round-to-nearest intrinsic so that no FMA contraction can break them.  The
// additions are the "sloppy" float-float sum (the error is bounded by
// ~2^-44 (|a| + |b|), not by |a + b|), which is what the all-pairs sum needs:
// its tolerance is relative to the sum of absolute terms.
struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_from(double d)
{
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}

__device__ __forceinline__ ff ff_fast2(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_two_sum(a.h, b.h);
    return ff_fast2(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ ff ff_addf(ff a, float b)   // b exact
{
    const ff s = ff_two_sum(a.h, b);
    return ff_fast2(s.h, __fadd_rn(s.l, a.l));
}

// the accurate sum (both halves two-summed): for the running totals
__device__ __forceinline__ ff ff_add_acc(ff a, ff b)
{
    const ff s = ff_two_sum(a.h, b.h);
    const ff t = ff_two_sum(a.l, b.l);
    const ff u = ff_fast2(s.h, __fadd_rn(s.l, t.h));
    return ff_fast2(u.h, __fadd_rn(u.l, t.l));
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_fast2(p, e);
}

__device__ __forceinline__ ff ff_mulf(ff a, float b)   // b exact
{
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return ff_fast2(p, e);
}

// 1/sqrt(x): the FP32 hardware approximation y (relative error ~2^-23) and one
// Newton step y (1 + (1 - x y^2) / 2), with x y^2 formed in float-float (its
// first difference from 1 is exact), giving ~2^-46 relative.
__device__ __forceinline__ ff ff_rsqrt(ff x)
{
    const float y = rsqrt_ftz(x.h);
    const ff t = ff_mulf(ff_mulf(x, y), y);
    const float r = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
    return ff_fast2(y, __fmul_rn(__fmul_rn(0.5f, y), r));
}

// Source record of the float-float kernel (converted from the FP64 record when
// staged): coordinates and fields split into hi + lo.
struct __align__(16) SrcFF {
    ff x, z, zx, zy, g, w, zxw, pad;
};

// The all-pairs sum in float-float, structured as k_pairs_r64 (source-row
// terms hoisted; dy, dy' and their squares are exact small integers in units
// of dy).  Running totals use the accurate sum every 64 sources.
template <int R>
__global__ void __launch_bounds__(128)
k_pairs_ff(int T_, int S_, int chunk, int N, const SrcRec64 *__restrict__ src, TgtArrays64 tg,
           double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 256;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcFF sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    ff ntx[R], ntz[R], ntg[R], ntzw[R], A[R], B[R], C[R], sum[R];
    float ty[R], dy[R], mdyp[R], dy2[R], dyp2[R];
    ff Bdy[R], mBdyp[R], Cdy2[R], Cdyp2[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = min(tb + r * nth, T_ - 1);
        ntx[r] = ff_from(-tg.x[t]); ty[r] = (float)tg.y[t]; ntz[r] = ff_from(-tg.zeta[t]);
        ntg[r] = ff_from(-tg.g[t]); ntzw[r] = ff_from(-tg.zxw[t]);
        A[r] = ff_from(tg.A[t]); B[r] = ff_from(tg.B[t]); C[r] = ff_from(tg.C[t]);
        sum[r] = {0.f, 0.f};
    }
    int row = -1;
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) {
            const SrcRec64 q = src[base + i];
            SrcFF r;
            r.x = ff_from(q.x); r.z = ff_from(q.zeta); r.zx = ff_from(q.zx); r.zy = ff_from(q.zy);
            r.g = ff_from(q.g); r.w = ff_from(q.w); r.zxw = ff_from(q.zxw); r.pad = {0.f, 0.f};
            sh[i] = r;
        }
        __syncthreads();
        int j = base / N;
        int row_end = (j + 1) * N - base;
        for (int sb = 0; sb < nt; sb += kSub) {
            const int se = min(sb + kSub, nt);
            ff loc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) loc[r] = {0.f, 0.f};
            int s = sb;
            while (s < se) {
                while (s >= row_end) { ++j; row_end += N; }
                if (j != row) {
                    row = j;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        dy[r] = (float)j - ty[r];              // exact (integers)
                        mdyp[r] = -(float)j - ty[r];            // -(y_j + y*)
                        dy2[r] = dy[r] * dy[r];
                        dyp2[r] = mdyp[r] * mdyp[r];
                        Bdy[r] = ff_mulf(B[r], dy[r]);
                        mBdyp[r] = ff_mulf(B[r], mdyp[r]);
                        Cdy2[r] = ff_mulf(C[r], dy2[r]);
                        Cdyp2[r] = ff_mulf(C[r], dyp2[r]);
                    }
                }
                const int send = min(se, row_end);
#pragma unroll 1
                for (; s < send; ++s) {
                    const SrcFF q = sh[s];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const ff p = ff_add(q.x, ntx[r]);
                        const ff dz = ff_add(q.z, ntz[r]);
                        const ff bs = ff_add(ff_mul(p, p), ff_mul(dz, dz));
                        const ff r1s = ff_addf(bs, dy2[r]);
                        const ff r2s = ff_addf(bs, dyp2[r]);
                        const ff nc = ff_add(dz, ff_neg(ff_mul(p, q.zx)));
                        const ff n1 = ff_add(nc, ff_neg(ff_mulf(q.zy, dy[r])));
                        const ff n2 = ff_add(nc, ff_mulf(q.zy, mdyp[r]));
                        const ff i1 = ff_rsqrt(r1s), i2 = ff_rsqrt(r2s);
                        const ff i1c = ff_mul(ff_mul(i1, i1), i1), i2c = ff_mul(ff_mul(i2, i2), i2);
                        const ff K1 = ff_add(ff_mul(n1, i1c), ff_mul(n2, i2c));
                        const ff K2 = ff_add(i1, i2);
                        const ff Ap = ff_mul(A[r], p);
                        const ff Q1 = ff_add(ff_mul(ff_add(Ap, Bdy[r]), p), Cdy2[r]);
                        const ff Q2 = ff_add(ff_mul(ff_add(Ap, mBdyp[r]), p), Cdyp2[r]);
                        const ff S2 = ff_add(ff_rsqrt(Q1), ff_rsqrt(Q2));
                        const ff f = ff_add(q.g, ntg[r]);
                        const ff inner = ff_add(ff_add(ff_mul(q.zxw, K2), ff_mul(f, K1)), ff_mul(ntzw[r], S2));
                        loc[r] = ff_add(loc[r], ff_mul(q.w, inner));
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) sum[r] = ff_add_acc(sum[r], loc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = tb + r * nth;
        if (t < T_) partial[(size_t)blockIdx.y * T_ + t] = (double)sum[r].h + (double)sum[r].l;
    }
}

// ------------------------------------------------------- float-float, packed
// The same float-float arithmetic on two targets at once: every value of a
// target pair is an ff2 (the hi and lo floats of both targets, each a float2)
// and every error-free transformation is the packed instruction
// (__fadd2_rn, __fmul2_rn, __ffma2_rn: one rounding per lane, as the scalar
// intrinsics), so each lane computes what k_pairs_ff computes for its target
// over the same sources, with half the FP32 instructions (the source chunking
// follows from the kernel's occupancy, as for every variant).  Subtractions
// are an FMA with -1 (exact product, one rounding).
struct ff2 {
    float2 h, l;
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ ff2 ff2_fast2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    return {s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 ff2_two_sum(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    return {s, __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b)
{
    const ff2 s = ff2_two_sum(a.h, b.h);
    return ff2_fast2(s.h, __fadd2_rn(s.l, __fadd2_rn(a.l, b.l)));
}

__device__ __forceinline__ ff2 ff2_addf(ff2 a, float2 b)   // b exact
{
    const ff2 s = ff2_two_sum(a.h, b);
    return ff2_fast2(s.h, __fadd2_rn(s.l, a.l));
}

__device__ __forceinline__ ff2 ff2_add_acc(ff2 a, ff2 b)
{
    const ff2 s = ff2_two_sum(a.h, b.h);
    const ff2 t = ff2_two_sum(a.l, b.l);
    const ff2 u = ff2_fast2(s.h, __fadd2_rn(s.l, t.h));
    return ff2_fast2(u.h, __fadd2_rn(u.l, t.l));
}

__device__ __forceinline__ ff2 ff2_neg(ff2 a)
{
    return {make_float2(-a.h.x, -a.h.y), make_float2(-a.l.x, -a.l.y)};
}

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b)
{
    const float2 p = __fmul2_rn(a.h, b.h);
    float2 e = __ffma2_rn(a.h, b.h, make_float2(-p.x, -p.y));
    e = __ffma2_rn(a.h, b.l, e);
    e = __ffma2_rn(a.l, b.h, e);
    return ff2_fast2(p, e);
}

__device__ __forceinline__ ff2 ff2_mulf(ff2 a, float2 b)   // b exact
{
    const float2 p = __fmul2_rn(a.h, b);
    float2 e = __ffma2_rn(a.h, b, make_float2(-p.x, -p.y));
    e = __ffma2_rn(a.l, b, e);
    return ff2_fast2(p, e);
}

__device__ __forceinline__ ff2 ff2_rsqrt(ff2 x)
{
    const float2 y = make_float2(rsqrt_ftz(x.h.x), rsqrt_ftz(x.h.y));
    const ff2 t = ff2_mulf(ff2_mulf(x, y), y);
    const float2 r = sub2(sub2(make_float2(1.f, 1.f), t.h), t.l);
    return ff2_fast2(y, __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), y), r));
}

__device__ __forceinline__ ff2 ff2_bc(ff v) { return {make_float2(v.h, v.h), make_float2(v.l, v.l)}; }

// source record of the packed kernel: every field broadcast to both lanes
struct __align__(16) SrcFF2 {
    ff2 x, z, zx, zy, g, w, zxw;
};

// RP packed pairs of targets per thread (target 2m + h of the thread is
// tb + (2m + h) 128, in lane h of pair m); otherwise k_pairs_ff.
template <int RP>
__global__ void __launch_bounds__(128)
k_pairs_ff2(int T_, int S_, int chunk, int N, const SrcRec64 *__restrict__ src, TgtArrays64 tg,
            double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 128;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcFF2 sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(S_, s0 + chunk);
    ff2 ntx[RP], ntz[RP], ntg[RP], ntzw[RP], A[RP], B[RP], C[RP], sum[RP];
    float2 ty[RP], dy[RP], mdyp[RP], dy2[RP], dyp2[RP];
    ff2 Bdy[RP], mBdyp[RP], Cdy2[RP], Cdyp2[RP];
    const int tb = blockIdx.x * 2 * RP * nth + tid;
    auto pair = [&](const double *a, int ta, int tc, bool neg) {
        const ff u = ff_from(neg ? -a[ta] : a[ta]), v = ff_from(neg ? -a[tc] : a[tc]);
        return ff2{make_float2(u.h, v.h), make_float2(u.l, v.l)};
    };
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = min(tb + 2 * m * nth, T_ - 1), tc = min(tb + (2 * m + 1) * nth, T_ - 1);
        ntx[m] = pair(tg.x, ta, tc, true); ntz[m] = pair(tg.zeta, ta, tc, true);
        ntg[m] = pair(tg.g, ta, tc, true); ntzw[m] = pair(tg.zxw, ta, tc, true);
        A[m] = pair(tg.A, ta, tc, false); B[m] = pair(tg.B, ta, tc, false); C[m] = pair(tg.C, ta, tc, false);
        ty[m] = make_float2((float)tg.y[ta], (float)tg.y[tc]);
        sum[m] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
    int row = -1;
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) {
            const SrcRec64 q = src[base + i];
            SrcFF2 r;
            r.x = ff2_bc(ff_from(q.x)); r.z = ff2_bc(ff_from(q.zeta)); r.zx = ff2_bc(ff_from(q.zx));
            r.zy = ff2_bc(ff_from(q.zy)); r.g = ff2_bc(ff_from(q.g)); r.w = ff2_bc(ff_from(q.w));
            r.zxw = ff2_bc(ff_from(q.zxw));
            sh[i] = r;
        }
        __syncthreads();
        int j = base / N;
        int row_end = (j + 1) * N - base;
        for (int sb = 0; sb < nt; sb += kSub) {
            const int se = min(sb + kSub, nt);
            ff2 loc[RP];
#pragma unroll
            for (int m = 0; m < RP; ++m) loc[m] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            int s = sb;
            while (s < se) {
                while (s >= row_end) { ++j; row_end += N; }
                if (j != row) {
                    row = j;
#pragma unroll
                    for (int m = 0; m < RP; ++m) {
                        dy[m] = make_float2((float)j - ty[m].x, (float)j - ty[m].y);        // exact (integers)
                        mdyp[m] = make_float2(-(float)j - ty[m].x, -(float)j - ty[m].y);    // -(y_j + y*)
                        dy2[m] = make_float2(dy[m].x * dy[m].x, dy[m].y * dy[m].y);
                        dyp2[m] = make_float2(mdyp[m].x * mdyp[m].x, mdyp[m].y * mdyp[m].y);
                        Bdy[m] = ff2_mulf(B[m], dy[m]);
                        mBdyp[m] = ff2_mulf(B[m], mdyp[m]);
                        Cdy2[m] = ff2_mulf(C[m], dy2[m]);
                        Cdyp2[m] = ff2_mulf(C[m], dyp2[m]);
                    }
                }
                const int send = min(se, row_end);
#pragma unroll 1
                for (; s < send; ++s) {
                    const SrcFF2 q = sh[s];
#pragma unroll
                    for (int m = 0; m < RP; ++m) {
                        const ff2 p = ff2_add(q.x, ntx[m]);
                        const ff2 dz = ff2_add(q.z, ntz[m]);
                        const ff2 bs = ff2_add(ff2_mul(p, p), ff2_mul(dz, dz));
                        const ff2 r1s = ff2_addf(bs, dy2[m]);
                        const ff2 r2s = ff2_addf(bs, dyp2[m]);
                        const ff2 nc = ff2_add(dz, ff2_neg(ff2_mul(p, q.zx)));
                        const ff2 n1 = ff2_add(nc, ff2_neg(ff2_mulf(q.zy, dy[m])));
                        const ff2 n2 = ff2_add(nc, ff2_mulf(q.zy, mdyp[m]));
                        const ff2 i1 = ff2_rsqrt(r1s), i2 = ff2_rsqrt(r2s);
                        const ff2 i1c = ff2_mul(ff2_mul(i1, i1), i1), i2c = ff2_mul(ff2_mul(i2, i2), i2);
                        const ff2 K1 = ff2_add(ff2_mul(n1, i1c), ff2_mul(n2, i2c));
                        const ff2 K2 = ff2_add(i1, i2);
                        const ff2 Ap = ff2_mul(A[m], p);
                        const ff2 Q1 = ff2_add(ff2_mul(ff2_add(Ap, Bdy[m]), p), Cdy2[m]);
                        const ff2 Q2 = ff2_add(ff2_mul(ff2_add(Ap, mBdyp[m]), p), Cdyp2[m]);
                        const ff2 S2 = ff2_add(ff2_rsqrt(Q1), ff2_rsqrt(Q2));
                        const ff2 f = ff2_add(q.g, ntg[m]);
                        const ff2 inner =
                            ff2_add(ff2_add(ff2_mul(q.zxw, K2), ff2_mul(f, K1)), ff2_mul(ntzw[m], S2));
                        loc[m] = ff2_add(loc[m], ff2_mul(q.w, inner));
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < RP; ++m) sum[m] = ff2_add_acc(sum[m], loc[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = tb + 2 * m * nth, tc = tb + (2 * m + 1) * nth;
        if (ta < T_) partial[(size_t)blockIdx.y * T_ + ta] = (double)sum[m].h.x + (double)sum[m].l.x;
        if (tc < T_) partial[(size_t)blockIdx.y * T_ + tc] = (double)sum[m].h.y + (double)sum[m].l.y;
    }
}

// Source-chunk count P for (tiles) target tiles: (tiles x P) blocks should fill
// whole waves of `slots` resident blocks; chunks keep at least 64 sources.
PairPlan make_plan(int T, int S, int slots, int tpb, int R, int v)
{
    PairPlan p;
    p.tpb = tpb;
    p.R = R;
    p.v = v;
    p.tiles = (T + tpb * R - 1) / (tpb * R);
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

typedef void (*PairLaunch)(dim3, cudaStream_t, int, int, int, int, const void *, const void *,
                           double *, const int *);

struct PairVariant {
    const void *kernel;
    int tpb, R;
    PairLaunch launch;
    const char *name;
};

template <typename T, int R, int TPB> struct ScalarLaunch;
template <typename T, int R> struct ScalarLaunch<T, R, 128> {
    static void go(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int, const void *src,
                   const void *tg, double *partial, const int *act)
    {
        k_pairs_s<T, R><<<g, 128, 0, st>>>(T_, S_, chunk, (const SrcRecS<T> *)src,
                                           *(const TgtArraysS<T> *)tg, partial, act);
    }
};

template <int R>
void launch_ff(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int N, const void *src,
               const void *tg, double *partial, const int *act)
{
    k_pairs_ff<R><<<g, 128, 0, st>>>(T_, S_, chunk, N, (const SrcRec64 *)src, *(const TgtArrays64 *)tg,
                                     partial, act);
}

template <int RP>
void launch_ff2(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int N, const void *src,
                const void *tg, double *partial, const int *act)
{
    k_pairs_ff2<RP><<<g, 128, 0, st>>>(T_, S_, chunk, N, (const SrcRec64 *)src, *(const TgtArrays64 *)tg,
                                       partial, act);
}

template <int R>
void launch_r64(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int N, const void *src,
                const void *tg, double *partial, const int *act)
{
    k_pairs_r64<R><<<g, 128, 0, st>>>(T_, S_, chunk, N, (const SrcRec64 *)src,
                                            *(const TgtArrays64 *)tg, partial, act);
}

template <int RP, int TPB, int MINB, bool LEAN, int UNR>
void launch_x2r(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int N, const void *src,
                const void *tg, double *partial, const int *act)
{
    k_pairs_x2r<RP, TPB, MINB, LEAN, UNR><<<g, TPB, 0, st>>>(T_, S_, chunk, N, (const SrcRec32 *)src,
                                                  *(const TgtArrays32 *)tg, partial, act);
}

template <int RP, int TPB, int MINB>
void launch_x2(dim3 g, cudaStream_t st, int T_, int S_, int chunk, int, const void *src, const void *tg,
               double *partial, const int *act)
{
    k_pairs_x2<RP, TPB, MINB><<<g, TPB, 0, st>>>(T_, S_, chunk, (const SrcRec32 *)src,
                                          *(const TgtArrays32 *)tg, partial, act);
}

// Compiled tile shapes; index 0 of each table is the untuned default.  Only
// shapes that compile without register spills are candidates (a spilling
// shape reads and writes its spill slots through the memory system).
const PairVariant kVar32[] = {
    {(const void *)k_pairs_s<float, 4>, 128, 4, ScalarLaunch<float, 4, 128>::go, "k_pairs_s<float,4>"},
    {(const void *)k_pairs_x2<2, 128, 1>, 128, 4, launch_x2<2, 128, 1>, "k_pairs_x2<2,128,1>"},
    {(const void *)k_pairs_x2<3, 128, 1>, 128, 6, launch_x2<3, 128, 1>, "k_pairs_x2<3,128,1>"},
    {(const void *)k_pairs_x2<4, 128, 1>, 128, 8, launch_x2<4, 128, 1>, "k_pairs_x2<4,128,1>"},
    {(const void *)k_pairs_x2<2, 256, 1>, 256, 4, launch_x2<2, 256, 1>, "k_pairs_x2<2,256,1>"},
    {(const void *)k_pairs_x2<4, 64, 1>, 64, 8, launch_x2<4, 64, 1>, "k_pairs_x2<4,64,1>"},
    {(const void *)k_pairs_x2<3, 256, 2>, 256, 6, launch_x2<3, 256, 2>, "k_pairs_x2<3,256,2>"},
    {(const void *)k_pairs_x2<1, 256, 4>, 256, 2, launch_x2<1, 256, 4>, "k_pairs_x2<1,256,4>"},
    {(const void *)k_pairs_x2r<2, 256, 2, false, 1>, 256, 4, launch_x2r<2, 256, 2, false, 1>, "k_pairs_x2r<2,256,2,0,1>"},
    {(const void *)k_pairs_x2r<2, 256, 2, true, 1>, 256, 4, launch_x2r<2, 256, 2, true, 1>, "k_pairs_x2r<2,256,2,1,1>"},
    {(const void *)k_pairs_x2r<3, 128, 2, true, 1>, 128, 6, launch_x2r<3, 128, 2, true, 1>, "k_pairs_x2r<3,128,2,1,1>"},
    {(const void *)k_pairs_x2r<1, 256, 4, true, 1>, 256, 2, launch_x2r<1, 256, 4, true, 1>, "k_pairs_x2r<1,256,4,1,1>"},
    {(const void *)k_pairs_x2r<1, 256, 4, true, 2>, 256, 2, launch_x2r<1, 256, 4, true, 2>, "k_pairs_x2r<1,256,4,1,2>"},
    {(const void *)k_pairs_x2r<1, 256, 3, true, 2>, 256, 2, launch_x2r<1, 256, 3, true, 2>, "k_pairs_x2r<1,256,3,1,2>"},
    {(const void *)k_pairs_x2r<2, 256, 2, false, 2>, 256, 4, launch_x2r<2, 256, 2, false, 2>, "k_pairs_x2r<2,256,2,0,2>"},
};
const PairVariant kVar64[] = {
    {(const void *)k_pairs_r64<2>, 128, 2, launch_r64<2>, "k_pairs_r64<2>"},
    {(const void *)k_pairs_r64<4>, 128, 4, launch_r64<4>, "k_pairs_r64<4>"},
    {(const void *)k_pairs_s<double, 2>, 128, 2, ScalarLaunch<double, 2, 128>::go, "k_pairs_s<double,2>"},
    {(const void *)k_pairs_s<double, 4>, 128, 4, ScalarLaunch<double, 4, 128>::go, "k_pairs_s<double,4>"},
};
const PairVariant kVarFF[] = {
    {(const void *)k_pairs_ff2<1>, 128, 2, launch_ff2<1>, "k_pairs_ff2<1>"},
    {(const void *)k_pairs_ff<2>, 128, 2, launch_ff<2>, "k_pairs_ff<2>"},
    {(const void *)k_pairs_ff<1>, 128, 1, launch_ff<1>, "k_pairs_ff<1>"},
    {(const void *)k_pairs_ff<4>, 128, 4, launch_ff<4>, "k_pairs_ff<4>"},
    {(const void *)k_pairs_ff2<2>, 128, 4, launch_ff2<2>, "k_pairs_ff2<2>"},
};
constexpr int kNVar32 = sizeof(kVar32) / sizeof(kVar32[0]);
constexpr int kNVar64 = sizeof(kVar64) / sizeof(kVar64[0]);
constexpr int kNVarFF = sizeof(kVarFF) / sizeof(kVarFF[0]);

const PairVariant &variant(int precision, int v)
{
    return precision == SWJ_FP64 ? kVar64[v] : (precision == SWJ_FF ? kVarFF[v] : kVar32[v]);
}

int n_variants(int precision) { return precision == SWJ_FP64 ? kNVar64 : (precision == SWJ_FF ? kNVarFF : kNVar32); }

// tuned variant per (T, S, precision, SM count), shared by every context
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, int> g_tuned;

int tuned_variant(const swj_ctx *c, int precision)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(std::make_tuple(c->T, c->S, precision, c->num_sms));
    return it == g_tuned.end() ? -1 : it->second;
}

}  // namespace

PairPlan swj_pair_plan_variant(const swj_ctx *c, int precision, int v)
{
    const PairVariant &pv = variant(precision, v);
    int slots = c->num_sms * resident_blocks(pv.kernel, pv.tpb);
    return make_plan(c->T, c->S, slots, pv.tpb, pv.R, v);
}

PairPlan swj_pair_plan(const swj_ctx *c, int precision)
{
    int v = tuned_variant(c, precision);
    return swj_pair_plan_variant(c, precision, v < 0 ? 0 : v);
}

int swj_pair_max_chunks(const swj_ctx *c)
{
    int P = 1;
    for (int prec = 0; prec < 3; ++prec)
        for (int v = 0; v < n_variants(prec); ++v) {
            PairPlan pl = swj_pair_plan_variant(c, prec, v);
            if (pl.P > P) P = pl.P;
        }
    return P;
}

static void launch_plan(swj_ctx *c, const PairPlan &pl, int precision, const int *act)
{
    dim3 grid(pl.tiles, pl.P, c->nb);
    SWJ_COUNT_LAUNCH();
    if (precision == SWJ_FP64)
        kVar64[pl.v].launch(grid, c->stream, c->T, c->S, pl.chunk, c->N, c->src64, &c->tgt64, c->partial,
                            act);
    else if (precision == SWJ_FF)
        kVarFF[pl.v].launch(grid, c->stream, c->T, c->S, pl.chunk, c->N, c->src64, &c->tgt64, c->partial,
                            act);
    else
        kVar32[pl.v].launch(grid, c->stream, c->T, c->S, pl.chunk, c->N, c->src32, &c->tgt32, c->partial,
                            act);
}

// One launch covers every instance (grid.z); each instance uses the chunking
// of the single-instance plan, so its result does not depend on the batch.
void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl, const int *act) { launch_plan(c, pl, SWJ_FP64, act); }
void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl, const int *act) { launch_plan(c, pl, SWJ_FP32, act); }
void swj_launch_pairs_ff(swj_ctx *c, const PairPlan &pl, const int *act) { launch_plan(c, pl, SWJ_FF, act); }

// Pick the context's plan for `precision`: the variant already tuned for this
// mesh size, else (FP32, autotune on, stream not capturing) time every variant on
// the current source/target records (one warm-up launch, then the mean of
// three) and keep the fastest for the whole process.
int swj_pair_autotune(swj_ctx *c, int precision, const int *act)
{
    int &done = swj_tuned_of(c, precision);
    if (done) return SWJ_OK;
    PairPlan &plan = swj_plan_of(c, precision);
    int v = tuned_variant(c, precision);
    // FP64 shapes differ by a few percent while timing them costs a dozen FP64
    // residuals: only the FP32 kernel is tuned, FP64 takes its default shape
    if (v < 0 && c->opts.autotune && precision == SWJ_FP32) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
            return SWJ_OK;   // untuned for now; tried again on a later residual
        cudaEvent_t e0, e1;
        SWJ_CUDA_TRY(cudaEventCreate(&e0));
        SWJ_CUDA_TRY(cudaEventCreate(&e1));
        float best = 0.f;
        int bv = 0;
        for (int k = 0; k < n_variants(precision); ++k) {
            PairPlan pl = swj_pair_plan_variant(c, precision, k);
            if ((size_t)pl.P * c->T * c->nb > c->partial_cap) continue;
            launch_plan(c, pl, precision, act);
            cudaEventRecord(e0, c->stream);
            for (int rep = 0; rep < 3; ++rep) launch_plan(c, pl, precision, act);
            cudaEventRecord(e1, c->stream);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return SWJ_ECUDA;
            }
            if (k == 0 || ms < best) { best = ms; bv = k; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto key = std::make_tuple(c->T, c->S, precision, c->num_sms);
        auto it = g_tuned.find(key);
        if (it == g_tuned.end()) g_tuned[key] = bv;   // first finished tuning wins
        else bv = it->second;
        v = bv;
    }
    if (v < 0) v = 0;
    plan = swj_pair_plan_variant(c, precision, v);
    done = 1;
    return SWJ_OK;
}

const char *swj_pair_variant_name(int precision, int v)
{
    if (!swj_valid_precision(precision) || v < 0 || v >= n_variants(precision)) return "";
    return variant(precision, v).name;
}

int swj_pair_variant_info(int precision, int v, int *tpb, int *R, int *packed)
{
    if (!swj_valid_precision(precision)) return SWJ_EINVAL;
    if (v < 0 || v >= n_variants(precision)) return SWJ_EINVAL;
    const PairVariant &pv = variant(precision, v);
    if (tpb) *tpb = pv.tpb;
    if (R) *R = pv.R;
    if (packed) *packed = (precision == SWJ_FP32 && v > 0) ? 1 : 0;
    return SWJ_OK;
}
