// Exact Jacobian-vector products J(u) v of the discrete residual E(u):
// forward-mode differentiation of every step of Section 3 along the
// direction v, the analytic alternative to the difference quotient of
// Eq. JvApprox.  No step size, no truncation error; the all-pairs part is
// computed in FP64 or in FP32 (Kahan-compensated per 64-source sub-tile,
// like the residual).
//
// With a dot for d/dt of a quantity along u + t v:
//   mesh step: the trapezoid rule and the spline are affine in u, so their
//     tangents are the same rules applied to v without the constants
//     (mesh.cu, swj_launch_mesh_tangent);
//   per target: E1' from the quotient rule on Eq. freeSurfCond; A' = 2 zx zx',
//     B' = 2 (zx' zy + zx zy'), C' = 2 zy zy'; I' from the closed form of
//     Eq. IS2 evaluated on dual numbers; the source term's derivative
//     -eps (zeta* + 1) zeta*' / r^3; E3'..E6' (linear rows) on v;
//   per pair (Eq. IntegroEqn kernels, Eq. S2), with e = dz dz':
//     (1/r)' = -e / r^3,  (1/r^3)' = -3 e / r^5,
//     K1' = n1' / r1^3 + n2' / r2^3 - 3 e (n1 / r1^5 + n2 / r2^5),
//     n' = dz' - dx zx' - dy zy' (dy' for the image),
//     K2' = -e (1 / r1^3 + 1 / r2^3),
//     S2' = -(Q1' / Q1^(3/2) + Q2' / Q2^(3/2)) / 2,  Q' = A' dx^2 +- B' dx dy + C' dy^2,
//     (w [f K1 + zx K2 - zx* S2])' = w [f' K1 + f K1' + zx' K2 + zx K2' - zx*' S2 - zx* S2'];
//   E2' = 2 pi g*' + src' - zx*' I - zx* I' - sum of the pair tangents.
#include "swj_internal.h"
#include <math.h>

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
// (value, derivative) with the rules of differentiation, for the closed form of I
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double k, Dual a) { return {k * a.v, k * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual dsqrt(Dual a)
{
    const double s = sqrt(a.v);
    return {s, 0.5 * a.d / s};
}
__device__ __forceinline__ Dual dasinh(Dual a) { return {asinh(a.v), a.d / sqrt(1.0 + a.v * a.v)}; }

// the corner function G(s, t) of the closed form (see closed_form.cuh) on
// dual A, B, C; s and t are geometry (constant)
__device__ Dual G_corner(Dual A, Dual B, Dual C, Dual sD, Dual rsA, Dual rsC, double s, double t)
{
    Dual v = {0.0, 0.0};
    if (s != 0.0) v = v + s * (rsC * dasinh((s * B + (2.0 * t) * C) / (fabs(s) * sD)));
    if (t != 0.0) v = v + t * (rsA * dasinh(((2.0 * s) * A + t * B) / (fabs(t) * sD)));
    return v;
}

__device__ Dual rect_int(Dual A, Dual B, Dual C, double s1, double s2, double t1, double t2)
{
    const Dual sD = dsqrt(4.0 * (A * C) - B * B);
    const Dual one = {1.0, 0.0};
    const Dual rsA = one / dsqrt(A), rsC = one / dsqrt(C);
    return G_corner(A, B, C, sD, rsA, rsC, s2, t2) - G_corner(A, B, C, sD, rsA, rsC, s1, t2) -
           G_corner(A, B, C, sD, rsA, rsC, s2, t1) + G_corner(A, B, C, sD, rsA, rsC, s1, t1);
}

// I of Eq. IS2 (direct + image part) and its derivative for target (k + 1/2, l)
__device__ Dual I_S2(Dual A, Dual B, Dual C, int N, int M, int k, int l, double dx, double dy)
{
    const double s1 = -((double)k + 0.5) * dx;
    const double s2 = ((double)(N - 1 - k) - 0.5) * dx;
    const double yt = (double)l * dy, yM = (double)(M - 1) * dy;
    return rect_int(A, B, C, s1, s2, -yt, yM - yt) + rect_int(A, -B, C, s1, s2, yt, yM + yt);
}

// ---------------------------------------------------------------- per target
// Thread per half-mesh target: the local rows of Jv (E1', E3'..E6'), the
// per-target part of E2', and the tangent target records.  Primal node arrays
// and target records come from the mesh step on u that precedes it.
__global__ void k_targets_tan(int N, int M, int H, double x1, double dx, double dy, const double *__restrict__ Fv,
                              const double *__restrict__ epsv, double nrad, int forcing, const double *__restrict__ u,
                              const double *__restrict__ v, const double *__restrict__ zeta,
                              const double *__restrict__ g, const double *__restrict__ zetay,
                              const double *__restrict__ gy, const double *__restrict__ dnode,
                              const double *__restrict__ Ival, double *__restrict__ Jv,
                              double *__restrict__ de2part, TgtArrays64 d64, TgtArrays32 d32,
                              const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int T = (N - 1) * M;
    if (t >= T) return;
    const int nb = gridDim.y;
    const size_t S = (size_t)N * M, NS = (size_t)nb * S;
    const double F = Fv[inst], eps = epsv[inst];
    const size_t on = (size_t)inst * S, ov = (size_t)inst * 2 * H, ot = (size_t)inst * T;
    u += ov; v += ov; Jv += ov;
    zeta += on; g += on; zetay += on; gy += on;
    const double *dz = dnode + on, *dg = dnode + NS + on, *dzy = dnode + 2 * NS + on, *dgy = dnode + 3 * NS + on;
    const int k = t % (N - 1), l = t / (N - 1);
    const size_t n0 = (size_t)l * N + k;
    const double *up = u + (size_t)l * (N + 1), *uz = u + H + (size_t)l * (N + 1);
    const double *vp = v + (size_t)l * (N + 1), *vz = v + H + (size_t)l * (N + 1);
    // primal half-mesh values (as in the residual's target step)
    const double zs = 0.5 * (zeta[n0] + zeta[n0 + 1]);
    const double zy = 0.5 * (zetay[n0] + zetay[n0 + 1]);
    const double py = 0.5 * (gy[n0] + gy[n0 + 1]);
    const double zx = 0.5 * (uz[1 + k] + uz[2 + k]);
    const double px = 0.5 * (up[1 + k] + up[2 + k]);
    // their tangents
    const double dzs = 0.5 * (dz[n0] + dz[n0 + 1]);
    const double dgs = 0.5 * (dg[n0] + dg[n0 + 1]);
    const double dzy_ = 0.5 * (dzy[n0] + dzy[n0 + 1]);
    const double dpy = 0.5 * (dgy[n0] + dgy[n0 + 1]);
    const double dzx = 0.5 * (vz[1 + k] + vz[2 + k]);
    const double dpx = 0.5 * (vp[1 + k] + vp[2 + k]);
    // E1' (quotient rule on 0.5 num / den + zeta* / F^2 - 0.5)
    const double zx2 = zx * zx, zy2 = zy * zy;
    const double num = (1.0 + zx2) * py * py + (1.0 + zy2) * px * px - 2.0 * zx * zy * px * py;
    const double dnum = 2.0 * zx * dzx * py * py + 2.0 * (1.0 + zx2) * py * dpy + 2.0 * zy * dzy_ * px * px +
                        2.0 * (1.0 + zy2) * px * dpx -
                        2.0 * (dzx * zy * px * py + zx * dzy_ * px * py + zx * zy * dpx * py + zx * zy * px * dpy);
    const double den = 1.0 + zx2 + zy2, dden = 2.0 * (zx * dzx + zy * dzy_);
    Jv[(size_t)l * (N + 1) + 2 + k] = 0.5 * (dnum * den - num * dden) / (den * den) + dzs / (F * F);
    // I' through the closed form on dual numbers
    const Dual A = {1.0 + zx2, 2.0 * zx * dzx};
    const Dual B = {2.0 * zx * zy, 2.0 * (dzx * zy + zx * dzy_)};
    const Dual C = {1.0 + zy2, 2.0 * zy * dzy_};
    const Dual I = I_S2(A, B, C, N, M, k, l, dx, dy);
    // source term eps / r, r^2 = x*^2 + y*^2 + (zeta* + 1)^2
    const double xt = x1 + ((double)k + 0.5) * dx, yt = (double)l * dy, zp1 = zs + 1.0;
    const double r2 = xt * xt + yt * yt + zp1 * zp1;
    // (the applied pressure of the pressure forcing does not depend on u)
    const double dsrc = (forcing == SWJ_FORCING_PRESSURE) ? 0.0 : -eps * zp1 * dzs / (r2 * sqrt(r2));
    de2part[ot + t] = 2.0 * kPi * dgs + dsrc - (dzx * Ival[ot + t] + zx * I.d);
    // tangent target records (units of L = dy, as the primal records)
    const size_t q = ot + t;
    d64.zeta[q] = dzs / dy; d64.g[q] = dgs; d64.zxw[q] = dzx * dy; d64.A[q] = A.d; d64.B[q] = B.d; d64.C[q] = C.d;
    d32.zeta[q] = (float)(dzs / dy); d32.g[q] = (float)dgs; d32.zxw[q] = (float)(dzx * dy);
    d32.A[q] = (float)A.d; d32.B[q] = (float)B.d; d32.C[q] = (float)C.d;
    if (k == 0) {
        // radiation rows: linear in u, so J v applies them to v without constants
        const double dphi1 = vp[0], dpxa = vp[1], dpxb = vp[2];
        const double dz1 = vz[0], dzxa = vz[1], dzxb = vz[2];
        Jv[(size_t)l * (N + 1)] = x1 * dpxa + nrad * dphi1;
        Jv[(size_t)l * (N + 1) + 1] = x1 * (dpxb - dpxa) / dx + nrad * dpxa;
        Jv[H + (size_t)l * (N + 1)] = x1 * dzxa + nrad * dz1;
        Jv[H + (size_t)l * (N + 1) + 1] = x1 * (dzxb - dzxa) / dx + nrad * dzxa;
    }
}

// Thread per mesh node: tangent source records (zeta'/L, zeta_x', zeta_y',
// g', L zeta_x'; x, y, w unused).
__global__ void k_sources_tan(int N, int M, int H, double dy, const double *__restrict__ v,
                              const double *__restrict__ dnode, SrcRec64 *__restrict__ t64,
                              SrcRec32 *__restrict__ t32, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t S = (size_t)N * M;
    if (s >= (int)S) return;
    const size_t NS = (size_t)gridDim.y * S, on = (size_t)inst * S;
    const int i = s % N, j = s / N;
    SrcRec64 r;
    r.x = 0.0; r.y = 0.0; r.w = 0.0;
    r.zeta = dnode[on + s] / dy;
    r.zx = v[(size_t)inst * 2 * H + H + (size_t)j * (N + 1) + 1 + i];
    r.zy = dnode[2 * NS + on + s];
    r.g = dnode[NS + on + s];
    r.zxw = r.zx * dy;
    t64[on + s] = r;
    SrcRec32 f;
    f.x = 0.f; f.y = 0.f; f.w = 0.f;
    f.zeta = (float)r.zeta; f.zx = (float)r.zx; f.zy = (float)r.zy; f.g = (float)r.g; f.zxw = (float)r.zxw;
    t32[on + s] = f;
}

// ---------------------------------------------------------------- all pairs
__device__ __forceinline__ float rsq(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename T> struct TanCfg;
template <> struct TanCfg<float> { static constexpr int tile = 256; static constexpr bool kahan = true; };
template <> struct TanCfg<double> { static constexpr int tile = 128; static constexpr bool kahan = false; };
constexpr int kTanSub = 64;   // sources per compensated sub-tile

// FP32 tangent pair sum on packed instructions: RP pairs of targets per
// thread (target 2m + h of the thread is tb + (2m + h) 128, in lane h of pair
// m), each formula of k_pairs_tan<float> as paired FFMA2/FMUL2/FADD2 with the
// source values broadcast to both lanes (negated copies where a formula
// subtracts them); the reciprocal square roots stay scalar.
struct __align__(16) TanX2 {
    float2 x, y, z, nzx, nzy, g, w, zxw, nzxw, dz, ndzx, ndzy, dg, dzxw;
};

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 rsq2(float2 v) { return make_float2(rsq(v.x), rsq(v.y)); }

template <int RP>
__global__ void __launch_bounds__(128)
k_pairs_tan_x2(int T_, int S_, int chunk, const SrcRecS<float> *__restrict__ src,
               const SrcRecS<float> *__restrict__ dsrc, TgtArraysS<float> tg, TgtArraysS<float> dtg,
               double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = 256;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        dsrc += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        dtg.zeta += ot; dtg.g += ot; dtg.zxw += ot; dtg.A += ot; dtg.B += ot; dtg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ TanX2 sh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk, s1 = min(S_, s0 + chunk);
    float2 ntx[RP], nty[RP], ty[RP], ntz[RP], ndtz[RP], ntg[RP], ndtg[RP], ntzw[RP], ndtzw[RP];
    float2 A[RP], B[RP], nB[RP], C[RP], dA[RP], dB[RP], ndB[RP], dC[RP], sum[RP], comp[RP];
    const int tb = blockIdx.x * 2 * RP * nth + tid;
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = min(tb + 2 * m * nth, T_ - 1), tc = min(tb + (2 * m + 1) * nth, T_ - 1);
        ntx[m] = make_float2(-tg.x[ta], -tg.x[tc]);
        ty[m] = make_float2(tg.y[ta], tg.y[tc]);
        nty[m] = make_float2(-tg.y[ta], -tg.y[tc]);
        ntz[m] = make_float2(-tg.zeta[ta], -tg.zeta[tc]);
        ndtz[m] = make_float2(-dtg.zeta[ta], -dtg.zeta[tc]);
        ntg[m] = make_float2(-tg.g[ta], -tg.g[tc]);
        ndtg[m] = make_float2(-dtg.g[ta], -dtg.g[tc]);
        ntzw[m] = make_float2(-tg.zxw[ta], -tg.zxw[tc]);
        ndtzw[m] = make_float2(-dtg.zxw[ta], -dtg.zxw[tc]);
        A[m] = make_float2(tg.A[ta], tg.A[tc]);
        B[m] = make_float2(tg.B[ta], tg.B[tc]);
        nB[m] = make_float2(-tg.B[ta], -tg.B[tc]);
        C[m] = make_float2(tg.C[ta], tg.C[tc]);
        dA[m] = make_float2(dtg.A[ta], dtg.A[tc]);
        dB[m] = make_float2(dtg.B[ta], dtg.B[tc]);
        ndB[m] = make_float2(-dtg.B[ta], -dtg.B[tc]);
        dC[m] = make_float2(dtg.C[ta], dtg.C[tc]);
        sum[m] = bc2(0.f);
        comp[m] = bc2(0.f);
    }
    const float2 m1 = bc2(-1.f), m3 = bc2(-3.f), mh = bc2(-0.5f);
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) {
            const SrcRecS<float> q = src[base + i], d = dsrc[base + i];
            TanX2 r;
            r.x = bc2(q.x); r.y = bc2(q.y); r.z = bc2(q.zeta); r.nzx = bc2(-q.zx); r.nzy = bc2(-q.zy);
            r.g = bc2(q.g); r.w = bc2(q.w); r.zxw = bc2(q.zxw); r.nzxw = bc2(-q.zxw);
            r.dz = bc2(d.zeta); r.ndzx = bc2(-d.zx); r.ndzy = bc2(-d.zy); r.dg = bc2(d.g); r.dzxw = bc2(d.zxw);
            sh[i] = r;
        }
        __syncthreads();
        for (int sb = 0; sb < nt; sb += kTanSub) {
            const int se = min(sb + kTanSub, nt);
            float2 loc[RP];
#pragma unroll
            for (int m = 0; m < RP; ++m) loc[m] = bc2(0.f);
            for (int s = sb; s < se; ++s) {
                const TanX2 q = sh[s];
#pragma unroll
                for (int m = 0; m < RP; ++m) {
                    const float2 p = __fadd2_rn(q.x, ntx[m]);
                    const float2 qq = __fadd2_rn(q.y, nty[m]), qp = __fadd2_rn(q.y, ty[m]);
                    const float2 dz = __fadd2_rn(q.z, ntz[m]), ddz = __fadd2_rn(q.dz, ndtz[m]);
                    const float2 p2 = __fmul2_rn(p, p);
                    const float2 bs = __ffma2_rn(dz, dz, p2);
                    const float2 r1s = __ffma2_rn(qq, qq, bs), r2s = __ffma2_rn(qp, qp, bs);
                    const float2 nc = __ffma2_rn(p, q.nzx, dz);
                    const float2 n1 = __ffma2_rn(qq, q.nzy, nc), n2 = __ffma2_rn(qp, q.nzy, nc);
                    const float2 dnc = __ffma2_rn(p, q.ndzx, ddz);
                    const float2 dn1 = __ffma2_rn(qq, q.ndzy, dnc), dn2 = __ffma2_rn(qp, q.ndzy, dnc);
                    const float2 i1 = rsq2(r1s), i2 = rsq2(r2s);
                    const float2 i1s = __fmul2_rn(i1, i1), i2s = __fmul2_rn(i2, i2);
                    const float2 i1c = __fmul2_rn(i1s, i1), i2c = __fmul2_rn(i2s, i2);
                    const float2 e = __fmul2_rn(dz, ddz);
                    const float2 a1 = __fmul2_rn(n1, i1c), a2 = __fmul2_rn(n2, i2c);
                    const float2 K1 = __fadd2_rn(a1, a2);
                    const float2 dK1 = __ffma2_rn(__fmul2_rn(m3, e), __ffma2_rn(a1, i1s, __fmul2_rn(a2, i2s)),
                                                  __ffma2_rn(dn1, i1c, __fmul2_rn(dn2, i2c)));
                    const float2 K2 = __fadd2_rn(i1, i2);
                    const float2 eK = __fmul2_rn(e, __fadd2_rn(i1c, i2c));   // -dK2
                    const float2 Ap2 = __fmul2_rn(A[m], p2), Bp = __fmul2_rn(B[m], p), nBp = __fmul2_rn(nB[m], p);
                    const float2 dAp2 = __fmul2_rn(dA[m], p2), dBp = __fmul2_rn(dB[m], p),
                                 ndBp = __fmul2_rn(ndB[m], p);
                    const float2 Q1 = __ffma2_rn(__ffma2_rn(C[m], qq, Bp), qq, Ap2);
                    const float2 Q2 = __ffma2_rn(__ffma2_rn(C[m], qp, nBp), qp, Ap2);
                    const float2 dQ1 = __ffma2_rn(__ffma2_rn(dC[m], qq, dBp), qq, dAp2);
                    const float2 dQ2 = __ffma2_rn(__ffma2_rn(dC[m], qp, ndBp), qp, dAp2);
                    const float2 j1 = rsq2(Q1), j2 = rsq2(Q2);
                    const float2 S2 = __fadd2_rn(j1, j2);
                    const float2 j1c = __fmul2_rn(__fmul2_rn(j1, j1), j1), j2c = __fmul2_rn(__fmul2_rn(j2, j2), j2);
                    const float2 dS2 = __fmul2_rn(mh, __ffma2_rn(j1c, dQ1, __fmul2_rn(j2c, dQ2)));
                    const float2 f = __fadd2_rn(q.g, ntg[m]), df = __fadd2_rn(q.dg, ndtg[m]);
                    float2 inner = __ffma2_rn(q.dzxw, K2, __fmul2_rn(q.nzxw, eK));
                    inner = __ffma2_rn(df, K1, inner);
                    inner = __ffma2_rn(f, dK1, inner);
                    inner = __ffma2_rn(ndtzw[m], S2, inner);
                    inner = __ffma2_rn(ntzw[m], dS2, inner);
                    loc[m] = __ffma2_rn(q.w, inner, loc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < RP; ++m) {
                const float2 y = __ffma2_rn(comp[m], m1, loc[m]);
                const float2 t2 = __fadd2_rn(sum[m], y);
                comp[m] = __ffma2_rn(y, m1, __ffma2_rn(sum[m], m1, t2));
                sum[m] = t2;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        const int ta = tb + 2 * m * nth, tc = tb + (2 * m + 1) * nth;
        if (ta < T_) partial[(size_t)blockIdx.y * T_ + ta] = (double)sum[m].x - (double)comp[m].x;
        if (tc < T_) partial[(size_t)blockIdx.y * T_ + tc] = (double)sum[m].y - (double)comp[m].y;
    }
}

// The sum over sources of the pair tangents above, per target and source
// chunk (grid: target tiles x chunks x instances; R targets per thread in
// registers, sources with their tangents through shared memory).
template <typename T, int R>
__global__ void __launch_bounds__(128)
k_pairs_tan(int T_, int S_, int chunk, const SrcRecS<T> *__restrict__ src, const SrcRecS<T> *__restrict__ dsrc,
            TgtArraysS<T> tg, TgtArraysS<T> dtg, double *__restrict__ partial, const int *__restrict__ act)
{
    constexpr int TILE = TanCfg<T>::tile;
    const int inst = blockIdx.z;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    {
        const size_t ot = (size_t)inst * T_;
        src += (size_t)inst * S_;
        dsrc += (size_t)inst * S_;
        tg.x += ot; tg.y += ot; tg.zeta += ot; tg.g += ot; tg.zxw += ot; tg.A += ot; tg.B += ot; tg.C += ot;
        dtg.zeta += ot; dtg.g += ot; dtg.zxw += ot; dtg.A += ot; dtg.B += ot; dtg.C += ot;
        partial += (size_t)inst * gridDim.y * T_;
    }
    __shared__ SrcRecS<T> sh[TILE], dsh[TILE];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int s0 = blockIdx.y * chunk, s1 = min(S_, s0 + chunk);
    T tx[R], ty[R], tz[R], tgv[R], tzw[R], A[R], B[R], C[R];
    T dtz[R], dtgv[R], dtzw[R], dA[R], dB[R], dC[R], sum[R], comp[R];
    const int tb = blockIdx.x * R * nth + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = min(tb + r * nth, T_ - 1);
        tx[r] = tg.x[t]; ty[r] = tg.y[t]; tz[r] = tg.zeta[t]; tgv[r] = tg.g[t];
        tzw[r] = tg.zxw[t]; A[r] = tg.A[t]; B[r] = tg.B[t]; C[r] = tg.C[t];
        dtz[r] = dtg.zeta[t]; dtgv[r] = dtg.g[t]; dtzw[r] = dtg.zxw[t];
        dA[r] = dtg.A[t]; dB[r] = dtg.B[t]; dC[r] = dtg.C[t];
        sum[r] = T(0); comp[r] = T(0);
    }
    for (int base = s0; base < s1; base += TILE) {
        const int nt = min(TILE, s1 - base);
        __syncthreads();
        for (int i = tid; i < nt; i += nth) {
            sh[i] = src[base + i];
            dsh[i] = dsrc[base + i];
        }
        __syncthreads();
        for (int sb = 0; sb < nt; sb += kTanSub) {
            const int se = min(sb + kTanSub, nt);
            T loc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) loc[r] = T(0);
            for (int s = sb; s < se; ++s) {
                const SrcRecS<T> q = sh[s];
                const SrcRecS<T> d = dsh[s];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T p = q.x - tx[r], qq = q.y - ty[r], qp = q.y + ty[r];
                    const T dz = q.zeta - tz[r], ddz = d.zeta - dtz[r];
                    const T p2 = p * p;
                    const T bs = fma(dz, dz, p2);
                    const T r1s = fma(qq, qq, bs), r2s = fma(qp, qp, bs);
                    const T nc = fma(-p, q.zx, dz);
                    const T n1 = fma(-qq, q.zy, nc), n2 = fma(-qp, q.zy, nc);
                    const T dnc = fma(-p, d.zx, ddz);
                    const T dn1 = fma(-qq, d.zy, dnc), dn2 = fma(-qp, d.zy, dnc);
                    const T i1 = rsq(r1s), i2 = rsq(r2s);
                    const T i1s = i1 * i1, i2s = i2 * i2;
                    const T i1c = i1s * i1, i2c = i2s * i2;
                    const T e = dz * ddz;
                    const T a1 = n1 * i1c, a2 = n2 * i2c;
                    const T K1 = a1 + a2;
                    const T dK1 = fma(dn1, i1c, dn2 * i2c) - T(3) * e * fma(a1, i1s, a2 * i2s);
                    const T K2 = i1 + i2;
                    const T dK2 = -e * (i1c + i2c);
                    const T Ap2 = A[r] * p2, Bp = B[r] * p;
                    const T dAp2 = dA[r] * p2, dBp = dB[r] * p;
                    const T Q1 = fma(fma(C[r], qq, Bp), qq, Ap2), Q2 = fma(fma(C[r], qp, -Bp), qp, Ap2);
                    const T dQ1 = fma(fma(dC[r], qq, dBp), qq, dAp2), dQ2 = fma(fma(dC[r], qp, -dBp), qp, dAp2);
                    const T j1 = rsq(Q1), j2 = rsq(Q2);
                    const T S2 = j1 + j2;
                    const T dS2 = T(-0.5) * fma(j1 * j1 * j1, dQ1, j2 * j2 * j2 * dQ2);
                    const T f = q.g - tgv[r], df = d.g - dtgv[r];
                    T inner = fma(d.zxw, K2, q.zxw * dK2);
                    inner = fma(df, K1, inner);
                    inner = fma(f, dK1, inner);
                    inner = fma(-dtzw[r], S2, inner);
                    inner = fma(-tzw[r], dS2, inner);
                    loc[r] = fma(q.w, inner, loc[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (TanCfg<T>::kahan) {
                    const T y = loc[r] - comp[r];
                    const T t2 = sum[r] + y;
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
        const int t = tb + r * nth;
        if (t < T_) partial[(size_t)blockIdx.y * T_ + t] = (double)sum[r] - (double)comp[r];
    }
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

int swj_jvp_exact_impl(swj_ctx *c, const double *u, const double *v, double *Jv, int precision,
                       const int *act)
{
    if (precision != SWJ_FP64 && precision != SWJ_FP32) return SWJ_EINVAL;
    const swj_mesh &m = c->mesh;
    cudaStream_t st = c->stream;
    const int nb = c->nb;
    // primal mesh step at u (node arrays, records, I); its E rows go to scratch
    swj_launch_mesh_step(c, u, c->E_tmp, act);
    swj_launch_mesh_tangent(c, v, act);
    SWJ_COUNT_LAUNCH();
    k_targets_tan<<<dim3(nblk(c->T, kFp64Block), nb), kFp64Block, 0, st>>>(
        c->N, c->M, c->H, m.x1, m.dx, m.dy, c->Fd, c->epsd, m.n_rad, c->opts.forcing, u, v, c->zeta, c->g,
        c->zetay, c->gy,
        c->dnode, c->Ival, Jv, c->de2part, c->ttgt64, c->ttgt32, act);
    SWJ_COUNT_LAUNCH();
    k_sources_tan<<<dim3(nblk(c->S, 256), nb), 256, 0, st>>>(c->N, c->M, c->H, m.dy, v, c->dnode, c->tsrc64,
                                                             c->tsrc32, act);
    // the launch geometry of the scalar residual kernel of the same precision
    // (128 threads; 2 FP64 or 4 FP32 targets per thread)
    const PairPlan pl = swj_pair_plan_variant(c, precision, precision == SWJ_FP64 ? 2 : 0);
    const dim3 grid(pl.tiles, pl.P, nb);
    SWJ_COUNT_LAUNCH();
    if (precision == SWJ_FP64) {
        if (pl.R != 2 || pl.tpb != 128) return SWJ_EINVAL;
        k_pairs_tan<double, 2><<<grid, 128, 0, st>>>(c->T, c->S, pl.chunk, c->src64, c->tsrc64, c->tgt64,
                                                      c->ttgt64, c->partial, act);
    } else {
        if (pl.R != 4 || pl.tpb != 128) return SWJ_EINVAL;
        k_pairs_tan_x2<2><<<grid, 128, 0, st>>>(c->T, c->S, pl.chunk, c->src32, c->tsrc32, c->tgt32,
                                                 c->ttgt32, c->partial, act);
    }
    swj_launch_assemble(c, Jv, pl.P, act, c->de2part);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}
