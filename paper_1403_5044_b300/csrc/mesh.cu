// Mesh step of the residual E(u), all in FP64 (Section 3):
//   * zeta and g = phi - x along x by the trapezoidal rule (Eq. zetaapprox),
//     as a warp-wide prefix sum per mesh row;
//   * zeta_y and g_y (= phi_y) at the nodes from the cubic spline along y,
//     clamped (zero slope) at y1 = 0 and not-a-knot at y_M, one Thomas sweep
//     per mesh column;
//   * half-mesh values, the free-surface rows E1 (Eq. freeSurfCond), the
//     radiation rows E3..E6 (Eq. numUpRadiation), and the per-target part of
//     E2 that needs no pair sum: 2 pi g* + eps / r_source - zeta_x* I, with I
//     the closed-form integral of S2 over the mesh rectangle (Eq. IS2);
//   * the source and target records read by the all-pairs kernels;
//   * assembly of E2 = (that part) - (all-pairs sum) in Appendix A order.
#include "swj_internal.h"
#include "closed_form.cuh"
#include <math.h>
#include <cuda_pipeline.h>

namespace {

constexpr double kPi = 3.14159265358979323846;

// Warp per mesh row.  Rows 0..M-1 integrate phi_x - 1 from g_1 = phi_1 - x1
// (so the result is g = phi - x exactly as the trapezoidal rule integrates
// the constant 1 exactly); rows M..2M-1 integrate zeta_x from zeta_1.  With
// `tangent` the input is a direction v and the rule is applied without the
// constants (the derivative of the map, which is affine in u).
__global__ void k_integrate(int N, int M, int H, double x1, double dx,
                            const double *__restrict__ u, double *__restrict__ zeta,
                            double *__restrict__ g, const int *__restrict__ act, bool tangent = false)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    u += (size_t)inst * 2 * H;
    zeta += (size_t)inst * N * M;
    g += (size_t)inst * N * M;
    int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (warp >= 2 * M) return;
    bool isz = warp >= M;
    int l = isz ? warp - M : warp;
    const double *row = u + (isz ? H : 0) + (size_t)l * (N + 1);
    double *out = (isz ? zeta : g) + (size_t)l * N;
    double shift = (isz || tangent) ? 0.0 : 1.0;
    double f1 = (isz || tangent) ? row[0] : row[0] - x1;
    double hdx = 0.5 * dx;
    int per = (N + 31) / 32;
    int k0 = lane * per, k1 = min(k0 + per, N);
    // increment from node k to node k+1 (0-based, k <= N-2)
    auto inc = [&](int k) { return hdx * ((row[1 + k] - shift) + (row[2 + k] - shift)); };
    double run = 0.0;
    for (int k = k0; k < k1; ++k)
        if (k <= N - 2) run += inc(k);
    double incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    double v = f1 + (incl - run);
    for (int k = k0; k < k1; ++k) {
        out[k] = v;
        if (k <= N - 2) v += inc(k);
    }
}

// Slopes m_j of the cubic spline through f_0..f_{M-1} along y (uniform
// spacing h), for every mesh column (columns 0..N-1: zeta, N..2N-1: g):
//   m_0 = 0                                          (even extension at y = 0)
//   m_{j-1} + 4 m_j + m_{j+1} = 3 (f_{j+1} - f_{j-1}) / h     (C2 continuity)
//   2 m_{M-2} + m_{M-1} = (d_{M-3} + 5 d_{M-2}) / 2,  d_j = (f_{j+1} - f_j)/h
// (the last row is the not-a-knot condition at y_{M-2} with m_{M-3}
// eliminated through the row above it).  cp, a, inv are the forward-sweep
// coefficients of this fixed matrix (Thomas algorithm).
//
// 32 columns per block, a column per lane of each of its four warps.  The
// warps first copy the columns into shared memory (all M rows in flight at
// once) and form the right-hand sides d_j of every row there, rows dealt over
// the four warps: B300 issues FP64 at 0.5 lanes per clock per SM
// sub-partition, so this off-chain work spreads over four sub-partitions.
// Warp 0 then runs the forward sweep (the chain of M dependent steps, now
// only its own two FP64 operations per step; m'_j overwrites d_j) and the
// backward sweep, writing each slope to global memory as it is found
// (coalesced across the warp).  The operations per value are those of the
// one-warp form, so the slopes are the same bit for bit.
constexpr int kSplineCols = 32, kSplineWarps = 4;

__global__ void __launch_bounds__(kSplineCols * kSplineWarps)
k_spline(int N, int M, double hy, const double *__restrict__ cp,
         const double *__restrict__ a, const double *__restrict__ inv,
         const double *__restrict__ zeta, const double *__restrict__ g,
         double *__restrict__ zetay, double *__restrict__ gy,
         const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const size_t off = (size_t)inst * N * M;
    zeta += off; g += off; zetay += off; gy += off;
    extern __shared__ double sp[];
    const int lane = threadIdx.x & (kSplineCols - 1), w = threadIdx.x / kSplineCols;
    const int t = blockIdx.x * kSplineCols + lane;
    const bool live = t < 2 * N;
    const int k = live ? t % N : 0;
    const double *f = (t < N ? zeta : g) + k;
    double *F = sp + lane;                      // f_j of this column at F[j * kSplineCols]
    double *D = sp + (size_t)M * kSplineCols + lane;   // d_j, then m'_j
    if (live)
        for (int j = w; j < M; j += kSplineWarps) __pipeline_memcpy_async(F + j * kSplineCols, f + (size_t)j * N, 8);
    __pipeline_commit();
    __pipeline_wait_prior(0);
    __syncthreads();
    const double rh = 1.0 / hy;
    if (live) {
        for (int j = 1 + w; j < M; j += kSplineWarps) {
            double d;
            if (j < M - 1) {
                d = 3.0 * (F[(j + 1) * kSplineCols] - F[(j - 1) * kSplineCols]) * rh;
            } else {
                const double d3 = (F[(M - 2) * kSplineCols] - F[(M - 3) * kSplineCols]) * rh;
                const double d2 = (F[(M - 1) * kSplineCols] - F[(M - 2) * kSplineCols]) * rh;
                d = 0.5 * (d3 + 5.0 * d2);
            }
            D[j * kSplineCols] = d;
        }
    }
    __syncthreads();
    if (w != 0 || !live) return;
    double *m = (t < N ? zetay : gy) + k;
    double dp = 0.0;
    for (int j = 1; j < M; ++j) {
        dp = (D[j * kSplineCols] - __ldg(a + j) * dp) * __ldg(inv + j);
        D[j * kSplineCols] = dp;
    }
    double next = dp;
    m[(size_t)(M - 1) * N] = next;
    for (int j = M - 2; j >= 1; --j) {
        next = D[j * kSplineCols] - __ldg(cp + j) * next;
        m[(size_t)j * N] = next;
    }
    m[0] = 0.0;
}

// The same slopes, thread per column straight from global memory: for meshes
// whose columns do not fit in shared memory.
__global__ void k_spline_global(int N, int M, double hy, const double *__restrict__ cp,
                                const double *__restrict__ a, const double *__restrict__ inv,
                                const double *__restrict__ zeta, const double *__restrict__ g,
                                double *__restrict__ zetay, double *__restrict__ gy,
                                const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const size_t off = (size_t)inst * N * M;
    zeta += off; g += off; zetay += off; gy += off;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * N) return;
    int k = t % N;
    const double *f = (t < N ? zeta : g) + k;
    double *m = (t < N ? zetay : gy) + k;
    double rh = 1.0 / hy;
    double dp = 0.0;
    m[0] = 0.0;
    for (int j = 1; j < M; ++j) {
        double d;
        if (j < M - 1) {
            d = 3.0 * (f[(size_t)(j + 1) * N] - f[(size_t)(j - 1) * N]) * rh;
        } else {
            double d3 = (f[(size_t)(M - 2) * N] - f[(size_t)(M - 3) * N]) * rh;
            double d2 = (f[(size_t)(M - 1) * N] - f[(size_t)(M - 2) * N]) * rh;
            d = 0.5 * (d3 + 5.0 * d2);
        }
        dp = (d - a[j] * dp) * inv[j];
        m[(size_t)j * N] = dp;
    }
    double next = m[(size_t)(M - 1) * N];
    for (int j = M - 2; j >= 1; --j) {
        next = m[(size_t)j * N] - cp[j] * next;
        m[(size_t)j * N] = next;
    }
}

// Thread per half-mesh target t = l (N-1) + k.
// Applied surface pressure of the pressure forcing: exp(2 + 1/(x^2-1) + 1/(y^2-1))
// on |x|, |y| < 1, else 0 (1 at the centre; smooth, compact support).
__device__ __forceinline__ double surface_pressure(double x, double y)
{
    if (!(fabs(x) < 1.0 && fabs(y) < 1.0)) return 0.0;
    return exp(2.0 + 1.0 / (x * x - 1.0) + 1.0 / (y * y - 1.0));
}

__global__ void k_targets(int N, int M, int H, double x1, double dx, double dy,
                          const double *__restrict__ Fv, const double *__restrict__ epsv,
                          double nrad, int forcing, const double *__restrict__ u,
                          const double *__restrict__ zeta, const double *__restrict__ g,
                          const double *__restrict__ zetay, const double *__restrict__ gy,
                          double *__restrict__ E, double *__restrict__ e2part,
                          double *__restrict__ Ival, TgtArrays64 t64, TgtArrays32 t32,
                          const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int T = (N - 1) * M;
    if (t >= T) return;
    const double F = Fv[inst], eps = epsv[inst];
    {
        const size_t on = (size_t)inst * N * M, ov = (size_t)inst * 2 * H, ot = (size_t)inst * T;
        u += ov; E += ov; zeta += on; g += on; zetay += on; gy += on; e2part += ot; Ival += ot;
        t64.x += ot; t64.y += ot; t64.zeta += ot; t64.g += ot; t64.zxw += ot; t64.A += ot; t64.B += ot; t64.C += ot;
        t32.x += ot; t32.y += ot; t32.zeta += ot; t32.g += ot; t32.zxw += ot; t32.A += ot; t32.B += ot; t32.C += ot;
    }
    int k = t % (N - 1), l = t / (N - 1);
    size_t n0 = (size_t)l * N + k;
    const double *urow_p = u + (size_t)l * (N + 1);
    const double *urow_z = u + H + (size_t)l * (N + 1);
    double zs = 0.5 * (zeta[n0] + zeta[n0 + 1]);
    double gs = 0.5 * (g[n0] + g[n0 + 1]);
    double zy = 0.5 * (zetay[n0] + zetay[n0 + 1]);
    double py = 0.5 * (gy[n0] + gy[n0 + 1]);
    double zx = 0.5 * (urow_z[1 + k] + urow_z[2 + k]);
    double px = 0.5 * (urow_p[1 + k] + urow_p[2 + k]);
    // E1: free-surface condition at the half-mesh point
    double zx2 = zx * zx, zy2 = zy * zy;
    double num = (1.0 + zx2) * py * py + (1.0 + zy2) * px * px - 2.0 * zx * zy * px * py;
    double E1 = 0.5 * num / (1.0 + zx2 + zy2) + zs / (F * F) - 0.5;
    // I: closed-form integral of S2 over [x1, xN] x [0, yM], direct + image
    double A = 1.0 + zx2, B = 2.0 * zx * zy, C = 1.0 + zy2;
    double xt = x1 + ((double)k + 0.5) * dx;
    double yt = (double)l * dy;
    double I = swj_I_S2(A, B, C, N, M, k, l, dx, dy);
    double zp1 = zs + 1.0;
    double src = 0.0;
    if (forcing == SWJ_FORCING_PRESSURE) E1 += eps * surface_pressure(xt, yt);
    else src = eps / sqrt(xt * xt + yt * yt + zp1 * zp1);
    e2part[t] = 2.0 * kPi * gs + src - zx * I;
    Ival[t] = I;
    E[(size_t)l * (N + 1) + 2 + k] = E1;
    // records of the pair kernels (units of L = dy, see SrcRecS)
    const double xs = ((double)k + 0.5) * (dx / dy);
    t64.x[t] = xs; t64.y[t] = (double)l; t64.zeta[t] = zs / dy; t64.g[t] = gs; t64.zxw[t] = zx * dy;
    t64.A[t] = A; t64.B[t] = B; t64.C[t] = C;
    t32.x[t] = (float)xs; t32.y[t] = (float)l; t32.zeta[t] = (float)(zs / dy); t32.g[t] = (float)gs;
    t32.zxw[t] = (float)(zx * dy); t32.A[t] = (float)A; t32.B[t] = (float)B; t32.C[t] = (float)C;
    if (k == 0) {
        // radiation rows at x = x1 (forward difference for the second derivative)
        double phi1 = urow_p[0], pxa = urow_p[1], pxb = urow_p[2];
        double z1 = urow_z[0], zxa = urow_z[1], zxb = urow_z[2];
        E[(size_t)l * (N + 1)] = x1 * (pxa - 1.0) + nrad * (phi1 - x1);
        E[(size_t)l * (N + 1) + 1] = x1 * (pxb - pxa) / dx + nrad * (pxa - 1.0);
        E[H + (size_t)l * (N + 1)] = x1 * zxa + nrad * z1;
        E[H + (size_t)l * (N + 1) + 1] = x1 * (zxb - zxa) / dx + nrad * zxa;
    }
}

// Thread per mesh node s = j N + i.
__global__ void k_sources(int N, int M, int H, double dx, double dy, const double *__restrict__ u,
                          const double *__restrict__ zeta, const double *__restrict__ g,
                          const double *__restrict__ zetay, SrcRec64 *__restrict__ s64,
                          SrcRec32 *__restrict__ s32, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N * M) return;
    {
        const size_t on = (size_t)inst * N * M;
        u += (size_t)inst * 2 * H; zeta += on; g += on; zetay += on; s64 += on; s32 += on;
    }
    int i = s % N, j = s / N;
    double ci = (i == 0 || i == N - 1) ? 0.5 : 1.0;
    double cj = (j == 0 || j == M - 1) ? 0.5 : 1.0;
    SrcRec64 r;
    r.x = (double)i * (dx / dy);
    r.y = (double)j;
    r.zeta = zeta[s] / dy;
    r.zx = u[H + (size_t)j * (N + 1) + 1 + i];
    r.zy = zetay[s];
    r.g = g[s];
    r.w = (dx / dy) * ci * cj;
    r.zxw = r.zx * dy;
    s64[s] = r;
    SrcRec32 q;
    q.x = (float)r.x; q.y = (float)j; q.zeta = (float)r.zeta; q.zx = (float)r.zx;
    q.zy = (float)r.zy; q.g = (float)r.g; q.w = (float)r.w; q.zxw = (float)r.zxw;
    s32[s] = q;
}

// Thread per target: E2 = (2 pi g* + src - zx* I) - sum over source chunks.
__global__ void k_assemble(int N, int M, int H, int P, const double *__restrict__ partial,
                           const double *__restrict__ e2part, double *__restrict__ E,
                           const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int T = (N - 1) * M;
    if (t >= T) return;
    partial += (size_t)inst * P * T;
    e2part += (size_t)inst * T;
    E += (size_t)inst * 2 * H;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += partial[(size_t)p * T + t];
    int k = t % (N - 1), l = t / (N - 1);
    E[H + (size_t)l * (N + 1) + 2 + k] = e2part[t] - s;
}

__global__ void k_flat(int N, int M, int H, double x1, double *__restrict__ u)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * H) return;
    u += (size_t)blockIdx.y * 2 * H;
    int r = i % (N + 1);
    double v;
    if (i < H) v = (r == 0) ? x1 : 1.0;
    else v = 0.0;
    u[i] = v;
}

__global__ void k_unpack(int N, int M, double x1, double dx, const double *__restrict__ zeta,
                         const double *__restrict__ g, double *__restrict__ zo,
                         double *__restrict__ po)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N * M) return;
    const size_t on = (size_t)blockIdx.y * N * M;
    zeta += on; g += on;
    if (zo) zo += on;
    if (po) po += on;
    int i = s % N;
    if (zo) zo[s] = zeta[s];
    if (po) po[s] = g[s] + (x1 + (double)i * dx);
}

__global__ void k_surface(int N, int M, double dy, const double *zeta, const double *g,
                          const double *zetay, const double *gy, TgtArrays64 t64,
                          const double *Ival, double *out)
{
    int S = N * M, T = (N - 1) * M;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S) {
        out[i] = zeta[i];
        out[S + i] = g[i];
        out[2 * S + i] = zetay[i];
        out[3 * S + i] = gy[i];
    }
    if (i < T) {
        double *o = out + 4 * (size_t)S;
        o[i] = t64.zeta[i] * dy;
        o[T + i] = t64.g[i];
        o[2 * T + i] = t64.zxw[i] / dy;
        int k = i % (N - 1), l = i / (N - 1);
        size_t n0 = (size_t)l * N + k;
        o[3 * T + i] = 0.5 * (zetay[n0] + zetay[n0 + 1]);
        o[4 * T + i] = Ival[i];
    }
}

// Mesh bootstrapping: thread per unknown slot (l, k), k = 0..Nd, of the
// destination mesh; bilinear interpolation of the source's node fields
// (coordinates clamped to the source mesh).  k = 0: phi_1 = g(x1, y) + x1 and
// zeta_1 = zeta(x1, y); k >= 1: phi_x and zeta_x at node k - 1.
__global__ void k_resample(int Ns, int Ms, int Hs, double x1s, double dxs, double dys,
                           const double *__restrict__ zeta_s, const double *__restrict__ g_s,
                           const double *__restrict__ u_s, int Nd, int Md, int Hd, double x1d, double dxd,
                           double dyd, double *__restrict__ u_d)
{
    const int inst = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Hd) return;
    zeta_s += (size_t)inst * Ns * Ms;
    g_s += (size_t)inst * Ns * Ms;
    u_s += (size_t)inst * 2 * Hs;
    u_d += (size_t)inst * 2 * Hd;
    const int l = e / (Nd + 1), k = e % (Nd + 1);
    const double x = (k == 0) ? x1d : x1d + (double)(k - 1) * dxd;
    const double y = (double)l * dyd;
    const double fi = fmin(fmax((x - x1s) / dxs, 0.0), (double)(Ns - 1));
    const double fj = fmin(fmax(y / dys, 0.0), (double)(Ms - 1));
    const int i0 = min((int)floor(fi), Ns - 2), j0 = min((int)floor(fj), Ms - 2);
    const double a = fi - i0, b = fj - j0;
    const double w00 = (1.0 - a) * (1.0 - b), w01 = a * (1.0 - b), w10 = (1.0 - a) * b, w11 = a * b;
    if (k == 0) {
        auto bil = [&](const double *f) {
            const double *r0 = f + (size_t)j0 * Ns + i0, *r1 = r0 + Ns;
            return w00 * r0[0] + w01 * r0[1] + w10 * r1[0] + w11 * r1[1];
        };
        u_d[e] = bil(g_s) + x1d;
        u_d[Hd + e] = bil(zeta_s);
    } else {
        // node field f[j][i] = u_s[base + j (Ns + 1) + 1 + i]
        auto bil = [&](const double *base) {
            const double *r0 = base + (size_t)j0 * (Ns + 1) + 1 + i0, *r1 = r0 + (Ns + 1);
            return w00 * r0[0] + w01 * r0[1] + w10 * r1[0] + w11 * r1[1];
        };
        u_d[e] = bil(u_s);
        u_d[Hd + e] = bil(u_s + Hs);
    }
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

// Shared memory of k_spline: two arrays of M rows of kSplineCols columns.  Up
// to 160 KB (M <= 320) it runs; above, k_spline_global does.
constexpr size_t kSplineSmemMax = 160 * 1024;

void launch_spline(swj_ctx *c, cudaStream_t st, const double *f1, const double *f2, double *m1, double *m2,
                   const int *act)
{
    const size_t smem = 2 * (size_t)c->M * kSplineCols * sizeof(double);
    if (smem <= kSplineSmemMax) {
        static const bool attr = cudaFuncSetAttribute(k_spline, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)kSplineSmemMax) == cudaSuccess;
        (void)attr;
        k_spline<<<dim3(nblk(2L * c->N, kSplineCols), c->nb), kSplineCols * kSplineWarps, smem, st>>>(
            c->N, c->M, c->mesh.dy, c->spl_cp, c->spl_a, c->spl_inv, f1, f2, m1, m2, act);
    } else {
        k_spline_global<<<dim3(nblk(2L * c->N, 128), c->nb), 128, 0, st>>>(
            c->N, c->M, c->mesh.dy, c->spl_cp, c->spl_a, c->spl_inv, f1, f2, m1, m2, act);
    }
}

}  // namespace

void swj_spline_coeffs(int M, double *cp, double *a, double *inv)
{
    // tridiagonal matrix of k_spline: row 0 (1 | 0), rows 1..M-2 (1 4 1), row M-1 (2 1 | -)
    cp[0] = 0.0; a[0] = 0.0; inv[0] = 1.0;
    for (int j = 1; j < M; ++j) {
        double aj = (j < M - 1) ? 1.0 : 2.0;
        double bj = (j < M - 1) ? 4.0 : 1.0;
        double cj = (j < M - 1) ? 1.0 : 0.0;
        double den = bj - aj * cp[j - 1];
        a[j] = aj;
        inv[j] = 1.0 / den;
        cp[j] = cj / den;
    }
}

void swj_launch_mesh_step(swj_ctx *c, const double *u, double *E, const int *act)
{
    const swj_mesh &m = c->mesh;
    cudaStream_t st = c->stream;
    const int nb = c->nb;
    SWJ_COUNT_LAUNCH();
    k_integrate<<<dim3(nblk(2L * c->M * 32, kFp64Block), nb), kFp64Block, 0, st>>>(c->N, c->M, c->H, m.x1, m.dx, u,
                                                                     c->zeta, c->g, act);
    SWJ_COUNT_LAUNCH();
    launch_spline(c, st, c->zeta, c->g, c->zetay, c->gy, act);
    SWJ_COUNT_LAUNCH();
    k_targets<<<dim3(nblk(c->T, kFp64Block), nb), kFp64Block, 0, st>>>(c->N, c->M, c->H, m.x1, m.dx, m.dy, c->Fd,
                                                          c->epsd, m.n_rad, c->opts.forcing, u, c->zeta, c->g,
                                                          c->zetay, c->gy, E, c->e2part, c->Ival,
                                                          c->tgt64, c->tgt32, act);
    SWJ_COUNT_LAUNCH();
    k_sources<<<dim3(nblk(c->S, 256), nb), 256, 0, st>>>(c->N, c->M, c->H, m.dx, m.dy, u, c->zeta,
                                                         c->g, c->zetay, c->src64, c->src32, act);
}

void swj_launch_assemble(swj_ctx *c, double *E, int P, const int *act, const double *e2part)
{
    SWJ_COUNT_LAUNCH();
    k_assemble<<<dim3(nblk(c->T, kFp64Block), c->nb), kFp64Block, 0, c->stream>>>(c->N, c->M, c->H, P, c->partial,
                                                                     e2part ? e2part : c->e2part, E, act);
}

// Tangent of the trapezoid and spline steps for a direction v: zeta', g',
// zeta_y', g_y' into c->dnode ([4][nb][S]).
void swj_launch_mesh_tangent(swj_ctx *c, const double *v, const int *act)
{
    const swj_mesh &m = c->mesh;
    cudaStream_t st = c->stream;
    const size_t NS = (size_t)c->nb * c->S;
    double *dz = c->dnode, *dg = dz + NS, *dzy = dg + NS, *dgy = dzy + NS;
    SWJ_COUNT_LAUNCH();
    k_integrate<<<dim3(nblk(2L * c->M * 32, kFp64Block), c->nb), kFp64Block, 0, st>>>(c->N, c->M, c->H, m.x1, m.dx, v, dz,
                                                                        dg, act, true);
    SWJ_COUNT_LAUNCH();
    launch_spline(c, st, dz, dg, dzy, dgy, act);
}

void swj_launch_flat(swj_ctx *c, double *u)
{
    SWJ_COUNT_LAUNCH();
    k_flat<<<dim3(nblk(c->nu, 256), c->nb), 256, 0, c->stream>>>(c->N, c->M, c->H, c->mesh.x1, u);
}

void swj_launch_unpack(swj_ctx *c, const double *u, double *zo, double *po)
{
    const swj_mesh &m = c->mesh;
    SWJ_COUNT_LAUNCH();
    k_integrate<<<dim3(nblk(2L * c->M * 32, kFp64Block), c->nb), kFp64Block, 0, c->stream>>>(
        c->N, c->M, c->H, m.x1, m.dx, u, c->zeta, c->g, nullptr);
    SWJ_COUNT_LAUNCH();
    k_unpack<<<dim3(nblk(c->S, 256), c->nb), 256, 0, c->stream>>>(c->N, c->M, m.x1, m.dx, c->zeta,
                                                                  c->g, zo, po);
}

void swj_launch_surface(swj_ctx *c, double *out)
{
    int n = c->S > c->T ? c->S : c->T;
    SWJ_COUNT_LAUNCH();
    k_surface<<<nblk(n, 256), 256, 0, c->stream>>>(c->N, c->M, c->mesh.dy, c->zeta, c->g, c->zetay,
                                                    c->gy, c->tgt64, c->Ival, out);
}

// u_dst (on dst's mesh) from u_src (on src's mesh), instance by instance, on
// dst's stream; src's node arrays serve as scratch (src must be idle).
void swj_launch_resample(swj_ctx *src, const double *u_src, swj_ctx *dst, double *u_dst)
{
    const swj_mesh &ms = src->mesh, &md = dst->mesh;
    cudaStream_t st = dst->stream;
    SWJ_COUNT_LAUNCH();
    k_integrate<<<dim3(nblk(2L * src->M * 32, kFp64Block), src->nb), kFp64Block, 0, st>>>(src->N, src->M, src->H, ms.x1, ms.dx,
                                                                            u_src, src->zeta, src->g, nullptr);
    SWJ_COUNT_LAUNCH();
    k_resample<<<dim3(nblk(dst->H, 256), dst->nb), 256, 0, st>>>(src->N, src->M, src->H, ms.x1, ms.dx, ms.dy,
                                                                  src->zeta, src->g, u_src, dst->N, dst->M,
                                                                  dst->H, md.x1, md.dx, md.dy, u_dst);
}
