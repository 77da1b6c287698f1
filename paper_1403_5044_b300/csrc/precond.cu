// Preconditioner of Section 4.2 / Appendices B-C.
//
// P is the Jacobian of the linearised discrete system (the eps -> 0 problem
// of Section 2.3 discretised as in Section 3), in Appendix A order:
//
//   P = [ A  B ]   rows  (E3, E4, E1) per y-row      columns (phi_1, phi_x) per y-row
//       [ C  D ]         (E5, E6, E2) per y-row              (zeta_1, zeta_x) per y-row
//
// A, B, C are block diagonal with one repeated (N+1) x (N+1) block
// (Eqs. PreA, PreB, PreC plus the radiation rows); D is dense (Eq. PreD) and
// is truncated to |l - m| <= h = (b - 1)/2 blocks.  The entries of B and C
// are written from the trapezoidal rule itself: d zeta*_k / d (zeta_x)_n =
// dx/2 (c_k(n) + c_{k+1}(n)) with c_m(n) the trapezoid coefficient of
// (zeta_x)_n in zeta_m (Eq. zetaapprox), which reproduces the case lists of
// PreB/PreC.  The diagonal correction of PreD needs, per target, the
// trapezoid sum of w K3 over all sources and I of the flat surface.
//
// Factorisation (Appendix C): S = D - C A^-1 B differs from D only in its
// diagonal blocks, by the one block G = C A^-1 B.  S is factored by a block
// LU that keeps the block band (no fill outside it), with partial pivoting
// inside each diagonal block.  Step i inverts the updated pivot block
// (inv_i), forms W_ik = inv_i S_ik for the blocks right of it, updates
// S_jk -= S_ji W_ik below it and replaces the blocks left of the diagonal by
// L_ij = inv_i S_ij, so the solve is
//   forward   z_i = inv_i t_i - sum_{j<i} L_ij z_j
//   backward  x_i = z_i - sum_{k>i} W_ik x_k.
// Everything is FP64.
//
// Elimination order.  Top-down, the M steps form a chain (each diagonal block
// waits for the update from the step before).  A one-instance context
// instead eliminates the top mt block rows downwards and the bottom mb rows
// upwards at the same time (mt + mb = M - h, mt - mb = 0 or 1), then the h
// rows between them: the two halves do not couple (they are h + 1 rows
// apart), each only updates the separator's blocks, and the separator's
// Schur complement is D minus both halves' updates.  Both halves run as the
// two instances of the batched code (the bottom one with its block order
// reversed, padded to mt rows), so the chain has mt + h steps instead of M.
// It is the same factorisation of S with the rows taken in another order;
// the solve visits the halves, then the separator, in that order.
//
// Apply, r = P^-1 b, by the three stages of Appendix C:
//   t2 = b2 - C A^-1 b1;  s2 = S^-1 t2;  r1 = A^-1 b1 - A^-1 B s2;  r2 = s2.
// Because A, B, C repeat per y-row, each stage with them is a product of the
// M x (N+1) matrix of per-row vectors with one (N+1)^2 block, computed as
// row-by-row dot products (one warp per output) so that all SMs share it.
#include "swj_internal.h"
#include <cuda.h>
#include <algorithm>
#include "closed_form.cuh"
#include <vector>
#include <string.h>
#include <stdlib.h>
#include <cuda_pipeline.h>

namespace {

constexpr double kPi = 3.14159265358979323846;

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

// coefficient of (zeta_x)_n in zeta_m / dx (1-based m, n): Eq. zetaapprox
// gives zeta_m = zeta_1 + dx (zx_1/2 + zx_2 + ... + zx_{m-1} + zx_m/2), m >= 2.
__device__ __forceinline__ double trap_coef(int m, int n)
{
    if (m == 1) return 0.0;
    if (n == 1 || n == m) return 0.5;
    return (n < m) ? 1.0 : 0.0;
}

// Dense (N+1)^2 blocks A, B, C (row-major).  Rows: 0 = E3 (E5), 1 = E4 (E6),
// 1 + k = E1_k (E2_k), k = 1..N-1.  Columns: 0 = phi_1 (zeta_1), n = phi_x,n (zeta_x,n).
__global__ void k_build_ABC(int N, double x1, double dx, double nrad, double F,
                            double *__restrict__ A, double *__restrict__ B,
                            double *__restrict__ C)
{
    int n1 = N + 1;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n1 * n1) return;
    int r = e / n1, c = e % n1;
    double a = 0.0, b = 0.0, cc = 0.0;
    if (r == 0) {
        if (c == 0) a = nrad;
        if (c == 1) a = x1;
    } else if (r == 1) {
        if (c == 1) a = nrad - x1 / dx;
        if (c == 2) a = x1 / dx;
    } else {
        int k = r - 1;
        if (c == k || c == k + 1) a = 0.5;                 // E1_k = phi_x*_k + ...
        double s = (c == 0) ? 1.0 : 0.5 * dx * (trap_coef(k, c) + trap_coef(k + 1, c));
        b = s / (F * F);                                    // zeta*_k / F^2 in E1_k
        cc = 2.0 * kPi * s;                                 // 2 pi phi*_k in E2_k
    }
    A[e] = a;
    B[e] = b;
    C[e] = cc;
}

// Forward-sweep coefficients of the tridiagonal block A (one thread): c'_r,
// the sub-diagonal a_r and 1 / den_r, den_r = b_r - a_r c'_{r-1} (Thomas
// algorithm), at coef[r], coef[n1 + r], coef[2 n1 + r].
__global__ void k_tri_coef(int n1, const double *__restrict__ A, double *__restrict__ coef)
{
    // the three diagonals into shared memory at once, then the recurrence on
    // one thread (a dependent division per row)
    extern __shared__ double dg[];   // sub, dia, sup: 3 n1
    for (int r = threadIdx.x; r < n1; r += blockDim.x) {
        dg[r] = r > 0 ? A[r * n1 + r - 1] : 0.0;
        dg[n1 + r] = A[r * n1 + r];
        dg[2 * n1 + r] = r + 1 < n1 ? A[r * n1 + r + 1] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double prev = 0.0;
    for (int r = 0; r < n1; ++r) {
        double sub = dg[r];
        double dia = dg[n1 + r];
        double sup = dg[2 * n1 + r];
        double rd = 1.0 / (dia - sub * prev);
        prev = sup * rd;
        coef[r] = prev;
        coef[n1 + r] = sub;
        coef[2 * n1 + r] = rd;
    }
}

// X = A^-1 Rhs for all ncol columns (Rhs == nullptr means the identity); X and
// Rhs are n1 x ncol row-major.  A column per thread, blockDim.x columns per
// block: the block's columns are copied into shared memory first (all rows
// in flight), both sweeps run there, and X is written as it is found.
// blockIdx.y selects (Rhs0, X0) or (Rhs1, X1): two systems in one launch.
__global__ void k_tri_cols(int n1, int ncol, const double *__restrict__ coef, const double *Rhs0, double *X0,
                           const double *Rhs1, double *X1)
{
    extern __shared__ double sc[];
    const double *Rhs = blockIdx.y ? Rhs1 : Rhs0;
    double *X = blockIdx.y ? X1 : X0;
    const int nc = blockDim.x, lane = threadIdx.x;
    const int col = blockIdx.x * nc + lane;
    if (col >= ncol) return;
    const double *cp = coef, *sub = coef + n1, *rden = coef + 2 * n1;
    double *Y = sc + lane;   // row r of this column at Y[r * nc]
    if (Rhs) {
        for (int r = 0; r < n1; ++r) __pipeline_memcpy_async(Y + (size_t)r * nc, Rhs + (size_t)r * ncol + col, 8);
        __pipeline_commit();
        __pipeline_wait_prior(0);
    } else {
        for (int r = 0; r < n1; ++r) Y[(size_t)r * nc] = (r == col) ? 1.0 : 0.0;
    }
    double dprev = 0.0;
    for (int r = 0; r < n1; ++r) {
        dprev = (Y[(size_t)r * nc] - sub[r] * dprev) * rden[r];
        Y[(size_t)r * nc] = dprev;
    }
    double next = dprev;
    X[(size_t)(n1 - 1) * ncol + col] = next;
    for (int r = n1 - 2; r >= 0; --r) {
        next = Y[(size_t)r * nc] - cp[r] * next;
        X[(size_t)r * ncol + col] = next;
    }
}

// columns per block of k_tri_cols: 32 while they fit in 160 KB of shared memory
inline int tri_cols_per_block(int n1)
{
    const int fit = (int)((160 * 1024) / ((size_t)n1 * sizeof(double)));
    return fit >= 32 ? 32 : (fit < 1 ? 1 : fit);
}

// Records of the flat state (zeta = 0, g = 0, zeta_x = 1 at the sources,
// zeta_x* = 0, A = C = 1, B = 0 at the targets) in the units of SrcRecS, for
// which the pair kernel's sum is sum_s w_s K2 = sum_s w_s K3.
template <typename T>
__global__ void k_flat_records(int N, int M, double dx, double dy, SrcRecS<T> *src, TgtArraysS<T> tg)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int S = N * M, Tn = (N - 1) * M;
    double rho = dx / dy;
    if (e < S) {
        int i = e % N, j = e / N;
        double ci = (i == 0 || i == N - 1) ? 0.5 : 1.0;
        double cj = (j == 0 || j == M - 1) ? 0.5 : 1.0;
        SrcRecS<T> r;
        r.x = (T)(i * rho); r.y = (T)j; r.zeta = T(0); r.zx = T(1); r.zy = T(0); r.g = T(0);
        r.w = (T)(rho * ci * cj); r.zxw = (T)dy;
        src[e] = r;
    }
    if (e < Tn) {
        int k = e % (N - 1), l = e / (N - 1);
        tg.x[e] = (T)((k + 0.5) * rho); tg.y[e] = (T)l;
        tg.zeta[e] = T(0); tg.g[e] = T(0); tg.zxw[e] = T(0);
        tg.A[e] = T(1); tg.B[e] = T(0); tg.C[e] = T(1);
    }
}

// I of the flat surface at every target (the closed form of the S2 integral
// with A = C = 1, B = 0), into out[t]; k_diag_corr completes it in place.
__global__ void k_flat_I(int N, int M, double dx, double dy, double *__restrict__ out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int Tn = (N - 1) * M;
    if (t >= Tn) return;
    int k = t % (N - 1), l = t / (N - 1);
    out[t] = swj_I_S2(1.0, 0.0, 1.0, N, M, k, l, dx, dy);
}

// diag[t] = (1/2) sum_s w K3 - (1/2) I_flat, the PreD correction of target t
// (I_flat read from diag[t], written there by k_flat_I).
__global__ void k_diag_corr(int N, int M, int P, const double *__restrict__ partial, double *__restrict__ diag)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int Tn = (N - 1) * M;
    if (t >= Tn) return;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += partial[(size_t)p * Tn + t];
    double I = diag[t];
    diag[t] = 0.5 * s - 0.5 * I;
}

// Kernel values 1 / sqrt(ddx^2 + ddy^2) of D's entries: row di = i - k + N - 1
// (ddx = (i - k + 1/2) dx, source column i, target k - 1/2), column dj = |ddy| / dy,
// for di < 2N - 2, dj < 2M - 1.
__global__ void k_k3_table(int N, int M, double dx, double dy, double *__restrict__ tab)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nj = 2 * M - 1;
    if (e >= (2 * N - 2) * nj) return;
    const int di = e / nj, dj = e % nj;
    const int i = di, k = N - 1;   // any pair with i - k = di - (N - 1)
    const double ddx = ((double)i - ((double)(k - 1) + 0.5)) * dx;
    const double ddy = (double)dj * dy;
    tab[e] = 1.0 / sqrt(ddx * ddx + ddy * ddy);
}

// Block (l, m) of D, the zeta-zeta block of P (block rows l, m of the mesh; it
// does not depend on F), row-major n1 x n1 at `out`; tab from k_k3_table.
//   row 0 (E5_l: x1 zeta_x,1 + n zeta_1) and row 1 (E6_l: x1 (zx_2 - zx_1)/dx +
//   n zx_1) on the diagonal block only;
//   row r = k + 1 >= 2, column c = i + 1 >= 1 (E2_k,l versus (zeta_x)_{i, m}):
//   -w K3 with w = dx dy ci cj (trapezoid weight of source (i, m)) and K3 =
//   1/|x - x'| + 1/|x - x'_image| at ddx = (i - k + 1/2) dx, ddy = (m - l) dy,
//   (m + l) dy, plus the PreD correction diag at columns k and k + 1 of the
//   diagonal block.
// -w K3 depends on the column only through i - k and ci, so the block first
// tabulates it (V[ci][i - k + N - 1], 2 (2N - 2) values, dynamic shared
// memory) and every entry is then a look-up: each value is formed by the same
// operations as entry by entry, and B300's FP64 pipe (two FMAs per clock per
// SM) does 45x less work.  With G1 != nullptr the diagonal block also gets
// -f G1 (S = D - G / F^2).  The calling CTA's threads all take part.
__device__ __forceinline__ void d_block(int N, int M, int l, int m, double x1, double dx, double dy, double nrad,
                                        const double *__restrict__ diag, const double *__restrict__ tab,
                                        const double *__restrict__ G1, double f, double *__restrict__ out,
                                        double *V)
{
    const int n1 = N + 1, nd = 2 * N - 2;
    const double cj = (m == 0 || m == M - 1) ? 0.5 : 1.0;
    const int ja = m > l ? m - l : l - m, jb = m + l;
    for (int q = threadIdx.x; q < 2 * nd; q += blockDim.x) {
        const int cs = q >= nd, di = q - cs * nd;
        const double ci = cs ? 0.5 : 1.0;
        const double w = dx * dy * ci * cj;
        const double *trow = tab + (size_t)di * (2 * M - 1);
        const double K3 = trow[ja] + trow[jb];
        V[q] = -w * K3;
    }
    __syncthreads();
    // Off the diagonal block every entry is a look-up (no FP64 instruction: B300
    // issues a predicated-off one at full cost); the diagonal block also
    // takes the E5/E6 rows, the PreD correction and -f G1.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (m != l) {
        for (int r = warp; r < n1; r += nw) {
            double *orow = out + (size_t)r * n1;
            for (int c = lane; c < n1; c += 32) {
                const int cs = (c == 1 || c == N) ? 1 : 0;   // ci = 1/2 at the end columns i = 0, N - 1
                orow[c] = (r >= 2 && c >= 1) ? V[cs * nd + (c - r + N - 1)] : 0.0;
            }
        }
        return;
    }
    for (int r = warp; r < n1; r += nw) {
        double *orow = out + (size_t)r * n1;
        const double dg = r >= 2 ? diag[(size_t)l * (N - 1) + (r - 2)] : 0.0;
        for (int c = lane; c < n1; c += 32) {
            double v = 0.0;
            if (r == 0) {
                v = (c == 0) ? nrad : (c == 1 ? x1 : 0.0);
            } else if (r == 1) {
                v = (c == 1) ? nrad - x1 / dx : (c == 2 ? x1 / dx : 0.0);
            } else if (c >= 1) {
                const int cs = (c == 1 || c == N) ? 1 : 0;
                v = V[cs * nd + (c - r + N - 1)];
                if (c == r - 1 || c == r) v += dg;
            }
            if (G1) v -= f * G1[(size_t)r * n1 + c];
            orow[c] = v;
        }
    }
}

// zero (or identity) n1 x n1 block
__device__ __forceinline__ void const_block(int n1, bool identity, double *__restrict__ out)
{
    const size_t n2 = (size_t)n1 * n1;
    for (size_t e = threadIdx.x; e < n2; e += blockDim.x) out[e] = (identity && e % (n1 + 1) == 0) ? 1.0 : 0.0;
}

// D of one instance (the band of D): block (l, m = l - h + slot), a CTA per
// block, blockIdx.x = l (2h + 1) + slot.
__global__ void k_fill_D(int N, int M, int h, double x1, double dx, double dy, double nrad,
                         const double *__restrict__ diag, const double *__restrict__ tab,
                         double *__restrict__ band)
{
    extern __shared__ double V[];
    const int n1 = N + 1, nb = 2 * h + 1;
    const int slot = blockIdx.x % nb, l = blockIdx.x / nb, m = l - h + slot;
    double *out = band + (size_t)blockIdx.x * n1 * n1;
    if (m >= 0 && m < M) d_block(N, M, l, m, x1, dx, dy, nrad, diag, tab, nullptr, 0.0, out, V);
    else const_block(n1, false, out);
}

// The two band instances of the two-sided order, S = D - G / F^2 on the
// diagonal blocks: instance 0 row l is block row l (columns below Mv only);
// instance 1 row l >= dB is block row M - 1 - (l - dB), the block order
// reversed (its columns likewise), and rows and columns below dB are padding
// (identity diagonal block, nothing else).  A CTA per block, blockIdx.x =
// (instance Mv + l) (2h + 1) + slot.
__global__ void k_fill_S_two_sided(int N, int M, int h, int Mv, int dB, double x1, double dx, double dy,
                                   double nrad, const double *__restrict__ diag, const double *__restrict__ tab,
                                   const double *__restrict__ G1, const double *__restrict__ invF2,
                                   double *__restrict__ band)
{
    extern __shared__ double V[];
    const int n1 = N + 1, nb = 2 * h + 1;
    const int slot = blockIdx.x % nb, l = (blockIdx.x / nb) % Mv, inst = blockIdx.x / (nb * Mv);
    const int m = l - h + slot;
    double *out = band + (size_t)blockIdx.x * n1 * n1;
    if (m < 0 || m >= Mv) {
        const_block(n1, false, out);
    } else if (inst == 1 && (l < dB || m < dB)) {
        const_block(n1, l == m, out);
    } else {
        const int pl = inst == 0 ? l : M - 1 - (l - dB);
        const int pm = inst == 0 ? m : M - 1 - (m - dB);
        d_block(N, M, pl, pm, x1, dx, dy, nrad, diag, tab, G1, invF2[0], out, V);
    }
}

// The h x h separator blocks of the two-sided order (block rows and columns
// Mv-h..Mv-1 of band instance 0, Mv-1..Mv-h of instance 1).  mode 0:
// sep0 <- instance 0's (D's, before any elimination); mode 1: instance 0's +=
// instance 1's - sep0, i.e. D minus the Schur updates of both halves.
__global__ void k_sep_blocks(int n1, int h, int Mv, double *__restrict__ band, size_t bst,
                             double *__restrict__ sep0, int mode)
{
    const size_t n2 = (size_t)n1 * n1, nb = 2 * h + 1;
    const size_t total = (size_t)h * h * n2;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t rc = e % n2;
        const int ab = (int)(e / n2), a = ab / h, b = ab % h;
        double *t = band + ((size_t)(Mv - h + a) * nb + (b - a + h)) * n2 + rc;
        if (mode == 0) {
            sep0[e] = *t;
        } else {
            const double u = band[bst + ((size_t)(Mv - 1 - a) * nb + (a - b + h)) * n2 + rc];
            *t = *t + (u - sep0[e]);
        }
    }
}

// Two-sided apply: tv = the right-hand side in the two band instances' row
// orders (padding rows 0); x = the solution from them.
__global__ void k_nd_scatter(int n1, int M, int Mv, int dB, const double *__restrict__ t, double *__restrict__ tv)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)Mv * n1;
    if (e >= 2 * per) return;
    const int inst = (int)(e / per), l = (int)((e % per) / n1), k = (int)(e % n1);
    tv[e] = inst == 0 ? t[(size_t)l * n1 + k] : (l < dB ? 0.0 : t[(size_t)(M - 1 - (l - dB)) * n1 + k]);
}

__global__ void k_nd_gather(int n1, int M, int Mv, int dB, const double *__restrict__ xv, double *__restrict__ x)
{
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)M * n1) return;
    const int l = (int)(e / n1), k = (int)(e % n1);
    x[e] = l < Mv ? xv[(size_t)l * n1 + k] : xv[(size_t)Mv * n1 + (size_t)(M - 1 - l + dB) * n1 + k];
}

// y_a = sum_j S_{s,j} z_j over the bottom half's block rows j next to separator
// row s (band instance 1 row Mv-1-a, the blocks left of its diagonal below
// row Mv-h), a warp per (a, row).
__global__ void k_sep_y(int n1, int h, int Mv, const double *__restrict__ bandB, const double *__restrict__ zB,
                        double *__restrict__ y)
{
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= h * n1) return;
    const size_t n2 = (size_t)n1 * n1, nb = 2 * h + 1;
    const int a = warp / n1, r = warp % n1, rp = Mv - 1 - a;
    double s = 0.0;
    for (int d = h; d >= 1; --d) {
        const int j = rp - d;
        if (j < 0 || j >= Mv - h) continue;
        const double *row = bandB + ((size_t)rp * nb + (h - d)) * n2 + (size_t)r * n1;
        for (int k = lane; k < n1; k += 32) s = fma(row[k], zB[(size_t)j * n1 + k], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[(size_t)a * n1 + r] = s;
}

// p_s -= inv_s y_a for separator row s = Mv-h+a of band instance 0
__global__ void k_sep_p(int n1, int h, int Mv, const double *__restrict__ bandT, const double *__restrict__ y,
                        double *__restrict__ pT)
{
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= h * n1) return;
    const size_t n2 = (size_t)n1 * n1, nb = 2 * h + 1;
    const int a = warp / n1, r = warp % n1, l = Mv - h + a;
    const double *row = bandT + ((size_t)l * nb + h) * n2 + (size_t)r * n1;
    double s = 0.0;
    for (int k = lane; k < n1; k += 32) s = fma(row[k], y[(size_t)a * n1 + k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) pT[(size_t)l * n1 + r] -= s;
}

// x of the separator rows, from band instance 0 into band instance 1
__global__ void k_sep_x(int n1, int h, int Mv, double *__restrict__ xv)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= h * n1) return;
    const int a = e / n1, k = e % n1;
    xv[(size_t)Mv * n1 + (size_t)(Mv - 1 - a) * n1 + k] = xv[(size_t)(Mv - h + a) * n1 + k];
}

// dst[b] = src for instances b = 1..nb-1 (src is instance 0's band)
__global__ void k_replicate(size_t n, const double *__restrict__ src, double *__restrict__ base,
                            size_t stride)
{
    const int inst = blockIdx.y + 1;
    double *dst = base + (size_t)inst * stride;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// S = D - G / F^2 on every diagonal block of every instance (G = C A^-1 B at F = 1)
__global__ void k_sub_G(int n1, int M, int h, const double *__restrict__ G1,
                        const double *__restrict__ invF2, double *__restrict__ band, size_t stride)
{
    const int inst = blockIdx.y;
    const size_t n2 = (size_t)n1 * n1, nb = 2 * h + 1;
    const double f = invF2[inst];
    double *b0 = band + (size_t)inst * stride;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)M * n2;
         e += (size_t)gridDim.x * blockDim.x) {
        size_t l = e / n2, rc = e % n2;
        b0[(l * nb + h) * n2 + rc] -= f * G1[rc];
    }
}

// copy `count` blocks of n doubles between strided locations
__global__ void k_copy_blocks(size_t n, const double *__restrict__ src, size_t sstride,
                              double *__restrict__ dst, size_t dstride)
{
    const int b = blockIdx.y;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dst[(size_t)b * dstride + e] = src[(size_t)b * sstride + e];
}

// Y[l][c] = alpha f dot(X[l, :], Mat[c, :]) + beta Y[l][c] for the M rows of
// every instance (X, Y at instance strides xs, ys; f = scale[inst] or 1)
__global__ void k_rowdot(int M, int n, const double *__restrict__ X, size_t xs,
                         const double *__restrict__ Mat, double alpha, const double *__restrict__ scale,
                         double beta, double *__restrict__ Y, size_t ys, const int *__restrict__ act)
{
    // Y[l, c] = a (X[l, :] . Mat[c, :]) + beta Y[l, c], 8 lanes per output (four
    // outputs per warp, consecutive c of one row l): each lane sums every 8th k,
    // then three butterfly steps within the group.  B300 issues FP64 per warp
    // instruction, so 8-lane groups need about half the FP64 instructions per
    // output of a warp per output (six FMAs and a five-step reduction at n = 182).
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long out = gid >> 3;
    const int sub = threadIdx.x & 7;
    if (out >= (long)M * n) return;   // whole 8-lane groups leave together
    const int l = (int)(out / n), c = (int)(out % n);
    const double *x = X + (size_t)inst * xs + (size_t)l * n, *mr = Mat + (size_t)c * n;
    double s = 0.0;
    for (int k = sub; k < n; k += 8) s = fma(x[k], mr[k], s);
    const unsigned grp = 0xFFu << (threadIdx.x & 24);
    s += __shfl_xor_sync(grp, s, 4, 8);
    s += __shfl_xor_sync(grp, s, 2, 8);
    s += __shfl_xor_sync(grp, s, 1, 8);
    if (sub == 0) {
        double a = scale ? alpha * scale[inst] : alpha;
        double *y = Y + (size_t)inst * ys + (size_t)l * n + c;
        *y = (beta == 0.0) ? a * s : fma(a, s, beta * *y);
    }
}

// y_inst = x_inst for vectors at different instance strides
__global__ void k_copy_vec(int n, const double *__restrict__ x, size_t xs, double *__restrict__ y,
                           size_t ys, const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[(size_t)inst * ys + i] = x[(size_t)inst * xs + i];
}

inline void rowdot(swj_ctx *c, const double *X, size_t xs, const double *Mat, double alpha,
                   const double *scale, double beta, double *Y, size_t ys, const int *act)
{
    SWJ_COUNT_LAUNCH();
    k_rowdot<<<dim3(nblk((long)c->M * c->n1 * 8, 256), c->nb), 256, 0, c->stream>>>(
        c->M, c->n1, X, xs, Mat, alpha, scale, beta, Y, ys, act);
}

inline size_t band_stride(const swj_ctx *c)
{
    return (size_t)c->pc_M * c->pc_nb * c->n1 * c->n1;
}

// block (l, m) of band instance inst (rows and columns of that instance)
inline double *blk(swj_ctx *c, int inst, int l, int m)
{
    size_t n2 = (size_t)c->n1 * c->n1;
    int slot = m - l + c->pc_h;
    return c->pc_band + inst * band_stride(c) + ((size_t)l * c->pc_nb + slot) * n2;
}

inline double *wblk(swj_ctx *c, int inst, int i, int k)
{
    size_t n2 = (size_t)c->n1 * c->n1;
    return c->pc_W + ((size_t)inst * c->pc_M * c->pc_h + (size_t)i * c->pc_h + (k - i - 1)) * n2;
}

// ---- SM partitions of the band LU (opts.sm_partition) -------------------------
// Two CUDA green contexts of the device: 32 to 48 SMs (40 on B300) that hold
// the Gauss-Jordan chain's clusters, the other SMs for the bulk block products
// (pc_partitions).  Unpartitioned,
// the bulk kernels share the chain's SMs and slow each pivot step of the
// latency-bound chain.  The driver functions come through the runtime's
// entry-point query (the library links only the runtime).
typedef CUresult (*PfnDevGet)(CUdevice *, int);
typedef CUresult (*PfnGetRes)(CUdevice, CUdevResource *, CUdevResourceType);
typedef CUresult (*PfnSplit)(CUdevResource *, unsigned int *, const CUdevResource *, CUdevResource *, unsigned int,
                             unsigned int);
typedef CUresult (*PfnDesc)(CUdevResourceDesc *, CUdevResource *, unsigned int);
typedef CUresult (*PfnGcCreate)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int);
typedef CUresult (*PfnGcDestroy)(CUgreenCtx);
typedef CUresult (*PfnGcStream)(CUstream *, CUgreenCtx, unsigned int, int);
typedef CUresult (*PfnCtxFromGc)(CUcontext *, CUgreenCtx);
typedef CUresult (*PfnCtxPush)(CUcontext);
typedef CUresult (*PfnCtxPop)(CUcontext *);
struct GreenApi {
    PfnDevGet dev_get = nullptr;
    PfnGetRes get_res = nullptr;
    PfnSplit split = nullptr;
    PfnDesc desc = nullptr;
    PfnGcCreate create = nullptr;
    PfnGcDestroy destroy = nullptr;
    PfnGcStream stream = nullptr;
    PfnCtxFromGc ctx_of = nullptr;
    PfnCtxPush push = nullptr;
    PfnCtxPop pop = nullptr;
    bool ok = false;
};
const GreenApi &green_api()
{
    static GreenApi g = [] {
        GreenApi a;
        auto get = [](const char *name, void **fn) {
            cudaDriverEntryPointQueryResult q;
            return cudaGetDriverEntryPointByVersion(name, fn, 12080, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fn;
        };
        a.ok = get("cuDeviceGet", (void **)&a.dev_get) && get("cuDeviceGetDevResource", (void **)&a.get_res) &&
               get("cuDevSmResourceSplitByCount", (void **)&a.split) &&
               get("cuDevResourceGenerateDesc", (void **)&a.desc) && get("cuGreenCtxCreate", (void **)&a.create) &&
               get("cuGreenCtxDestroy", (void **)&a.destroy) && get("cuGreenCtxStreamCreate", (void **)&a.stream) &&
               get("cuCtxFromGreenCtx", (void **)&a.ctx_of) && get("cuCtxPushCurrent", (void **)&a.push) &&
               get("cuCtxPopCurrent", (void **)&a.pop);
        cudaGetLastError();
        return a;
    }();
    return g;
}
constexpr size_t kGJOneCtaSmem = 116 * 1024;   // above half an SM's shared memory: one CTA per SM

void free_partitions(swj_ctx *c)
{
    if (c->pc_gchain) cudaStreamDestroy(c->pc_gchain);
    if (c->pc_gbulk) cudaStreamDestroy(c->pc_gbulk);
    c->pc_gchain = c->pc_gbulk = nullptr;
    const GreenApi &g = green_api();
    for (void *&h : c->pc_gctx) {
        if (h && g.ok) g.destroy((CUgreenCtx)h);
        h = nullptr;
    }
    cudaGetLastError();
    c->pc_green = 0;
}

// Create the partitions (once per context): the smallest chain partition of
// 32, 40 or 48 SMs whose SMs hold the chain's nv clusters of n1 x n1 blocks at
// once at one CTA per SM (a partition's SMs need not form whole GPCs), the
// rest of the device for the bulk work.  True if that worked.
bool pc_partitions(swj_ctx *c, int n1, int nv)
{
    if (c->pc_green) return c->pc_green > 0;
    c->pc_green = -1;
    // a tool injected into the process (a profiler, a sanitizer) may not follow
    // green contexts (Nsight Compute fails to prepare the chain's launches): the
    // set-up then runs unpartitioned (the factors are the same).  The tools
    // announce themselves through their injection variables.
    for (const char *var : {"CUDA_INJECTION64_PATH", "NV_NSIGHT_INJECTION_TRANSPORT_TYPE",
                            "NV_COMPUTE_PROFILER_PERFWORKS_DIR"}) {
        const char *v = getenv(var);
        if (v && *v) return false;
    }
    const GreenApi &g = green_api();
    if (!g.ok) return false;
    int ord = 0, lo = 0, hi = 0;
    CUdevice dev;
    CUdevResource all;
    if (cudaGetDevice(&ord) != cudaSuccess || g.dev_get(&dev, ord) != CUDA_SUCCESS ||
        g.get_res(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) {
        cudaGetLastError();
        return false;
    }
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (unsigned int want : {32u, 40u, 48u}) {
        CUdevResource grp[1], rest;
        unsigned int ng = 1;
        CUdevResourceDesc dc, db;
        CUgreenCtx gc = nullptr, gb = nullptr;
        CUstream sc = nullptr, sb = nullptr;
        bool ok = g.split(grp, &ng, &all, &rest, CU_DEV_SM_RESOURCE_SPLIT_MAX_POTENTIAL_CLUSTER_SIZE, want) ==
                      CUDA_SUCCESS &&
                  ng == 1 && grp[0].sm.smCount >= want && rest.sm.smCount >= 2 * want &&
                  g.desc(&dc, grp, 1) == CUDA_SUCCESS && g.desc(&db, &rest, 1) == CUDA_SUCCESS &&
                  g.create(&gc, dc, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
                  g.create(&gb, db, dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS &&
                  g.stream(&sc, gc, CU_STREAM_NON_BLOCKING, hi) == CUDA_SUCCESS &&
                  g.stream(&sb, gb, CU_STREAM_NON_BLOCKING, lo) == CUDA_SUCCESS;
        c->pc_gctx[0] = gc;
        c->pc_gctx[1] = gb;
        c->pc_gchain = (cudaStream_t)sc;
        c->pc_gbulk = (cudaStream_t)sb;
        if (ok) {
            CUcontext cc = nullptr, popped = nullptr;
            int ncl = 0;
            if (g.ctx_of(&cc, gc) == CUDA_SUCCESS && g.push(cc) == CUDA_SUCCESS) {
                ncl = swj_gj_cluster_capacity(n1, kGJOneCtaSmem);
                g.pop(&popped);
            }
            ok = ncl >= nv;
        }
        cudaGetLastError();
        if (ok) {
            c->pc_green = 1;
            c->pc_gsms = (int)grp[0].sm.smCount;
            return true;
        }
        free_partitions(c);
    }
    c->pc_green = -1;
    return false;
}

void delete_plan(void *plan);

void free_pc(swj_ctx *c)
{
    delete_plan(c->pc_plan);
    c->pc_plan = nullptr;
    double **bufs[] = {&c->pc_Ainv, &c->pc_AinvB1, &c->pc_CAinv, &c->pc_G1, &c->pc_A, &c->pc_B1,
                       &c->pc_C, &c->pc_invF2, &c->pc_band, &c->pc_W, &c->pc_sumK3, &c->pc_t1,
                       &c->pc_t2, &c->pc_z, &c->pc_work, &c->pc_lt, &c->pc_mc_buf, &c->pc_nd_buf,
                       &c->pc_k3};
    for (double **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    if (c->pc_info) cudaFree(c->pc_info);
    c->pc_info = nullptr;
    if (c->pc_ptrs) cudaFree(c->pc_ptrs);
    c->pc_ptrs = nullptr;
    c->pc_ptrs_cap = 0;
    if (c->pc_mc_err) cudaFree(c->pc_mc_err);
    c->pc_mc_err = nullptr;
    void *oz[] = {c->oz_sa, c->oz_sb, c->oz_ea, c->oz_eb, c->oz_P, c->oz_err, c->oz_desc};
    for (void *q : oz)
        if (q) cudaFree(q);
    c->oz_sa = c->oz_sb = nullptr;
    c->oz_ea = c->oz_eb = nullptr;
    c->oz_P = nullptr;
    c->oz_err = nullptr;
    c->oz_desc = nullptr;
    c->pc_mc = 0;
    if (c->pc_chain) {
        cudaStreamSynchronize(c->pc_chain);
        cudaStreamSynchronize(c->pc_bulk);
        for (cudaEvent_t &e : c->pc_ev) cudaEventDestroy(e);
        cudaStreamDestroy(c->pc_chain);
        cudaStreamDestroy(c->pc_bulk);
        c->pc_chain = c->pc_bulk = nullptr;
    }
    if (c->pc_gchain) cudaStreamSynchronize(c->pc_gchain);
    if (c->pc_gbulk) cudaStreamSynchronize(c->pc_gbulk);
    free_partitions(c);
    c->pc_ready = 0;
    c->bytes -= c->pc_bytes;
    c->pc_bytes = 0;
}

// block half bandwidth of the option block_bw (0 = the whole matrix, -1 = by
// mesh: b = 11 up to 48 block rows, 15 above, the fastest set-up + solve
// measured on the 61x21, 121x41, 181x61 and 361x121 meshes)
int half_band(int block_bw, int M)
{
    if (block_bw < 0) block_bw = (M <= 48) ? 11 : 15;
    int h = (block_bw == 0) ? M - 1 : (block_bw - 1) / 2;
    return h > M - 1 ? M - 1 : h;
}

// Layout of the band LU (see swj_ctx::pc_M): half bandwidth h, pc_nv band
// instances of Mv block rows, the two-sided split.  Step i of the
// factorisation runs on band instances 0..insts(i)-1.
struct PcShape {
    int h, Mv, nv, dB, split;
    bool nd;
    int insts(int i) const { return i < split ? nv : 1; }
};

PcShape pc_shape(int M, int nb, int h, int lu_order)
{
    PcShape s = {h, M, nb, 0, M, false};
    if (nb == 1 && h >= 1 && lu_order == SWJ_LU_TWO_SIDED && M - h >= 2) {
        const int mt = (M - h + 1) / 2, mb = M - h - mt;
        s.nd = true;
        s.Mv = mt + h;
        s.nv = 2;
        s.dB = mt - mb;
        s.split = mt;
    }
    return s;
}

// multi-cluster apply scratch (h >= 2; one instance, or the two band instances of
// the two-sided order): per band instance z [Mv][n1], then the term slots cf, cb
// [Mv][h+1][n1] (0 where it does not apply)
size_t pc_mc_doubles(int n1, const PcShape &sh)
{
    return (sh.h >= 2 && (sh.nd || sh.nv == 1)) ? (size_t)sh.nv * sh.Mv * n1 * (1 + 2 * (size_t)(sh.h + 1)) : 0;
}

constexpr int kPcBufs = 19;

// doubles of each preconditioner buffer, in the order of free_pc's list
// (0: not allocated)
void pc_sizes(int n1, int M, int T, int H, int nb, const PcShape &sh, bool gj_inplace, size_t sz[kPcBufs])
{
    const size_t n2 = (size_t)n1 * n1, h = sh.h, Mv = sh.Mv, nv = sh.nv;
    const size_t work_blocks = gj_inplace ? 1 : nv * (h == 0 ? Mv : 1);
    const size_t vz = std::max((size_t)nb * H, nv * Mv * n1);
    const size_t nd = sh.nd ? 2 * nv * Mv * n1 + h * h * n2 + h * n1 : 0;
    const size_t v[kPcBufs] = {n2, n2, n2, n2, n2, n2, n2, (size_t)nb,
                               nv * Mv * (2 * h + 1) * n2, nv * Mv * (h > 0 ? h : 1) * n2,
                               (size_t)T, (size_t)nb * H, (size_t)nb * H, vz, work_blocks * n2,
                               nv * h * n2, pc_mc_doubles(n1, sh), nd, (size_t)(2 * n1 - 4) * (2 * M - 1)};
    for (int i = 0; i < kPcBufs; ++i) sz[i] = v[i];
}

// block products of the band LU (pointer triples of the batched GEMMs)
size_t pc_gemm_count(const PcShape &sh)
{
    const int h = sh.h, M = sh.Mv;
    if (h == 0) return 0;
    size_t np = 0;
    for (int i = 0; i < M; ++i) {
        size_t k = (size_t)(i + h < M - 1 ? h : M - 1 - i);
        np += (size_t)sh.insts(i) * (k + k * k + (size_t)std::min(i, h));
    }
    return np;
}

// ---- sliced (bf16 tensor-core) block products of the bulk stream (ozaki.cu)
// Per step i and instance: the A factors split by rows (slot 0 = inv_i,
// slot 1 + (j - i - 1) = S_ji, j = i+1..kmax), the B factors split by columns
// (S_ik, k = i+2..kmax at [0, h-1); W_ik, k = i+1..kmax at [h, 2h); S_ij,
// j < i, at [2h, 3h)), and the products of the groups Wb, B1, B2, L.
struct OzLayout {
    OzScheme z;
    int np, beta, s;
    size_t nsa, nsb;          // slice slots (A, B)
    size_t maxP;              // block products per batched call
    size_t nptr, nprod;       // split-list and product-list entries of all steps
    size_t bytes_desc;        // descriptor buffer
    size_t bytes;             // every buffer of the sliced path
};

constexpr size_t kOzPBytes = (size_t)256 << 20;   // slice products of one batched call

size_t oz_align(size_t b) { return (b + 255) & ~(size_t)255; }

OzLayout oz_layout(int n1, const PcShape &sh)
{
    OzLayout L = {};
    const int h = sh.h, M = sh.Mv, nb = sh.nv;
    swj_ozaki_scheme(n1, &L.z);
    L.np = L.z.np;
    L.beta = L.z.beta;
    L.s = L.z.s;
    const size_t n2 = (size_t)L.np * L.np;
    L.nsa = (size_t)nb * (h + 1);
    L.nsb = (size_t)nb * 3 * h;
    const size_t per = (size_t)L.z.nout * n2 * sizeof(float);   // the outputs of one block product
    size_t cap = kOzPBytes / per;
    if (cap < 1) cap = 1;
    const size_t most = (size_t)nb * h * h;
    L.maxP = cap < most ? cap : most;
    for (int i = 0; i < M; ++i) {
        const size_t kr = (size_t)(i + h < M - 1 ? h : M - 1 - i), nt = (size_t)(i < h ? i : h);
        const size_t q = (size_t)sh.insts(i);
        L.nptr += q * ((1 + kr) + (kr > 0 ? kr - 1 : 0) + kr + nt);
        L.nprod += q * ((kr > 0 ? kr - 1 : 0) + (kr > 0 ? kr * kr - 1 : 0) + nt);
    }
    L.bytes_desc = oz_align(L.nptr * sizeof(double *)) + oz_align(L.nptr * sizeof(int)) +
                   oz_align(L.nprod * sizeof(OzProd));
    L.bytes = (L.nsa + L.nsb) * L.s * n2 * 2 + (L.nsa + L.nsb) * L.np * sizeof(int) + L.maxP * per + sizeof(int) +
              L.bytes_desc;
    return L;
}

// One step's entries in the sliced path's split and product lists.
struct OzStep {
    size_t a, wb, u, l, pwb, pb1, pb2, pl;
    int na, nwb, nu, nl, cwb, cb1, cb2, cl;
};

// The band LU's host-side plan, built once per allocation of the buffers (the
// lists hold device addresses of blocks, fixed until the buffers are freed):
// per step and group the offset and count into the pointer triples of the
// batched FP64 products (uploaded to pc_ptrs), and the sliced path's split and
// product lists (uploaded to oz_desc).
struct PcPlan {
    int np = 0;
    std::vector<int> off, cnt;
    std::vector<OzStep> zo;
    OzLayout OL = {};
};

void delete_plan(void *plan) { delete (PcPlan *)plan; }

}  // namespace

void swj_pc_free(swj_ctx *c) { free_pc(c); }

size_t swj_pc_bytes(int N, int M, int nb, int block_bw, int lu_products, int lu_order)
{
    const int n1 = N + 1;
    const PcShape sh = pc_shape(M, nb, half_band(block_bw, M), lu_order);
    size_t sz[kPcBufs], tot = 0;
    pc_sizes(n1, M, (N - 1) * M, n1 * M, nb, sh, swj_gj_inplace(n1), sz);
    for (size_t v : sz) tot += v * sizeof(double);
    tot += (size_t)sh.nv * sh.Mv * sizeof(int);
    tot += 3 * pc_gemm_count(sh) * sizeof(double *);
    if (pc_mc_doubles(n1, sh)) tot += sizeof(int);
    if (lu_products == SWJ_LU_SLICED && sh.h > 0) tot += oz_layout(n1, sh).bytes;
    return tot;
}

// S x = pc_t2 on h clusters into x (one instance, top-down order): p into
// pc_z, the scratch and x set to "not yet written", then the sweep
static int mc_solve(swj_ctx *c, double *x)
{
    const int M = c->pc_M, n1 = c->n1, h = c->pc_h;
    const size_t mn = (size_t)M * n1;
    double *z = c->pc_mc_buf, *cf = z + mn, *cb = cf + mn * (h + 1);
    int rc = swj_block_p(c->stream, 1, n1, M, h, c->pc_band, band_stride(c), c->pc_t2, mn, c->pc_z, mn,
                         nullptr, c->pc_mc_buf, mn * (1 + 2 * (size_t)(h + 1)), x, mn);
    if (rc) return rc;
    return swj_band_sweep_mc(c->stream, n1, M, h, c->pc_band, c->pc_W, c->pc_z, z, x, cf, cb, c->pc_mc_err, false,
                             swj_waits(c, true));
}

// S x = t for the two-sided order (one instance; t, x [M][n1]).  With
// F = Mv - h block rows per half:
//   1. t in both band instances' row orders, p = inv t for every row of both;
//   2. the forward recurrence of both halves (rows 0..F-1 of both instances);
//   3. each separator row's p loses inv_s sum_j S_sj z_j over the bottom rows
//      j next to it (those blocks of instance 1, left as they were at the
//      bottom half's steps);
//   4. the separator rows of instance 0: forward, then backward;
//   5. the separator's x into instance 1, the backward recurrence of both
//      halves (rows F-1..0 of both instances, the rows above given);
//   6. x from both instances.
// mode 2: steps 2 and 5 each one multi-cluster launch for both instances (a
// critical cluster each, shared helpers); mode 1: multi-cluster launches for
// one instance at a time (bottom forward, the whole of instance 0, bottom
// backward); mode 0: the same order with one cluster per launch.
static int nd_solve(swj_ctx *c, const double *t, double *x, int mode)
{
    const int n1 = c->n1, Mv = c->pc_M, h = c->pc_h, M = c->M, F = Mv - h;
    const size_t per = (size_t)Mv * n1, n2 = (size_t)n1 * n1, bst = band_stride(c), wst = (size_t)Mv * h * n2;
    const size_t sst = per * (h + 1);   // term slots of one band instance
    cudaStream_t st = c->stream;
    double *tv = c->pc_nd_buf, *xv = tv + 2 * per, *y = xv + 2 * per + (size_t)h * h * n2;
    const double *bandT = c->pc_band, *bandB = c->pc_band + bst, *WT = c->pc_W, *WB = c->pc_W + wst;
    double *pz = c->pc_z;   // p of both band instances (the one-cluster sweep turns it into z)
    const int nw = nblk((long)h * n1 * 32, 256);
    int *err = c->pc_mc_err;
    const SwjWaits wt = swj_waits(c, true);
    SWJ_COUNT_LAUNCH();
    k_nd_scatter<<<nblk((long)(2 * per), 256), 256, 0, st>>>(n1, M, Mv, c->pc_dB, t, tv);
    int rc;
    auto sep_p = [&](const double *zB) {
        SWJ_COUNT_LAUNCH();
        k_sep_y<<<nw, 256, 0, st>>>(n1, h, Mv, bandB, zB, y);
        SWJ_COUNT_LAUNCH();
        k_sep_p<<<nw, 256, 0, st>>>(n1, h, Mv, bandT, y, pz);
    };
    auto sep_x = [&]() {
        SWJ_COUNT_LAUNCH();
        k_sep_x<<<nblk((long)h * n1, 256), 256, 0, st>>>(n1, h, Mv, xv);
    };
    if (mode > 0) {
        // multi-cluster scratch: z of both instances, then cf of both, then cb of both
        double *zv = c->pc_mc_buf, *cf = zv + 2 * per, *cb = cf + 2 * sst;
        if ((rc = swj_block_p(st, 2, n1, Mv, h, c->pc_band, bst, tv, per, pz, per, nullptr, c->pc_mc_buf,
                              2 * (per + 2 * sst), xv, 2 * per)))
            return rc;
        if (mode == 2) {
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 2, c->pc_band, bst, c->pc_W, wst, pz, zv, xv, per, cf,
                                               cb, sst, err, false, 0, F, -1, 0, wt)))
                return rc;
            sep_p(zv + per);
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 1, bandT, 0, WT, 0, pz, zv, xv, 0, cf, cb, 0, err,
                                               false, F, Mv, Mv - 1, F, wt)))
                return rc;
            sep_x();
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 2, c->pc_band, bst, c->pc_W, wst, zv, zv, xv, per, cf,
                                               cb, sst, err, false, 0, 0, F - 1, 0, wt)))
                return rc;
        } else {
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 1, bandB, 0, WB, 0, pz + per, zv + per, xv + per, 0,
                                               cf + sst, cb + sst, 0, err, false, 0, F, -1, 0, wt)))
                return rc;
            sep_p(zv + per);
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 1, bandT, 0, WT, 0, pz, zv, xv, 0, cf, cb, 0, err,
                                               false, 0, Mv, Mv - 1, 0, wt)))
                return rc;
            sep_x();
            if ((rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, 1, bandB, 0, WB, 0, zv + per, zv + per, xv + per, 0,
                                               cf + sst, cb + sst, 0, err, false, 0, 0, F - 1, 0, wt)))
                return rc;
        }
    } else {
        if ((rc = swj_block_p(st, 2, n1, Mv, h, c->pc_band, bst, tv, per, pz, per, nullptr))) return rc;
        if ((rc = swj_band_sweep_cluster(st, 1, n1, Mv, h, bandB, bst, WB, wst, pz + per, per, xv + per, per,
                                         nullptr, false, F, -1)))
            return rc;
        sep_p(pz + per);
        if ((rc = swj_band_sweep_cluster(st, 1, n1, Mv, h, bandT, bst, WT, wst, pz, per, xv, per, nullptr)))
            return rc;
        sep_x();
        if ((rc = swj_band_sweep_cluster(st, 1, n1, Mv, h, bandB, bst, WB, wst, pz + per, per, xv + per, per,
                                         nullptr, false, 0, F - 1)))
            return rc;
    }
    SWJ_COUNT_LAUNCH();
    k_nd_gather<<<nblk((long)M * n1, 256), 256, 0, st>>>(n1, M, Mv, c->pc_dB, xv, x);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_pc_setup(swj_ctx *c)
{
    const int N = c->N, M = c->M, n1 = c->n1, nb = c->nb;
    const swj_mesh &m = c->mesh;
    cudaStream_t st = c->stream;
    const int h = half_band(c->opts.block_bw, M);
    const PcShape sh = pc_shape(M, nb, h, c->opts.lu_order);
    const int Mv = sh.Mv, nv = sh.nv;
    // the band sweep stages h vectors of n1 doubles in shared memory
    if ((size_t)(h + 1) * n1 * sizeof(double) > 200 * 1024) return SWJ_EINVAL;
    const size_t n2 = (size_t)n1 * n1;
    const int nbs = 2 * h + 1;
    const bool gj_inplace = swj_gj_inplace(n1);
    const bool sliced = c->opts.lu_products == SWJ_LU_SLICED && h > 0;
    if (!c->pc_band || c->pc_h != h || (c->oz_sa != nullptr) != sliced || c->pc_nd != (int)sh.nd) {
        free_pc(c);
        c->pc_h = h;
        c->pc_nb = nbs;
        c->pc_nd = sh.nd;
        c->pc_M = Mv;
        c->pc_nv = nv;
        c->pc_dB = sh.dB;
        c->pc_split = sh.split;
        size_t sz[kPcBufs];
        pc_sizes(n1, M, c->T, c->H, nb, sh, gj_inplace, sz);
        double **bufs[] = {&c->pc_Ainv, &c->pc_AinvB1, &c->pc_CAinv, &c->pc_G1, &c->pc_A,
                           &c->pc_B1, &c->pc_C, &c->pc_invF2, &c->pc_band, &c->pc_W,
                           &c->pc_sumK3, &c->pc_t1, &c->pc_t2, &c->pc_z, &c->pc_work,
                           &c->pc_lt, &c->pc_mc_buf, &c->pc_nd_buf, &c->pc_k3};
        static_assert(sizeof(bufs) / sizeof(bufs[0]) == kPcBufs, "buffer list");
        for (int i = 0; i < kPcBufs; ++i) {
            if (!sz[i]) continue;
            if (cudaMalloc(bufs[i], sz[i] * sizeof(double)) != cudaSuccess) {
                free_pc(c);
                return SWJ_ENOMEM;
            }
            c->pc_bytes += sz[i] * sizeof(double);
            c->bytes += sz[i] * sizeof(double);
        }
        if (cudaMalloc(&c->pc_info, (size_t)nv * Mv * sizeof(int)) != cudaSuccess) {
            free_pc(c);
            return SWJ_ENOMEM;
        }
        c->pc_bytes += (size_t)nv * Mv * sizeof(int);
        c->bytes += (size_t)nv * Mv * sizeof(int);
        if (c->pc_mc_buf) {
            if (cudaMalloc(&c->pc_mc_err, sizeof(int)) != cudaSuccess) {
                free_pc(c);
                return SWJ_ENOMEM;
            }
            c->pc_bytes += sizeof(int);
            c->bytes += sizeof(int);
        }
        if (sliced) {
            const OzLayout L = oz_layout(n1, sh);
            void **ozb[] = {&c->oz_sa, &c->oz_sb, (void **)&c->oz_ea, (void **)&c->oz_eb, (void **)&c->oz_P,
                            (void **)&c->oz_err, &c->oz_desc};
            const size_t p2 = (size_t)L.np * L.np;
            const size_t ozs[] = {L.nsa * L.s * p2 * 2, L.nsb * L.s * p2 * 2, L.nsa * L.np * sizeof(int),
                                  L.nsb * L.np * sizeof(int), L.maxP * L.z.nout * p2 * sizeof(float), sizeof(int),
                                  L.bytes_desc};
            for (int i = 0; i < 7; ++i) {
                if (cudaMalloc(ozb[i], ozs[i]) != cudaSuccess) {
                    free_pc(c);
                    return SWJ_ENOMEM;
                }
                c->pc_bytes += ozs[i];
                c->bytes += ozs[i];
            }
        }
    }
    c->pc_ready = 0;
    c->pc_chain_sms = 0;
    if (!c->pc_chain) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        SWJ_CUDA_TRY(cudaStreamCreateWithPriority(&c->pc_chain, cudaStreamNonBlocking, hi));
        SWJ_CUDA_TRY(cudaStreamCreateWithPriority(&c->pc_bulk, cudaStreamNonBlocking, lo));
        for (cudaEvent_t &e : c->pc_ev) SWJ_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // Two independent branches, joined before the band is filled: on the side
    // stream A, B (at F = 1), C, A^-1, A^-1 B, C A^-1, G = C A^-1 B (Appendix
    // C), the K3 table and I of the flat surface; on the context's stream the
    // trapezoid sum of w K3 of the flat surface (the pair kernel).
    cudaStream_t sa = c->pc_chain;
    cudaEvent_t evFork = c->pc_ev[10], evJoin = c->pc_ev[11];
    SWJ_CUDA_TRY(cudaEventRecord(evFork, st));
    SWJ_CUDA_TRY(cudaStreamWaitEvent(sa, evFork, 0));
    std::vector<double> invF2(nb);
    for (int i = 0; i < nb; ++i) invF2[i] = 1.0 / (c->F[i] * c->F[i]);
    SWJ_CUDA_TRY(cudaMemcpyAsync(c->pc_invF2, invF2.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st));
    // --- repeated blocks A, B (at F = 1), C and their products (Appendix C)
    SWJ_COUNT_LAUNCH();
    k_build_ABC<<<nblk((long)n2, 256), 256, 0, sa>>>(N, m.x1, m.dx, m.n_rad, 1.0, c->pc_A,
                                                     c->pc_B1, c->pc_C);
    double *cpv = c->pc_t1;   // 3 n1 scratch (pc_t1 holds M n1, M >= 3)
    SWJ_COUNT_LAUNCH();
    k_tri_coef<<<1, 256, 3 * (size_t)n1 * sizeof(double), sa>>>(n1, c->pc_A, cpv);
    {
        const int tc = tri_cols_per_block(n1);
        const size_t tsm = (size_t)tc * n1 * sizeof(double);
        static const bool tri_attr = cudaFuncSetAttribute(k_tri_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          160 * 1024) == cudaSuccess;
        if (!tri_attr) cudaGetLastError();
        SWJ_COUNT_LAUNCH();
        k_tri_cols<<<dim3(nblk(n1, tc), 2), tc, tsm, sa>>>(n1, n1, cpv, nullptr, c->pc_Ainv, c->pc_B1,
                                                          c->pc_AinvB1);
    }
    swj_dgemm(sa, n1, n1, n1, 1.0, c->pc_C, n1, c->pc_Ainv, n1, 0.0, c->pc_CAinv, n1);
    swj_dgemm(sa, n1, n1, n1, 1.0, c->pc_C, n1, c->pc_AinvB1, n1, 0.0, c->pc_G1, n1);
    SWJ_COUNT_LAUNCH();
    k_k3_table<<<nblk((long)(2 * N - 2) * (2 * M - 1), 256), 256, 0, sa>>>(N, M, m.dx, m.dy, c->pc_k3);
    SWJ_COUNT_LAUNCH();
    k_flat_I<<<nblk(c->T, kFp64Block), kFp64Block, 0, sa>>>(N, M, m.dx, m.dy, c->pc_sumK3);
    SWJ_CUDA_TRY(cudaEventRecord(evJoin, sa));
    // --- PreD diagonal correction: trapezoid sum of w K3 and I of the flat surface
    //     (instance 0's record buffers serve as scratch; every residual rewrites them)
    int prec = (c->opts.solve_mode == SWJ_SOLVE_FP64) ? SWJ_FP64 : SWJ_FP32;
    // the default tile shape, whatever the autotuner picked: the preconditioner of
    // a mesh and F must not depend on when it was built
    PairPlan pl = swj_pair_plan_variant(c, prec, 0);
    int ne = c->S > c->T ? c->S : c->T;
    std::vector<int> only0(nb, 0);
    only0[0] = 1;
    int *act0 = c->act_d;
    for (int i = 0; i < nb; ++i) c->act_h[i] = only0[i];
    SWJ_CUDA_TRY(cudaMemcpyAsync(act0, c->act_h, nb * sizeof(int), cudaMemcpyHostToDevice, st));
    if (prec == SWJ_FP64) {
        SWJ_COUNT_LAUNCH();
        k_flat_records<double><<<nblk(ne, 256), 256, 0, st>>>(N, M, m.dx, m.dy, c->src64, c->tgt64);
        swj_launch_pairs64(c, pl, act0);
    } else {
        SWJ_COUNT_LAUNCH();
        k_flat_records<float><<<nblk(ne, 256), 256, 0, st>>>(N, M, m.dx, m.dy, c->src32, c->tgt32);
        swj_launch_pairs32(c, pl, act0);
    }
    SWJ_CUDA_TRY(cudaStreamWaitEvent(st, evJoin, 0));
    SWJ_COUNT_LAUNCH();
    k_diag_corr<<<nblk(c->T, kFp64Block), kFp64Block, 0, st>>>(N, M, pl.P, c->partial, c->pc_sumK3);
    // --- band of S for every instance: D (shared) minus G / F^2 on the diagonal blocks
    const size_t bst = band_stride(c);
    double *sep0 = sh.nd ? c->pc_nd_buf + 2 * (size_t)nv * Mv * n1 : nullptr;   // D's separator blocks
    const size_t vsm = (size_t)2 * (2 * N - 2) * sizeof(double);   // the fill kernels' value table
    if (vsm > 48 * 1024) {                                           // N > 1537
        SWJ_CUDA_TRY(cudaFuncSetAttribute(k_fill_D, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
        SWJ_CUDA_TRY(cudaFuncSetAttribute(k_fill_S_two_sided, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
    }
    if (sh.nd) {
        SWJ_COUNT_LAUNCH();
        k_fill_S_two_sided<<<2 * Mv * nbs, 256, vsm, st>>>(N, M, h, Mv, sh.dB, m.x1, m.dx, m.dy, m.n_rad,
                                                            c->pc_sumK3, c->pc_k3, c->pc_G1, c->pc_invF2,
                                                            c->pc_band);
        SWJ_COUNT_LAUNCH();
        k_sep_blocks<<<2 * c->num_sms, 256, 0, st>>>(n1, h, Mv, c->pc_band, bst, sep0, 0);
    } else {
        SWJ_COUNT_LAUNCH();
        k_fill_D<<<M * nbs, 256, vsm, st>>>(N, M, h, m.x1, m.dx, m.dy, m.n_rad, c->pc_sumK3, c->pc_k3,
                                            c->pc_band);
        if (nb > 1) {
            SWJ_COUNT_LAUNCH();
            k_replicate<<<dim3(2 * c->num_sms, nb - 1), 256, 0, st>>>(bst, c->pc_band, c->pc_band, bst);
        }
        SWJ_COUNT_LAUNCH();
        k_sub_G<<<dim3(nblk((long)M * n2, 256) < 4096 ? nblk((long)M * n2, 256) : 4096, nb), 256, 0, st>>>(
            n1, M, h, c->pc_G1, c->pc_invF2, c->pc_band, bst);
    }
    // --- block LU of every band instance, step by step
    SWJ_CUDA_TRY(cudaMemsetAsync(c->pc_info, 0, (size_t)nv * Mv * sizeof(int), st));
    int rc;
    if (h == 0) {
        // all M diagonal blocks of all instances are independent
        if (gj_inplace) {
            rc = swj_gj_inverse_cluster(st, n1, nb * M, c->pc_band, n2, c->pc_band, n2, c->pc_info,
                                        swj_waits(c, false).spin_limit);
        } else {
            SWJ_CUDA_TRY(cudaMemcpyAsync(c->pc_work, c->pc_band, (size_t)nb * M * n2 * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
            rc = swj_gj_inverse_cluster(st, n1, nb * M, c->pc_work, n2, c->pc_band, n2, c->pc_info,
                                        swj_waits(c, false).spin_limit);
        }
        if (rc) return rc;
    } else {
        // device pointer triples of the batched GEMMs of every step, all instances,
        // in groups (kmax = min(i + h, M - 1)):
        //   Wc  W_{i,i+1} = inv_i S_{i,i+1}
        //   Uc  S_{i+1,i+1} -= S_{i+1,i} W_{i,i+1}
        //   Wb  W_ik = inv_i S_ik, k = i+2..kmax
        //   B1  S_jk -= S_ji W_ik for (j,k) = (i+1,i+2), (i+2,i+1), (i+2,i+2)
        //   B2  S_jk -= S_ji W_ik for the other j, k = i+1..kmax
        //   L   L_ij = inv_i S_ij, j = i-h..i-1, into the scratch pc_lt
        enum { gWc, gUc, gWb, gB1, gB2, gL, kGroups };
        auto chain_b1 = [&](int i, int j, int k) {
            return (j == i + 1 && k == i + 1) || (j == i + 1 && k == i + 2) || (j == i + 2 && k == i + 1) ||
                   (j == i + 2 && k == i + 2);
        };
        if (!c->pc_plan) {
        PcPlan *plan = new PcPlan();
        c->pc_plan = plan;
        std::vector<const double *> PA, PB;
        std::vector<double *> PC;
        std::vector<int> &off = plan->off, &cnt = plan->cnt;
        off.assign((size_t)Mv * kGroups, 0);
        cnt.assign((size_t)Mv * kGroups, 0);
        auto begin = [&](int i, int g) { off[(size_t)i * kGroups + g] = (int)PA.size(); };
        auto end = [&](int i, int g) {
            cnt[(size_t)i * kGroups + g] = (int)PA.size() - off[(size_t)i * kGroups + g];
        };
        auto add = [&](const double *a, const double *b, double *cc) {
            PA.push_back(a); PB.push_back(b); PC.push_back(cc);
        };
        for (int i = 0; i < Mv; ++i) {
            const int kmax = i + h < Mv - 1 ? i + h : Mv - 1;
            begin(i, gWc);
            for (int q = 0; q < sh.insts(i); ++q)
                if (kmax >= i + 1) add(blk(c, q, i, i), blk(c, q, i, i + 1), wblk(c, q, i, i + 1));
            end(i, gWc);
            begin(i, gUc);
            for (int q = 0; q < sh.insts(i); ++q)
                if (kmax >= i + 1) add(blk(c, q, i + 1, i), wblk(c, q, i, i + 1), blk(c, q, i + 1, i + 1));
            end(i, gUc);
            begin(i, gWb);
            for (int q = 0; q < sh.insts(i); ++q)
                for (int k = i + 2; k <= kmax; ++k) add(blk(c, q, i, i), blk(c, q, i, k), wblk(c, q, i, k));
            end(i, gWb);
            for (int g : {gB1, gB2}) {
                begin(i, g);
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int j = i + 1; j <= kmax; ++j)
                        for (int k = i + 1; k <= kmax; ++k) {
                            if (j == i + 1 && k == i + 1) continue;   // Uc
                            if (chain_b1(i, j, k) != (g == gB1)) continue;
                            add(blk(c, q, j, i), wblk(c, q, i, k), blk(c, q, j, k));
                        }
                end(i, g);
            }
            const int j0 = std::max(0, i - h);
            begin(i, gL);
            for (int q = 0; q < sh.insts(i); ++q)
                for (int j = j0; j < i; ++j)
                    add(blk(c, q, i, i), blk(c, q, i, j), c->pc_lt + ((size_t)q * h + (j - j0)) * n2);
            end(i, gL);
        }
        const int np = (int)PA.size();
        plan->np = np;
        if (c->pc_ptrs_cap < np) {
            if (c->pc_ptrs) {
                cudaFree(c->pc_ptrs);
                c->pc_bytes -= (size_t)3 * c->pc_ptrs_cap * sizeof(double *);
                c->bytes -= (size_t)3 * c->pc_ptrs_cap * sizeof(double *);
            }
            c->pc_ptrs = nullptr;
            if (cudaMalloc(&c->pc_ptrs, (size_t)3 * np * sizeof(double *)) != cudaSuccess) {
                c->pc_ptrs_cap = 0;
                return SWJ_ENOMEM;
            }
            c->pc_ptrs_cap = np;
            c->pc_bytes += (size_t)3 * np * sizeof(double *);
            c->bytes += (size_t)3 * np * sizeof(double *);
        }
        std::vector<double *> all((size_t)3 * np);
        for (int q = 0; q < np; ++q) {
            all[q] = const_cast<double *>(PA[q]);
            all[np + q] = const_cast<double *>(PB[q]);
            all[2 * np + q] = PC[q];
        }
        SWJ_CUDA_TRY(cudaMemcpyAsync(c->pc_ptrs, all.data(), all.size() * sizeof(double *),
                                     cudaMemcpyHostToDevice, st));
        SWJ_CUDA_TRY(cudaStreamSynchronize(st));   // `all` must outlive the copy
        // the sliced path: split lists and product lists of every step (see OzLayout)
        std::vector<OzStep> &zo = plan->zo;
        zo.assign(sliced ? Mv : 0, OzStep{});
        if (sliced) {
            OzLayout &OL = plan->OL;
            OL = oz_layout(n1, sh);
            std::vector<const double *> zp;
            std::vector<int> zs;
            std::vector<OzProd> zq;
            const int hs = h + 1, hb = 3 * h;
            for (int i = 0; i < Mv; ++i) {
                const int kmax = i + h < Mv - 1 ? i + h : Mv - 1, j0 = std::max(0, i - h);
                OzStep &o = zo[i];
                o.a = zp.size();
                for (int q = 0; q < sh.insts(i); ++q) {
                    zp.push_back(blk(c, q, i, i)); zs.push_back(q * hs);
                    for (int j = i + 1; j <= kmax; ++j) { zp.push_back(blk(c, q, j, i)); zs.push_back(q * hs + (j - i)); }
                }
                o.na = (int)(zp.size() - o.a);
                // the factors right (S_ik, k >= i + 2) and left (S_ij, j < i) of the
                // diagonal, one split; their products with inv_i, one batched call
                o.wb = zp.size();
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int k = i + 2; k <= kmax; ++k) { zp.push_back(blk(c, q, i, k)); zs.push_back(q * hb + (k - i - 2)); }
                o.nwb = (int)(zp.size() - o.wb);
                o.l = zp.size();
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int j = j0; j < i; ++j) { zp.push_back(blk(c, q, i, j)); zs.push_back(q * hb + 2 * h + (j - j0)); }
                o.nl = (int)(zp.size() - o.l);
                o.u = zp.size();
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int k = i + 1; k <= kmax; ++k) { zp.push_back(wblk(c, q, i, k)); zs.push_back(q * hb + h + (k - i - 1)); }
                o.nu = (int)(zp.size() - o.u);
                o.pwb = zq.size();
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int k = i + 2; k <= kmax; ++k) zq.push_back({q * hs, q * hb + (k - i - 2), wblk(c, q, i, k), 0});
                o.cwb = (int)(zq.size() - o.pwb);
                // L_ij = inv_i S_ij straight into the band: S_ij was split above, the
                // product reads only the slices
                o.pl = zq.size();
                for (int q = 0; q < sh.insts(i); ++q)
                    for (int j = j0; j < i; ++j) zq.push_back({q * hs, q * hb + 2 * h + (j - j0), blk(c, q, i, j), 0});
                o.cl = (int)(zq.size() - o.pl);
                for (int g = 0; g < 2; ++g) {
                    (g ? o.pb2 : o.pb1) = zq.size();
                    for (int q = 0; q < sh.insts(i); ++q)
                        for (int j = i + 1; j <= kmax; ++j)
                            for (int k = i + 1; k <= kmax; ++k) {
                                if (j == i + 1 && k == i + 1) continue;   // the chain's update
                                if (chain_b1(i, j, k) != (g == 0)) continue;
                                zq.push_back({q * hs + (j - i), q * hb + h + (k - i - 1), blk(c, q, j, k), 1});
                            }
                    (g ? o.cb2 : o.cb1) = (int)(zq.size() - (g ? o.pb2 : o.pb1));
                }
            }
            if (zp.size() != OL.nptr || zq.size() != OL.nprod) return SWJ_EINVAL;   // layout and lists disagree
            char *base = (char *)c->oz_desc;
            const size_t offS = oz_align(OL.nptr * sizeof(double *)), offQ = offS + oz_align(OL.nptr * sizeof(int));
            SWJ_CUDA_TRY(cudaMemcpyAsync(base, zp.data(), zp.size() * sizeof(double *), cudaMemcpyHostToDevice, st));
            SWJ_CUDA_TRY(cudaMemcpyAsync(base + offS, zs.data(), zs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            SWJ_CUDA_TRY(cudaMemcpyAsync(base + offQ, zq.data(), zq.size() * sizeof(OzProd), cudaMemcpyHostToDevice, st));
            SWJ_CUDA_TRY(cudaStreamSynchronize(st));   // the host lists must outlive the copies
        }
        }
        const PcPlan &PL = *(const PcPlan *)c->pc_plan;
        const std::vector<int> &off = PL.off, &cnt = PL.cnt;
        const std::vector<OzStep> &zo = PL.zo;
        const OzLayout &OL = PL.OL;
        const int np = PL.np;
        double **dA = c->pc_ptrs, **dB = c->pc_ptrs + np, **dC = c->pc_ptrs + 2 * np;
        const double *const *zP = nullptr;
        const int *zS = nullptr;
        const OzProd *zQ = nullptr;
        if (sliced) {
            char *base = (char *)c->oz_desc;
            const size_t offS = oz_align(OL.nptr * sizeof(double *)), offQ = offS + oz_align(OL.nptr * sizeof(int));
            zP = (const double *const *)base;
            zS = (const int *)(base + offS);
            zQ = (const OzProd *)(base + offQ);
        }
        // Look-ahead factorisation.  The chain stream (high priority) runs only
        // what the next diagonal block waits for: at step i it inverts S_ii,
        // forms W_{i,i+1} and applies the one update S_{i+1,i+1} -= S_{i+1,i}
        // W_{i,i+1}, then goes on with step i + 1.  The bulk stream forms the
        // other W_ik, first the three updates step i + 1 of the chain reads
        // (B1, event evB1), then all the others (B2), then replaces block row
        // i's left blocks by L_ij = inv_i S_ij (the forward substitution's
        // factors; nothing of the set-up reads them after step i - 1; the
        // sliced path forms them with the W_ik, in one batched call).  The
        // chain waits for B1 of step i - 1 before W_{i,i+1}; every other
        // update a chain product reads was enqueued on the bulk stream before
        // that B1.  Every block receives its updates in the order of the steps,
        // so the factors do not depend on timing.  Events: evW[i % 4] after
        // W_{i,i+1}, evB1[i % 4] after B1 of step i (rings of 4: a wait is
        // always enqueued before its event is recorded again).
        // With SM partitions (two-sided order, opts.sm_partition) the Gauss-Jordan
        // launches run on the chain partition's stream sg at one CTA per SM, the
        // bulk work on the other partition's stream; the chain's two FP64 block
        // products stay on sc, which may use every SM (evG: the inverse of step i
        // is done; evU: the update of S_{i+1,i+1} is done).
        const bool part = c->opts.sm_partition && sh.nd && pc_partitions(c, n1, nv);
        c->pc_chain_sms = part ? c->pc_gsms : 0;
        cudaStream_t sc = c->pc_chain, sb = part ? c->pc_gbulk : c->pc_bulk, sg = part ? c->pc_gchain : sc;
        const size_t gj_smem = part ? kGJOneCtaSmem : 0;
        cudaEvent_t *evW = c->pc_ev, *evB1 = c->pc_ev + 4, evStart = c->pc_ev[8], evEnd = c->pc_ev[9],
                    *evG = c->pc_ev + 12, *evU = c->pc_ev + 16;
        // Output tile of a batched product launch: the largest of 64, 32, 16 that
        // still gives every SM a few CTAs.  One CTA of a 64-wide tile runs for
        // ~0.2 ms on B300's FP64 pipe (two FMAs per clock per SM), so a launch of
        // a few such CTAs leaves most SMs idle; the arithmetic of every output
        // element is the same for all three tiles.
        auto tile_for = [&](int products) {
            const long t64 = (long)products * ((n1 + 63) / 64) * ((n1 + 63) / 64);
            const long t32 = (long)products * ((n1 + 31) / 32) * ((n1 + 31) / 32);
            if (t64 >= 4L * c->num_sms) return 64;
            if (t32 >= 2L * c->num_sms) return 32;
            return 16;
        };
        auto gemm = [&](cudaStream_t s, int i, int g, double alpha, double beta) {
            const int o = off[(size_t)i * kGroups + g], n = cnt[(size_t)i * kGroups + g];
            if (!n) return SWJ_OK;
            swj_dgemm_batched(s, n1, n1, n1, alpha, (const double *const *)(dA + o), n1,
                              (const double *const *)(dB + o), n1, beta, dC + o, n1, n, tile_for(n));
            return SWJ_OK;
        };
        // a bounded wait of the slice GEMM that runs out sets oz_err (checked at the end)
        if (sliced) SWJ_CUDA_TRY(cudaMemsetAsync(c->oz_err, 0, sizeof(int), st));
        // steps [i0, i1) of the factorisation on both streams, joined into st at the end
        auto run_steps = [&](int i0, int i1) -> int {
        if (i0 >= i1) return SWJ_OK;
        int rc = SWJ_OK;
        SWJ_CUDA_TRY(cudaEventRecord(evStart, st));
        SWJ_CUDA_TRY(cudaStreamWaitEvent(sc, evStart, 0));
        SWJ_CUDA_TRY(cudaStreamWaitEvent(sb, evStart, 0));
        if (part) SWJ_CUDA_TRY(cudaStreamWaitEvent(sg, evStart, 0));
        for (int i = i0; i < i1; ++i) {
            double *diag0 = blk(c, 0, i, i);
            const int nq = sh.insts(i);
            if (part && i > i0) SWJ_CUDA_TRY(cudaStreamWaitEvent(sg, evU[(i - 1) % 4], 0));
            if (gj_inplace) {
                rc = swj_gj_inverse_cluster(sg, n1, nq, diag0, bst, diag0, bst, c->pc_info + (size_t)i * nv,
                                            swj_waits(c, false).spin_limit, gj_smem);
            } else {
                SWJ_COUNT_LAUNCH();
                k_copy_blocks<<<dim3(64, nq), 256, 0, sg>>>(n2, diag0, bst, c->pc_work, n2);
                rc = swj_gj_inverse_cluster(sg, n1, nq, c->pc_work, n2, diag0, bst, c->pc_info + (size_t)i * nv,
                                            swj_waits(c, false).spin_limit, gj_smem);
            }
            if (rc) return rc;
            if (part) {
                SWJ_CUDA_TRY(cudaEventRecord(evG[i % 4], sg));
                SWJ_CUDA_TRY(cudaStreamWaitEvent(sc, evG[i % 4], 0));
            }
            if (i >= 1) SWJ_CUDA_TRY(cudaStreamWaitEvent(sc, evB1[(i - 1) % 4], 0));
            if ((rc = gemm(sc, i, gWc, 1.0, 0.0))) return rc;
            SWJ_CUDA_TRY(cudaEventRecord(evW[i % 4], sc));
            if ((rc = gemm(sc, i, gUc, -1.0, 1.0))) return rc;
            if (part) SWJ_CUDA_TRY(cudaEventRecord(evU[i % 4], sc));
            SWJ_CUDA_TRY(cudaStreamWaitEvent(sb, evW[i % 4], 0));
            if (sliced) {
                const OzStep &o = zo[i];
                auto split = [&](bool rows, size_t off, int n_) {
                    return swj_ozaki_split(sb, rows, n1, OL.np, OL.s, OL.beta, n_, zP + off, zS + off,
                                           rows ? c->oz_sa : c->oz_sb, rows ? c->oz_ea : c->oz_eb);
                };
                auto prods = [&](size_t off, int n_, double alpha) {
                    for (int c0 = 0; c0 < n_; c0 += (int)OL.maxP) {
                        const int cc = std::min((int)OL.maxP, n_ - c0);
                        const int r_ = swj_ozaki_products(sb, n1, OL.z, cc, zQ + off + c0,
                                                          c->oz_sa, OL.nsa, c->oz_ea, c->oz_sb, OL.nsb, c->oz_eb,
                                                          alpha, c->oz_P, c->oz_err);
                        if (r_) return r_;
                    }
                    return (int)SWJ_OK;
                };
                // (the plan lists S_ij, j < i, right after S_ik and L_ij right after W_ik)
                if ((rc = split(true, o.a, o.na)) || (rc = split(false, o.wb, o.nwb + o.nl)) ||
                    (rc = prods(o.pwb, o.cwb + o.cl, 1.0)) || (rc = split(false, o.u, o.nu)) ||
                    (rc = prods(o.pb1, o.cb1, -1.0)))
                    return rc;
                SWJ_CUDA_TRY(cudaEventRecord(evB1[i % 4], sb));
                if ((rc = prods(o.pb2, o.cb2, -1.0))) return rc;
                continue;
            }
            if ((rc = gemm(sb, i, gWb, 1.0, 0.0))) return rc;
            if ((rc = gemm(sb, i, gB1, -1.0, 1.0))) return rc;
            SWJ_CUDA_TRY(cudaEventRecord(evB1[i % 4], sb));
            if ((rc = gemm(sb, i, gB2, -1.0, 1.0))) return rc;
            if (cnt[(size_t)i * kGroups + gL]) {
                if ((rc = gemm(sb, i, gL, 1.0, 0.0))) return rc;
                const int nt = std::min(i, h);
                SWJ_COUNT_LAUNCH();
                k_copy_blocks<<<dim3(64, nq), 256, 0, sb>>>((size_t)nt * n2, c->pc_lt, (size_t)h * n2,
                                                            blk(c, 0, i, i - nt), bst);
            }
        }
        SWJ_CUDA_TRY(cudaEventRecord(evEnd, sb));
        SWJ_CUDA_TRY(cudaStreamWaitEvent(st, evEnd, 0));
        SWJ_CUDA_TRY(cudaEventRecord(evEnd, sc));
        SWJ_CUDA_TRY(cudaStreamWaitEvent(st, evEnd, 0));
        if (part) {
            SWJ_CUDA_TRY(cudaEventRecord(evEnd, sg));
            SWJ_CUDA_TRY(cudaStreamWaitEvent(st, evEnd, 0));
        }
        return SWJ_OK;
        };
        // Two-sided order: both halves first (steps 0..split-1 of both band
        // instances), then the separator blocks of instance 0 become D minus the
        // Schur updates of both halves, then instance 0 alone eliminates the
        // separator rows.  Top-down: split = Mv, one phase.
        if ((rc = run_steps(0, sh.split))) return rc;
        if (sh.nd) {
            SWJ_COUNT_LAUNCH();
            k_sep_blocks<<<2 * c->num_sms, 256, 0, st>>>(n1, h, Mv, c->pc_band, bst, sep0, 1);
        }
        if ((rc = run_steps(sh.split, Mv))) return rc;
    }
    std::vector<int> info((size_t)nv * Mv);
    SWJ_CUDA_TRY(cudaMemcpyAsync(info.data(), c->pc_info, info.size() * sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
    int oz_err = 0;
    if (c->oz_err) SWJ_CUDA_TRY(cudaMemcpyAsync(&oz_err, c->oz_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SWJ_CUDA_TRY(cudaStreamSynchronize(st));
    SWJ_CUDA_TRY(cudaGetLastError());
    if (oz_err) return SWJ_ETIMEOUT;
    for (size_t i = 0; i < info.size(); ++i)
        if (info[i] < 0) return SWJ_ETIMEOUT;
        else if (info[i] != 0) return SWJ_ESINGULAR;
    if (h > 0) {
        int rc = swj_band_sweep_cluster(st, nv, n1, Mv, h, c->pc_band, band_stride(c), c->pc_W,
                                        (size_t)Mv * h * n2, c->pc_z, (size_t)Mv * n1, c->pc_t2,
                                        (size_t)Mv * n1, nullptr, true);
        if (rc) return rc;
    }
    // one instance: the multi-cluster apply where the device holds its h
    // clusters, after one trial solve (of t = 0) shows that the launch forms
    // them
    //  (two-sided order: both halves at once where ni + h - 1 = h + 1 clusters fit,
    //  else one half at a time)
    //  (a launch with empty row ranges only checks that the clusters form; it
    //  runs at every set-up, since a profiler that replays launches one by one
    //  may break them up at any time)
    c->pc_mc = 0;
    if (c->pc_mc_buf && swj_band_sweep_mc(st, n1, Mv, h, c->pc_band, c->pc_W, nullptr, nullptr, nullptr, nullptr,
                                          nullptr, nullptr, true) == SWJ_OK) {
        int best = 1;
        if (sh.nd && swj_band_sweep_mc_ranges(st, n1, Mv, h, 2, nullptr, 0, nullptr, 0, nullptr, nullptr, nullptr,
                                              0, nullptr, nullptr, 0, nullptr, true, 0, 0, -1, 0) == SWJ_OK)
            best = 2;
        const size_t per = (size_t)Mv * n1, sst = per * (h + 1);
        double *zv = c->pc_mc_buf, *cf = zv + nv * per, *cb = cf + nv * sst;
        for (int mode = best; mode >= 1 && !c->pc_mc; --mode) {
            const int ni = mode == 2 ? 2 : 1;
            SWJ_CUDA_TRY(cudaMemsetAsync(c->pc_mc_err, 0, sizeof(int), st));
            int rc = swj_band_sweep_mc_ranges(st, n1, Mv, h, ni, c->pc_band, bst, c->pc_W, (size_t)Mv * h * n2,
                                              c->pc_z, zv, zv, per, cf, cb, sst, c->pc_mc_err, false, 0, 0, -1, 0,
                                              swj_waits(c, false));
            int err = 1;
            if (rc == SWJ_OK) {
                SWJ_CUDA_TRY(cudaMemcpyAsync(&err, c->pc_mc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
                SWJ_CUDA_TRY(cudaStreamSynchronize(st));
            }
            if (rc == SWJ_OK && err == 0) c->pc_mc = sh.nd ? mode : 1;
        }
        SWJ_CUDA_TRY(cudaMemsetAsync(c->pc_mc_err, 0, sizeof(int), st));
    }
    c->pc_ready = 1;
    return SWJ_OK;
}

// SWJ_ETIMEOUT if a wait of the multi-cluster apply gave up since the set-up
// (synchronises the stream)
int swj_pc_status(swj_ctx *c)
{
    if (!c->pc_mc) return SWJ_OK;
    int err = 0;
    SWJ_CUDA_TRY(cudaMemcpyAsync(&err, c->pc_mc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return err ? SWJ_ETIMEOUT : SWJ_OK;
}

int swj_pc_apply(swj_ctx *c, const double *b, double *r, const int *act)
{
    const int M = c->M, n1 = c->n1, H = c->H, h = c->pc_h, nb = c->nb;
    const size_t nu = c->nu;
    cudaStream_t st = c->stream;
    const size_t n2 = (size_t)n1 * n1;
    double *t1 = c->pc_t1, *t2 = c->pc_t2;
    // t2 = b2 - C A^-1 b1 ; t1 = A^-1 b1   (per-row vectors are the rows of M x n1 matrices)
    SWJ_COUNT_LAUNCH();
    k_copy_vec<<<dim3(nblk(H, 256), nb), 256, 0, st>>>(H, b + H, nu, t2, H, act);
    rowdot(c, b, nu, c->pc_CAinv, -1.0, nullptr, 1.0, t2, H, act);
    rowdot(c, b, nu, c->pc_Ainv, 1.0, nullptr, 0.0, t1, H, act);
    // s2 = S^-1 t2 into r2 (= r + H of every instance)
    int rc = SWJ_EINVAL;
    if (c->pc_mc) {
        rc = c->pc_nd ? nd_solve(c, t2, r + H, c->pc_mc) : mc_solve(c, r + H);
        if (rc == SWJ_EINVAL) c->pc_mc = 0;   // the launch was refused: one cluster from now on
        else if (rc) return rc;
    }
    if (rc && c->pc_nd) {
        rc = nd_solve(c, t2, r + H, 0);
        if (rc) return rc;
    } else if (rc) {
        rc = swj_block_p(st, nb, n1, M, h, c->pc_band, band_stride(c), t2, H, h ? c->pc_z : r + H,
                         h ? H : nu, act);
        if (rc) return rc;
        if (h > 0) {
            rc = swj_band_sweep_cluster(st, nb, n1, M, h, c->pc_band, band_stride(c), c->pc_W,
                                        (size_t)M * h * n2, c->pc_z, H, r + H, nu, act);
            if (rc) return rc;
        }
    }
    // r1 = A^-1 b1 - (A^-1 B) s2, A^-1 B = (A^-1 B at F = 1) / F^2
    rowdot(c, r + H, nu, c->pc_AinvB1, -1.0, c->pc_invF2, 1.0, t1, H, act);
    SWJ_COUNT_LAUNCH();
    k_copy_vec<<<dim3(nblk(H, 256), nb), 256, 0, st>>>(H, t1, H, r, nu, act);
    return SWJ_OK;
}
