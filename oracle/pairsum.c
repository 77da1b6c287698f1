/*
 * oracle/pairsum.c -- plain FP64 CPU evaluation of the discretised
 * boundary-integral sum of the nonlinear ship-wave residual.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the CPU oracle that the
 * tests, the smoke check and the CPU-baseline leg of the benchmark use to
 * check the CUDA path.  Nothing in the product library calls, links or
 * shares code with it.
 *
 * What it computes (Section 3, after Eq. S2/IS2, with the kernels K1, K2 of
 * Eq. IntegroEqn and S2 of Eq. S2, discretised by the trapezoidal rule):
 *
 *   for every half-mesh target (x*_k, y*_l), k = 1..N-1, l = 1..M,
 *     sum_{i=1..N} sum_{j=1..M} w(i,j) [ (g_ij - g*) K1 + zx_ij K2 - zx* S2 ]
 *
 * with g = phi - x (so that phi - phi* - x + x* = g - g*), w(i,j) the
 * trapezoidal product weights, and
 *   K1 = (dz - dx zx_ij - dy  zy_ij) / r1^3 + (dz - dx zx_ij - dy' zy_ij) / r2^3
 *   K2 = 1/r1 + 1/r2
 *   S2 = (A dx^2 + B dx dy + C dy^2)^(-1/2) + (A dx^2 - B dx dy' + C dy'^2)^(-1/2)
 *   dx = x_i - x*, dy = y_j - y*, dy' = y_j + y*, dz = zeta_ij - zeta*,
 *   r1^2 = dx^2 + dy^2 + dz^2,  r2^2 = dx^2 + dy'^2 + dz^2,
 *   A = 1 + zx*^2, B = 2 zx* zy*, C = 1 + zy*^2  (target values).
 *
 * Readings of the paper used here:
 *  - the image part of K1 has (y + y*)^2 in its denominator (the printed
 *    (y - y*)^2 is read as a typo: K2's and S2's image parts and the mirror
 *    argument both require y + y*);
 *  - zeta_x, zeta_y inside K1 are the slopes at the integration (source)
 *    point (x_i, y_j): they belong to the normal of the integration surface;
 *  - w(i,j) = dx dy c_i c_j with c = 1/2 on the first and last index in each
 *    direction and 1 elsewhere (product trapezoidal rule).
 *
 * Everything is IEEE double with plain left-to-right accumulation over the
 * sources in (j, i) order; targets are independent and run in parallel with
 * OpenMP when it is enabled at compile time.
 */
#include <math.h>
#include <complex.h>

/* The three kernel values of one (source, target) pair.  Exposed so the
 * tests can pin each kernel against its geometric definition. */
void oracle_pair_kernels(double dx, double dy, double dyp, double dz,
                         double zx_s, double zy_s,
                         double A, double B, double C, double out[3])
{
    double r1 = sqrt(dx * dx + dy * dy + dz * dz);
    double r2 = sqrt(dx * dx + dyp * dyp + dz * dz);
    double K1 = (dz - dx * zx_s - dy * zy_s) / (r1 * r1 * r1)
              + (dz - dx * zx_s - dyp * zy_s) / (r2 * r2 * r2);
    double K2 = 1.0 / r1 + 1.0 / r2;
    double S2 = 1.0 / sqrt(A * dx * dx + B * dx * dy + C * dy * dy)
              + 1.0 / sqrt(A * dx * dx - B * dx * dyp + C * dyp * dyp);
    out[0] = K1;
    out[1] = K2;
    out[2] = S2;
}

/*
 * Grid values are [M][N] row-major (index j*N + i), target values are
 * [M][N-1] row-major (index l*(N-1) + k).  Outputs, per target:
 *   sum[t]  = the trapezoidal sum above,
 *   asum[t] = sum over sources of |w (g-g*) K1| + |w zx K2| + |w zx* S2|
 *             (the scale that the parity tolerance is measured against).
 */
static void one_target(int t, int N, int M, double x1, double dxm, double dym,
                       const double *zeta, const double *zetax,
                       const double *zetay, const double *g,
                       const double *zeta_t, const double *zetax_t,
                       const double *zetay_t, const double *g_t,
                       double *sum_out, double *asum_out)
{
    int k = t % (N - 1);
    int l = t / (N - 1);
    double xt = x1 + ((double)k + 0.5) * dxm;
    double yt = (double)l * dym;
    double zt = zeta_t[t], zxt = zetax_t[t], zyt = zetay_t[t], gt = g_t[t];
    double A = 1.0 + zxt * zxt;
    double B = 2.0 * zxt * zyt;
    double C = 1.0 + zyt * zyt;
    double s = 0.0, a = 0.0;
    for (int j = 0; j < M; ++j) {
        double yj = (double)j * dym;
        double cj = (j == 0 || j == M - 1) ? 0.5 : 1.0;
        for (int i = 0; i < N; ++i) {
            double xi = x1 + (double)i * dxm;
            double ci = (i == 0 || i == N - 1) ? 0.5 : 1.0;
            double w = dxm * dym * ci * cj;
            int p = j * N + i;
            double kv[3];
            oracle_pair_kernels(xi - xt, yj - yt, yj + yt, zeta[p] - zt,
                                zetax[p], zetay[p], A, B, C, kv);
            double t1 = w * (g[p] - gt) * kv[0];
            double t2 = w * zetax[p] * kv[1];
            double t3 = w * zxt * kv[2];
            s += t1 + t2 - t3;
            a += fabs(t1) + fabs(t2) + fabs(t3);
        }
    }
    *sum_out = s;
    *asum_out = a;
}

void oracle_pairsum(int N, int M, double x1, double dxm, double dym,
                    const double *zeta, const double *zetax,
                    const double *zetay, const double *g,
                    const double *zeta_t, const double *zetax_t,
                    const double *zetay_t, const double *g_t,
                    double *sum, double *asum)
{
    int T = (N - 1) * M;
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < T; ++t)
        one_target(t, N, M, x1, dxm, dym, zeta, zetax, zetay, g, zeta_t, zetax_t,
                   zetay_t, g_t, &sum[t], &asum[t]);
}

/* The same sum for the listed targets only (tidx[q], q < nt); outputs are
 * indexed by q. */
void oracle_pairsum_targets(int N, int M, double x1, double dxm, double dym,
                            const double *zeta, const double *zetax,
                            const double *zetay, const double *g,
                            const double *zeta_t, const double *zetax_t,
                            const double *zetay_t, const double *g_t,
                            int nt, const int *tidx, double *sum, double *asum)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nt; ++q)
        one_target(tidx[q], N, M, x1, dxm, dym, zeta, zetax, zetay, g, zeta_t,
                   zetax_t, zetay_t, g_t, &sum[q], &asum[q]);
}

/*
 * Complex-step form of the same sum, for the exact directional derivative:
 * every grid and target value is a complex number (arrays of interleaved
 * re, im pairs, the layout of C99 double complex).  The kernels K1, K2, S2
 * are analytic in every value, so for inputs u + i h v with h tiny,
 * Im(sum) / h equals d sum(u + t v) / dt at t = 0 to rounding (the
 * complex-step derivative; no subtractive cancellation).  aim[t] is the sum
 * over sources of |Im| of the three terms, the scale of the derivative.
 */
static void one_target_cs(int t, int N, int M, double x1, double dxm, double dym,
                          const double complex *zeta, const double complex *zetax,
                          const double complex *zetay, const double complex *g,
                          const double complex *zeta_t, const double complex *zetax_t,
                          const double complex *zetay_t, const double complex *g_t,
                          double complex *sum_out, double *aim_out)
{
    int k = t % (N - 1);
    int l = t / (N - 1);
    double xt = x1 + ((double)k + 0.5) * dxm;
    double yt = (double)l * dym;
    double complex zt = zeta_t[t], zxt = zetax_t[t], zyt = zetay_t[t], gt = g_t[t];
    double complex A = 1.0 + zxt * zxt;
    double complex B = 2.0 * zxt * zyt;
    double complex C = 1.0 + zyt * zyt;
    double complex s = 0.0;
    double a = 0.0;
    for (int j = 0; j < M; ++j) {
        double yj = (double)j * dym;
        double cj = (j == 0 || j == M - 1) ? 0.5 : 1.0;
        for (int i = 0; i < N; ++i) {
            double xi = x1 + (double)i * dxm;
            double ci = (i == 0 || i == N - 1) ? 0.5 : 1.0;
            double w = dxm * dym * ci * cj;
            int p = j * N + i;
            double dx = xi - xt, dy = yj - yt, dyp = yj + yt;
            double complex dz = zeta[p] - zt;
            double complex r1 = csqrt(dx * dx + dy * dy + dz * dz);
            double complex r2 = csqrt(dx * dx + dyp * dyp + dz * dz);
            double complex K1 = (dz - dx * zetax[p] - dy * zetay[p]) / (r1 * r1 * r1)
                              + (dz - dx * zetax[p] - dyp * zetay[p]) / (r2 * r2 * r2);
            double complex K2 = 1.0 / r1 + 1.0 / r2;
            double complex S2 = 1.0 / csqrt(A * dx * dx + B * dx * dy + C * dy * dy)
                              + 1.0 / csqrt(A * dx * dx - B * dx * dyp + C * dyp * dyp);
            double complex t1 = w * (g[p] - gt) * K1;
            double complex t2 = w * zetax[p] * K2;
            double complex t3 = w * zxt * S2;
            s += t1 + t2 - t3;
            a += fabs(cimag(t1)) + fabs(cimag(t2)) + fabs(cimag(t3));
        }
    }
    *sum_out = s;
    *aim_out = a;
}

void oracle_pairsum_cs(int N, int M, double x1, double dxm, double dym,
                       const double complex *zeta, const double complex *zetax,
                       const double complex *zetay, const double complex *g,
                       const double complex *zeta_t, const double complex *zetax_t,
                       const double complex *zetay_t, const double complex *g_t,
                       double complex *sum, double *aim)
{
    int T = (N - 1) * M;
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < T; ++t)
        one_target_cs(t, N, M, x1, dxm, dym, zeta, zetax, zetay, g, zeta_t, zetax_t,
                      zetay_t, g_t, &sum[t], &aim[t]);
}
