// Internal declarations of libswj: the context, device buffers and the
// launch wrappers of each kernel family.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "../../include/swj.h"

#define SWJ_VERSION_STRING "swj 0.1 (sm_103a)"

// ---------------------------------------------------------------- records
// Source record of the all-pairs sum (one per mesh node (i, j)), lengths in
// units of L = dy (rho = dx / dy):
//   x = i rho, y = j (exact when rho is a short binary fraction, e.g. 1),
//   zeta = zeta_ij / L, zx, zy = slopes, g = g_ij, w = rho c_i c_j (= w(i,j) / L^2),
//   zxw = L (zeta_x)_ij.
// With r' = r / L the pair term w [(g - g*) K1 + zx K2 - zx* S2] equals
// w' [(g - g*) K1' + zxw K2' - zxw* S2'] where K1', K2', S2' are the kernels
// evaluated in these units, so no coordinate is rescaled per pair and every
// coordinate difference is exact.
template <typename T> struct SrcRecS {
    T x, y, zeta, zx, zy, g, w, zxw;
};

// Target arrays in the same units, structure of arrays of length T each:
// x = (k + 1/2) rho, y = l, zeta* / L, g*, L zeta_x*, and the dimensionless
// A = 1 + zx*^2, B = 2 zx* zy*, C = 1 + zy*^2.
template <typename T> struct TgtArraysS {
    T *x, *y, *zeta, *g, *zxw, *A, *B, *C;
};

typedef SrcRecS<float> SrcRec32;
typedef TgtArraysS<float> TgtArrays32;
typedef SrcRecS<double> SrcRec64;
typedef TgtArraysS<double> TgtArrays64;

struct PairPlan {
    int tpb;      // threads per block
    int R;        // targets per thread
    int P;        // source chunks (grid.y)
    int chunk;    // sources per chunk
    int tiles;    // target tiles (grid.x)
};

// ---------------------------------------------------------------- context
struct swj_ctx {
    swj_mesh mesh;
    double F, eps;
    swj_opts opts;
    cudaStream_t stream;
    int dev, num_sms;

    int N, M;          // mesh
    int n1;            // N + 1 (block size)
    int H;             // (N + 1) M (half of the unknowns)
    int nu;            // 2 (N + 1) M
    int T;             // (N - 1) M targets
    int S;             // N M sources

    // mesh step (FP64), node arrays [M][N]
    double *zeta, *g, *zetay, *gy;
    double *spl_cp, *spl_a, *spl_inv;   // Thomas coefficients along y (M each)
    // per-target E2 terms that do not need the pair sum: 2 pi g* + src - zx* I
    double *e2part;
    double *Ival;      // I per target (diagnostics)
    // records for the two precisions
    SrcRec64 *src64;
    SrcRec32 *src32;
    TgtArrays64 tgt64;
    TgtArrays32 tgt32;
    double *tgt64_base; float *tgt32_base;
    // partial sums [P][T]
    double *partial;
    size_t partial_cap;   // doubles
    PairPlan plan64, plan32;

    // JVP / solver temporaries (length nu)
    double *u_tmp, *E_tmp;           // JVP: u + h v and E(u + h v)
    double *E_cur, *u_try, *E_try;   // Newton: current residual, line-search trial
    double *E_base32;                // MIXED refinement: FP32 residual at u (JVP base)
    double *du, *rvec;               // Newton step, GMRES right-hand side
    double *dscal;        // device scalars (norms, FD step, Arnoldi coefficients)
    double *red;          // reduction scratch
    double *hpin;         // pinned host mirror of device scalars

    // Krylov basis (m + 1) x nu and preconditioned basis m x nu
    double *V, *Z;
    int kry_m;

    // preconditioner
    int pc_ready, pc_h, pc_nb;   // built flag, block half bandwidth, blocks per band row
    double *pc_Ainv, *pc_AinvB, *pc_CAinv, *pc_G, *pc_A, *pc_B, *pc_C, *pc_tmp;
    double *pc_band;             // [M][2h+1][n1][n1]
    double *pc_sumK3;            // [T] sum_s w K3 (flat-state trapezoid sum)
    int *pc_info;                // device status of the factorisation
    double **pc_ptrs;            // device pointer arrays for batched block GEMMs
    int pc_ptrs_cap;
    double *pc_t1, *pc_t2;       // apply temporaries [H]
    double *pc_work;             // Gauss-Jordan work copy: M blocks (h = 0) or one block
    double *pc_W;                // W_ik = inv_i S_ik, [M][h][n1][n1]
    double *pc_z;                // z_i = inv_i y_i of the forward sweep [H]

    size_t bytes;                // device bytes held
    cudaEvent_t ev0, ev1;
    // optional timing of every all-pairs launch (events on the context's stream)
    int time_pairs;
    int n_timed;
    cudaEvent_t *tev;            // 2 * SWJ_MAX_TIMED events, created on first enable
    int *tev_prec;               // precision of each timed launch (host array)
};

// ---------------------------------------------------------------- launches
// mesh.cu
void swj_launch_mesh_step(swj_ctx *c, const double *u, double *E);
void swj_launch_assemble(swj_ctx *c, double *E, int P);
void swj_spline_coeffs(int M, double *cp, double *a, double *inv);  // host helper
void swj_launch_flat(swj_ctx *c, double *u);
void swj_launch_unpack(swj_ctx *c, const double *u, double *zeta_out, double *phi_out);
void swj_launch_surface(swj_ctx *c, double *out);

// pairs.cu
PairPlan swj_pair_plan(const swj_ctx *c, int precision);
void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl);
void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl);

// linalg.cu
void swj_axpby(cudaStream_t st, int n, double a, const double *x, double b, double *y);      // y = a x + b y
void swj_axpy_dev(cudaStream_t st, int n, const double *a_dev, double a_scale,
                  const double *x, double *y);                                             // y += (a_scale * *a_dev) x
void swj_scale_dev(cudaStream_t st, int n, const double *num_dev, double *x, int invert);  // x *= *num (or 1/ *num)
void swj_copy(cudaStream_t st, int n, const double *x, double *y);
void swj_fill(cudaStream_t st, int n, double v, double *x);
// out[0] = ||x||_2^2, out[1] = ||x||_inf (NaN if any entry is NaN/Inf)
void swj_norms(cudaStream_t st, int n, const double *x, double *red, double *out);
// out[r] = sum_i V[r*ld + i] w[i], r = 0..rows-1
void swj_mdot(cudaStream_t st, int n, int rows, const double *V, size_t ld, const double *w,
              double *red, double *out);
// w -= sum_r coef[r] V[r*ld + :]
void swj_mgemv_sub(cudaStream_t st, int n, int rows, const double *V, size_t ld,
                   const double *coef, double *w);
// x = sum_r coef_host[r] Z[r*ld + :]  (coefficients from host)
void swj_combine(cudaStream_t st, int n, int rows, const double *Z, size_t ld,
                 const double *coef_dev, double *x, int accumulate);
// C(mxn) = alpha A(mxk) B(kxn) + beta C, row-major with leading dims; batched by pointer arrays
void swj_dgemm_batched(cudaStream_t st, int m, int n, int k, double alpha,
                       const double *const *A, int lda, const double *const *B, int ldb,
                       double beta, double *const *C, int ldc, int batch);
void swj_dgemm(cudaStream_t st, int m, int n, int k, double alpha, const double *A, int lda,
               const double *B, int ldb, double beta, double *C, int ldc);
// in-place inverse of `count` n x n blocks (stride `stride` doubles) by Gauss-Jordan with
// partial pivoting; info[b] = 0 or 1 + failing column.
void swj_block_inverse(cudaStream_t st, int n, int count, double *blocks, size_t stride, int *info);

// cluster.cu
int swj_gj_inverse_cluster(cudaStream_t st, int n, int count, double *work, size_t wstride,
                           double *out, size_t ostride, int *info);
int swj_band_sweep_cluster(cudaStream_t st, int n1, int M, int h, const double *band,
                           const double *W, double *y, double *z, double *x);

// precond.cu
int swj_pc_setup(swj_ctx *c);
int swj_pc_apply(swj_ctx *c, const double *b, double *r);
void swj_pc_free(swj_ctx *c);

// solver.cu
int swj_residual_impl(swj_ctx *c, const double *u, double *E, int precision);
int swj_jvp_impl(swj_ctx *c, const double *u, const double *Eu, const double *v, double *Jv,
                 int precision, double h_fixed);
int swj_solve_impl(swj_ctx *c, double *u, swj_stats *st);

// Running count of kernel launches issued by the library (all contexts;
// not synchronised across host threads).
extern unsigned long long g_swj_launches;
#define SWJ_COUNT_LAUNCH() (++g_swj_launches)

#define SWJ_MAX_TIMED 2048   // pair-kernel launches whose duration can be recorded

#define SWJ_CUDA_TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return SWJ_ECUDA; } while (0)
