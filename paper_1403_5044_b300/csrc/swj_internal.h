// Internal declarations of libswj: the context, device buffers and the
// launch wrappers of each kernel family.  Not part of the public ABI.
//
// A context holds nb >= 1 instances of one mesh, each with its own (F, eps)
// and its own unknowns, residual, Krylov space and preconditioner factors.
// Every per-instance buffer is nb consecutive copies with a fixed stride, and
// every kernel runs over all instances at once (the instance index is a grid
// dimension).  A device array of per-instance flags (`act`, nullable = all)
// lets converged instances drop out without changing any launch shape, so a
// captured CUDA graph stays valid whatever the mix of active instances.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <stdint.h>
#include <stddef.h>
#include "../../include/swj.h"

#define SWJ_VERSION_STRING "swj 0.2 (sm_103a)"

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

// Target arrays in the same units, structure of arrays (each field holds nb
// blocks of T values): x = (k + 1/2) rho, y = l, zeta* / L, g*, L zeta_x*, and
// the dimensionless A = 1 + zx*^2, B = 2 zx* zy*, C = 1 + zy*^2.
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
    int v;        // compiled tile shape (index into the variant table)
};

// One FP64 block product of the sliced (tensor-core) path, ozaki.cu:
// C = alpha A_slot(a) B_slot(b) (+ C when accumulate)
struct OzProd {
    int a, b;
    double *C;
    int accumulate;
};

// is instance `inst` active (act = device flags, or nullptr for all)
#define SWJ_INST_ACTIVE(act, inst) ((act) == nullptr || (act)[inst] != 0)

// ---------------------------------------------------------------- context
struct swj_ctx {
    swj_mesh mesh;
    swj_opts opts;
    cudaStream_t stream;
    int dev, num_sms;

    int nb;            // instances
    double *F, *eps;   // host, per instance
    double *Fd, *epsd; // device copies
    int *act_d;        // device per-instance flags (1 = active)
    int *act_h;        // pinned host mirror

    int N, M;          // mesh
    int n1;            // N + 1 (block size)
    int H;             // (N + 1) M (half of the unknowns)
    int nu;            // 2 (N + 1) M
    int T;             // (N - 1) M targets
    int S;             // N M sources

    // mesh step (FP64), node arrays [nb][M][N]
    double *zeta, *g, *zetay, *gy;
    double *spl_cp, *spl_a, *spl_inv;   // Thomas coefficients along y (M each, shared)
    // per-target E2 terms that do not need the pair sum: 2 pi g* + src - zx* I  [nb][T]
    double *e2part;
    double *Ival;      // I per target (diagnostics)  [nb][T]
    // records for the two precisions, [nb][S] / fields of [nb][T]
    SrcRec64 *src64;
    SrcRec32 *src32;
    TgtArrays64 tgt64;
    TgtArrays32 tgt32;
    double *tgt64_base; float *tgt32_base;
    // partial sums [nb][P][T]
    double *partial;
    size_t partial_cap;   // doubles
    PairPlan plan64, plan32, planff;
    int tuned64, tuned32, tunedff;   // plan settled (autotuned or taken from the process cache)

    // JVP / solver temporaries, [nb][nu]
    double *u_tmp, *E_tmp;           // JVP: u + h v and E(u + h v)
    double *hs_buf;                  // swj_solve_host staging: u [nu], zeta [S], phi [S] (first call)
    double *u_tmp2, *E_tmp2;         // central-difference JVP: u - h v and E(u - h v)
    double *E_cur, *u_try, *E_try;   // Newton: current residual, line-search trial
    double *E_base32;                // MIXED refinement: FP32 residual at u (JVP base)
    double *du, *rvec;               // Newton step, GMRES right-hand side
    double *dscal;        // device scalars [nb][SWJ_DS]
    double *red;          // reduction scratch [nb][SWJ_RED]
    double *hpin;         // pinned host mirror of dscal

    // Krylov bases [nb][m + 1][nu] and preconditioned [nb][m][nu]
    double *V, *Z;
    int kry_m;
    // captured Arnoldi steps, one per Krylov index and per kind of linear solve
    // (FP64 Newton, FP32 Newton, FP32-JVP refinement), valid for one address of u
    cudaGraphExec_t *arn_graph;   // [3][kry_m], null until captured
    const double *arn_u;          // the u the graphs were captured with
    int graphs_enabled;

    // preconditioner: blocks that do not depend on F are shared, the factors are per instance
    int pc_ready, pc_h, pc_nb;   // built flag, block half bandwidth, blocks per band row
    double *pc_Ainv, *pc_AinvB1, *pc_CAinv, *pc_G1, *pc_A, *pc_B1, *pc_C;   // (n1 x n1), "1" = at F = 1
    double *pc_invF2;            // [nb] 1 / F^2 (scales B, G, A^-1 B)
    // Block rows of the factors: pc_nv band instances of pc_M block rows.  Top-down
    // order: pc_nv = nb, pc_M = M.  Two-sided order (pc_nd, one instance, M - h = mt + mb
    // with mt = mb or mb + 1): band instance 0 holds block rows 0..mt+h-1 (the top half
    // and the h separator rows), instance 1 holds rows M-1 down to mt (the bottom half
    // and the separator rows, reversed) after pc_dB = mt - mb padding rows; pc_split = mt
    // is the first step that instance 0 takes alone (pc_M when top-down).
    int pc_nd, pc_M, pc_nv, pc_dB, pc_split;
    double *pc_band;             // [pc_nv][pc_M][2h+1][n1][n1]
    double *pc_W;                // [pc_nv][pc_M][h][n1][n1]  W_ik = inv_i S_ik
    double *pc_sumK3;            // [T] PreD correction (flat-state sums; F-independent)
    int *pc_info;                // [pc_nv][pc_M] status of the block inverses
    double *pc_k3;               // [2N-2][2M-1] kernel values of D's entries (set-up scratch)
    double *pc_nd_buf;           // two-sided apply: right-hand sides and solutions [2][pc_M][n1],
                                 // separator blocks of D [h][h][n1][n1], separator sums [h][n1]
    double **pc_ptrs;            // device pointer arrays for batched block GEMMs
    void *pc_plan;               // host plan of the band LU's block products (precond.cu)
    int pc_ptrs_cap;
    double *pc_t1, *pc_t2, *pc_z;   // apply temporaries [nb][H]
    double *pc_work;             // Gauss-Jordan work copies [nb][(h == 0 ? M : 1)][n1][n1]
    // look-ahead factorisation: the critical chain (Gauss-Jordan, W, next block row)
    // on a high-priority stream, the other Schur updates on a low-priority one
    cudaStream_t pc_chain, pc_bulk;
    cudaEvent_t pc_ev[20];
    // SM partitions of the set-up's band LU (opts.sm_partition): green contexts
    // (CUgreenCtx) for the Gauss-Jordan chain and the bulk products, a stream in
    // each; pc_green 1 in use, -1 unavailable, 0 not tried
    void *pc_gctx[2];
    cudaStream_t pc_gchain, pc_gbulk;
    int pc_green;
    int pc_gsms;                 // SMs of the chain partition
    int pc_chain_sms;            // SMs of the chain partition the last set-up used (0: none)
    // multi-cluster apply (one instance): z, then the term slots cf, cb, and the error word
    double *pc_mc_buf;
    int *pc_mc_err;
    int pc_mc;                   // apply on h clusters: 0 no, 1 one instance (or half) per launch, 2 both
    int test_hooks;              // SWJ_TEST_* flags (swj_set_test_hooks)
                                 // halves of the two-sided order in one launch
    double *pc_lt;               // set-up scratch: inv_i S_ij (j < i) of one block row, every instance
    // sliced (bf16 tensor-core) block products of the band LU (lu_products = SWJ_LU_SLICED)
    void *oz_sa, *oz_sb;         // bf16 slices of the A (row-split) and B (column-split) factors
    int *oz_ea, *oz_eb;          // their row / column exponents
    float *oz_P;                 // slice products of one batch of block products
    int *oz_err;                 // set by the slice GEMM when a bounded wait ran out
    void *oz_desc;               // split lists and product lists of every step (device)
    size_t oz_desc_cap;

    // exact JVP (jvp.cu): tangents of the node arrays [4][nb][S] (zeta, g,
    // zeta_y, g_y), of the source records and target arrays (same layouts
    // as the primal ones; x, y, w unused), and of the per-target part of E2
    double *dnode;
    SrcRec64 *tsrc64;
    SrcRec32 *tsrc32;
    double *ttgt64_base;
    float *ttgt32_base;
    TgtArrays64 ttgt64;
    TgtArrays32 ttgt32;
    double *de2part;

    size_t pc_bytes;             // device bytes of the preconditioner buffers
    size_t bytes;                // device bytes held (workspace + preconditioner)
    cudaEvent_t ev0, ev1;
    // optional timing of every all-pairs launch (events on the context's stream)
    int time_pairs;
    int n_timed;
    cudaEvent_t *tev;            // 2 * SWJ_MAX_TIMED events, created on first enable
    int *tev_prec;               // precision of each timed launch (host array)
};

enum { SWJ_DS = 512, SWJ_RED = 64 * 64 + 1024 };

inline bool swj_valid_precision(int p) { return p == SWJ_FP64 || p == SWJ_FP32 || p == SWJ_FF; }
inline PairPlan &swj_plan_of(swj_ctx *c, int prec)
{
    return prec == SWJ_FP64 ? c->plan64 : (prec == SWJ_FF ? c->planff : c->plan32);
}
inline int &swj_tuned_of(swj_ctx *c, int prec)
{
    return prec == SWJ_FP64 ? c->tuned64 : (prec == SWJ_FF ? c->tunedff : c->tuned32);
}

// ---------------------------------------------------------------- launches
// mesh.cu (act: device per-instance flags or nullptr for all)
void swj_launch_mesh_step(swj_ctx *c, const double *u, double *E, const int *act);
// E2 rows = e2part (c->e2part when null) - sum over the P source chunks
void swj_launch_assemble(swj_ctx *c, double *E, int P, const int *act, const double *e2part = nullptr);
void swj_launch_mesh_tangent(swj_ctx *c, const double *v, const int *act);
void swj_launch_resample(swj_ctx *src, const double *u_src, swj_ctx *dst, double *u_dst);
// jvp.cu: Jv = J(u) v exactly (forward-mode derivative of E), all-pairs part in
// `precision` (SWJ_FP64 or SWJ_FP32)
int swj_jvp_exact_impl(swj_ctx *c, const double *u, const double *v, double *Jv, int precision,
                       const int *act);
void swj_spline_coeffs(int M, double *cp, double *a, double *inv);  // host helper
void swj_launch_flat(swj_ctx *c, double *u);
void swj_launch_unpack(swj_ctx *c, const double *u, double *zeta_out, double *phi_out);
void swj_launch_surface(swj_ctx *c, double *out);

// pairs.cu
// plan of the tuned tile shape for this mesh size (the default shape if none yet)
PairPlan swj_pair_plan(const swj_ctx *c, int precision);
PairPlan swj_pair_plan_variant(const swj_ctx *c, int precision, int v);
int swj_pair_max_chunks(const swj_ctx *c);     // largest P over every compiled shape
int swj_pair_autotune(swj_ctx *c, int precision, const int *act);
int swj_pair_variant_info(int precision, int v, int *tpb, int *R, int *packed);
void swj_launch_pairs64(swj_ctx *c, const PairPlan &pl, const int *act);
void swj_launch_pairs32(swj_ctx *c, const PairPlan &pl, const int *act);
void swj_launch_pairs_ff(swj_ctx *c, const PairPlan &pl, const int *act);

// linalg.cu: batched vector operations on nb vectors of length n at stride ld
// (one instance per grid row; act: per-instance flags or nullptr), with
// per-instance scalars in device arrays at stride sstride.
void swj_bcopy(cudaStream_t st, int nb, int n, const double *x, double *y, size_t ld, const int *act);
void swj_bfill(cudaStream_t st, int nb, int n, double v, double *x, size_t ld, const int *act);
// y = a x + y with a = a_scale * a_dev[inst * sstride] (a_dev may be null: a = a_scale)
void swj_baxpy(cudaStream_t st, int nb, int n, const double *a_dev, size_t sstride, double a_scale,
               const double *x, double *y, size_t ld, const int *act);
// y = s x with s = s_scale * s_dev[inst * sstride] (or 1 / that if invert; s_dev null: s_scale)
void swj_bscale(cudaStream_t st, int nb, int n, const double *s_dev, size_t sstride, double s_scale,
                int invert, const double *x, double *y, size_t ld, const int *act);
// out[inst*sstride + 0] = ||x||_2^2, [1] = ||x||_inf (NaN if any entry is NaN/Inf)
void swj_bnorms(cudaStream_t st, int nb, int n, const double *x, size_t ld, double *red,
                double *out, size_t sstride, const int *act);
// out[inst*sstride + r] = <V_inst[r], w_inst>, r < rows; rows of V_inst at ld, V_inst at vstride
void swj_bmdot(cudaStream_t st, int nb, int n, int rows, const double *V, size_t ld, size_t vstride,
               const double *w, size_t wstride, double *red, double *out, size_t sstride, const int *act);
// w_inst -= sum_r coef[inst*sstride + r] V_inst[r]
void swj_bmgemv_sub(cudaStream_t st, int nb, int n, int rows, const double *V, size_t ld,
                    size_t vstride, const double *coef, size_t sstride, double *w, size_t wstride,
                    const int *act);
// x_inst (+)= sum_r coef[inst*sstride + r] Z_inst[r]
void swj_bcombine(cudaStream_t st, int nb, int n, int rows, const double *Z, size_t ld,
                  size_t zstride, const double *coef, size_t sstride, double *x, size_t xstride,
                  int accumulate, const int *act);
// C(mxn) = alpha A(mxk) B(kxn) + beta C, row-major with leading dims; batched by pointer
// arrays; output tiles of `tile` (64, or 32 for small products that must spread over SMs)
void swj_dgemm_batched(cudaStream_t st, int m, int n, int k, double alpha,
                       const double *const *A, int lda, const double *const *B, int ldb,
                       double beta, double *const *C, int ldc, int batch, int tile = 64);   // tile 16, 32 or 64
// Block size of the thread-per-item kernels that run long chains of FP64
// instructions (the per-target closed forms, the residual assembly, the row
// integrations): one-warp blocks spread their few warps over every SM instead
// of a few SMs' sub-partitions (181x61: 344 target warps on 148 SMs rather than
// 86).  Each FP64 warp instruction holds its sub-partition for 64 cycles, so a
// warp's own chain bounds these kernels (targets 57 -> 54.5 us).
constexpr int kFp64Block = 32;
// ozaki.cu: FP64-accurate block products from bf16 slices (see there).
// The digit scheme of n x n products: np = n padded to a multiple of 8, s
// digits of beta bits; the GEMM's nout outputs of one block product, output
// o summing a_p b_(d-p) over p in [p0[o], p1[o]] (T_d of level d = o: p0 = 0,
// p1 = d); order[] lists the outputs by decreasing length (the GEMM's tile
// order).
constexpr int kOzMaxOut = 16;
struct OzScheme {
    int np, beta, s, nout;
    unsigned char d[kOzMaxOut], p0[kOzMaxOut], p1[kOzMaxOut], order[kOzMaxOut];
};
void swj_ozaki_scheme(int n, OzScheme *z);
// Slot layout of both factors, K-major: [np rows (A) or columns (B)][s][np]
// bf16, plus [np] row or column exponents
int swj_ozaki_split(cudaStream_t st, bool by_rows, int n, int np, int s, int beta, int count,
                    const double *const *mats, const int *slots, void *slices, int *ex);
// the count block products prods (device list): the T_d of every product on
// the tensor cores into P (count * s * np^2 floats), then the exact combine
// into each C; err (device word) is set if a bounded wait of the GEMM ran out
int swj_ozaki_products(cudaStream_t st, int n, const OzScheme &z, int count, const OzProd *prods,
                       const void *sa, size_t nsa, const int *ea, const void *sb, size_t nsb, const int *eb,
                       double alpha, float *P, int *err);
// umma.cu: the outputs of every product (tcgen05 bf16 MMAs, FP32
// accumulators; exact for the sliced operands); nsa, nsb: slots in sa, sb
int swj_oz_gemm(cudaStream_t st, const OzScheme &z, int count, const OzProd *prods, const void *sa, size_t nsa,
                const void *sb, size_t nsb, float *P, int *err);
void swj_dgemm(cudaStream_t st, int m, int n, int k, double alpha, const double *A, int lda,
               const double *B, int ldb, double beta, double *C, int ldc);

// cluster.cu
bool swj_gj_inplace(int n);
// Limits of the bounded device waits of the preconditioner kernels, from
// opts.wait_limit (0: the built-in ones), and whether the multi-cluster
// substitution is launched without its helper clusters (test hook).
struct SwjWaits {
    long long spin_limit;   // Gauss-Jordan flag waits
    int poll_limit;         // multi-cluster substitution: polls of another cluster's values
    int no_helpers;
};
constexpr long long kSwjSpinLimit = 1ll << 26;
constexpr int kSwjPollLimit = 1 << 21;
inline SwjWaits swj_waits(const swj_ctx *c, bool hooks)
{
    const int w = c->opts.wait_limit;
    return SwjWaits{w > 0 ? (long long)w : kSwjSpinLimit, w > 0 ? w : kSwjPollLimit,
                    hooks && (c->test_hooks & SWJ_TEST_WITHHOLD_HELPERS) ? 1 : 0};
}
inline SwjWaits swj_default_waits() { return SwjWaits{kSwjSpinLimit, kSwjPollLimit, 0}; }

// min_smem: shared memory per CTA at least (the kernel ignores the rest; the
// set-up's SM partition asks for one CTA per SM)
int swj_gj_inverse_cluster(cudaStream_t st, int n, int count, double *work, size_t wstride,
                           double *out, size_t ostride, int *info, long long spin_limit = kSwjSpinLimit,
                           size_t min_smem = 0);
// clusters of the Gauss-Jordan launch for n x n blocks (with min_smem) that the
// current context's SMs hold at once
int swj_gj_cluster_capacity(int n, size_t min_smem);
// cluster size (16, else 8) for `kern` with `smem` bytes of dynamic shared
// memory per CTA; raises the kernel's shared-memory limit to `smem`
int swj_cluster_for(const void *kern, int threads, size_t smem);

// sweep.cu: the solve S x = t with the band LU factors (see sweep.cu).
// p_i = inv_i t_i for every block row of every active instance; fill1/fill2
// (optional, instance 0's launch) are set to the multi-cluster sweep's
// "not yet written" pattern.
int swj_block_p(cudaStream_t st, int nb, int n1, int M, int h, const double *band, size_t band_stride,
                const double *t, size_t ts, double *p, size_t ps, const int *act,
                double *fill1 = nullptr, size_t nfill1 = 0, double *fill2 = nullptr, size_t nfill2 = 0);
// One cluster per instance: z (p on entry) -> z, then x.  prepare = true only
// settles the kernel's attributes (no launch); call it once before any launch
// that may be captured into a graph.  The forward recurrence covers block rows
// 0..F-1 and the backward one rows Bs..0 (the rows of x above Bs are inputs);
// F = -1, Bs = -2: the whole band.
int swj_band_sweep_cluster(cudaStream_t st, int nb, int n1, int M, int h, const double *band,
                           size_t band_stride, const double *W, size_t w_stride, double *z, size_t zs,
                           double *x, size_t xs, const int *act, bool prepare = false, int F = -1,
                           int Bs = -2);
// One instance on h clusters (a critical one and h - 1 helpers, cooperative
// launch): p -> z -> x.  z, x and cf, cb ([M][h+1][n1]) must hold the "not yet
// written" pattern (swj_block_p's fill) where the launch writes them; err: set
// to 1 when a poll gave up, 2 when the launch did not form clusters of the
// expected size.  SWJ_EINVAL when h < 2 or the device cannot hold h clusters
// at once (nothing launched).
int swj_band_sweep_mc(cudaStream_t st, int n1, int M, int h, const double *band, const double *W,
                      const double *p, double *z, double *x, double *cf, double *cb, int *err,
                      bool prepare = false, SwjWaits waits = swj_default_waits());
// The same for ni = 1 or 2 instances at once (instance q's band, W, vectors and
// term slots at q bst, q wst, q vst, q sst; one critical cluster each, the h - 1
// helper clusters shared) over forward rows F0..F1-1 and backward rows B1 down to
// B0: the rows of z below F0 and of x above B1 are inputs, zs starts from p (pass
// z as p for a launch without forward rows).  SWJ_EINVAL when the device cannot
// hold ni + h - 1 clusters at once (nothing launched); SWJ_ECUDA when the launch
// met an invalidated stream capture.
int swj_band_sweep_mc_ranges(cudaStream_t st, int n1, int M, int h, int ni, const double *band, size_t bst,
                             const double *W, size_t wst, const double *p, double *z, double *x, size_t vst,
                             double *cf, double *cb, size_t sst, int *err, bool prepare, int F0, int F1, int B1,
                             int B0, SwjWaits waits = swj_default_waits());

// precond.cu
int swj_pc_setup(swj_ctx *c);
int swj_pc_apply(swj_ctx *c, const double *b, double *r, const int *act);
int swj_pc_status(swj_ctx *c);   // SWJ_ETIMEOUT if a bounded wait of the apply gave up
void swj_pc_free(swj_ctx *c);
// device bytes the preconditioner of an nb-instance context holds after set-up
size_t swj_pc_bytes(int N, int M, int nb, int block_bw, int lu_products, int lu_order);

// solver.cu
int swj_residual_impl(swj_ctx *c, const double *u, double *E, int precision, const int *act);
// Eu = E(u) in `precision`: forward difference (E(u + h v) - E(u)) / h;
// Eu = nullptr: central difference (E(u + h v) - E(u - h v)) / (2 h)
int swj_jvp_impl(swj_ctx *c, const double *u, const double *Eu, const double *v, double *Jv,
                 int precision, double h_fixed, const int *act);
int swj_solve_impl(swj_ctx *c, double *u, swj_stats *st);
void swj_graphs_free(swj_ctx *c);

// Running count of kernel launches issued by the library (all contexts and
// host threads).
extern std::atomic<unsigned long long> g_swj_launches;
#define SWJ_COUNT_LAUNCH() (g_swj_launches.fetch_add(1, std::memory_order_relaxed))

#define SWJ_MAX_TIMED 2048   // pair-kernel launches whose duration can be recorded

#define SWJ_CUDA_TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return SWJ_ECUDA; } while (0)
