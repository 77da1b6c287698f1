/*
 * swj.h -- C ABI of libswj, a B300 (sm_103a) library for steady nonlinear
 * free-surface flow past a submerged source, solved with the preconditioned
 * Jacobian-free Newton-Krylov method of Pethiyagoda, McCue, Moroney & Back
 * (arXiv 1403.5044).
 *
 * Problem (Section 2): infinite-depth flow with unit upstream speed past a
 * source of strength eps at depth 1 under a free surface z = zeta(x, y);
 * F is the depth Froude number.  Discretisation (Section 3): an N x M mesh
 * x_i = x1 + (i-1) dx, y_j = (j-1) dy (y1 = 0, only y >= 0 is meshed), the
 * 2(N+1)M unknowns
 *     u = [phi_{1,l}, (phi_x)_{1..N,l}]_{l=1..M}, [zeta_{1,l}, (zeta_x)_{1..N,l}]_{l=1..M}
 * (Eq. unknowns) and the 2(N+1)M equations E(u) = 0 ordered as
 *     [E3_l, E4_l, E1_{1..N-1,l}]_{l=1..M}, [E5_l, E6_l, E2_{1..N-1,l}]_{l=1..M}
 * (Appendix A): E1 is the free-surface condition (Eq. freeSurfCond) and E2 the
 * boundary-integral equation (Eq. IntegroEqn) at the (N-1)M half-mesh points,
 * E3..E6 the upstream radiation conditions (Eq. numUpRadiation).
 *
 * Conventions for every entry point:
 *  - Vectors u, E, v, ... are caller-owned DEVICE pointers to IEEE double,
 *    length 2(N+1)M unless stated; they must not alias unless stated.
 *  - Work is queued on the context's CUDA stream (the one given to
 *    swj_create).  Entry points marked "async" return before the device has
 *    finished; the others synchronise that stream before returning.
 *  - Every entry point returns SWJ_OK (0) or a negative status; nothing
 *    throws across the ABI.  swj_strerror() names a status.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - The context owns all device workspace it needs (allocated in
 *    swj_create, freed in swj_destroy).
 */
#ifndef SWJ_H
#define SWJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SWJ_OK           0
#define SWJ_EINVAL      -1   /* bad argument (size, pointer, option)          */
#define SWJ_ENOMEM      -2   /* device or pinned-host allocation failed       */
#define SWJ_ECUDA       -3   /* a CUDA runtime call failed                    */
#define SWJ_ENOTCONV    -4   /* Newton iteration cap reached                  */
#define SWJ_ELINESEARCH -5   /* line search could not reduce ||E||_2         */
#define SWJ_EGMRES      -6   /* Krylov iteration cap reached with no progress */
#define SWJ_ENAN        -7   /* NaN or Inf met in E or in a Krylov vector     */
#define SWJ_ETIMEOUT    -8   /* a bounded device-side wait gave up            */
#define SWJ_ESINGULAR   -9   /* zero pivot in the preconditioner factorisation */
#define SWJ_ESIZE      -10   /* the mesh does not fit the no-allocation scratch */
#define SWJ_PENDING      1   /* serving: request not finished yet             */

/* ---- precision of the all-pairs boundary-integral sum ---- */
#define SWJ_FP64 0   /* every step in IEEE double                                  */
#define SWJ_FP32 1   /* all-pairs sum in FP32 with compensated accumulation; the   */
                     /* mesh step, per-target terms and assembly stay in FP64      */
#define SWJ_FF   2   /* all-pairs sum in float-float: FP32 arithmetic with error-  */
                     /* free transformations (~2^-44 relative, close to FP64), at  */
                     /* FP32 speed; residual only (not swj_jvp)                    */

/* ---- solve modes ---- */
#define SWJ_SOLVE_FP64  0  /* Newton-GMRES with the FP64 residual throughout       */
#define SWJ_SOLVE_MIXED 1  /* FP32 residual inside Newton/GMRES, then FP64         */
                           /* residual refinement steps (Newton on the FP64        */
                           /* residual with exact Jacobian-vector products whose   */
                           /* all-pairs part is FP32, as swj_jvp_exact)            */

/* Mesh (Section 3).  N >= 4 points in x, M >= 3 in y; dx, dy > 0; y1 = 0.
 * n_rad is the decay rate n of the radiation condition (0.05 in Section 3). */
typedef struct swj_mesh {
    int N, M;
    double x1, dx, dy;
    double n_rad;
} swj_mesh;

/* Solver options.  swj_default_opts() fills the defaults noted here. */
typedef struct swj_opts {
    int    solve_mode;     /* SWJ_SOLVE_FP64 | SWJ_SOLVE_MIXED (MIXED)               */
    int    block_bw;       /* preconditioner block bandwidth b: odd >= 1, 0 for the  */
                           /* untruncated linear Jacobian (Section 4.2), or -1: by  */
                           /* mesh, 11 for M <= 48 block rows, else 15 (-1)         */
    int    gmres_restart;  /* GMRES restart length m (30)                            */
    int    max_newton;     /* Newton iteration cap (60)                              */
    int    max_krylov;     /* GMRES iterations per Newton step (300)                 */
    double ftol_inf;       /* stop when ||E||_inf < ftol_inf (1e-10)                 */
    double eta_max;        /* cap of the Eisenstat-Walker forcing term (0.1)         */
    double eta_min;        /* floor of the forcing term (1e-6)                        */
    double fd_h;           /* FD step of Eq. JvApprox; 0: h = sqrt(eps_mach)          */
                           /* max(1,||u||_2)/||P^-1 v||_2 (0)                         */
    int    refine_max;     /* MIXED: cap on FP64 refinement Newton steps (4)          */
    double mixed_tol_inf;  /* MIXED: the FP32 phase stops at ||E_fp32||_inf below     */
                           /* this, or when it stalls (2e-6)                          */
    double refine_tol_inf; /* MIXED: the FP64 refinement stops at ||E_fp64||_inf      */
                           /* below this (1e-9)                                       */
    int    verbose;        /* 1: one line per Newton step on stderr (0)               */
    int    autotune;       /* 1: on the first FP32 residual of a mesh size, time      */
                           /* every compiled FP32 tile shape of the all-pairs kernel  */
                           /* and keep the fastest for the process (1)                */
    int    refine_precision; /* MIXED: all-pairs precision of the refinement          */
                           /* residuals: SWJ_FF (float-float, as accurate as FP64 and */
                           /* ~8x faster on this GPU) or SWJ_FP64 (SWJ_FF)            */
    int    jvp;            /* Jacobian-vector products of GMRES: SWJ_JVP_FD (the      */
                           /* difference quotient of Eq. JvApprox) or SWJ_JVP_EXACT   */
                           /* (swj_jvp_exact, all-pairs part in the phase's precision)*/
                           /* (SWJ_JVP_FD)                                            */
    int    forcing;        /* SWJ_FORCING_SOURCE: the submerged source of strength   */
                           /* eps (Section 2); SWJ_FORCING_PRESSURE: an applied      */
                           /* surface pressure eps p(x, y) in Bernoulli's condition, */
                           /* p = exp(2 + 1/(x^2-1) + 1/(y^2-1)) on |x|, |y| < 1,    */
                           /* else 0, and no source (SWJ_FORCING_SOURCE)             */
    int    lu_products;    /* block products of the band LU's bulk updates:          */
                           /* SWJ_LU_FP64 (FP64 CUDA-core kernel) or SWJ_LU_SLICED    */
                           /* (FP64-accurate: bf16 slices of each factor multiplied   */
                           /* exactly on the tensor cores, Ozaki's splitting, summed */
                           /* in FP64) (SWJ_LU_SLICED)                                */
    int    lu_order;       /* elimination order of the band LU of a one-instance     */
                           /* context: SWJ_LU_TOP_DOWN (block rows 0..M-1) or        */
                           /* SWJ_LU_TWO_SIDED (the top half downwards and the bottom */
                           /* half upwards at the same time, then the h block rows    */
                           /* between them: the same factorisation of P up to         */
                           /* rounding in about half the sequential steps); batched   */
                           /* contexts always go top-down (SWJ_LU_TWO_SIDED)          */
    int    wait_limit;     /* iterations after which a bounded device-side wait of    */
                           /* the preconditioner gives up and reports SWJ_ETIMEOUT    */
                           /* (the Gauss-Jordan chain's flag waits in the set-up, the */
                           /* multi-cluster substitution's polls in the apply); 0:    */
                           /* the built-in limits, 2^26 and 2^21 (about a second     */
                           /* each) (0)                                               */
    int    sm_partition;   /* 1: the band LU of a two-sided one-instance context runs */
                           /* its Gauss-Jordan chain on a partition of 32 SMs and the */
                           /* bulk block products on the other SMs (two CUDA green    */
                           /* contexts of the device, created at the first set-up),   */
                           /* so that neither slows the other; where the device or    */
                           /* driver offers no such partition, or a tool is injected  */
                           /* into the process (CUDA_INJECTION64_PATH or Nsight's     */
                           /* injection variables set: profilers, sanitizers), the    */
                           /* set-up runs unpartitioned.  The                         */
                           /* factors do not change.  0: every kernel may run on      */
                           /* every SM (1)                                            */
} swj_opts;

#define SWJ_LU_FP64   0
#define SWJ_LU_SLICED 1

#define SWJ_LU_TOP_DOWN  0
#define SWJ_LU_TWO_SIDED 1

#define SWJ_FORCING_SOURCE   0
#define SWJ_FORCING_PRESSURE 1

#define SWJ_JVP_FD    0
#define SWJ_JVP_EXACT 1

/* Counters and timings of one solve (KINSOL-style counters). */
typedef struct swj_stats {
    int    status;               /* final status code                                */
    int    newton_iters;         /* Newton steps taken (both phases)                 */
    int    refine_iters;         /* of which FP64 refinement steps (MIXED)           */
    int    residual_evals;       /* all residual evaluations                         */
    int    residual_evals_fp64;  /* of which with the FP64 all-pairs sum             */
    int    krylov_iters;         /* GMRES iterations (= FD Jacobian-vector products) */
    int    precond_applies;
    int    line_search_cuts;     /* halvings of the Newton step                      */
    double final_norm_inf;       /* ||E||_inf at the returned u, in the precision    */
                                 /* of the last residual evaluated                   */
    double final_norm_inf_fp64;  /* ||E||_inf at the returned u with an FP64-accurate */
                                 /* all-pairs sum (FP64, or float-float in MIXED mode */
                                 /* with refine_precision SWJ_FF); -1 if never        */
    double t_total_ms;           /* wall time of swj_solve                           */
    double t_setup_ms;           /* preconditioner set-up                            */
    int    pairs_per_residual_hi, pairs_per_residual_lo;  /* (N-1)M*NM as 2x31 bits */
    int    residual_evals_ff;    /* of which with the float-float all-pairs sum (the */
                                 /* right-hand side of the MIXED refinement)         */
    int    exact_jvps;           /* GMRES iterations that used swj_jvp_exact (opts.jvp) */
} swj_stats;

typedef struct swj_ctx swj_ctx;

/* Fill *o with the defaults listed in swj_opts. */
void swj_default_opts(swj_opts *o);

/* Create a context for one mesh and one (F, eps), working on `stream`
 * (a cudaStream_t; NULL = the legacy default stream) of the current device.
 * Allocates all device workspace.  F > 0, eps >= 0.  opts may be NULL
 * (defaults).  Returns SWJ_EINVAL for a bad mesh/option, SWJ_ENOMEM when the
 * workspace does not fit. */
int swj_create(swj_ctx **ctx, const swj_mesh *mesh, double F, double eps,
               const swj_opts *opts, void *stream);

/* ---- batches of instances on one mesh ----
 * A batch context holds `count` >= 1 independent problems on the same mesh,
 * instance i with its own F[i] > 0 and eps[i] >= 0 (copied).  Every vector
 * argument of the entry points below is then `count` consecutive vectors of
 * the single-instance length (u, E, v: count * 2(N+1)M doubles; zeta/phi of
 * swj_unpack: count * NM).  All instances advance together in the same
 * kernel launches (the instance index is a grid dimension), so one launch
 * sequence serves the whole batch; instances that have converged are masked
 * out on the device.  swj_solve takes `stats` as an array of `count`
 * entries (or NULL), fills one per instance and returns SWJ_OK when every
 * instance converged, else the status of the first instance that did not.
 * swj_surface reports instance 0 only.  swj_create is swj_batch_create with
 * count = 1. */
int swj_batch_create(swj_ctx **ctx, const swj_mesh *mesh, int count, const double *F,
                     const double *eps, const swj_opts *opts, void *stream);

/* Number of instances of the context (0 for NULL). */
int swj_batch_count(const swj_ctx *ctx);

/* Per-instance F[count], eps[count] (see swj_set_params). */
int swj_batch_set_params(swj_ctx *ctx, const double *F, const double *eps);

/* Free the context and its device workspace (synchronises its stream). */
void swj_destroy(swj_ctx *ctx);

/* Change F and eps (of every instance of a batch).  A new F invalidates the preconditioner (it depends on
 * the mesh and F only, Appendix B); the next solve or precond call rebuilds
 * it. */
int swj_set_params(swj_ctx *ctx, double F, double eps);

/* Replace the options (same validation as swj_create).  A new block_bw
 * invalidates the preconditioner. */
int swj_set_opts(swj_ctx *ctx, const swj_opts *opts);

/* Bytes of device workspace the context holds (its buffers and, once built,
 * the preconditioner's). */
size_t swj_workspace_bytes(const swj_ctx *ctx);

/* Device bytes a context of `count` instances of `mesh` with `opts` (NULL =
 * defaults) holds after its preconditioner is built, i.e. what
 * swj_workspace_bytes reports for it then (allocator rounding not included).
 * Uses the current device's SM count.  0 for an invalid mesh or option. */
size_t swj_footprint_bytes(const swj_mesh *mesh, int count, const swj_opts *opts);

/* u_dev <- the flat-surface initial guess of Section 4.1: phi_{1,l} = x1,
 * (phi_x)_{k,l} = 1, zeta_{1,l} = 0, (zeta_x)_{k,l} = 0.  Async. */
int swj_initial_guess_flat(swj_ctx *ctx, double *u_dev);

/* u_dev <- the solution of the linearised problem (Section 2.3, the weak-
 * source limit), the other initial guess of Section 4.1:
 * u0 - P^-1 E(u0), u0 the flat state, P the context's preconditioner (the
 * linear Jacobian of Appendix B; with block_bw = 0 this is the exact solution
 * of the discretised linear problem, with b > 0 its block-banded
 * approximation).  E(u0) uses an FP64-accurate all-pairs sum (FP64, or the
 * refinement precision in MIXED mode).  Builds P if needed.  Every instance
 * of a batch.  u_dev: device, count * 2(N+1)M.  Synchronous when it builds P,
 * else async; SWJ_ETIMEOUT as swj_sync. */
int swj_initial_guess_linear(swj_ctx *ctx, double *u_dev);

/* Bootstrapping in eps (Section 4.1): solve at eps_k = eps k / steps,
 * k = 1..steps, each from the previous solution, starting from u_dev as
 * given (e.g. the flat or linear guess); every instance of a batch scales
 * its own eps.  F is unchanged, so the preconditioner is built once.  The
 * context's eps is restored at return.  stats (optional, count entries)
 * accumulate the counts and times of all steps and keep the final norms and
 * status of the last one.  Returns the first failing step's status.
 * Synchronous. */
int swj_solve_continuation(swj_ctx *ctx, double *u_dev, int steps, swj_stats *stats);

/* Mesh bootstrapping: u_dst (on dst's mesh) from u_src (a solution on src's
 * mesh) by bilinear interpolation of src's node fields zeta, g = phi - x,
 * zeta_x, phi_x at dst's nodes, coordinates clamped to src's mesh; phi_1 and
 * zeta_1 from g and zeta at dst's x1.  Instance i of dst from instance i of
 * src (equal counts).  src's scratch node arrays are used, so src must not
 * be in use on another stream; runs on dst's stream and returns when done.
 * src may equal dst (then u_dst must differ from u_src). */
int swj_resample(swj_ctx *src, const double *u_src, swj_ctx *dst, double *u_dst);

/* E_dev <- E(u_dev) (Section 3, Appendix A order), with the all-pairs sum in
 * `precision` (SWJ_FP64, SWJ_FP32 or SWJ_FF).  Steps: trapezoidal integration of
 * zeta and phi along x (Eq. zetaapprox), cubic-spline slopes along y
 * (clamped zero slope at y1 = 0, not-a-knot at y_M), half-mesh values,
 * E1 (Eq. freeSurfCond), the singularity-subtracted boundary integral with
 * the closed-form integral I of S2 (Eqs. IntegroEqn, S2, IS2) and trapezoid
 * weights, E3..E6 (Eq. numUpRadiation).  u_dev and E_dev may not alias.
 * Async. */
int swj_residual(swj_ctx *ctx, const double *u_dev, double *E_dev, int precision);

/* Jv_dev <- (E(u + h v) - E(u)) / h, Eq. JvApprox with the caller's v
 * (apply swj_precond_apply first for J P^-1 v).  Eu_dev must hold E(u) in
 * the same precision; h = opts.fd_h, or when 0 the rule noted in swj_opts
 * with eps_mach of `precision`.  Async. */
int swj_jvp(swj_ctx *ctx, const double *u_dev, const double *Eu_dev,
            const double *v_dev, double *Jv_dev, int precision);

/* Jv_dev <- J(u) v exactly: the derivative d E(u + t v) / dt at t = 0, by
 * forward-mode differentiation of every step of E (mesh step, per-target
 * terms, the closed form of I, the all-pairs sum), the analytic counterpart
 * of the difference quotient of Eq. JvApprox: no step size, no truncation
 * error.  The all-pairs part is computed in `precision` (SWJ_FP64, or SWJ_FP32
 * with Kahan compensation); everything else in FP64.  u_dev, v_dev, Jv_dev:
 * device, count * 2(N+1)M doubles, Appendix A order; Jv_dev must not alias u
 * or v.  Async.  SWJ_EINVAL for a null pointer or another precision. */
int swj_jvp_exact(swj_ctx *ctx, const double *u_dev, const double *v_dev, double *Jv_dev,
                  int precision);

/* Columns col0 .. col0 + ncols - 1 of the preconditioned Jacobian J(u) P^-1
 * (the matrix whose spectrum Section 4.2 wants clustered; Figs. 2-3), for
 * spectral diagnostics on small meshes: column j = swj_jvp_exact(u, P^-1 e_j)
 * with the all-pairs part in `precision`.  out_dev: device, column-major,
 * 2(N+1)M x ncols (leading dimension 2(N+1)M).  Single-instance contexts
 * only.  Builds P if needed.  Synchronous.  SWJ_EINVAL for a batch context,
 * a bad range or precision. */
int swj_preconditioned_jacobian(swj_ctx *ctx, const double *u_dev, int col0, int ncols,
                                double *out_dev, int precision);

/* Build and factor the preconditioner P for the context's mesh, F and
 * block_bw: the linear Jacobian of Appendix B (Eqs. PreA-PreD plus the
 * radiation rows), its zeta-zeta block truncated to the block band, factored
 * through the Schur complement S = D - C A^-1 B (Appendix C) with a block LU
 * of S in FP64.  Synchronous. */
int swj_precond_setup(swj_ctx *ctx);

/* r_dev <- P^-1 b_dev by the three-stage Schur solve of Appendix C.  Builds
 * P first if needed.  b_dev and r_dev may alias.  Async (synchronous when it
 * had to build P). */
int swj_precond_apply(swj_ctx *ctx, const double *b_dev, double *r_dev);

/* Clusters the block substitution of the apply runs on: h (the block half
 * bandwidth) when a single-instance context spreads it over one critical and
 * h - 1 helper clusters, 1 for one cluster per instance, 0 before the
 * preconditioner is built.  Both give identical results. */
int swj_precond_sweep_clusters(const swj_ctx *ctx);

/* SMs of the partition the set-up's Gauss-Jordan chain ran on
 * (opts.sm_partition: 32 on B300; the bulk block products ran on the other
 * SMs), 0 when the last set-up ran unpartitioned or none has run yet. */
int swj_precond_chain_sms(const swj_ctx *ctx);

/* Solve E(u) = 0 by damped inexact Newton (Section 4.1) with right-
 * preconditioned restarted GMRES and FD Jacobian-vector products
 * (Eq. JvApprox), starting from u_dev_inout; on return it holds the last
 * iterate.  stats may be NULL.  Returns SWJ_OK when ||E||_inf < ftol_inf
 * (FP64 mode) or refine_tol_inf (MIXED mode, measured on the FP64 residual),
 * else SWJ_ENOTCONV / SWJ_ELINESEARCH / SWJ_ENAN.  Synchronous. */
int swj_solve(swj_ctx *ctx, double *u_dev_inout, swj_stats *stats);

/* The whole solve from and to HOST memory, for callers whose data live on the
 * host: u0_host (2(N+1)M doubles; pinned host memory copies fastest, pageable
 * works) is copied to the device as the initial guess; with setup != 0 the
 * preconditioner is rebuilt first (with setup = 0 it is built only if the
 * context has none); then the solve of swj_solve runs, and the result is
 * copied back: u_host the final iterate (may be NULL; may alias u0_host),
 * zeta_host and phi_host the surface and potential at the nodes ([M][N]
 * row-major, x fastest; either may be NULL).  The first call allocates the
 * context's device staging, 2(N+1)M + 2NM doubles, counted by
 * swj_workspace_bytes.  Single-instance contexts only (SWJ_EINVAL for a
 * batch).  Synchronous.  Returns swj_solve's status, or SWJ_EINVAL /
 * SWJ_ENOMEM / SWJ_ECUDA / a set-up status. */
int swj_solve_host(swj_ctx *ctx, const double *u0_host, int setup, double *u_host, double *zeta_host,
                   double *phi_host, swj_stats *stats);

/* zeta_dev, phi_dev <- zeta and phi on the mesh ([M][N] row-major, index
 * (l-1) N + (k-1)) rebuilt from u by Eq. zetaapprox.  Either may be NULL.
 * Async. */
int swj_unpack(swj_ctx *ctx, const double *u_dev, double *zeta_dev, double *phi_dev);

/* Diagnostic view of the mesh step for u_dev: out_dev receives, each as an
 * [M][N] array in this order, zeta, g = phi - x, zeta_y, g_y (= phi_y), and
 * then, each as an [M][N-1] array, zeta*, g*, zeta_x*, zeta_y* and I (the
 * closed-form integral of S2, Eq. IS2), all FP64.  out_dev must hold
 * 4NM + 5(N-1)M doubles.  Async. */
int swj_surface(swj_ctx *ctx, const double *u_dev, double *out_dev);

/* ---- tile shapes of the all-pairs kernel ----
 * Several tile shapes (threads per block, targets per thread, FP32 packed
 * pair instructions or not) are compiled per precision; index 0 is the
 * default.  With opts.autotune the first FP32 residual of each mesh size
 * times the FP32 shapes and every context of that size in the process uses
 * the fastest; FP64 residuals use the default shape unless one is pinned. */

/* Number of compiled shapes for `precision`. */
int swj_pair_variants(int precision);

/* The shape the context uses for `precision`: its index, threads per block,
 * targets per thread and whether it uses packed FP32 pair instructions (any
 * pointer may be NULL). */
int swj_pair_config(const swj_ctx *ctx, int precision, int *variant, int *threads,
                    int *targets_per_thread, int *packed);

/* Name of compiled shape `variant` (kernel and template arguments, e.g.
 * "k_pairs_x2r<2,256,2,0,1>"; "" for an unknown index).  Static storage. */
const char *swj_pair_variant_name(int precision, int variant);

/* Pin shape `variant` for `precision` on this context (synchronises its
 * stream; drops captured graphs).  SWJ_EINVAL for an unknown index. */
int swj_set_pair_config(swj_ctx *ctx, int precision, int variant);

/* ---- serving: a request loop over concurrent solves ----
 * A server owns worker threads, one CUDA stream per running group, and the
 * contexts it creates, all on the device current at swj_server_create.
 * Requests (mesh, F, eps; flat initial guess, the server's swj_opts) queue
 * in FIFO order.  A request is admitted when one of max_active worker slots
 * is free and the footprint of its context (swj_footprint_bytes) fits the
 * memory budget; later queued requests on the same mesh are admitted with it
 * as one batch context (a power of two of them, at most max_group).  Groups
 * on different streams run concurrently on the device; each finished group
 * frees its slot for the next admission at once.  Finished contexts are kept
 * for reuse by later groups of the same mesh and size when keep_contexts is
 * set (evicted least recently used when memory is needed).  A result is the
 * same whether its request ran alone or in a group.  All server entry points
 * are thread-safe. */
typedef struct swj_server swj_server;

typedef struct {
    size_t   hbm_budget_bytes; /* device bytes for contexts (0: 80% of free memory)   */
    int      max_active;       /* groups running at once, 1..256 (default 4)          */
    int      max_group;        /* requests per batch context, 1..1024 (default 8)     */
    int      keep_contexts;    /* reuse finished contexts (default 1)                 */
    swj_opts opts;             /* solve options of every request                      */
} swj_server_opts;

typedef struct {
    long long submitted, completed, failed;
    int       queued, active, peak_active;
    size_t    bytes_held, peak_bytes_held, budget_bytes;
    long long contexts_created, contexts_reused, contexts_evicted;
} swj_server_info;

typedef struct {
    double queue_ms;     /* submit -> admission                      */
    double run_ms;       /* admission -> result copied to the host   */
    double latency_ms;   /* submit -> result copied to the host      */
    int    group_size;   /* requests in the batch context it ran in  */
} swj_request_times;

void swj_server_default_opts(swj_server_opts *opts);

/* Start a server (threads and budget; no context is created yet).  opts may
 * be NULL.  SWJ_EINVAL for bad options. */
int swj_server_create(swj_server **srv, const swj_server_opts *opts);

/* Queue one solve; *id receives its handle.  SWJ_ENOMEM if its context could
 * never fit the budget, SWJ_EINVAL for a bad mesh or parameter. */
int swj_server_submit(swj_server *srv, const swj_mesh *mesh, double F, double eps, long long *id);

/* SWJ_PENDING while request `id` runs or waits (wait = 0); with wait = 1
 * block until it is done.  When done: fill stats, zeta_host (N*M doubles,
 * [M][N] as swj_unpack), times (each may be NULL), forget the request and
 * return its status (SWJ_OK or the solver's error).  SWJ_EINVAL for an
 * unknown or already collected id. */
int swj_server_poll(swj_server *srv, long long id, int wait, swj_stats *stats,
                    double *zeta_host, swj_request_times *times);

/* Counters and memory of the server. */
int swj_server_get_info(swj_server *srv, swj_server_info *info);

/* Block until no request is queued or running. */
int swj_server_drain(swj_server *srv);

/* Drop queued requests, wait for running groups, free everything. */
void swj_server_destroy(swj_server *srv);

/* Block until the context's stream is idle; returns SWJ_ECUDA if a kernel
 * failed, SWJ_ETIMEOUT if a bounded device-side wait of the preconditioner
 * apply gave up since the last set-up. */
int swj_sync(swj_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *swj_strerror(int status);

/* Library version string. */
const char *swj_version(void);

/* ---- test hooks ---- */

/* Test hook for the failure path of the bounded device waits: with
 * SWJ_TEST_WITHHOLD_HELPERS set, the multi-cluster substitution of
 * swj_precond_apply is launched without its helper clusters, so the terms the
 * critical clusters poll for are never written; every poll gives up after
 * opts.wait_limit iterations, the kernel returns, and the apply reports
 * SWJ_ETIMEOUT (its result is then meaningless).  Nothing faults, traps or
 * waits without bound.  hooks = 0 restores normal launches; the next
 * swj_precond_setup clears the timeout status.  Applies only to contexts whose
 * apply runs on several clusters (swj_sweep_clusters > 1).  Returns SWJ_OK or
 * SWJ_EINVAL. */
#define SWJ_TEST_WITHHOLD_HELPERS 1
int swj_set_test_hooks(swj_ctx *ctx, int hooks);

/* ---- residual without allocation ---- */

/* Bytes of the device array that swj_residual_noalloc works in. */
#define SWJ_NOALLOC_SCRATCH_BYTES (16u << 20)

/* E_dev <- E(u_dev) as swj_residual computes it with default options (source
 * forcing; precision SWJ_FP64 or SWJ_FP32, the same kernels), for callers
 * that cannot allocate device memory: no context, no cudaMalloc, cudaFree or
 * allocating library call.  The paper has no counterpart; it exists for hosts
 * such as a serving loop with a fixed latency budget (cudaMalloc/cudaFree
 * synchronise the whole device) or a framework that budgets all device memory
 * up front.  The result equals swj_residual's within the residual parity
 * tolerance (10^-12 of the row scale in FP64, 2*10^-6 in FP32); it can differ
 * in the last bits where the scratch forces fewer source chunks than the
 * context's launch plan, which changes the summation order.
 *
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default) of the
 * current device; the call returns before it finishes.  u_dev and E_dev are
 * caller-owned device buffers of 2(N+1)M doubles and may not alias.
 *
 * Scratch: one file-scope device array of SWJ_NOALLOC_SCRATCH_BYTES (16 MiB)
 * per GPU that loads the library, held until the process exits.  A mesh
 * needs about 128 NM + 120 (N-1)M bytes plus 8 (N-1)M per source chunk (at
 * least one): 361 x 121 fits (with fewer chunks than a context uses), and
 * with N = 361 the largest that fits is 361 x 187 (one chunk).  A mesh that does not fit returns SWJ_ESIZE before any work is
 * queued.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture.  All calls on a device share the array and leave
 * their data in it; nothing needs clearing between calls (every byte a call
 * reads it wrote first), but calls that overlap on the GPU race on it, so
 * serialise them.
 * Returns SWJ_OK, SWJ_EINVAL (bad argument), SWJ_ESIZE or SWJ_ECUDA. */
int swj_residual_noalloc(const swj_mesh *mesh, double F, double eps, const double *u_dev,
                         double *E_dev, int precision, void *stream);

/* ---- instrumentation ---- */

/* Kernel launches the library has issued since it was loaded (all
 * contexts; a plain counter, not synchronised across host threads). */
unsigned long long swj_kernel_launches(void);

/* enable != 0: record a CUDA event pair around every launch of the all-pairs
 * kernel on the context's stream (up to 2048 launches until the next reset),
 * so its device time can be read back; 0: stop recording.  Either way the
 * record is cleared.  Returns SWJ_ENOMEM / SWJ_ECUDA if the events cannot be
 * created. */
int swj_set_kernel_timing(swj_ctx *ctx, int enable);

/* Synchronise the stream and report the summed device time (ms) and count of
 * the recorded all-pairs launches of the given precision since the last
 * reset. */
int swj_pair_timing(swj_ctx *ctx, int precision, double *total_ms, int *launches);

/* Clear the record of timed launches (synchronises the stream). */
int swj_reset_pair_timing(swj_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SWJ_H */
