// Residual, Jacobian-vector product, GMRES and the Newton driver (Section 4).
//
//  * residual: mesh step (FP64) -> all-pairs sum (FP64 or FP32) -> assembly.
//  * JVP (Eq. JvApprox): J v ~ (E(u + h v) - E(u)) / h, with the FD step
//    h = sqrt(eps_mach) max(1, ||u||_2) / ||v||_2 computed on the device.
//  * GMRES (Saad & Schultz) with right preconditioning: the Krylov space is
//    K_m(J P^-1, r); the preconditioned directions z_j = P^-1 v_j are kept
//    (so the step is sum_j y_j z_j without one more P^-1 apply); the Arnoldi
//    vectors are orthogonalised by classical Gram-Schmidt applied twice
//    (as stable as modified Gram-Schmidt, two block reductions per step
//    instead of j + 1 dependent ones); Givens rotations and the small
//    triangular solve are done on the host in FP64.
//  * Damped inexact Newton (Eqs. newtonstep0, newtonstep): the step is
//    halved until ||E||_2 decreases by the Armijo factor (1 - 1e-4 lambda);
//    the GMRES tolerance is the Eisenstat-Walker forcing term (choice 1 with
//    its safeguard), kept in [eta_min, eta_max].
//  * MIXED mode: Newton on the FP32-sum residual until it reaches its noise
//    floor, then Newton steps on the FP64 residual whose linear solves use
//    FP32 JVPs (a defect correction: the root is the FP64 one).
#include "swj_internal.h"
#include <math.h>
#include <stdio.h>
#include <chrono>
#include <string.h>
#include <vector>

namespace {

enum {
    DS_NU = 0, DS_NV = 2, DS_H = 4, DS_NW = 6, DS_NE = 8, DS_NT = 10, DS_NR = 12,
    DS_H1 = 64, DS_H2 = 128, DS_Y = 192, DS_C = 256
};

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

__global__ void k_fd_h(const double *__restrict__ nu2, const double *__restrict__ nv2,
                       double epsm, double hfix, double *__restrict__ h)
{
    if (threadIdx.x || blockIdx.x) return;
    if (hfix > 0.0) { h[0] = hfix; return; }
    double nv = sqrt(nv2[0]);
    double nu = sqrt(nu2[0]);
    h[0] = (nv > 0.0) ? sqrt(epsm) * fmax(1.0, nu) / nv : 1.0;
}

__global__ void k_perturb(int n, const double *__restrict__ u, const double *__restrict__ v,
                          const double *__restrict__ h, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fma(h[0], v[i], u[i]);
}

__global__ void k_fd_diff(int n, const double *__restrict__ Ep, const double *__restrict__ Eu,
                          const double *__restrict__ h, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (Ep[i] - Eu[i]) / h[0];
}

__global__ void k_scale_to(int n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}

__global__ void k_add_rows(int rows, double *__restrict__ a, const double *__restrict__ b)
{
    int i = threadIdx.x;
    if (i < rows) a[i] += b[i];
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int read_scalars(swj_ctx *c, int off, int count)
{
    SWJ_CUDA_TRY(cudaMemcpyAsync(c->hpin + off, c->dscal + off, (size_t)count * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SWJ_OK;
}

struct Norms { double two, inf; };

int norms_of(swj_ctx *c, const double *x, int slot, Norms *out)
{
    swj_norms(c->stream, c->nu, x, c->red, c->dscal + slot);
    int rc = read_scalars(c, slot, 2);
    if (rc) return rc;
    out->two = sqrt(c->hpin[slot]);
    out->inf = c->hpin[slot + 1];
    return SWJ_OK;
}

int residual_counted(swj_ctx *c, const double *u, double *E, int prec, swj_stats *st)
{
    if (st) {
        st->residual_evals++;
        if (prec == SWJ_FP64) st->residual_evals_fp64++;
    }
    return swj_residual_impl(c, u, E, prec);
}

// Right-preconditioned restarted GMRES for J x = rhs, J v from FD-JVPs about
// (u, Ebase) in precision `prec`.  Stops when the (rotated) residual estimate
// is <= rtol ||rhs||_2 or after maxit iterations.
struct GmresResult { int iters; double res, bnorm; };

int gmres(swj_ctx *c, const double *u, const double *Ebase, int prec, const double *rhs,
          double *x, double rtol, int maxit, GmresResult *res, swj_stats *st)
{
    const int n = c->nu, m = c->kry_m;
    const size_t ld = (size_t)n;
    cudaStream_t s = c->stream;
    Norms nb;
    int rc = norms_of(c, rhs, DS_NR, &nb);
    if (rc) return rc;
    res->iters = 0;
    res->bnorm = nb.two;
    res->res = nb.two;
    swj_fill(s, n, 0.0, x);
    if (!isfinite(nb.two)) return SWJ_ENAN;
    if (nb.two == 0.0) return SWJ_OK;
    SWJ_COUNT_LAUNCH();
    k_scale_to<<<nblk(n, 256), 256, 0, s>>>(n, 1.0 / nb.two, rhs, c->V);
    double beta = nb.two;
    const double target = rtol * nb.two;
    std::vector<double> R((size_t)(m + 1) * m), Hraw((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    int total = 0;
    for (;;) {
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int k = 0;
        double est = beta;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            double *Vj = c->V + (size_t)j * ld, *Zj = c->Z + (size_t)j * ld;
            double *w = c->V + (size_t)(j + 1) * ld;
            rc = swj_pc_apply(c, Vj, Zj);
            if (rc) return rc;
            if (st) { st->precond_applies++; st->krylov_iters++; }
            if (st) { st->residual_evals++; if (prec == SWJ_FP64) st->residual_evals_fp64++; }
            rc = swj_jvp_impl(c, u, Ebase, Zj, w, prec, c->opts.fd_h);
            if (rc) return rc;
            // classical Gram-Schmidt, twice
            swj_mdot(s, n, j + 1, c->V, ld, w, c->red, c->dscal + DS_H1);
            swj_mgemv_sub(s, n, j + 1, c->V, ld, c->dscal + DS_H1, w);
            swj_mdot(s, n, j + 1, c->V, ld, w, c->red, c->dscal + DS_H2);
            swj_mgemv_sub(s, n, j + 1, c->V, ld, c->dscal + DS_H2, w);
            SWJ_COUNT_LAUNCH();
            k_add_rows<<<1, 64, 0, s>>>(j + 1, c->dscal + DS_H1, c->dscal + DS_H2);
            swj_norms(s, n, w, c->red, c->dscal + DS_NW);
            SWJ_CUDA_TRY(cudaMemcpyAsync(c->hpin + DS_H1, c->dscal + DS_H1, (size_t)(j + 1) * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
            SWJ_CUDA_TRY(cudaMemcpyAsync(c->hpin + DS_NW, c->dscal + DS_NW, 2 * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
            SWJ_CUDA_TRY(cudaStreamSynchronize(s));
            double hn = sqrt(c->hpin[DS_NW]);
            if (!isfinite(hn)) return SWJ_ENAN;
            double *col = &R[(size_t)j * (m + 1)];
            for (int i = 0; i <= j; ++i) {
                col[i] = c->hpin[DS_H1 + i];
                Hraw[(size_t)j * (m + 1) + i] = col[i];
            }
            col[j + 1] = hn;
            Hraw[(size_t)j * (m + 1) + j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            double a = col[j], b2 = col[j + 1];
            double rr = hypot(a, b2);
            cs[j] = (rr > 0) ? a / rr : 1.0;
            sn[j] = (rr > 0) ? b2 / rr : 0.0;
            col[j] = rr;
            col[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            est = fabs(gv[j + 1]);
            ++total;
            k = j + 1;
            if (hn > 0.0) {
                SWJ_COUNT_LAUNCH();
                k_scale_to<<<nblk(n, 256), 256, 0, s>>>(n, 1.0 / hn, w, w);
            }
            if (est <= target || hn == 0.0 || total >= maxit) { done = true; break; }
        }
        // y = R^-1 g (upper triangular k x k)
        for (int i = k - 1; i >= 0; --i) {
            double v = gv[i];
            for (int q = i + 1; q < k; ++q) v -= R[(size_t)q * (m + 1) + i] * y[q];
            y[i] = v / R[(size_t)i * (m + 1) + i];
            if (!isfinite(y[i])) return SWJ_ENAN;
        }
        for (int i = 0; i < k; ++i) c->hpin[DS_Y + i] = y[i];
        SWJ_CUDA_TRY(cudaMemcpyAsync(c->dscal + DS_Y, c->hpin + DS_Y, (size_t)k * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        swj_combine(s, n, k, c->Z, ld, c->dscal + DS_Y, x, 1);
        res->iters = total;
        res->res = est;
        if (done && (est <= target || total >= maxit)) break;
        if (done) break;   // happy breakdown: exact in the Krylov space
        // restart: r = V_{k+1} (beta e1 - Hraw y)
        std::vector<double> cvec(k + 1, 0.0);
        cvec[0] = beta;
        for (int q = 0; q < k; ++q)
            for (int i = 0; i <= q + 1; ++i) cvec[i] -= Hraw[(size_t)q * (m + 1) + i] * y[q];
        for (int i = 0; i <= k; ++i) c->hpin[DS_C + i] = cvec[i];
        SWJ_CUDA_TRY(cudaMemcpyAsync(c->dscal + DS_C, c->hpin + DS_C, (size_t)(k + 1) * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        swj_combine(s, n, k + 1, c->V, ld, c->dscal + DS_C, c->rvec, 0);
        Norms nr;
        rc = norms_of(c, c->rvec, DS_NT, &nr);
        if (rc) return rc;
        if (!isfinite(nr.two)) return SWJ_ENAN;
        beta = nr.two;
        if (beta <= target) break;
        SWJ_COUNT_LAUNCH();
        k_scale_to<<<nblk(n, 256), 256, 0, s>>>(n, 1.0 / beta, c->rvec, c->V);
    }
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

struct PhaseResult { double finf, f2; int status; };

// Damped inexact Newton in one residual precision; E_cur holds E(u) on entry
// (norms in *ph) and on exit.
int newton_phase(swj_ctx *c, double *u, int prec, double tol, int max_it, PhaseResult *ph,
                 swj_stats *st, bool stop_on_stall)
{
    const int n = c->nu;
    cudaStream_t s = c->stream;
    const swj_opts &o = c->opts;
    double eta = o.eta_max;
    for (int it = 0; it < max_it; ++it) {
        if (!isfinite(ph->finf)) { ph->status = SWJ_ENAN; return SWJ_ENAN; }
        if (ph->finf < tol) { ph->status = SWJ_OK; return SWJ_OK; }
        SWJ_COUNT_LAUNCH();
        k_scale_to<<<nblk(n, 256), 256, 0, s>>>(n, -1.0, c->E_cur, c->rvec);
        GmresResult gr;
        int rc = gmres(c, u, c->E_cur, prec, c->rvec, c->du, eta, o.max_krylov, &gr, st);
        if (rc) { ph->status = rc; return rc; }
        double f2 = ph->f2, lam = 1.0;
        Norms nt;
        for (;;) {
            swj_copy(s, n, u, c->u_try);
            swj_axpby(s, n, lam, c->du, 1.0, c->u_try);
            rc = residual_counted(c, c->u_try, c->E_try, prec, st);
            if (rc) { ph->status = rc; return rc; }
            rc = norms_of(c, c->E_try, DS_NE, &nt);
            if (rc) { ph->status = rc; return rc; }
            if (isfinite(nt.two) && nt.two <= (1.0 - 1e-4 * lam) * f2) break;
            lam *= 0.5;
            if (st) st->line_search_cuts++;
            if (lam < 1.0 / 1024.0) { ph->status = SWJ_ELINESEARCH; return SWJ_ELINESEARCH; }
        }
        // Eisenstat-Walker choice 1 with safeguard
        double lin = (1.0 - lam) * f2 + lam * gr.res;
        double eta_new = fabs(nt.two - lin) / f2;
        double safe = pow(eta, 0.5 * (1.0 + sqrt(5.0)));
        if (safe > 0.1 && eta_new < safe) eta_new = safe;
        if (eta_new > o.eta_max) eta_new = o.eta_max;
        if (eta_new < o.eta_min) eta_new = o.eta_min;
        eta = eta_new;
        swj_copy(s, n, c->u_try, u);
        double *tmp = c->E_cur; c->E_cur = c->E_try; c->E_try = tmp;
        double prev_inf = ph->finf;
        ph->f2 = nt.two;
        ph->finf = nt.inf;
        if (st) st->newton_iters++;
        if (o.verbose)
            fprintf(stderr, "[swj] newton %s it=%d |E|inf=%.3e |E|2=%.3e lam=%.3g gmres=%d eta=%.2e\n",
                    prec == SWJ_FP64 ? "fp64" : "fp32", it + 1, nt.inf, nt.two, lam, gr.iters, eta);
        if (stop_on_stall && nt.inf > 0.5 * prev_inf && nt.inf < 100.0 * tol) {
            ph->status = SWJ_OK;
            return SWJ_OK;
        }
    }
    ph->status = (ph->finf < tol) ? SWJ_OK : SWJ_ENOTCONV;
    return ph->status;
}

}  // namespace

int swj_residual_impl(swj_ctx *c, const double *u, double *E, int precision)
{
    swj_launch_mesh_step(c, u, E);
    const bool rec = c->time_pairs && c->tev && c->n_timed < SWJ_MAX_TIMED;
    if (rec) cudaEventRecord(c->tev[2 * c->n_timed], c->stream);
    if (precision == SWJ_FP64) swj_launch_pairs64(c, c->plan64);
    else swj_launch_pairs32(c, c->plan32);
    if (rec) {
        cudaEventRecord(c->tev[2 * c->n_timed + 1], c->stream);
        c->tev_prec[c->n_timed++] = precision;
    }
    swj_launch_assemble(c, E, precision == SWJ_FP64 ? c->plan64.P : c->plan32.P);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_jvp_impl(swj_ctx *c, const double *u, const double *Eu, const double *v, double *Jv,
                 int precision, double h_fixed)
{
    cudaStream_t s = c->stream;
    const int n = c->nu;
    if (!(h_fixed > 0.0)) {
        swj_norms(s, n, u, c->red, c->dscal + DS_NU);
        swj_norms(s, n, v, c->red, c->dscal + DS_NV);
    }
    double epsm = (precision == SWJ_FP64) ? 2.220446049250313e-16 : 1.1920928955078125e-07;
    SWJ_COUNT_LAUNCH();
    k_fd_h<<<1, 1, 0, s>>>(c->dscal + DS_NU, c->dscal + DS_NV, epsm, h_fixed, c->dscal + DS_H);
    SWJ_COUNT_LAUNCH();
    k_perturb<<<nblk(n, 256), 256, 0, s>>>(n, u, v, c->dscal + DS_H, c->u_tmp);
    int rc = swj_residual_impl(c, c->u_tmp, c->E_tmp, precision);
    if (rc) return rc;
    SWJ_COUNT_LAUNCH();
    k_fd_diff<<<nblk(n, 256), 256, 0, s>>>(n, c->E_tmp, Eu, c->dscal + DS_H, Jv);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_solve_impl(swj_ctx *c, double *u, swj_stats *stats)
{
    swj_stats local;
    swj_stats *st = stats ? stats : &local;
    memset(st, 0, sizeof(*st));
    st->final_norm_inf_fp64 = -1.0;
    long long pairs = (long long)c->T * c->S;
    st->pairs_per_residual_hi = (int)(pairs >> 31);
    st->pairs_per_residual_lo = (int)(pairs & 0x7fffffffLL);
    double t0 = now_ms();
    const swj_opts &o = c->opts;
    int rc;
    if (!c->pc_ready) {
        double ts = now_ms();
        rc = swj_pc_setup(c);
        st->t_setup_ms = now_ms() - ts;
        if (rc) { st->status = rc; st->t_total_ms = now_ms() - t0; return rc; }
    }
    const bool mixed = (o.solve_mode == SWJ_SOLVE_MIXED);
    const int prec = mixed ? SWJ_FP32 : SWJ_FP64;
    rc = residual_counted(c, u, c->E_cur, prec, st);
    if (rc) { st->status = rc; return rc; }
    Norms n0;
    rc = norms_of(c, c->E_cur, DS_NE, &n0);
    if (rc) { st->status = rc; return rc; }
    PhaseResult ph{n0.inf, n0.two, SWJ_OK};
    rc = newton_phase(c, u, prec, mixed ? o.mixed_tol_inf : o.ftol_inf, o.max_newton, &ph, st, mixed);
    st->final_norm_inf = ph.finf;
    if (!mixed) {
        st->final_norm_inf_fp64 = ph.finf;
        st->status = rc;
        st->t_total_ms = now_ms() - t0;
        return rc;
    }
    if (rc == SWJ_ENAN || rc == SWJ_ECUDA || rc == SWJ_ENOMEM || rc == SWJ_ESINGULAR) {
        st->status = rc;
        st->t_total_ms = now_ms() - t0;
        return rc;
    }
    // FP64 refinement: Newton on E_fp64 with FP32 JVPs about the same u
    const int n = c->nu;
    cudaStream_t s = c->stream;
    rc = residual_counted(c, u, c->E_cur, SWJ_FP64, st);
    if (rc) { st->status = rc; return rc; }
    Norms e64;
    rc = norms_of(c, c->E_cur, DS_NE, &e64);
    if (rc) { st->status = rc; return rc; }
    int status = SWJ_ENOTCONV;
    for (int r = 0; r <= o.refine_max; ++r) {
        if (!isfinite(e64.inf)) { status = SWJ_ENAN; break; }
        if (e64.inf < o.refine_tol_inf) { status = SWJ_OK; break; }
        if (r == o.refine_max) break;
        rc = residual_counted(c, u, c->E_base32, SWJ_FP32, st);
        if (rc) { status = rc; break; }
        SWJ_COUNT_LAUNCH();
        k_scale_to<<<nblk(n, 256), 256, 0, s>>>(n, -1.0, c->E_cur, c->rvec);
        GmresResult gr;
        rc = gmres(c, u, c->E_base32, SWJ_FP32, c->rvec, c->du, 1e-3, o.max_krylov, &gr, st);
        if (rc) { status = rc; break; }
        double lam = 1.0;
        Norms nt;
        bool ok = false;
        for (int cut = 0; cut < 4; ++cut) {
            swj_copy(s, n, u, c->u_try);
            swj_axpby(s, n, lam, c->du, 1.0, c->u_try);
            rc = residual_counted(c, c->u_try, c->E_try, SWJ_FP64, st);
            if (rc) break;
            rc = norms_of(c, c->E_try, DS_NE, &nt);
            if (rc) break;
            if (isfinite(nt.two) && nt.two < e64.two) { ok = true; break; }
            lam *= 0.5;
            st->line_search_cuts++;
        }
        if (rc) { status = rc; break; }
        if (!ok) { status = SWJ_ELINESEARCH; break; }
        swj_copy(s, n, c->u_try, u);
        double *tmp = c->E_cur; c->E_cur = c->E_try; c->E_try = tmp;
        e64 = nt;
        st->newton_iters++;
        st->refine_iters++;
        if (o.verbose)
            fprintf(stderr, "[swj] refine fp64 it=%d |E|inf=%.3e lam=%.3g gmres=%d\n", r + 1, nt.inf,
                    lam, gr.iters);
    }
    st->final_norm_inf = e64.inf;
    st->final_norm_inf_fp64 = e64.inf;
    st->status = status;
    st->t_total_ms = now_ms() - t0;
    return status;
}
