// Residual, Jacobian-vector product, GMRES and the Newton driver (Section 4),
// for the nb instances of a context at once.
//
//  * residual: mesh step (FP64) -> all-pairs sum (FP64 or FP32) -> assembly,
//    each one launch over every active instance.
//  * JVP (Eq. JvApprox): J v ~ (E(u + h v) - E(u)) / h, with the FD step
//    h = sqrt(eps_mach) max(1, ||u||_2) / ||v||_2 per instance, on the device.
//  * GMRES (Saad & Schultz) with right preconditioning: the Krylov space is
//    K_m(J P^-1, r); the preconditioned directions z_j = P^-1 v_j are kept
//    (the step is sum_j y_j z_j without one more P^-1 apply); the Arnoldi
//    vectors are orthogonalised by classical Gram-Schmidt applied twice (as
//    stable as modified Gram-Schmidt, two block reductions per step instead
//    of j + 1 dependent ones).  The device part of one Arnoldi step (apply,
//    JVP, CGS2, normalisation, copy of the new Hessenberg column to the host)
//    is captured once per Krylov index as a CUDA graph and replayed; Givens
//    rotations and the small triangular solves are done on the host in FP64.
//  * Damped inexact Newton (Eqs. newtonstep0, newtonstep): the step is
//    halved until ||E||_2 decreases by the Armijo factor (1 - 1e-4 lambda);
//    the GMRES tolerance is the Eisenstat-Walker forcing term (choice 1 with
//    its safeguard), kept in [eta_min, eta_max].
//  * MIXED mode: Newton on the FP32-sum residual until it reaches its noise
//    floor, then Newton steps on an FP64-accurate residual (the float-float or
//    the FP64 all-pairs sum) whose linear solves use FP32 JVPs (a defect
//    correction: the root is the FP64 one).
// Instances advance in lock step; a per-instance flag array on the device
// masks those that have finished (or whose GMRES has converged), so every
// launch keeps its shape.
#include "swj_internal.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <chrono>
#include <string.h>
#include <vector>
#include <algorithm>

namespace {

// slots of the per-instance device scalars (dscal[inst * SWJ_DS + slot])
enum {
    DS_NU = 0, DS_NV = 2, DS_H = 4, DS_NW = 6, DS_NE = 8, DS_NT = 10, DS_NR = 12, DS_SC = 14,
    DS_LAM = 15, DS_H1 = 64, DS_H2 = 128, DS_Y = 192, DS_C = 256
};

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

// FD step: h = sqrt(eps_mach) max(1, ||u||_2) / ||v||_2 (||u|| is dominated by
// the phi_x ~ 1 entries, so h ||v|| is already ~0.05 of a mesh-wide unit; a
// larger step for the central difference would make its truncation error, not
// the rounding, the larger term)
__global__ void k_fd_h(double *__restrict__ ds, double rel, double hfix, const int *__restrict__ act,
                       int nb)
{
    int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= nb || !SWJ_INST_ACTIVE(act, inst)) return;
    double *d = ds + (size_t)inst * SWJ_DS;
    if (hfix > 0.0) { d[DS_H] = hfix; return; }
    double nv = sqrt(d[DS_NV]);
    double nu = sqrt(d[DS_NU]);
    d[DS_H] = (nv > 0.0) ? rel * fmax(1.0, nu) / nv : 1.0;
}

// out = u + sgn h v
__global__ void k_perturb(int n, const double *__restrict__ u, const double *__restrict__ v,
                          const double *__restrict__ ds, double sgn, double *__restrict__ out,
                          const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t o = (size_t)inst * n;
    if (i < n) out[o + i] = fma(sgn * ds[(size_t)inst * SWJ_DS + DS_H], v[o + i], u[o + i]);
}

// out = (Ep - Eu) / (span h): span 1 forward, 2 central (Eu = E(u - h v))
__global__ void k_fd_diff(int n, const double *__restrict__ Ep, const double *__restrict__ Eu,
                          const double *__restrict__ ds, double span, double *__restrict__ out,
                          const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t o = (size_t)inst * n;
    if (i < n) out[o + i] = (Ep[o + i] - Eu[o + i]) / (span * ds[(size_t)inst * SWJ_DS + DS_H]);
}

// v_{j+1} <- w / ||w||_2 (the squared norm is in slot DS_NW)
__global__ void k_normalise(int n, double *__restrict__ w, size_t stride, const double *__restrict__ ds,
                            const int *__restrict__ act)
{
    const int inst = blockIdx.y;
    if (!SWJ_INST_ACTIVE(act, inst)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double nn = ds[(size_t)inst * SWJ_DS + DS_NW];
    if (i < n && nn > 0.0) w[(size_t)inst * stride + i] *= 1.0 / sqrt(nn);
}

__global__ void k_add_rows(int rows, double *__restrict__ ds, const int *__restrict__ act, int nb)
{
    const int inst = blockIdx.x;
    if (inst >= nb || !SWJ_INST_ACTIVE(act, inst)) return;
    int i = threadIdx.x;
    if (i < rows) ds[(size_t)inst * SWJ_DS + DS_H1 + i] += ds[(size_t)inst * SWJ_DS + DS_H2 + i];
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// copy `count` per-instance scalars starting at `slot` of every instance to the host mirror
int read_scalars(swj_ctx *c, int slot, int count)
{
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->hpin + slot, SWJ_DS * sizeof(double), c->dscal + slot,
                                   SWJ_DS * sizeof(double), (size_t)count * sizeof(double), c->nb,
                                   cudaMemcpyDeviceToHost, c->stream));
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SWJ_OK;
}

int write_scalars(swj_ctx *c, int slot, int count)
{
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->dscal + slot, SWJ_DS * sizeof(double), c->hpin + slot,
                                   SWJ_DS * sizeof(double), (size_t)count * sizeof(double), c->nb,
                                   cudaMemcpyHostToDevice, c->stream));
    return SWJ_OK;
}

inline double &hs(swj_ctx *c, int inst, int slot) { return c->hpin[(size_t)inst * SWJ_DS + slot]; }

// make the device mask equal to `mask` (one flag per instance)
int set_mask(swj_ctx *c, const std::vector<int> &mask)
{
    bool same = true;
    for (int i = 0; i < c->nb; ++i)
        if (c->act_h[i] != mask[i]) { same = false; break; }
    if (same) return SWJ_OK;
    // the previous upload must have left the pinned mirror before it changes
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->nb; ++i) c->act_h[i] = mask[i];
    SWJ_CUDA_TRY(cudaMemcpyAsync(c->act_d, c->act_h, c->nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return SWJ_OK;
}

struct Norms { std::vector<double> two, inf; };

int norms_of(swj_ctx *c, const double *x, int slot, Norms *out, const int *act)
{
    swj_bnorms(c->stream, c->nb, c->nu, x, c->nu, c->red, c->dscal + slot, SWJ_DS, act);
    int rc = read_scalars(c, slot, 2);
    if (rc) return rc;
    out->two.resize(c->nb);
    out->inf.resize(c->nb);
    for (int i = 0; i < c->nb; ++i) {
        out->two[i] = sqrt(hs(c, i, slot));
        out->inf[i] = hs(c, i, slot + 1);
    }
    return SWJ_OK;
}

void count_residual(swj_stats *st, const std::vector<int> &mask, int prec)
{
    if (!st) return;
    for (size_t i = 0; i < mask.size(); ++i)
        if (mask[i]) {
            st[i].residual_evals++;
            if (prec == SWJ_FP64) st[i].residual_evals_fp64++;
            if (prec == SWJ_FF) st[i].residual_evals_ff++;
        }
}

// The device work of Arnoldi step j for the instances flagged in act_d.
// V and Z rows of instance i live at i * (rows * nu) + j * nu; the apply and
// the JVP work on [nb][nu] vectors, so v_j is gathered into E_try first.
int arnoldi_device_step(swj_ctx *c, int j, const double *u, const double *Ebase, int prec)
{
    const int n = c->nu, nb = c->nb;
    const size_t ld = (size_t)n;
    const size_t vst = (size_t)(c->kry_m + 1) * n, zst = (size_t)c->kry_m * n;
    cudaStream_t s = c->stream;
    const int *act = c->act_d;
    double *Vj = c->V + (size_t)j * ld, *Zj = c->Z + (size_t)j * ld;
    double *w = c->V + (size_t)(j + 1) * ld;
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->E_try, ld * sizeof(double), Vj, vst * sizeof(double),
                                   ld * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    int rc = swj_pc_apply(c, c->E_try, c->u_try, act);
    if (rc) return rc;
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(Zj, zst * sizeof(double), c->u_try, ld * sizeof(double),
                                   ld * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    // w = J z_j: exact, or the FD-JVP about (u, Ebase).  Refinement steps
    // (Ebase == nullptr) take the exact product in FP32: a central difference
    // of FP32 residuals costs as much (two residuals against one tangent) and
    // is ~100 times less accurate, which leaves one refinement step just short
    // of the FP64 tolerance.
    if (c->opts.jvp == SWJ_JVP_EXACT || !Ebase)
        rc = swj_jvp_exact_impl(c, u, c->u_try, c->E_try, prec == SWJ_FP64 ? SWJ_FP64 : SWJ_FP32, act);
    else
        rc = swj_jvp_impl(c, u, Ebase, c->u_try, c->E_try, prec, c->opts.fd_h, act);
    if (rc) return rc;
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(w, vst * sizeof(double), c->E_try, ld * sizeof(double),
                                   ld * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    // classical Gram-Schmidt, twice
    swj_bmdot(s, nb, n, j + 1, c->V, ld, vst, w, vst, c->red, c->dscal + DS_H1, SWJ_DS, act);
    swj_bmgemv_sub(s, nb, n, j + 1, c->V, ld, vst, c->dscal + DS_H1, SWJ_DS, w, vst, act);
    swj_bmdot(s, nb, n, j + 1, c->V, ld, vst, w, vst, c->red, c->dscal + DS_H2, SWJ_DS, act);
    swj_bmgemv_sub(s, nb, n, j + 1, c->V, ld, vst, c->dscal + DS_H2, SWJ_DS, w, vst, act);
    SWJ_COUNT_LAUNCH();
    k_add_rows<<<nb, 64, 0, s>>>(j + 1, c->dscal, act, nb);
    swj_bnorms(s, nb, n, w, vst, c->red, c->dscal + DS_NW, SWJ_DS, act);
    SWJ_COUNT_LAUNCH();
    k_normalise<<<dim3(nblk(n, 256), nb), 256, 0, s>>>(n, w, vst, c->dscal, act);
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->hpin + DS_H1, SWJ_DS * sizeof(double), c->dscal + DS_H1,
                                   SWJ_DS * sizeof(double), (size_t)(j + 1) * sizeof(double), nb,
                                   cudaMemcpyDeviceToHost, s));
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->hpin + DS_NW, SWJ_DS * sizeof(double), c->dscal + DS_NW,
                                   SWJ_DS * sizeof(double), 2 * sizeof(double), nb,
                                   cudaMemcpyDeviceToHost, s));
    return SWJ_OK;
}

// Run Arnoldi step j: replay its captured graph, capturing it on first use.
// `kind`: 0 FP64 Newton, 1 FP32 Newton, 2 FP32-JVP refinement (the graphs bake
// in u and the JVP base buffer, both fixed for one kind and one u).
int arnoldi_step(swj_ctx *c, int kind, int j, const double *u, const double *Ebase, int prec)
{
    if (!c->graphs_enabled || c->time_pairs || !c->arn_graph) return arnoldi_device_step(c, j, u, Ebase, prec);
    cudaGraphExec_t &ge = c->arn_graph[kind * c->kry_m + j];
    if (!ge) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            c->graphs_enabled = 0;
            return arnoldi_device_step(c, j, u, Ebase, prec);
        }
        int rc = arnoldi_device_step(c, j, u, Ebase, prec);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess || !g) {
            // The capture was invalidated, e.g. by a device-wide synchronisation
            // from another host thread (cudaFree of another context in a
            // server) while it ran; the errors the step met came from that.
            // Nothing was executed: run the step now, capture it next time.
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return arnoldi_device_step(c, j, u, Ebase, prec);
        }
        if (rc) {
            cudaGraphDestroy(g);
            c->graphs_enabled = 0;
            return rc;
        }
        if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            ge = nullptr;
            c->graphs_enabled = 0;
            return arnoldi_device_step(c, j, u, Ebase, prec);
        }
        cudaGraphDestroy(g);
    }
    SWJ_CUDA_TRY(cudaGraphLaunch(ge, c->stream));
    return SWJ_OK;
}

// Right-preconditioned restarted GMRES for J x = rhs (rhs = c->rvec, x = c->du,
// both [nb][nu]) about (u, Ebase) in precision `prec`, for the instances with
// on[i] = 1.  Per instance: stop when the rotated residual estimate is <=
// rtol[i] ||rhs_i||_2 or after maxit iterations.  res[i] gets the estimate;
// failed[i] = 1 for an instance that met a NaN or Inf (it drops out, the
// others go on).
int gmres(swj_ctx *c, int kind, const double *u, const double *Ebase, int prec,
          const std::vector<int> &on, const std::vector<double> &rtol, int maxit,
          std::vector<double> &res, std::vector<int> &iters, std::vector<int> &failed, swj_stats *st)
{
    const int n = c->nu, m = c->kry_m, nb = c->nb;
    const size_t ld = (size_t)n, vst = (size_t)(m + 1) * n, zst = (size_t)m * n;
    cudaStream_t s = c->stream;
    int rc = set_mask(c, on);
    if (rc) return rc;
    Norms nb0;
    rc = norms_of(c, c->rvec, DS_NR, &nb0, c->act_d);
    if (rc) return rc;
    swj_bfill(s, nb, n, 0.0, c->du, ld, c->act_d);
    res.assign(nb, 0.0);
    iters.assign(nb, 0);
    failed.assign(nb, 0);
    std::vector<int> live(nb, 0);
    std::vector<double> beta(nb, 0.0), target(nb, 0.0);
    for (int i = 0; i < nb; ++i) {
        if (!on[i]) continue;
        if (!isfinite(nb0.two[i])) { failed[i] = 1; continue; }
        res[i] = nb0.two[i];
        target[i] = rtol[i] * nb0.two[i];
        beta[i] = nb0.two[i];
        live[i] = nb0.two[i] > 0.0;
        hs(c, i, DS_SC) = live[i] ? 1.0 / nb0.two[i] : 0.0;
    }
    rc = set_mask(c, live);
    if (rc) return rc;
    rc = write_scalars(c, DS_SC, 1);
    if (rc) return rc;
    // v_0 = rhs / ||rhs|| into V row 0 of every instance
    swj_bscale(s, nb, n, c->dscal + DS_SC, SWJ_DS, 1.0, 0, c->rvec, c->E_try, ld, c->act_d);
    SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->V, vst * sizeof(double), c->E_try, ld * sizeof(double),
                                   ld * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    std::vector<std::vector<double>> R(nb), Hraw(nb), cs(nb), sn(nb), gv(nb), y(nb);
    for (int i = 0; i < nb; ++i) {
        R[i].assign((size_t)(m + 1) * m, 0.0);
        Hraw[i].assign((size_t)(m + 1) * m, 0.0);
        cs[i].assign(m, 0.0);
        sn[i].assign(m, 0.0);
        gv[i].assign(m + 1, 0.0);
        y[i].assign(m, 0.0);
    }
    std::vector<int> kk(nb, 0);
    for (;;) {
        std::vector<int> cyc = live;   // instances in this restart cycle
        for (int i = 0; i < nb; ++i) {
            if (!cyc[i]) continue;
            std::fill(gv[i].begin(), gv[i].end(), 0.0);
            gv[i][0] = beta[i];
            kk[i] = 0;
        }
        std::vector<int> step = cyc;
        for (int j = 0; j < m; ++j) {
            bool any = false;
            for (int i = 0; i < nb; ++i) any |= step[i] != 0;
            if (!any) break;
            rc = set_mask(c, step);
            if (rc) return rc;
            rc = arnoldi_step(c, kind, j, u, Ebase, prec);
            if (rc) return rc;
            SWJ_CUDA_TRY(cudaStreamSynchronize(s));
            if (c->opts.jvp == SWJ_JVP_EXACT || !Ebase) {
                for (int i = 0; st && i < c->nb; ++i)
                    if (step[i]) st[i].exact_jvps++;
            } else {
                count_residual(st, step, prec);
            }
            for (int i = 0; i < nb; ++i) {
                if (!step[i]) continue;
                if (st) { st[i].precond_applies++; st[i].krylov_iters++; }
                double hn = sqrt(hs(c, i, DS_NW));
                bool bad = !isfinite(hn);
                for (int q = 0; q <= j && !bad; ++q) bad = !isfinite(hs(c, i, DS_H1 + q));
                if (bad) { failed[i] = 1; step[i] = 0; cyc[i] = 0; continue; }
                double *col = &R[i][(size_t)j * (m + 1)];
                for (int q = 0; q <= j; ++q) {
                    col[q] = hs(c, i, DS_H1 + q);
                    Hraw[i][(size_t)j * (m + 1) + q] = col[q];
                }
                col[j + 1] = hn;
                Hraw[i][(size_t)j * (m + 1) + j + 1] = hn;
                for (int q = 0; q < j; ++q) {
                    double t = cs[i][q] * col[q] + sn[i][q] * col[q + 1];
                    col[q + 1] = -sn[i][q] * col[q] + cs[i][q] * col[q + 1];
                    col[q] = t;
                }
                double a = col[j], b2 = col[j + 1];
                double rr = hypot(a, b2);
                cs[i][j] = (rr > 0) ? a / rr : 1.0;
                sn[i][j] = (rr > 0) ? b2 / rr : 0.0;
                col[j] = rr;
                col[j + 1] = 0.0;
                gv[i][j + 1] = -sn[i][j] * gv[i][j];
                gv[i][j] = cs[i][j] * gv[i][j];
                res[i] = fabs(gv[i][j + 1]);
                iters[i]++;
                kk[i] = j + 1;
                if (res[i] <= target[i] || hn == 0.0 || iters[i] >= maxit) step[i] = 0;
            }
        }
        // x += Z y, y = R^-1 g per instance (upper triangular k x k)
        int kmax = 0;
        for (int i = 0; i < nb; ++i) {
            if (!cyc[i]) continue;
            int k = kk[i];
            kmax = std::max(kmax, k);
            for (int q = k - 1; q >= 0 && !failed[i]; --q) {
                double v = gv[i][q];
                for (int r = q + 1; r < k; ++r) v -= R[i][(size_t)r * (m + 1) + q] * y[i][r];
                y[i][q] = v / R[i][(size_t)q * (m + 1) + q];
                if (!isfinite(y[i][q])) failed[i] = 1;
            }
            if (failed[i]) { cyc[i] = 0; continue; }
            for (int q = 0; q < m; ++q) hs(c, i, DS_Y + q) = (q < k) ? y[i][q] : 0.0;
        }
        if (kmax > 0) {
            rc = set_mask(c, cyc);
            if (rc) return rc;
            rc = write_scalars(c, DS_Y, kmax);
            if (rc) return rc;
            swj_bcombine(s, nb, n, kmax, c->Z, ld, zst, c->dscal + DS_Y, SWJ_DS, c->du, ld, 1, c->act_d);
        }
        // restart the instances that neither converged nor ran out of iterations
        std::vector<int> again(nb, 0);
        bool any = false;
        for (int i = 0; i < nb; ++i) {
            if (!cyc[i]) continue;
            bool breakdown = kk[i] > 0 && Hraw[i][(size_t)(kk[i] - 1) * (m + 1) + kk[i]] == 0.0;
            if (res[i] > target[i] && iters[i] < maxit && !breakdown) { again[i] = 1; any = true; }
        }
        if (!any) break;
        // r = V_{k+1} (beta e1 - Hraw y)
        int kc = 0;
        for (int i = 0; i < nb; ++i) {
            if (!again[i]) continue;
            int k = kk[i];
            std::vector<double> cvec(m + 1, 0.0);
            cvec[0] = beta[i];
            for (int q = 0; q < k; ++q)
                for (int r = 0; r <= q + 1; ++r) cvec[r] -= Hraw[i][(size_t)q * (m + 1) + r] * y[i][q];
            for (int r = 0; r <= m; ++r) hs(c, i, DS_C + r) = (r <= k) ? cvec[r] : 0.0;
            kc = std::max(kc, k + 1);
        }
        rc = set_mask(c, again);
        if (rc) return rc;
        rc = write_scalars(c, DS_C, kc);
        if (rc) return rc;
        swj_bcombine(s, nb, n, kc, c->V, ld, vst, c->dscal + DS_C, SWJ_DS, c->rvec, ld, 0, c->act_d);
        Norms nr;
        rc = norms_of(c, c->rvec, DS_NT, &nr, c->act_d);
        if (rc) return rc;
        for (int i = 0; i < nb; ++i) {
            if (!again[i]) continue;
            if (!isfinite(nr.two[i])) { failed[i] = 1; again[i] = 0; continue; }
            beta[i] = nr.two[i];
            if (beta[i] <= target[i]) again[i] = 0;
            hs(c, i, DS_SC) = again[i] ? 1.0 / beta[i] : 0.0;
        }
        live = again;
        bool more = false;
        for (int i = 0; i < nb; ++i) more |= live[i] != 0;
        if (!more) break;
        rc = set_mask(c, live);
        if (rc) return rc;
        rc = write_scalars(c, DS_SC, 1);
        if (rc) return rc;
        swj_bscale(s, nb, n, c->dscal + DS_SC, SWJ_DS, 1.0, 0, c->rvec, c->E_try, ld, c->act_d);
        SWJ_CUDA_TRY(cudaMemcpy2DAsync(c->V, vst * sizeof(double), c->E_try, ld * sizeof(double),
                                       ld * sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
    }
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

// GMRES tolerance of the refinement steps: their JVPs (exact, FP32 all-pairs
// part) are accurate to ~1e-7 relative, so one step contracts the FP64
// residual by about this factor
constexpr double kRefineEta = 1e-4;

struct Phase {
    std::vector<double> finf, f2;
    std::vector<int> status;     // SWJ_PENDING while iterating
};

// Damped inexact Newton in one residual precision on the instances whose
// status is SWJ_PENDING; E_cur holds E(u) on entry (norms in ph) and on exit.
// refine: the FP64 residual with FP32 JVPs about the same u (MIXED mode).
int newton_phase(swj_ctx *c, double *u, int prec, double tol, int max_it, Phase &ph, swj_stats *st,
                 bool stop_on_stall, bool refine)
{
    const int n = c->nu, nb = c->nb;
    const size_t ld = (size_t)n;
    cudaStream_t s = c->stream;
    const swj_opts &o = c->opts;
    std::vector<double> eta(nb, refine ? kRefineEta : o.eta_max);
    const int kind = refine ? 2 : (prec == SWJ_FP64 ? 0 : 1);
    int rc;
    for (int it = 0; it <= max_it; ++it) {
        std::vector<int> on(nb, 0);
        bool any = false;
        for (int i = 0; i < nb; ++i) {
            if (ph.status[i] != SWJ_PENDING) continue;
            if (!isfinite(ph.finf[i])) { ph.status[i] = SWJ_ENAN; continue; }
            if (ph.finf[i] < tol) { ph.status[i] = SWJ_OK; continue; }
            if (it == max_it) { ph.status[i] = SWJ_ENOTCONV; continue; }
            on[i] = 1;
            any = true;
        }
        if (!any) break;
        rc = set_mask(c, on);
        if (rc) return rc;
        // refinement: exact JVPs with the FP32 all-pairs tangent (no FP32 base residual needed)
        const double *Ebase = refine ? nullptr : c->E_cur;
        const int jprec = refine ? SWJ_FP32 : prec;
        swj_bscale(s, nb, n, nullptr, 0, -1.0, 0, c->E_cur, c->rvec, ld, c->act_d);
        std::vector<double> gres;
        std::vector<int> giters, gfail;
        rc = gmres(c, kind, u, Ebase, jprec, on, eta, o.max_krylov, gres, giters, gfail, st);
        if (rc) return rc;
        for (int i = 0; i < nb; ++i)
            if (gfail[i]) { ph.status[i] = SWJ_ENAN; on[i] = 0; }
        // line search: lambda halves from 1 per instance
        std::vector<double> lam(nb, 1.0), tn(nb, 0.0), ti(nb, 0.0);
        std::vector<int> trying = on, accepted(nb, 0);
        Norms nt;
        for (;;) {
            rc = set_mask(c, trying);
            if (rc) return rc;
            for (int i = 0; i < nb; ++i) hs(c, i, DS_LAM) = trying[i] ? lam[i] : 0.0;
            rc = write_scalars(c, DS_LAM, 1);
            if (rc) return rc;
            swj_bcopy(s, nb, n, u, c->u_try, ld, c->act_d);
            swj_baxpy(s, nb, n, c->dscal + DS_LAM, SWJ_DS, 1.0, c->du, c->u_try, ld, c->act_d);
            rc = swj_residual_impl(c, c->u_try, c->E_try, prec, c->act_d);
            if (rc) return rc;
            count_residual(st, trying, prec);
            rc = norms_of(c, c->E_try, DS_NE, &nt, c->act_d);
            if (rc) return rc;
            bool more = false;
            for (int i = 0; i < nb; ++i) {
                if (!trying[i]) continue;
                double f2 = ph.f2[i];
                bool ok = isfinite(nt.two[i]) &&
                          (refine ? nt.two[i] < f2 : nt.two[i] <= (1.0 - 1e-4 * lam[i]) * f2);
                if (ok) {
                    accepted[i] = 1;
                    trying[i] = 0;
                    tn[i] = nt.two[i];
                    ti[i] = nt.inf[i];
                } else {
                    lam[i] *= 0.5;
                    if (st) st[i].line_search_cuts++;
                    if (lam[i] < (refine ? 1.0 / 8.0 : 1.0 / 1024.0)) {
                        trying[i] = 0;
                        ph.status[i] = SWJ_ELINESEARCH;
                    } else {
                        more = true;
                    }
                }
            }
            if (!more) break;
        }
        rc = set_mask(c, accepted);
        if (rc) return rc;
        swj_bcopy(s, nb, n, c->u_try, u, ld, c->act_d);
        swj_bcopy(s, nb, n, c->E_try, c->E_cur, ld, c->act_d);
        for (int i = 0; i < nb; ++i) {
            if (!accepted[i]) continue;
            double f2 = ph.f2[i];
            if (!refine) {
                // Eisenstat-Walker choice 1 with safeguard
                double lin = (1.0 - lam[i]) * f2 + lam[i] * gres[i];
                double e_new = fabs(tn[i] - lin) / f2;
                double safe = pow(eta[i], 0.5 * (1.0 + sqrt(5.0)));
                if (safe > 0.1 && e_new < safe) e_new = safe;
                eta[i] = std::min(o.eta_max, std::max(o.eta_min, e_new));
            }
            double prev = ph.finf[i];
            ph.f2[i] = tn[i];
            ph.finf[i] = ti[i];
            if (st) {
                st[i].newton_iters++;
                if (refine) st[i].refine_iters++;
            }
            if (o.verbose)
                fprintf(stderr, "[swj] %s inst=%d it=%d |E|inf=%.3e |E|2=%.3e lam=%.3g gmres=%d eta=%.2e\n",
                        refine ? (prec == SWJ_FF ? "refine ff" : "refine fp64")
                               : (prec == SWJ_FP64 ? "newton fp64" : "newton fp32"),
                        i, it + 1, ti[i], tn[i], lam[i], giters[i], eta[i]);
            if (stop_on_stall && ti[i] > 0.5 * prev && ti[i] < 100.0 * tol) ph.status[i] = SWJ_OK;
        }
    }
    return SWJ_OK;
}

}  // namespace

int swj_residual_impl(swj_ctx *c, const double *u, double *E, int precision, const int *act)
{
    swj_launch_mesh_step(c, u, E, act);
    if (!swj_tuned_of(c, precision)) {
        int rc = swj_pair_autotune(c, precision, act);
        if (rc) return rc;
    }
    const bool rec = c->time_pairs && c->tev && c->n_timed < SWJ_MAX_TIMED;
    if (rec) cudaEventRecord(c->tev[2 * c->n_timed], c->stream);
    if (precision == SWJ_FP64) swj_launch_pairs64(c, c->plan64, act);
    else if (precision == SWJ_FF) swj_launch_pairs_ff(c, c->planff, act);
    else swj_launch_pairs32(c, c->plan32, act);
    if (rec) {
        cudaEventRecord(c->tev[2 * c->n_timed + 1], c->stream);
        c->tev_prec[c->n_timed++] = precision;
    }
    swj_launch_assemble(c, E, swj_plan_of(c, precision).P, act);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_jvp_impl(swj_ctx *c, const double *u, const double *Eu, const double *v, double *Jv,
                 int precision, double h_fixed, const int *act)
{
    cudaStream_t s = c->stream;
    const int n = c->nu, nb = c->nb;
    const bool central = (Eu == nullptr);
    if (!(h_fixed > 0.0)) {
        swj_bnorms(s, nb, n, u, n, c->red, c->dscal + DS_NU, SWJ_DS, act);
        swj_bnorms(s, nb, n, v, n, c->red, c->dscal + DS_NV, SWJ_DS, act);
    }
    const double epsm = (precision == SWJ_FP64) ? 2.220446049250313e-16 : 1.1920928955078125e-07;
    SWJ_COUNT_LAUNCH();
    k_fd_h<<<nblk(nb, 64), 64, 0, s>>>(c->dscal, sqrt(epsm), h_fixed, act, nb);
    SWJ_COUNT_LAUNCH();
    k_perturb<<<dim3(nblk(n, 256), nb), 256, 0, s>>>(n, u, v, c->dscal, 1.0, c->u_tmp, act);
    int rc = swj_residual_impl(c, c->u_tmp, c->E_tmp, precision, act);
    if (rc) return rc;
    if (central) {
        SWJ_COUNT_LAUNCH();
        k_perturb<<<dim3(nblk(n, 256), nb), 256, 0, s>>>(n, u, v, c->dscal, -1.0, c->u_tmp2, act);
        rc = swj_residual_impl(c, c->u_tmp2, c->E_tmp2, precision, act);
        if (rc) return rc;
    }
    SWJ_COUNT_LAUNCH();
    k_fd_diff<<<dim3(nblk(n, 256), nb), 256, 0, s>>>(n, c->E_tmp, central ? c->E_tmp2 : Eu, c->dscal,
                                                      central ? 2.0 : 1.0, Jv, act);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

void swj_graphs_free(swj_ctx *c)
{
    if (!c->arn_graph) return;
    for (int i = 0; i < 3 * c->kry_m; ++i)
        if (c->arn_graph[i]) cudaGraphExecDestroy(c->arn_graph[i]);
    free(c->arn_graph);
    c->arn_graph = nullptr;
    c->arn_u = nullptr;
}

// stats: array of nb (may be null)
int swj_solve_impl(swj_ctx *c, double *u, swj_stats *stats)
{
    const int nb = c->nb;
    std::vector<swj_stats> local(stats ? 0 : nb);
    swj_stats *st = stats ? stats : local.data();
    long long pairs = (long long)c->T * c->S;
    for (int i = 0; i < nb; ++i) {
        memset(&st[i], 0, sizeof(swj_stats));
        st[i].final_norm_inf_fp64 = -1.0;
        st[i].pairs_per_residual_hi = (int)(pairs >> 31);
        st[i].pairs_per_residual_lo = (int)(pairs & 0x7fffffffLL);
    }
    double t0 = now_ms();
    const swj_opts &o = c->opts;
    int rc;
    auto finish = [&](int code) {
        double t = now_ms() - t0;
        for (int i = 0; i < nb; ++i) {
            st[i].t_total_ms = t;
            if (code) st[i].status = code;
        }
        return code;
    };
    if (!c->pc_ready) {
        double ts = now_ms();
        rc = swj_pc_setup(c);
        for (int i = 0; i < nb; ++i) st[i].t_setup_ms = now_ms() - ts;
        if (rc) return finish(rc);
    }
    // the Arnoldi graphs bake in the address of u: capture anew for another u
    if (c->arn_u != u || !c->arn_graph) {
        swj_graphs_free(c);
        c->arn_graph = (cudaGraphExec_t *)calloc(3 * c->kry_m, sizeof(cudaGraphExec_t));
        c->arn_u = u;
    }
    const bool mixed = (o.solve_mode == SWJ_SOLVE_MIXED);
    const int prec = mixed ? SWJ_FP32 : SWJ_FP64;
    std::vector<int> all(nb, 1);
    // (re)upload the mask: the preconditioner set-up uses the flags too
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < nb; ++i) c->act_h[i] = 1;
    SWJ_CUDA_TRY(cudaMemcpyAsync(c->act_d, c->act_h, nb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    rc = swj_residual_impl(c, u, c->E_cur, prec, c->act_d);
    if (rc) return finish(rc);
    count_residual(st, all, prec);
    Norms n0;
    rc = norms_of(c, c->E_cur, DS_NE, &n0, c->act_d);
    if (rc) return finish(rc);
    Phase ph{n0.inf, n0.two, std::vector<int>(nb, SWJ_PENDING)};
    rc = newton_phase(c, u, prec, mixed ? o.mixed_tol_inf : o.ftol_inf, o.max_newton, ph, st, mixed, false);
    if (rc) return finish(rc);
    if (!mixed) {
        for (int i = 0; i < nb; ++i) {
            st[i].final_norm_inf = ph.finf[i];
            st[i].final_norm_inf_fp64 = ph.finf[i];
            st[i].status = ph.status[i];
        }
        finish(0);
        rc = swj_pc_status(c);
        if (rc) return finish(rc);
        for (int i = 0; i < nb; ++i)
            if (st[i].status) return st[i].status;
        return SWJ_OK;
    }
    // FP64 refinement for every instance whose FP32 phase did not fail hard
    Phase rf;
    rf.finf.assign(nb, 0.0);
    rf.f2.assign(nb, 0.0);
    rf.status.assign(nb, SWJ_PENDING);
    std::vector<int> go(nb, 0);
    for (int i = 0; i < nb; ++i) {
        st[i].final_norm_inf = ph.finf[i];
        int s1 = ph.status[i];
        if (s1 == SWJ_ENAN || s1 == SWJ_ECUDA || s1 == SWJ_ENOMEM || s1 == SWJ_ESINGULAR) rf.status[i] = s1;
        else go[i] = 1;
    }
    rc = set_mask(c, go);
    if (rc) return finish(rc);
    const int rprec = o.refine_precision;   // FP64-accurate: float-float or FP64
    rc = swj_residual_impl(c, u, c->E_cur, rprec, c->act_d);
    if (rc) return finish(rc);
    count_residual(st, go, rprec);
    Norms e64;
    rc = norms_of(c, c->E_cur, DS_NE, &e64, c->act_d);
    if (rc) return finish(rc);
    for (int i = 0; i < nb; ++i) {
        if (!go[i]) continue;
        rf.finf[i] = e64.inf[i];
        rf.f2[i] = e64.two[i];
    }
    rc = newton_phase(c, u, rprec, o.refine_tol_inf, o.refine_max, rf, st, false, true);
    if (rc) return finish(rc);
    for (int i = 0; i < nb; ++i) {
        if (go[i]) {
            st[i].final_norm_inf = rf.finf[i];
            st[i].final_norm_inf_fp64 = rf.finf[i];
        }
        st[i].status = rf.status[i];
    }
    finish(0);
    rc = swj_pc_status(c);
    if (rc) return finish(rc);
    for (int i = 0; i < nb; ++i)
        if (st[i].status) return st[i].status;
    return SWJ_OK;
}
