// C ABI of libswj (declared in include/swj.h): context lifecycle, argument
// checks and dispatch to the kernel families.
#include "swj_internal.h"
#include <new>
#include <stdlib.h>
#include <string.h>
#include <vector>

std::atomic<unsigned long long> g_swj_launches{0};

namespace {

bool valid_mesh(const swj_mesh *m)
{
    return m && m->N >= 4 && m->M >= 3 && m->dx > 0.0 && m->dy > 0.0 && m->n_rad >= 0.0 &&
           (long long)2 * (m->N + 1) * m->M < (1LL << 31) && (long long)(m->N - 1) * m->M < (1LL << 30);
}

bool valid_opts(const swj_opts *o)
{
    if (!o) return false;
    if (o->solve_mode != SWJ_SOLVE_FP64 && o->solve_mode != SWJ_SOLVE_MIXED) return false;
    if (o->block_bw < -1 || (o->block_bw > 0 && o->block_bw % 2 == 0)) return false;
    if (o->gmres_restart < 1 || o->gmres_restart > 60) return false;
    if (o->max_newton < 0 || o->max_krylov < 1 || o->refine_max < 0) return false;
    if (!(o->ftol_inf > 0.0) || !(o->eta_max > 0.0) || o->eta_max >= 1.0) return false;
    if (!(o->eta_min > 0.0) || o->eta_min > o->eta_max) return false;
    if (o->fd_h < 0.0 || !(o->mixed_tol_inf > 0.0) || !(o->refine_tol_inf > 0.0)) return false;
    if (o->autotune != 0 && o->autotune != 1) return false;
    if (o->refine_precision != SWJ_FF && o->refine_precision != SWJ_FP64) return false;
    if (o->jvp != SWJ_JVP_FD && o->jvp != SWJ_JVP_EXACT) return false;
    if (o->forcing != SWJ_FORCING_SOURCE && o->forcing != SWJ_FORCING_PRESSURE) return false;
    if (o->lu_products != SWJ_LU_FP64 && o->lu_products != SWJ_LU_SLICED) return false;
    if (o->lu_order != SWJ_LU_TOP_DOWN && o->lu_order != SWJ_LU_TWO_SIDED) return false;
    if (o->wait_limit < 0) return false;
    if (o->sm_partition != 0 && o->sm_partition != 1) return false;
    return true;
}

template <typename T> int dalloc(swj_ctx *c, T **p, size_t count)
{
    size_t b = count * sizeof(T);
    if (b == 0) b = sizeof(T);
    if (cudaMalloc((void **)p, b) != cudaSuccess) { *p = nullptr; return SWJ_ENOMEM; }
    c->bytes += b;
    return SWJ_OK;
}

void free_all(swj_ctx *c)
{
    void *ptrs[] = {c->zeta, c->g, c->zetay, c->gy, c->spl_cp, c->spl_a, c->spl_inv, c->e2part,
                    c->Ival, c->src64, c->src32, c->tgt64_base, c->tgt32_base, c->partial,
                    c->u_tmp, c->E_tmp, c->u_tmp2, c->E_tmp2, c->E_cur, c->u_try, c->E_try, c->E_base32, c->du,
                    c->rvec, c->dscal, c->red, c->V, c->Z, c->Fd, c->epsd, c->act_d,
                    c->dnode, c->tsrc64, c->tsrc32, c->ttgt64_base, c->ttgt32_base, c->de2part, c->hs_buf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->hpin) cudaFreeHost(c->hpin);
    if (c->act_h) cudaFreeHost(c->act_h);
    free(c->F);
    free(c->eps);
    swj_graphs_free(c);
    swj_pc_free(c);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->tev) {
        for (int i = 0; i < 2 * SWJ_MAX_TIMED; ++i) cudaEventDestroy(c->tev[i]);
        free(c->tev);
        free(c->tev_prec);
    }
}

int alloc_all(swj_ctx *c)
{
    const size_t S = c->S, T = c->T, M = c->M, nu = c->nu, nb = c->nb;
    int rc = 0;
    rc |= dalloc(c, &c->zeta, nb * S);
    rc |= dalloc(c, &c->g, nb * S);
    rc |= dalloc(c, &c->zetay, nb * S);
    rc |= dalloc(c, &c->gy, nb * S);
    rc |= dalloc(c, &c->spl_cp, M);
    rc |= dalloc(c, &c->spl_a, M);
    rc |= dalloc(c, &c->spl_inv, M);
    rc |= dalloc(c, &c->e2part, nb * T);
    rc |= dalloc(c, &c->Ival, nb * T);
    rc |= dalloc(c, &c->src64, nb * S);
    rc |= dalloc(c, &c->src32, nb * S);
    rc |= dalloc(c, &c->tgt64_base, 8 * nb * T);
    rc |= dalloc(c, &c->tgt32_base, 8 * nb * T);
    rc |= dalloc(c, &c->Fd, nb);
    rc |= dalloc(c, &c->epsd, nb);
    rc |= dalloc(c, &c->act_d, nb);
    rc |= dalloc(c, &c->dnode, 4 * nb * S);
    rc |= dalloc(c, &c->tsrc64, nb * S);
    rc |= dalloc(c, &c->tsrc32, nb * S);
    rc |= dalloc(c, &c->ttgt64_base, 8 * nb * T);
    rc |= dalloc(c, &c->ttgt32_base, 8 * nb * T);
    rc |= dalloc(c, &c->de2part, nb * T);
    if (rc) return SWJ_ENOMEM;
    // each field of the target arrays holds nb blocks of T values
    const size_t NT = nb * T;
    double *b = c->tgt64_base;
    c->tgt64 = TgtArrays64{b, b + NT, b + 2 * NT, b + 3 * NT, b + 4 * NT, b + 5 * NT, b + 6 * NT, b + 7 * NT};
    float *f = c->tgt32_base;
    c->tgt32 = TgtArrays32{f, f + NT, f + 2 * NT, f + 3 * NT, f + 4 * NT, f + 5 * NT, f + 6 * NT, f + 7 * NT};
    b = c->ttgt64_base;
    c->ttgt64 = TgtArrays64{b, b + NT, b + 2 * NT, b + 3 * NT, b + 4 * NT, b + 5 * NT, b + 6 * NT, b + 7 * NT};
    f = c->ttgt32_base;
    c->ttgt32 = TgtArrays32{f, f + NT, f + 2 * NT, f + 3 * NT, f + 4 * NT, f + 5 * NT, f + 6 * NT, f + 7 * NT};
    c->plan64 = swj_pair_plan(c, SWJ_FP64);
    c->plan32 = swj_pair_plan(c, SWJ_FP32);
    c->planff = swj_pair_plan(c, SWJ_FF);
    // room for the partial sums of every compiled tile shape (the autotuner tries them all)
    const int P = swj_pair_max_chunks(c);
    c->partial_cap = (size_t)P * T * nb;
    rc |= dalloc(c, &c->partial, c->partial_cap);
    double **vecs[] = {&c->u_tmp, &c->E_tmp, &c->u_tmp2, &c->E_tmp2, &c->E_cur, &c->u_try, &c->E_try,
                       &c->E_base32, &c->du, &c->rvec};
    for (double **v : vecs) rc |= dalloc(c, v, nb * nu);
    rc |= dalloc(c, &c->dscal, nb * SWJ_DS);
    rc |= dalloc(c, &c->red, nb * SWJ_RED);
    c->kry_m = c->opts.gmres_restart;
    rc |= dalloc(c, &c->V, nb * (c->kry_m + 1) * nu);
    rc |= dalloc(c, &c->Z, nb * c->kry_m * nu);
    if (rc) return SWJ_ENOMEM;
    if (cudaMallocHost((void **)&c->hpin, nb * SWJ_DS * sizeof(double)) != cudaSuccess) {
        c->hpin = nullptr;
        return SWJ_ENOMEM;
    }
    if (cudaMallocHost((void **)&c->act_h, nb * sizeof(int)) != cudaSuccess) {
        c->act_h = nullptr;
        return SWJ_ENOMEM;
    }
    for (size_t i = 0; i < nb; ++i) c->act_h[i] = 1;
    double *cp = (double *)malloc(3 * M * sizeof(double));
    if (!cp) return SWJ_ENOMEM;
    swj_spline_coeffs((int)M, cp, cp + M, cp + 2 * M);
    cudaError_t e1 = cudaMemcpy(c->spl_cp, cp, M * sizeof(double), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(c->spl_a, cp + M, M * sizeof(double), cudaMemcpyHostToDevice);
    cudaError_t e3 = cudaMemcpy(c->spl_inv, cp + 2 * M, M * sizeof(double), cudaMemcpyHostToDevice);
    free(cp);
    if (e1 || e2 || e3) return SWJ_ECUDA;
    if (cudaMemcpy(c->Fd, c->F, nb * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->epsd, c->eps, nb * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->act_d, c->act_h, nb * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return SWJ_ECUDA;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
        return SWJ_ECUDA;
    c->graphs_enabled = 1;
    return SWJ_OK;
}

// device bytes alloc_all() requests for nb instances (plan from the current device)
int ctx_bytes(const swj_mesh *mesh, int nb, int kry_m, size_t *out)
{
    swj_ctx c;
    memset((void *)&c, 0, sizeof(c));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SWJ_ECUDA;
    c.N = mesh->N;
    c.M = mesh->M;
    c.T = (c.N - 1) * c.M;
    c.S = c.N * c.M;
    c.nu = 2 * (c.N + 1) * c.M;
    const size_t S = c.S, T = c.T, M = c.M, nu = c.nu, n = nb, d = sizeof(double);
    const size_t P = (size_t)swj_pair_max_chunks(&c);
    size_t b = 4 * n * S * d + 3 * M * d + 2 * n * T * d + n * S * sizeof(SrcRec64) +
               n * S * sizeof(SrcRec32) + 8 * n * T * d + 8 * n * T * sizeof(float) + 2 * n * d +
               n * sizeof(int) + P * T * n * d + 10 * n * nu * d + n * SWJ_DS * d + n * SWJ_RED * d +
               n * (size_t)(2 * kry_m + 1) * nu * d +
               // exact-JVP tangents
               4 * n * S * d + n * S * sizeof(SrcRec64) + n * S * sizeof(SrcRec32) + 8 * n * T * d +
               8 * n * T * sizeof(float) + n * T * d;
    *out = b;
    return SWJ_OK;
}

int create_ctx(swj_ctx **out, const swj_mesh *mesh, int nb, const double *F, const double *eps,
               const swj_opts *opts, void *stream)
{
    if (!out) return SWJ_EINVAL;
    *out = nullptr;
    if (!valid_mesh(mesh) || nb < 1 || !F || !eps) return SWJ_EINVAL;
    for (int i = 0; i < nb; ++i)
        if (!(F[i] > 0.0) || !(eps[i] >= 0.0)) return SWJ_EINVAL;
    swj_opts o;
    if (opts) o = *opts; else swj_default_opts(&o);
    if (!valid_opts(&o)) return SWJ_EINVAL;
    swj_ctx *c = new (std::nothrow) swj_ctx();
    if (!c) return SWJ_ENOMEM;
    memset((void *)c, 0, sizeof(*c));
    c->mesh = *mesh;
    c->opts = o;
    c->stream = (cudaStream_t)stream;
    c->nb = nb;
    c->F = (double *)malloc(nb * sizeof(double));
    c->eps = (double *)malloc(nb * sizeof(double));
    if (!c->F || !c->eps) {
        free(c->F);
        free(c->eps);
        delete c;
        return SWJ_ENOMEM;
    }
    memcpy(c->F, F, nb * sizeof(double));
    memcpy(c->eps, eps, nb * sizeof(double));
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
        free(c->F);
        free(c->eps);
        delete c;
        return SWJ_ECUDA;
    }
    c->N = mesh->N;
    c->M = mesh->M;
    c->n1 = c->N + 1;
    c->H = c->n1 * c->M;
    c->nu = 2 * c->H;
    c->T = (c->N - 1) * c->M;
    c->S = c->N * c->M;
    int rc = alloc_all(c);
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return SWJ_OK;
}

}  // namespace

extern "C" {

void swj_default_opts(swj_opts *o)
{
    if (!o) return;
    o->solve_mode = SWJ_SOLVE_MIXED;
    o->block_bw = -1;
    o->gmres_restart = 30;
    o->max_newton = 60;
    o->max_krylov = 300;
    o->ftol_inf = 1e-10;
    o->eta_max = 0.1;
    o->eta_min = 1e-6;
    o->fd_h = 0.0;
    o->refine_max = 4;
    o->mixed_tol_inf = 2e-6;
    o->refine_tol_inf = 1e-9;
    o->verbose = 0;
    o->autotune = 1;
    o->refine_precision = SWJ_FF;
    o->jvp = SWJ_JVP_FD;
    o->forcing = SWJ_FORCING_SOURCE;
    o->lu_products = SWJ_LU_SLICED;
    o->lu_order = SWJ_LU_TWO_SIDED;
    o->wait_limit = 0;
    o->sm_partition = 1;
}

int swj_set_test_hooks(swj_ctx *c, int hooks)
{
    if (!c || (hooks & ~SWJ_TEST_WITHHOLD_HELPERS)) return SWJ_EINVAL;
    c->test_hooks = hooks;
    return SWJ_OK;
}

int swj_create(swj_ctx **out, const swj_mesh *mesh, double F, double eps, const swj_opts *opts,
               void *stream)
{
    return create_ctx(out, mesh, 1, &F, &eps, opts, stream);
}

int swj_batch_create(swj_ctx **out, const swj_mesh *mesh, int count, const double *F,
                     const double *eps, const swj_opts *opts, void *stream)
{
    return create_ctx(out, mesh, count, F, eps, opts, stream);
}

int swj_batch_count(const swj_ctx *c) { return c ? c->nb : 0; }

void swj_destroy(swj_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

int swj_set_params(swj_ctx *c, double F, double eps)
{
    if (!c || !(F > 0.0) || !(eps >= 0.0)) return SWJ_EINVAL;
    for (int i = 0; i < c->nb; ++i) {
        if (F != c->F[i]) c->pc_ready = 0;
        c->F[i] = F;
        c->eps[i] = eps;
    }
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    SWJ_CUDA_TRY(cudaMemcpy(c->Fd, c->F, c->nb * sizeof(double), cudaMemcpyHostToDevice));
    SWJ_CUDA_TRY(cudaMemcpy(c->epsd, c->eps, c->nb * sizeof(double), cudaMemcpyHostToDevice));
    return SWJ_OK;
}

int swj_batch_set_params(swj_ctx *c, const double *F, const double *eps)
{
    if (!c || !F || !eps) return SWJ_EINVAL;
    for (int i = 0; i < c->nb; ++i)
        if (!(F[i] > 0.0) || !(eps[i] >= 0.0)) return SWJ_EINVAL;
    for (int i = 0; i < c->nb; ++i) {
        if (F[i] != c->F[i]) c->pc_ready = 0;
        c->F[i] = F[i];
        c->eps[i] = eps[i];
    }
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    SWJ_CUDA_TRY(cudaMemcpy(c->Fd, c->F, c->nb * sizeof(double), cudaMemcpyHostToDevice));
    SWJ_CUDA_TRY(cudaMemcpy(c->epsd, c->eps, c->nb * sizeof(double), cudaMemcpyHostToDevice));
    return SWJ_OK;
}

int swj_set_opts(swj_ctx *c, const swj_opts *o)
{
    if (!c || !valid_opts(o)) return SWJ_EINVAL;
    if (o->gmres_restart != c->kry_m) {
        double *V = nullptr, *Z = nullptr;
        if (cudaMalloc(&V, (size_t)c->nb * (o->gmres_restart + 1) * c->nu * sizeof(double)) != cudaSuccess)
            return SWJ_ENOMEM;
        if (cudaMalloc(&Z, (size_t)c->nb * o->gmres_restart * c->nu * sizeof(double)) != cudaSuccess) {
            cudaFree(V);
            return SWJ_ENOMEM;
        }
        cudaStreamSynchronize(c->stream);
        swj_graphs_free(c);
        c->bytes -= (size_t)c->nb * (2 * c->kry_m + 1) * c->nu * sizeof(double);
        cudaFree(c->V);
        cudaFree(c->Z);
        c->V = V;
        c->Z = Z;
        c->kry_m = o->gmres_restart;
        c->bytes += (size_t)c->nb * (2 * c->kry_m + 1) * c->nu * sizeof(double);
    }
    if (o->fd_h != c->opts.fd_h) swj_graphs_free(c);
    if (o->block_bw != c->opts.block_bw || o->solve_mode != c->opts.solve_mode ||
        o->lu_products != c->opts.lu_products || o->lu_order != c->opts.lu_order)
        c->pc_ready = 0;
    c->opts = *o;
    return SWJ_OK;
}

size_t swj_workspace_bytes(const swj_ctx *c) { return c ? c->bytes : 0; }

int swj_pair_variants(int precision)
{
    int n = 0;
    while (swj_pair_variant_info(precision, n, nullptr, nullptr, nullptr) == SWJ_OK) ++n;
    return n;
}

int swj_pair_config(const swj_ctx *c, int precision, int *variant, int *threads, int *targets,
                    int *packed)
{
    if (!c || !swj_valid_precision(precision)) return SWJ_EINVAL;
    const PairPlan &pl = swj_plan_of(const_cast<swj_ctx *>(c), precision);
    if (variant) *variant = pl.v;
    return swj_pair_variant_info(precision, pl.v, threads, targets, packed);
}

int swj_set_pair_config(swj_ctx *c, int precision, int variant)
{
    if (!c || !swj_valid_precision(precision)) return SWJ_EINVAL;
    if (swj_pair_variant_info(precision, variant, nullptr, nullptr, nullptr) != SWJ_OK) return SWJ_EINVAL;
    PairPlan pl = swj_pair_plan_variant(c, precision, variant);
    if ((size_t)pl.P * c->T * c->nb > c->partial_cap) return SWJ_EINVAL;
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    swj_graphs_free(c);   // captured steps bake in the old plan
    swj_plan_of(c, precision) = pl;
    swj_tuned_of(c, precision) = 1;
    return SWJ_OK;
}

size_t swj_footprint_bytes(const swj_mesh *mesh, int count, const swj_opts *opts)
{
    swj_opts o;
    if (opts) o = *opts; else swj_default_opts(&o);
    if (!valid_mesh(mesh) || count < 1 || !valid_opts(&o)) return 0;
    size_t b = 0;
    if (ctx_bytes(mesh, count, o.gmres_restart, &b) != SWJ_OK) return 0;
    return b + swj_pc_bytes(mesh->N, mesh->M, count, o.block_bw, o.lu_products, o.lu_order);
}

int swj_initial_guess_flat(swj_ctx *c, double *u)
{
    if (!c || !u) return SWJ_EINVAL;
    swj_launch_flat(c, u);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_initial_guess_linear(swj_ctx *c, double *u)
{
    if (!c || !u) return SWJ_EINVAL;
    // u0 - P^-1 E(u0), E with an FP64-accurate all-pairs sum
    const int prec = (c->opts.solve_mode == SWJ_SOLVE_FP64) ? SWJ_FP64 : c->opts.refine_precision;
    swj_launch_flat(c, u);
    int rc = swj_residual_impl(c, u, c->E_try, prec, nullptr);
    if (rc) return rc;
    if (!c->pc_ready && (rc = swj_pc_setup(c)) != SWJ_OK) return rc;
    if ((rc = swj_pc_apply(c, c->E_try, c->u_try, nullptr)) != SWJ_OK) return rc;
    swj_baxpy(c->stream, c->nb, (int)c->nu, nullptr, 0, -1.0, c->u_try, u, c->nu, nullptr);
    SWJ_CUDA_TRY(cudaGetLastError());
    return swj_pc_status(c);
}

int swj_solve_continuation(swj_ctx *c, double *u, int steps, swj_stats *stats)
{
    if (!c || !u || steps < 1) return SWJ_EINVAL;
    const int nb = c->nb;
    std::vector<double> eps0(c->eps, c->eps + nb), F(c->F, c->F + nb), epsk(nb);
    std::vector<swj_stats> acc(nb), one(nb);
    memset((void *)acc.data(), 0, nb * sizeof(swj_stats));
    int rc = SWJ_OK;
    for (int k = 1; k <= steps && rc == SWJ_OK; ++k) {
        for (int i = 0; i < nb; ++i) epsk[i] = eps0[i] * (double)k / (double)steps;
        if ((rc = swj_batch_set_params(c, F.data(), epsk.data())) != SWJ_OK) break;   // F unchanged: P is kept
        rc = swj_solve(c, u, one.data());
        for (int i = 0; i < nb; ++i) {
            swj_stats &a = acc[i], &o = one[i];
            a.status = o.status;
            a.newton_iters += o.newton_iters; a.refine_iters += o.refine_iters;
            a.residual_evals += o.residual_evals; a.residual_evals_fp64 += o.residual_evals_fp64;
            a.residual_evals_ff += o.residual_evals_ff; a.krylov_iters += o.krylov_iters;
            a.precond_applies += o.precond_applies; a.line_search_cuts += o.line_search_cuts;
            a.exact_jvps += o.exact_jvps;
            a.final_norm_inf = o.final_norm_inf; a.final_norm_inf_fp64 = o.final_norm_inf_fp64;
            a.t_total_ms += o.t_total_ms; a.t_setup_ms += o.t_setup_ms;
            a.pairs_per_residual_hi = o.pairs_per_residual_hi; a.pairs_per_residual_lo = o.pairs_per_residual_lo;
        }
    }
    const int rc2 = swj_batch_set_params(c, F.data(), eps0.data());
    if (stats) memcpy(stats, acc.data(), nb * sizeof(swj_stats));
    return rc ? rc : rc2;
}

int swj_resample(swj_ctx *src, const double *u_src, swj_ctx *dst, double *u_dst)
{
    if (!src || !dst || !u_src || !u_dst || src->nb != dst->nb || u_src == u_dst) return SWJ_EINVAL;
    if (src != dst) SWJ_CUDA_TRY(cudaStreamSynchronize(src->stream));   // its node arrays are reused
    swj_launch_resample(src, u_src, dst, u_dst);
    SWJ_CUDA_TRY(cudaGetLastError());
    if (src != dst) SWJ_CUDA_TRY(cudaStreamSynchronize(dst->stream));
    return SWJ_OK;
}

int swj_residual(swj_ctx *c, const double *u, double *E, int precision)
{
    if (!c || !u || !E || u == E) return SWJ_EINVAL;
    if (!swj_valid_precision(precision)) return SWJ_EINVAL;
    return swj_residual_impl(c, u, E, precision, nullptr);
}

int swj_jvp(swj_ctx *c, const double *u, const double *Eu, const double *v, double *Jv,
            int precision)
{
    if (!c || !u || !Eu || !v || !Jv) return SWJ_EINVAL;
    if (precision != SWJ_FP64 && precision != SWJ_FP32) return SWJ_EINVAL;
    return swj_jvp_impl(c, u, Eu, v, Jv, precision, c->opts.fd_h, nullptr);
}

int swj_jvp_exact(swj_ctx *c, const double *u, const double *v, double *Jv, int precision)
{
    if (!c || !u || !v || !Jv || Jv == u || Jv == v) return SWJ_EINVAL;
    if (precision != SWJ_FP64 && precision != SWJ_FP32) return SWJ_EINVAL;
    return swj_jvp_exact_impl(c, u, v, Jv, precision, nullptr);
}

int swj_preconditioned_jacobian(swj_ctx *c, const double *u, int col0, int ncols, double *out, int precision)
{
    if (!c || !u || !out || c->nb != 1) return SWJ_EINVAL;
    if (precision != SWJ_FP64 && precision != SWJ_FP32) return SWJ_EINVAL;
    if (col0 < 0 || ncols < 0 || (size_t)col0 + (size_t)ncols > c->nu) return SWJ_EINVAL;
    int rc;
    if (!c->pc_ready && (rc = swj_pc_setup(c)) != SWJ_OK) return rc;
    const int n = (int)c->nu;
    for (int j = 0; j < ncols; ++j) {
        swj_bfill(c->stream, 1, n, 0.0, c->E_try, c->nu, nullptr);
        swj_bfill(c->stream, 1, 1, 1.0, c->E_try + col0 + j, c->nu, nullptr);
        if ((rc = swj_pc_apply(c, c->E_try, c->u_try, nullptr)) != SWJ_OK) return rc;
        if ((rc = swj_jvp_exact_impl(c, u, c->u_try, out + (size_t)j * c->nu, precision, nullptr)) != SWJ_OK)
            return rc;
    }
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return swj_pc_status(c);
}

int swj_precond_setup(swj_ctx *c)
{
    if (!c) return SWJ_EINVAL;
    return swj_pc_setup(c);
}

int swj_precond_sweep_clusters(const swj_ctx *c)
{
    if (!c || !c->pc_ready) return 0;
    return c->pc_mc ? c->pc_h : 1;
}

int swj_precond_chain_sms(const swj_ctx *c)
{
    if (!c || !c->pc_ready) return 0;
    return c->pc_chain_sms;
}

int swj_precond_apply(swj_ctx *c, const double *b, double *r)
{
    if (!c || !b || !r) return SWJ_EINVAL;
    if (!c->pc_ready) {
        int rc = swj_pc_setup(c);
        if (rc) return rc;
    }
    return swj_pc_apply(c, b, r, nullptr);
}

int swj_solve(swj_ctx *c, double *u, swj_stats *st)
{
    if (!c || !u) return SWJ_EINVAL;
    int rc = swj_solve_impl(c, u, st);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SWJ_ECUDA;
    return rc;
}

int swj_solve_host(swj_ctx *c, const double *u0_host, int setup, double *u_host, double *zeta_host,
                   double *phi_host, swj_stats *st)
{
    if (!c || !u0_host || c->nb != 1) return SWJ_EINVAL;
    const size_t nu = (size_t)c->nu, S = (size_t)c->S;
    if (!c->hs_buf) {
        const size_t b = (nu + 2 * S) * sizeof(double);
        if (cudaMalloc(&c->hs_buf, b) != cudaSuccess) {
            c->hs_buf = nullptr;
            return SWJ_ENOMEM;
        }
        c->bytes += b;
    }
    double *u = c->hs_buf, *z = u + nu, *p = z + S;
    SWJ_CUDA_TRY(cudaMemcpyAsync(u, u0_host, nu * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (setup || !c->pc_ready) {
        const int rc = swj_pc_setup(c);
        if (rc) return rc;
    }
    const int src = swj_solve_impl(c, u, st);
    if (src == SWJ_ECUDA) return src;
    if (zeta_host || phi_host) swj_launch_unpack(c, u, zeta_host ? z : nullptr, phi_host ? p : nullptr);
    if (zeta_host) SWJ_CUDA_TRY(cudaMemcpyAsync(zeta_host, z, S * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (phi_host) SWJ_CUDA_TRY(cudaMemcpyAsync(phi_host, p, S * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u_host) SWJ_CUDA_TRY(cudaMemcpyAsync(u_host, u, nu * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    SWJ_CUDA_TRY(cudaGetLastError());
    return src;
}

int swj_unpack(swj_ctx *c, const double *u, double *zeta, double *phi)
{
    if (!c || !u) return SWJ_EINVAL;
    swj_launch_unpack(c, u, zeta, phi);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_surface(swj_ctx *c, const double *u, double *out)
{
    if (!c || !u || !out) return SWJ_EINVAL;
    // the mesh step also writes E1/E3..E6 rows; send them to a scratch vector
    swj_launch_mesh_step(c, u, c->E_tmp, nullptr);
    swj_launch_surface(c, out);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}

int swj_sync(swj_ctx *c)
{
    if (!c) return SWJ_EINVAL;
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    SWJ_CUDA_TRY(cudaGetLastError());
    return swj_pc_status(c);
}

const char *swj_strerror(int s)
{
    switch (s) {
    case SWJ_OK: return "ok";
    case SWJ_EINVAL: return "invalid argument";
    case SWJ_ENOMEM: return "out of memory";
    case SWJ_ECUDA: return "CUDA error";
    case SWJ_ENOTCONV: return "Newton iteration cap reached";
    case SWJ_ELINESEARCH: return "line search failed";
    case SWJ_EGMRES: return "GMRES failed";
    case SWJ_ENAN: return "NaN or Inf encountered";
    case SWJ_ETIMEOUT: return "device wait timed out";
    case SWJ_ESINGULAR: return "singular preconditioner block";
    case SWJ_ESIZE: return "mesh exceeds the no-allocation scratch";
    case SWJ_PENDING: return "pending";
    default: return "unknown status";
    }
}

const char *swj_version(void) { return SWJ_VERSION_STRING; }

unsigned long long swj_kernel_launches(void) { return g_swj_launches.load(); }

int swj_set_kernel_timing(swj_ctx *c, int enable)
{
    if (!c) return SWJ_EINVAL;
    if (enable && !c->tev) {
        c->tev = (cudaEvent_t *)calloc(2 * SWJ_MAX_TIMED, sizeof(cudaEvent_t));
        c->tev_prec = (int *)calloc(SWJ_MAX_TIMED, sizeof(int));
        if (!c->tev || !c->tev_prec) return SWJ_ENOMEM;
        for (int i = 0; i < 2 * SWJ_MAX_TIMED; ++i)
            if (cudaEventCreate(&c->tev[i]) != cudaSuccess) return SWJ_ECUDA;
    }
    c->time_pairs = enable ? 1 : 0;
    c->n_timed = 0;
    return SWJ_OK;
}

int swj_pair_timing(swj_ctx *c, int precision, double *total_ms, int *launches)
{
    if (!c || !total_ms || !launches) return SWJ_EINVAL;
    *total_ms = 0.0;
    *launches = 0;
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->n_timed; ++i) {
        if (c->tev_prec[i] != precision) continue;
        float ms = 0.f;
        SWJ_CUDA_TRY(cudaEventElapsedTime(&ms, c->tev[2 * i], c->tev[2 * i + 1]));
        *total_ms += ms;
        ++*launches;
    }
    return SWJ_OK;
}

int swj_reset_pair_timing(swj_ctx *c)
{
    if (!c) return SWJ_EINVAL;
    SWJ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->n_timed = 0;
    return SWJ_OK;
}

}  // extern "C"
