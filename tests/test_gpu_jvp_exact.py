"""The exact Jacobian-vector product (swj_jvp_exact, forward-mode derivative
of E) against the oracle's complex-step derivative, and Newton-GMRES solves
that use it in place of the difference quotient of Eq. JvApprox."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu


def omesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def gpu_jvp(spec, F, eps, u, v, prec):
    with swj.Context.from_spec(spec, F, eps) as ctx:
        J = ctx.vector()
        ctx.jvp_exact(dev(u), dev(v), J, prec)
        ctx.sync()
        return J.cpu().numpy()


# tolerance per row relative to max(1, the row's sum of |tangent terms|):
# FP64 differs from the oracle only in summation order; FP32 is the residual's
# few-ulp-per-term bound
TOL = {swj.FP64: 1e-12, swj.FP32: 2e-6}


@pytest.mark.parametrize("prec", [swj.FP64, swj.FP32])
@pytest.mark.parametrize("spec,seed", [(W.MeshSpec(4, 3, -1.5, 0.5, 0.4), 1), (W.MeshSpec(9, 5, -2.0, 0.5, 0.4), 2),
                                       (W.MeshSpec(37, 13, -8.0, 0.45, 0.35), 3), (W.MESH_41x21, 4),
                                       (W.MeshSpec(91, 31, -12.0, 0.3, 0.3), 5)])
def test_exact_jvp_matches_oracle_complex_step(spec, seed, prec):
    F, eps = 0.7, 0.3
    u = W.random_state(spec, seed=seed, amp=0.1)
    v = np.random.default_rng(100 + seed).normal(size=u.size)
    ref, scale = O.jvp_exact(omesh(spec), F, eps, u, v)
    got = gpu_jvp(spec, F, eps, u, v, prec)
    err = np.abs(got - ref) / np.maximum(1.0, scale)
    assert err.max() <= TOL[prec], (spec.N, spec.M, float(err.max()), int(err.argmax()))


@pytest.mark.parametrize("prec", [swj.FP64, swj.FP32])
def test_exact_jvp_181x61_workload(prec):
    spec, F, eps = W.SOLVE_181x61
    u = W.random_state(spec, seed=7, amp=0.05)
    v = np.random.default_rng(8).normal(size=u.size)
    ref, scale = O.jvp_exact(omesh(spec), F, eps, u, v)
    got = gpu_jvp(spec, F, eps, u, v, prec)
    assert (np.abs(got - ref) / np.maximum(1.0, scale)).max() <= TOL[prec]


def test_exact_jvp_of_a_batch_equals_single_instances():
    spec = W.MESH_41x21
    F, eps = [0.6, 0.8, 0.95], [0.1, 0.3, 0.5]
    us = [W.random_state(spec, seed=20 + i, amp=0.1) for i in range(3)]
    vs = [np.random.default_rng(30 + i).normal(size=spec.n_unknowns) for i in range(3)]
    with swj.BatchContext.from_spec(spec, F, eps) as ctx:
        J = ctx.vector()
        ctx.jvp_exact(dev(np.concatenate(us)), dev(np.concatenate(vs)), J, swj.FP64)
        ctx.sync()
        J = ctx.view(J).cpu().numpy()
    for i in range(3):
        one = gpu_jvp(spec, F[i], eps[i], us[i], vs[i], swj.FP64)
        assert np.array_equal(J[i], one)


def test_exact_jacobian_times_untruncated_preconditioner_is_identity_at_flat_state():
    """Two independent GPU components: at the flat state with eps = 0 the exact
    Jacobian is the linear Jacobian of Appendix B, which the untruncated
    preconditioner (block_bw = 0) inverts, so J (P^-1 b) = b."""
    spec = W.MESH_41x21
    b = np.random.default_rng(40).normal(size=spec.n_unknowns)
    with swj.Context.from_spec(spec, 0.7, 0.0, solve_mode="fp64", block_bw=0) as ctx:
        u0 = ctx.initial_guess_flat(ctx.vector())
        r, Jr = ctx.vector(), ctx.vector()
        ctx.precond_setup()
        ctx.precond_apply(dev(b), r)
        ctx.jvp_exact(u0, r, Jr, swj.FP64)
        ctx.sync()
        got = Jr.cpu().numpy()
    assert np.abs(got - b).max() <= 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_solves_with_exact_jvps_reach_the_fd_root(mode):
    spec, F, eps = W.MESH_41x21, 0.7, 0.1
    roots = {}
    for jvp in (swj.JVP_FD, swj.JVP_EXACT):
        with swj.Context.from_spec(spec, F, eps, solve_mode=mode, block_bw=5, jvp=jvp) as ctx:
            u = ctx.initial_guess_flat(ctx.vector())
            st = ctx.solve(u)
            assert st["rc"] == swj.OK
            if jvp == swj.JVP_EXACT:
                assert st["exact_jvps"] == st["krylov_iters"]
            elif mode == "fp64":
                assert st["exact_jvps"] == 0
            else:   # the Newton phase differences FP32 residuals, the FP64 refinement steps do not
                assert 0 < st["exact_jvps"] < st["krylov_iters"]
            roots[jvp] = u.cpu().numpy()
    m = omesh(spec)
    za, _ = O.zeta_phi(m, roots[swj.JVP_FD])
    zb, _ = O.zeta_phi(m, roots[swj.JVP_EXACT])
    assert np.abs(za - zb).max() <= 1e-8
    assert np.abs(O.residual(m, F, eps, roots[swj.JVP_EXACT])).max() < 1e-8


def test_181x61_mixed_solve_with_exact_jvps():
    spec, F, eps = W.SOLVE_181x61
    out = {}
    for jvp in (swj.JVP_FD, swj.JVP_EXACT):
        with swj.Context.from_spec(spec, F, eps, solve_mode="mixed", jvp=jvp) as ctx:
            u = ctx.initial_guess_flat(ctx.vector())
            st = ctx.solve(u)
            assert st["rc"] == swj.OK and st["final_norm_inf_fp64"] < 1e-9
            z = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
            ctx.unpack(u, z, None)
            ctx.sync()
            out[jvp] = z.cpu().numpy()
    assert np.abs(out[swj.JVP_FD] - out[swj.JVP_EXACT]).max() <= 1e-8
