"""The pressure-distribution forcing (an applied surface pressure eps p(x, y)
in Bernoulli's condition instead of the submerged source) on the GPU against
the oracle: residual, exact Jacobian-vector product, linear guess, solves."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

P = "pressure"


def omesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


MESHES = [W.MESH_41x21, W.MeshSpec(37, 13, -4.0, 0.25, 0.2), W.domain_mesh(121, 41)]


@pytest.mark.parametrize("prec,tol", [(swj.FP64, 1e-12), (swj.FP32, 2e-6)])
@pytest.mark.parametrize("spec", MESHES)
def test_pressure_residual_matches_oracle(spec, prec, tol):
    F, eps = 0.7, 0.4
    u = W.random_state(spec, seed=70, amp=0.1)
    m = omesh(spec)
    ref = O.residual(m, F, eps, u, forcing=P)
    scale = O.residual_scale(m, F, eps, u, forcing=P)
    with swj.Context.from_spec(spec, F, eps, forcing=swj.FORCING_PRESSURE) as ctx:
        E = ctx.vector()
        ctx.residual(dev(u), E, prec)
        ctx.sync()
        got = E.cpu().numpy()
    assert (np.abs(got - ref) / scale).max() <= tol


def test_pressure_flat_state_residual_is_the_pressure():
    spec = W.MESH_41x21
    m = omesh(spec)
    ref = O.residual(m, 0.7, 0.3, O.flat_guess(m), forcing=P)
    assert np.count_nonzero(ref) > 0
    with swj.Context.from_spec(spec, 0.7, 0.3, forcing=swj.FORCING_PRESSURE) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        E = ctx.vector()
        ctx.residual(u, E, swj.FP64)
        ctx.sync()
        got = E.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-14


def test_pressure_exact_jvp_matches_oracle():
    spec, F, eps = W.MESH_41x21, 0.7, 0.3
    u = W.random_state(spec, seed=71, amp=0.1)
    v = np.random.default_rng(72).normal(size=u.size)
    ref, scale = O.jvp_exact(omesh(spec), F, eps, u, v, forcing=P)
    with swj.Context.from_spec(spec, F, eps, forcing=swj.FORCING_PRESSURE) as ctx:
        J = ctx.vector()
        ctx.jvp_exact(dev(u), dev(v), J, swj.FP64)
        ctx.sync()
        got = J.cpu().numpy()
    assert (np.abs(got - ref) / np.maximum(1.0, scale)).max() <= 1e-12


def test_pressure_linear_guess_matches_oracle():
    spec, F, eps = W.MESH_41x21, 0.7, 0.2
    ref = O.linear_solution(omesh(spec), F, eps, 5, forcing=P)
    with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=5, forcing=swj.FORCING_PRESSURE) as ctx:
        u = ctx.initial_guess_linear(ctx.vector())
        ctx.sync()
        got = u.cpu().numpy()
    u0 = O.flat_guess(omesh(spec))
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref - u0).max()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_pressure_solve_reaches_the_oracle_root(mode):
    spec, F, eps = W.MESH_41x21, 0.7, 0.2
    m = omesh(spec)
    uo, _ = O.newton_gmres(m, F, eps, O.flat_guess(m), tol=1e-11, eta=1e-8, forcing=P)
    zo, _ = O.zeta_phi(m, uo)
    with swj.Context.from_spec(spec, F, eps, solve_mode=mode, forcing=swj.FORCING_PRESSURE) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        st = ctx.solve(u)
        assert st["rc"] == swj.OK
        ug = u.cpu().numpy()
    zg, _ = O.zeta_phi(m, ug)
    assert np.abs(zg - zo).max() <= (1e-8 if mode == "fp64" else 1e-6)
    assert np.abs(O.residual(m, F, eps, ug, forcing=P)).max() < 1e-8
    # a wave pattern trails the pressure patch: the surface is not flat downstream
    assert np.abs(zg[:, m.x() > 2.0]).max() > 0.01 * eps
