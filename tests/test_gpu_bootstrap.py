"""Initial guesses and bootstrapping (Section 4.1): the linear-problem guess,
continuation in eps, and resampling a solution onto another mesh, against
the oracle and against direct solves."""
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


@pytest.mark.parametrize("b", [0, 5])
def test_linear_guess_matches_oracle(b):
    spec, F, eps = W.MESH_41x21, 0.7, 0.2
    ref = O.linear_solution(omesh(spec), F, eps, None if b == 0 else b)
    with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=b) as ctx:
        u = ctx.initial_guess_linear(ctx.vector())
        ctx.sync()
        got = u.cpu().numpy()
    u0 = O.flat_guess(omesh(spec))
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref - u0).max()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_solve_from_the_linear_guess_reaches_the_flat_start_root(mode):
    spec, F, eps = W.SERVE_MESHES[1], 0.7, 0.3
    roots, iters = [], []
    for guess in ("flat", "linear"):
        with swj.Context.from_spec(spec, F, eps, solve_mode=mode) as ctx:
            u = ctx.vector()
            (ctx.initial_guess_flat if guess == "flat" else ctx.initial_guess_linear)(u)
            st = ctx.solve(u)
            assert st["rc"] == swj.OK
            roots.append(u.cpu().numpy())
            iters.append(st["newton_iters"])
    m = omesh(spec)
    za, _ = O.zeta_phi(m, roots[0])
    zb, _ = O.zeta_phi(m, roots[1])
    assert np.abs(za - zb).max() <= 1e-8
    assert iters[1] <= iters[0]


def test_continuation_reaches_the_direct_root():
    spec, F, eps = W.MESH_41x21, 0.7, 0.3
    with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=5) as ctx:
        u1 = ctx.initial_guess_flat(ctx.vector())
        s1 = ctx.solve(u1)
        u2 = ctx.initial_guess_flat(ctx.vector())
        s2 = ctx.solve_continuation(u2, 3)
        E = ctx.vector()
        ctx.residual(u2, E, swj.FP64)
        ctx.sync()
        assert np.abs(E.cpu().numpy()).max() < 1e-10
    assert s1["rc"] == s2["rc"] == swj.OK
    assert s2["newton_iters"] >= s1["newton_iters"]
    m = omesh(spec)
    assert np.abs(O.zeta_phi(m, u1.cpu().numpy())[0] - O.zeta_phi(m, u2.cpu().numpy())[0]).max() <= 1e-8


def test_continuation_of_a_batch_scales_each_instance():
    spec = W.MESH_41x21
    F, eps = [0.6, 0.8], [0.2, 0.4]
    with swj.BatchContext.from_spec(spec, F, eps, solve_mode="mixed") as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        st = (swj.Stats * 2)()
        rc = swj.lib().swj_solve_continuation(ctx._h, swj._ptr(u), 2, swj.ctypes.cast(st, swj._vp))
        assert rc == swj.OK
        ub = ctx.view(u).cpu().numpy()
    for i in range(2):
        with swj.Context.from_spec(spec, F[i], eps[i], solve_mode="mixed") as one:
            v = one.initial_guess_flat(one.vector())
            one.solve(v)
            m = omesh(spec)
            assert np.abs(O.zeta_phi(m, ub[i])[0] - O.zeta_phi(m, v.cpu().numpy())[0]).max() <= 1e-8


@pytest.mark.parametrize("src,dst", [((61, 21), (121, 41)), ((121, 41), (61, 21)), ((121, 41), (121, 41))])
def test_resample_matches_oracle(src, dst):
    ss, sd = W.domain_mesh(*src), W.domain_mesh(*dst)
    u = W.random_state(ss, seed=50, amp=0.1)
    ref = O.resample(omesh(ss), u, omesh(sd))
    with swj.Context.from_spec(ss, 0.7, 0.2) as a, swj.Context.from_spec(sd, 0.7, 0.2) as b:
        got = b.resample_from(a, dev(u), b.vector()).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_resample_onto_a_shifted_domain_clamps_to_the_source():
    ss = W.domain_mesh(61, 21)
    sd = W.MeshSpec(50, 30, ss.x1 - 3.0, 0.5, 0.5)    # extends beyond the source upstream and across
    u = W.random_state(ss, seed=51, amp=0.1)
    ref = O.resample(omesh(ss), u, omesh(sd))
    with swj.Context.from_spec(ss, 0.7, 0.2) as a, swj.Context.from_spec(sd, 0.7, 0.2) as b:
        got = b.resample_from(a, dev(u), b.vector()).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_mesh_bootstrapping_starts_closer_and_reaches_the_same_root():
    """Solve on the coarse mesh, resample the root onto the fine mesh, solve
    there: the guess has a smaller residual than the flat state, the solve
    takes no more Newton steps and reaches the flat start's root.  (From
    Delta = 0.6 to 0.3 the saving is within one Newton step: 4 and 4.)"""
    coarse, fine, F, eps = W.SERVE_MESHES[0], W.SERVE_MESHES[1], 0.7, 0.3
    with swj.Context.from_spec(coarse, F, eps, solve_mode="mixed") as a, \
            swj.Context.from_spec(fine, F, eps, solve_mode="mixed") as b:
        uc = a.initial_guess_flat(a.vector())
        assert a.solve(uc)["rc"] == swj.OK
        uf = b.resample_from(a, uc, b.vector())
        u0 = b.initial_guess_flat(b.vector())
        E = b.vector()
        b.residual(uf, E, swj.FP64)
        r_boot = float(E.abs().max())
        b.residual(u0, E, swj.FP64)
        r_flat = float(E.abs().max())
        assert r_boot < 0.5 * r_flat
        s_boot = b.solve(uf)
        s_flat = b.solve(u0)
        assert s_boot["rc"] == s_flat["rc"] == swj.OK
        assert s_boot["newton_iters"] <= s_flat["newton_iters"]
        m = omesh(fine)
        assert np.abs(O.zeta_phi(m, uf.cpu().numpy())[0] - O.zeta_phi(m, u0.cpu().numpy())[0]).max() <= 1e-8
