"""Batches of instances on one mesh (swj_batch_create): every kernel runs over
all instances at once, with per-instance F, eps, Newton/Krylov state and
convergence masks.  Each instance of a batch must give what it gives alone,
and the oracle's result, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {swj.FP64: 1e-12, swj.FP32: 2e-6}   # residual parity, relative to the oracle's term scale


def omesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


PARAMS_41 = [(0.7, 0.1), (0.55, 0.3), (0.9, 0.05), (0.8, 0.45), (0.65, 0.2)]


def states(spec, count, seed):
    return [W.random_state(spec, seed=seed + i, amp=0.04 + 0.02 * i) for i in range(count)]


@pytest.mark.parametrize("prec", [swj.FP64, swj.FP32])
def test_batch_residual_matches_oracle_per_instance(prec):
    spec = W.MESH_41x21
    F = [p[0] for p in PARAMS_41]
    eps = [p[1] for p in PARAMS_41]
    us = states(spec, len(F), 101)
    m = omesh(spec)
    with swj.BatchContext.from_spec(spec, F, eps) as ctx:
        assert swj.lib().swj_batch_count(ctx._h) == len(F)
        E = ctx.vector()
        ctx.residual(dev(np.concatenate(us)), E, prec)
        ctx.sync()
        got = ctx.view(E).cpu().numpy()
    for i, u in enumerate(us):
        ref = O.residual(m, F[i], eps[i], u)
        scale = np.maximum(1.0, O.residual_scale(m, F[i], eps[i], u))
        assert (np.abs(got[i] - ref) / scale).max() <= TOL[prec], i


def test_batch_jvp_and_precond_match_single_instances():
    """The batched FD-JVP and Schur preconditioner apply equal the single-
    instance ones (each instance has its own h, F and factors)."""
    spec = W.MESH_41x21
    F = [p[0] for p in PARAMS_41]
    eps = [p[1] for p in PARAMS_41]
    us = states(spec, len(F), 201)
    vs = [np.random.default_rng(300 + i).normal(size=spec.n_unknowns) for i in range(len(F))]
    with swj.BatchContext.from_spec(spec, F, eps, solve_mode="fp64", block_bw=3) as ctx:
        ub, vb = dev(np.concatenate(us)), dev(np.concatenate(vs))
        Eb, Jb, Rb = ctx.vector(), ctx.vector(), ctx.vector()
        ctx.residual(ub, Eb, swj.FP64)
        ctx.jvp(ub, Eb, vb, Jb, swj.FP64)
        ctx.precond_setup()
        ctx.precond_apply(vb, Rb)
        ctx.sync()
        Jb = ctx.view(Jb).cpu().numpy()
        Rb = ctx.view(Rb).cpu().numpy()
    for i in range(len(F)):
        with swj.Context.from_spec(spec, F[i], eps[i], solve_mode="fp64", block_bw=3,
                                   lu_order=swj.LU_TOP_DOWN) as one:
            u, v = dev(us[i]), dev(vs[i])
            E, J, R = one.vector(), one.vector(), one.vector()
            one.residual(u, E, swj.FP64)
            one.jvp(u, E, v, J, swj.FP64)
            one.precond_setup()
            one.precond_apply(v, R)
            one.sync()
            J, R = J.cpu().numpy(), R.cpu().numpy()
        # the residual differs from the single-instance one by summation order only
        # (1e-16 relative), and the FD quotient divides that by h ~ 1e-8
        assert np.abs(Jb[i] - J).max() <= 1e-6 * np.abs(J).max(), i
        assert np.abs(Rb[i] - R).max() <= 1e-12 * np.abs(R).max(), i


def unpack_zeta(ctx, u, spec):
    z = torch.empty(ctx.count * spec.N * spec.M, dtype=torch.float64, device="cuda")
    ctx.unpack(u, z, None)
    ctx.sync()
    return z.view(ctx.count, spec.M, spec.N).cpu().numpy()


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_batch_solve_matches_single_solves(mode):
    """Instances converge at different Newton steps; each must end where it
    ends alone.  eps = 0 makes the flat guess an exact root, so that instance
    is masked out before the first step and must come back untouched."""
    spec = W.MESH_41x21
    params = PARAMS_41[:4] + [(0.75, 0.0)]
    F = [p[0] for p in params]
    eps = [p[1] for p in params]
    with swj.BatchContext.from_spec(spec, F, eps, solve_mode=mode, block_bw=3) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        flat = ctx.view(u)[-1].clone()
        rc, stats = ctx.solve(u)
        assert rc == swj.OK
        zb = unpack_zeta(ctx, u, spec)
        ub = ctx.view(u).cpu().numpy()
    assert torch.equal(torch.tensor(ub[-1]), flat.cpu())
    assert stats[-1]["newton_iters"] == 0
    for i in range(len(F) - 1):
        assert stats[i]["status"] == swj.OK and stats[i]["newton_iters"] >= 2
        with swj.Context.from_spec(spec, F[i], eps[i], solve_mode=mode, block_bw=3) as one:
            u1 = one.initial_guess_flat(one.vector())
            st = one.solve(u1)
            z1 = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
            one.unpack(u1, z1, None)
            one.sync()
            z1 = z1.view(spec.M, spec.N).cpu().numpy()
        assert st["rc"] == swj.OK
        # both stop at ||E||_inf below 1e-9 (mixed) / 1e-10 (FP64) along different rounding paths
        tol = 1e-7 if mode == "mixed" else 1e-8
        assert np.abs(zb[i] - z1).max() <= tol, (i, np.abs(zb[i] - z1).max())
        assert np.abs(zb[i]).max() < F[i] ** 2 / 2


def test_batch_64x121x41_mixed_matches_fp64():
    """The batched workload (64 instances of 121 x 41, F ~ U[0.5, 1],
    eps ~ U[0.05, 0.6]): mixed-precision and FP64 batched solves reach the
    same surfaces to 1e-6, every instance converging."""
    spec = W.MESH_121x41
    params = W.batch_params()
    F = [p[0] for p in params]
    eps = [p[1] for p in params]
    z = {}
    for mode in ("mixed", "fp64"):
        with swj.BatchContext.from_spec(spec, F, eps, solve_mode=mode, block_bw=15) as ctx:
            u = ctx.initial_guess_flat(ctx.vector())
            rc, stats = ctx.solve(u, check=False)
            bad = [(i, s["status"]) for i, s in enumerate(stats) if s["status"] != swj.OK]
            assert rc == swj.OK and not bad, (mode, bad)
            z[mode] = unpack_zeta(ctx, u, spec)
    dz = np.abs(z["mixed"] - z["fp64"]).reshape(len(F), -1).max(axis=1)
    assert dz.max() <= 1e-6, dz.max()
    assert all(np.abs(z["fp64"][i]).max() < F[i] ** 2 / 2 for i in range(len(F)))
    # sampled instances against the oracle's own roots, stored by
    # tests/golden/make_roots.py (||E||_inf ~ 2e-14)
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sp = importlib.util.spec_from_file_location("make_roots", os.path.join(here, "make_roots.py"))
    mod = importlib.util.module_from_spec(sp)
    sp.loader.exec_module(mod)
    for head, zo, _ in mod.load(os.path.join(here, "oracle_root_121x41_batch.txt")):
        i = int(head["label"])
        assert (head["F"], head["eps"]) == (F[i], eps[i])
        zm = np.asarray(z["mixed"][i]).reshape(spec.M, spec.N)
        z6 = np.asarray(z["fp64"][i]).reshape(spec.M, spec.N)
        assert np.abs(z6 - zo).max() <= 1e-8, (i, np.abs(z6 - zo).max())
        assert np.abs(zm - zo).max() <= 1e-6, (i, np.abs(zm - zo).max())


def test_batch_instance_matches_oracle_root():
    """One instance of a mixed batch against the oracle's own Newton root on
    a small mesh (the batch neighbours must not leak into it)."""
    spec = W.MeshSpec(21, 9, -5.0, 0.5, 0.4)
    params = [(0.7, 0.15), (0.6, 0.35), (0.85, 0.25)]
    m = omesh(spec)
    with swj.BatchContext.from_spec(spec, [p[0] for p in params], [p[1] for p in params],
                                    solve_mode="mixed", block_bw=0) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        rc, _ = ctx.solve(u)
        ub = ctx.view(u).cpu().numpy()
    for i, (F, eps) in enumerate(params):
        ref, info = O.newton_dense(m, F, eps, O.flat_guess(m), tol=1e-11)
        zr, _ = O.zeta_phi(m, ref)
        zg, _ = O.zeta_phi(m, ub[i])
        assert np.abs(zg - zr).max() <= 1e-7, i
        assert np.abs(O.residual(m, F, eps, ub[i])).max() < 1e-8, i
