"""Parity of the CUDA residual path with the CPU oracle (element by element),
through the C ABI.

Tolerances (per row r, with s_r the oracle's sum of absolute term values of
that row, 1 for rows without an integral):
  FP64 all-pairs sum:  |E_gpu - E_oracle| <= 1e-12 max(1, s_r)
  FP32 all-pairs sum:  |E_gpu - E_oracle| <= 2e-6  max(1, s_r)
The FP32 bound is the worst case of a few-ulp relative error (~1.2e-6) on
every term, all of one sign, plus the rounding of the FP64 inputs to FP32;
compensated summation keeps the accumulation error at the level of the final
sum's last bits.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6
TOLFF = 1e-12   # float-float (~2^-44 per operation): the FP64 tolerance; measured 3e-15


def omesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


def oracle_E_and_scale(spec, F, eps, u):
    m = omesh(spec)
    p = O.residual_parts(m, F, eps, u)
    E = O.order(m, p["E1"], p["E2"], p["E3"], p["E4"], p["E5"], p["E6"])
    one, r = np.ones_like(p["E1"]), np.ones(spec.M)
    scale = O.order(m, one, p["scale2"], r, r, r, r)
    return E, np.maximum(1.0, scale), p


def gpu_residual(spec, F, eps, u, precision, **kw):
    with swj.Context.from_spec(spec, F, eps, **kw) as ctx:
        ud = torch.tensor(u, dtype=torch.float64, device="cuda")
        Ed = ctx.vector()
        ctx.residual(ud, Ed, precision)
        ctx.sync()
        return Ed.cpu().numpy()


# (mesh, F, eps, seed, amplitude): minimum size, tiny, a ragged single tile,
# the 41x21 workload, the paper's 91x31 mesh (several tiles, ragged tail)
CASES = [
    (W.MeshSpec(4, 3, -1.0, 0.5, 0.5), 0.7, 0.2, 1, 0.10),
    (W.MeshSpec(9, 5, -2.0, 0.5, 0.4), 0.7, 0.3, 4, 0.15),
    (W.MeshSpec(37, 13, -8.0, 0.45, 0.35), 0.8, 0.25, 5, 0.10),
    (W.MESH_41x21, 0.7, 0.1, 6, 0.05),
    (W.MeshSpec(91, 31, -9.0, 0.3, 0.3), 0.7, 1.0, 7, 0.10),
]


@pytest.mark.parametrize("spec,F,eps,seed,amp", CASES)
def test_residual_fp64_matches_oracle(spec, F, eps, seed, amp):
    u = W.random_state(spec, seed=seed, amp=amp)
    Eo, scale, _ = oracle_E_and_scale(spec, F, eps, u)
    Eg = gpu_residual(spec, F, eps, u, swj.FP64)
    err = np.abs(Eg - Eo) / scale
    assert err.max() <= TOL64, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("spec,F,eps,seed,amp", CASES)
def test_residual_fp32_matches_oracle(spec, F, eps, seed, amp):
    u = W.random_state(spec, seed=seed, amp=amp)
    Eo, scale, _ = oracle_E_and_scale(spec, F, eps, u)
    Eg = gpu_residual(spec, F, eps, u, swj.FP32)
    err = np.abs(Eg - Eo) / scale
    assert err.max() <= TOL32, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("spec,F,eps,seed,amp", [CASES[2], CASES[4]])
@pytest.mark.parametrize("prec", [swj.FP64, swj.FP32, swj.FF])
def test_every_tile_shape_matches_oracle(spec, F, eps, seed, amp, prec):
    """Each compiled tile shape of the all-pairs kernel (the autotuner's
    candidates, packed FP32 pair instructions included), pinned in turn."""
    u = W.random_state(spec, seed=seed, amp=amp)
    Eo, scale, _ = oracle_E_and_scale(spec, F, eps, u)
    n = swj.pair_variants(prec)
    assert n >= (6 if prec == swj.FP32 else 3)
    with swj.Context.from_spec(spec, F, eps) as ctx:
        ud = torch.tensor(u, dtype=torch.float64, device="cuda")
        for v in range(n):
            ctx.set_pair_config(prec, v)
            assert ctx.pair_config(prec)[0] == v
            Ed = ctx.vector()
            ctx.residual(ud, Ed, prec)
            ctx.sync()
            err = np.abs(Ed.cpu().numpy() - Eo) / scale
            assert err.max() <= {swj.FP64: TOL64, swj.FP32: TOL32, swj.FF: TOLFF}[prec], (v, err.max())


def test_autotuned_shape_is_shared_by_contexts_of_one_mesh_size():
    spec, F, eps = W.SOLVE_41x21
    u = torch.tensor(W.random_state(spec, seed=3, amp=0.05), dtype=torch.float64, device="cuda")
    cfg = []
    for _ in range(2):
        with swj.Context.from_spec(spec, F, eps) as ctx:
            E = ctx.vector()
            ctx.residual(u, E, swj.FP32)
            ctx.sync()
            cfg.append(ctx.pair_config(swj.FP32))
    assert cfg[0] == cfg[1]


@pytest.mark.parametrize("spec,F,eps,seed,amp", CASES)
def test_residual_ff_matches_oracle(spec, F, eps, seed, amp):
    u = W.random_state(spec, seed=seed, amp=amp)
    Eo, scale, _ = oracle_E_and_scale(spec, F, eps, u)
    Eg = gpu_residual(spec, F, eps, u, swj.FF)
    err = np.abs(Eg - Eo) / scale
    assert err.max() <= TOLFF, (err.max(), int(err.argmax()))


def test_residual_181x61_every_precision():
    """The 181x61, F = 0.7, eps = 0.4 workload, every row."""
    spec, F, eps = W.SOLVE_181x61
    u = W.random_state(spec, seed=11, amp=0.08)
    Eo, scale, _ = oracle_E_and_scale(spec, F, eps, u)
    for prec, tol in ((swj.FP64, TOL64), (swj.FP32, TOL32), (swj.FF, TOLFF)):
        err = np.abs(gpu_residual(spec, F, eps, u, prec) - Eo) / scale
        assert err.max() <= tol, (prec, err.max())


def test_residual_721x241_sampled():
    """The 721x241 workload: every local row (E1, E3..E6) in full, E2 at 48
    sampled targets (corners, edges, the source region, random)."""
    spec, F, eps = W.SOLVE_721x241
    m = omesh(spec)
    u = W.random_state(spec, seed=12, amp=0.1)
    p = O.residual_parts(m, F, eps, u, pairs=False)
    Tn = (spec.N - 1) * spec.M
    rng = np.random.default_rng(3)
    k_src = int(round(-spec.x1 / spec.dx))          # column of the source, x = 0
    picks = [0, spec.N - 2, Tn - 1, Tn - (spec.N - 1), k_src, k_src - 1, (spec.N - 1) + k_src]
    tidx = np.unique(np.concatenate([picks, rng.integers(0, Tn, 41)]))
    E2o, s2 = O.residual_E2_at(m, F, eps, u, tidx)
    H = (spec.N + 1) * spec.M
    for prec, tol in ((swj.FP64, TOL64), (swj.FP32, TOL32)):
        Eg = gpu_residual(spec, F, eps, u, prec)
        top = Eg[:H].reshape(spec.M, spec.N + 1)
        bot = Eg[H:].reshape(spec.M, spec.N + 1)
        assert np.abs(top[:, 2:] - p["E1"]).max() <= 1e-13
        assert np.abs(top[:, 0] - p["E3"]).max() <= 1e-13 and np.abs(top[:, 1] - p["E4"]).max() <= 1e-12
        assert np.abs(bot[:, 0] - p["E5"]).max() <= 1e-13 and np.abs(bot[:, 1] - p["E6"]).max() <= 1e-12
        k, l = tidx % (spec.N - 1), tidx // (spec.N - 1)
        err = np.abs(bot[l, 2 + k] - E2o) / np.maximum(1.0, s2)
        assert err.max() <= tol, (prec, err.max())


def test_flat_state_is_exact():
    spec = W.MESH_41x21
    with swj.Context.from_spec(spec, 0.7, 0.0) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        E = ctx.vector()
        ctx.sync()
        assert np.array_equal(u.cpu().numpy(), O.flat_guess(omesh(spec)))
        for prec in (swj.FP64, swj.FP32):
            ctx.residual(u, E, prec)
            ctx.sync()
            assert torch.count_nonzero(E).item() == 0
        ctx.set_params(0.7, 0.37)
        ctx.residual(u, E, swj.FP64)
        ctx.sync()
        p = O.residual_parts(omesh(spec), 0.7, 0.37, O.flat_guess(omesh(spec)))
        H = (spec.N + 1) * spec.M
        E2 = E.cpu().numpy()[H:].reshape(spec.M, spec.N + 1)[:, 2:]
        assert np.abs(E2 - p["E2"]).max() < 1e-15


def test_mesh_step_intermediates_match_oracle():
    spec = W.MeshSpec(37, 13, -8.0, 0.45, 0.35)
    u = W.random_state(spec, seed=21, amp=0.2)
    st = O.surface(omesh(spec), u)
    p = O.residual_parts(omesh(spec), 0.7, 0.2, u, pairs=False)
    S, T = spec.N * spec.M, (spec.N - 1) * spec.M
    with swj.Context.from_spec(spec, 0.7, 0.2) as ctx:
        out = torch.empty(4 * S + 5 * T, dtype=torch.float64, device="cuda")
        ctx.surface(torch.tensor(u, device="cuda"), out)
        ctx.sync()
        o = out.cpu().numpy()
    names = ["zeta", "g", "zetay", "phiy"]
    for q, name in enumerate(names):
        assert np.abs(o[q * S:(q + 1) * S].reshape(spec.M, spec.N) - st[name]).max() < 1e-13, name
    base = 4 * S
    for q, name in enumerate(["zeta_t", "g_t", "zetax_t", "zetay_t"]):
        got = o[base + q * T: base + (q + 1) * T].reshape(spec.M, spec.N - 1)
        assert np.abs(got - st[name]).max() < 1e-13, name
    I = o[base + 4 * T: base + 5 * T].reshape(spec.M, spec.N - 1)
    assert np.abs(I - p["I"]).max() < 1e-12 * np.abs(p["I"]).max()


def test_residual_is_bitwise_reproducible():
    spec, F, eps = W.SOLVE_181x61
    u = torch.tensor(W.random_state(spec, seed=2, amp=0.05), device="cuda")
    with swj.Context.from_spec(spec, F, eps) as ctx:
        for prec in (swj.FP64, swj.FP32):
            a, b = ctx.vector(), ctx.vector()
            ctx.residual(u, a, prec)
            ctx.residual(u, b, prec)
            ctx.sync()
            assert torch.equal(a, b)


def test_nan_input_propagates():
    spec = W.MeshSpec(9, 5, -2.0, 0.5, 0.4)
    u = W.random_state(spec, seed=1, amp=0.05)
    u[7] = np.nan
    Eg = gpu_residual(spec, 0.7, 0.1, u, swj.FP32)
    assert np.isnan(Eg).any()
