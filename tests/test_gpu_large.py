"""The 721x241 workload (x in [-16, 20], y in [0, 12], dx = dy = 0.05, F = 0.7,
eps = 0.8: a steep wave, 3.0e10 kernel pairs per residual): one mixed solve
from the flat state (FP32 Newton-GMRES, FP64 Krylov and band LU, float-float
refinement), checked against the oracle.  A full oracle solve at this size
takes hours on the host, so the root is checked as a root of the oracle's
residual: every local row (E1, E3..E6) in full and E2 at sampled targets
(corners, edges, the column over the source, random ones), computed one by one
by the oracle.  The crest stays below the limiting height F^2/2 (Section 6).
About a minute on one B300.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_721x241_mixed_solve_is_a_root_of_the_oracle_residual():
    spec, F, eps = W.SOLVE_721x241
    with swj.Context.from_spec(spec, F, eps, solve_mode="mixed", block_bw=-1) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        st = ctx.solve(u, check=False)
        zeta = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
        ctx.unpack(u, zeta, None)
        ctx.sync()
        ug = u.cpu().numpy()
        zg = zeta.cpu().numpy()
    assert st["rc"] == swj.OK, st
    assert st["final_norm_inf_fp64"] < 1e-9
    assert zg.max() < F ** 2 / 2
    m = O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    p = O.residual_parts(m, F, eps, ug, pairs=False)
    for name in ("E1", "E3", "E4", "E5", "E6"):
        assert np.abs(p[name]).max() < 1e-9, (name, np.abs(p[name]).max())
    Tn = (spec.N - 1) * spec.M
    k_src = int(round(-spec.x1 / spec.dx))
    picks = [0, spec.N - 2, Tn - 1, Tn - (spec.N - 1), k_src, k_src - 1, (spec.N - 1) + k_src]
    tidx = np.unique(np.concatenate([picks, np.random.default_rng(9).integers(0, Tn, 33)]))
    E2, scale = O.residual_E2_at(m, F, eps, ug, tidx)
    assert np.abs(E2).max() < 1e-9, np.abs(E2).max()
