"""The preconditioned Jacobian J(u) P^-1 formed on the GPU
(swj_preconditioned_jacobian) against the oracle, and the clustering of its
spectrum as the block bandwidth grows (Section 4.2, Figs. 2-3)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import diagnostics as D
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = W.MeshSpec(13, 7, -3.0, 0.5, 0.4)


def omesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


@pytest.mark.parametrize("b", [0, 1, 3])
def test_preconditioned_jacobian_matches_oracle(b):
    F, eps = 0.7, 0.2
    u = W.random_state(SMALL, seed=60, amp=0.08)
    ref = O.preconditioned_jacobian(omesh(SMALL), F, eps, u, None if b == 0 else b)
    with swj.Context.from_spec(SMALL, F, eps, solve_mode="fp64", block_bw=b) as ctx:
        got = D.preconditioned_jacobian(ctx, torch.tensor(u, device="cuda"))
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_column_range_and_fp32_columns():
    F, eps = 0.7, 0.2
    u = torch.tensor(W.random_state(SMALL, seed=61, amp=0.08), device="cuda")
    with swj.Context.from_spec(SMALL, F, eps, solve_mode="fp64", block_bw=3) as ctx:
        n = ctx.n_unknowns
        full = D.preconditioned_jacobian(ctx, u)
        part = torch.empty(n * 5, dtype=torch.float64, device="cuda")
        ctx.preconditioned_jacobian(u, part, 17, 5, swj.FP64)
        assert np.array_equal(part.view(5, n).t().cpu().numpy(), full[:, 17:22])
        ctx.preconditioned_jacobian(u, part, 17, 5, swj.FP32)
        p32 = part.view(5, n).t().cpu().numpy()
        assert np.abs(p32 - full[:, 17:22]).max() <= 1e-4 * np.abs(full).max()
        with pytest.raises(swj.SwjError):
            ctx.preconditioned_jacobian(u, part, n - 2, 5, swj.FP64)


def test_identity_at_the_linear_limit():
    with swj.Context.from_spec(SMALL, 0.7, 0.0, solve_mode="fp64", block_bw=0) as ctx:
        u0 = ctx.initial_guess_flat(ctx.vector())
        A = D.preconditioned_jacobian(ctx, u0)
    assert np.abs(A - np.eye(A.shape[0])).max() <= 1e-10


def test_spectrum_clusters_as_the_block_bandwidth_grows():
    """At the converged 41x21 solution the eigenvalues of J P^-1 move towards
    1 as b grows; the untruncated preconditioner clusters them tightest."""
    spec, F, eps = W.MESH_41x21, 0.7, 0.1
    with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=0) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        assert ctx.solve(u)["rc"] == swj.OK
    out = {}
    for b in (1, 5, 0):
        with swj.Context.from_spec(spec, F, eps, solve_mode="fp64", block_bw=b) as ctx:
            _, out[b] = D.spectrum(ctx, u)
    assert out[1]["max_dist_from_1"] > out[5]["max_dist_from_1"] > out[0]["max_dist_from_1"]
    assert out[0]["frac_within_0.5"] >= out[5]["frac_within_0.5"] >= out[1]["frac_within_0.5"]
