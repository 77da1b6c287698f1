"""The serving loop (swj_server_*): requests on uneven meshes admitted by
device-memory footprint into concurrent groups.  Each served result must be
the one the same request gives alone, and admission must respect the memory
budget and the slot count."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

MESH_61, MESH_121, MESH_181 = W.SERVE_MESHES[0], W.SERVE_MESHES[1], W.SERVE_MESHES[2]
BW = 15


def solve_alone(spec, F, eps, **kw):
    with swj.Context.from_spec(spec, F, eps, block_bw=BW, **kw) as ctx:
        u = ctx.initial_guess_flat(ctx.vector())
        st = ctx.solve(u, check=False)
        z = torch.empty(spec.N * spec.M, dtype=torch.float64, device="cuda")
        ctx.unpack(u, z, None)
        ctx.sync()
        return st["rc"], z.view(spec.M, spec.N).cpu().numpy()


def test_footprint_equals_workspace_after_setup():
    for spec, count, bw in [(MESH_61, 1, BW), (MESH_121, 3, BW), (MESH_181, 1, 7), (W.MESH_41x21, 2, 0)]:
        F = [0.7] * count
        with swj.BatchContext.from_spec(spec, F, [0.2] * count, block_bw=bw) as ctx:
            ctx.precond_setup()
            held = ctx.workspace_bytes()
        assert held == swj.footprint_bytes(spec, count, block_bw=bw), (spec, count, bw)


def test_served_mix_equals_each_request_alone():
    """A mix on three meshes, several requests per mesh (so groups form),
    with more groups than slots: every result equals the request solved
    alone in its own context."""
    rng = np.random.default_rng(77)
    meshes = [MESH_61] * 4 + [MESH_121] * 3 + [MESH_181] * 3
    order = rng.permutation(len(meshes))
    reqs = [(meshes[i], float(rng.uniform(0.55, 1.0)), float(rng.uniform(0.05, 0.45))) for i in order]
    with swj.Server(max_active=3, max_group=4, block_bw=BW) as srv:
        ids = [srv.submit(*r) for r in reqs]
        out = [srv.poll(i, wait=True) for i in ids]
        info = srv.info()
    assert info["completed"] == len(reqs) and info["failed"] == 0
    assert info["peak_active"] >= 2
    assert max(o["group_size"] for o in out) >= 2
    for (spec, F, eps), o in zip(reqs, out):
        assert o["rc"] == swj.OK, (spec, F, eps, o["rc"])
        rc, z = solve_alone(spec, F, eps)
        assert rc == swj.OK
        # a request served in a group of two or more runs in a batched context,
        # whose band LU goes top-down, and alone two-sided: the same P^-1 up to
        # rounding, so the two solves stop at different points of the
        # ||E||_inf < 1e-9 ball around the root
        tol = 1e-10 if o["group_size"] == 1 else 1e-8
        assert np.abs(o["zeta"] - z).max() <= tol, (spec.N, F, eps, o["group_size"])
        assert np.abs(o["zeta"]).max() < F ** 2 / 2


def test_served_result_is_the_oracle_root():
    spec, F, eps = MESH_61, 0.8, 0.3
    m = O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    uo, _ = O.newton_gmres(m, F, eps, O.flat_guess(m), tol=1e-11, eta=1e-8)
    zo, _ = O.zeta_phi(m, uo)
    with swj.Server(max_active=2, block_bw=BW) as srv:
        other = srv.submit(MESH_121, 0.7, 0.2)
        rid = srv.submit(spec, F, eps)
        o = srv.poll(rid, wait=True)
        assert srv.poll(other, wait=True)["rc"] == swj.OK
    assert o["rc"] == swj.OK
    assert np.abs(o["zeta"] - zo).max() <= 1e-6


def test_admission_respects_the_memory_budget():
    """A budget that holds one 181x61 context (not two): three such requests
    run one after another, and a request that can never fit is refused."""
    one = swj.footprint_bytes(MESH_181, 1, block_bw=BW)
    extra = 2 * (2 * 182 * 61 + 181 * 61) * 8          # the server's u and zeta buffers
    budget = one + extra + one // 4
    with swj.Server(hbm_budget_bytes=budget, max_active=4, max_group=1, block_bw=BW) as srv:
        ids = [srv.submit(MESH_181, 0.6 + 0.1 * k, 0.2) for k in range(3)]
        out = [srv.poll(i, wait=True) for i in ids]
        info = srv.info()
        with pytest.raises(swj.SwjError) as e:
            srv.submit(W.SERVE_MESHES[3], 0.7, 0.2)
        assert e.value.status == swj.ENOMEM
    assert all(o["rc"] == swj.OK for o in out)
    assert info["peak_active"] == 1 and info["peak_bytes_held"] <= budget
    # each waited for the one before it
    assert out[1]["queue_ms"] >= 0.5 * out[0]["run_ms"]
    assert out[2]["queue_ms"] >= out[1]["queue_ms"]


def test_requests_are_admitted_while_others_run():
    """With two slots, a request submitted while another is on the GPU is
    admitted at once (continuous admission), and a third waits only for the
    first free slot."""
    with swj.Server(max_active=2, max_group=1, keep_contexts=False, block_bw=BW) as srv:
        a = srv.submit(MESH_181, 0.7, 0.4)
        b = srv.submit(MESH_121, 0.8, 0.3)
        c = srv.submit(MESH_61, 0.9, 0.2)
        ra, rb, rc_ = (srv.poll(i, wait=True) for i in (a, b, c))
        info = srv.info()
    assert ra["rc"] == rb["rc"] == rc_["rc"] == swj.OK
    assert rb["queue_ms"] < 0.5 * ra["run_ms"]
    assert rc_["queue_ms"] <= min(ra["latency_ms"], rb["latency_ms"]) + 50.0
    assert info["peak_active"] == 2 and info["contexts_reused"] == 0


def test_kept_contexts_are_reused():
    with swj.Server(max_active=1, max_group=1, keep_contexts=True, block_bw=BW) as srv:
        ids = [srv.submit(MESH_61, 0.6 + 0.05 * k, 0.25) for k in range(4)]
        out = [srv.poll(i, wait=True) for i in ids]
        info = srv.info()
    assert all(o["rc"] == swj.OK for o in out)
    assert info["contexts_created"] == 1 and info["contexts_reused"] == 3
    for k, o in enumerate(out):
        rc, z = solve_alone(MESH_61, 0.6 + 0.05 * k, 0.25)
        assert np.abs(o["zeta"] - z).max() <= 1e-10
