"""The failure path of the preconditioner's bounded device waits.

Nothing here faults, traps or waits without bound.  The multi-cluster
substitution of the apply is launched without its helper clusters (test
hook), so the terms its critical clusters poll for are never written: every
poll gives up after opts.wait_limit reads, the kernel returns, and the status
read back is SWJ_ETIMEOUT.  The Gauss-Jordan chain of the set-up is run with
a wait limit of one iteration, so a CTA that finds the pivot step it waits for
not yet published gives up at once.  Afterwards the same context, with the
normal limits, sets up and applies P^-1 bit for bit as before.
"""
import time

import numpy as np
import pytest
import torch

from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

SPEC, F, EPS, BW = W.MESH_41x21, 0.7, 0.1, 5      # h = 2: one helper cluster per half


def _opts(**kw):
    return swj.default_opts(solve_mode="fp64", block_bw=BW, **kw)


def _reference(ctx, b):
    r = ctx.precond_apply(b, ctx.vector())
    ctx.sync()
    return r.clone()


def test_apply_poll_timeout_is_reported_and_the_context_recovers():
    b = torch.tensor(np.random.default_rng(7).normal(size=SPEC.n_unknowns), device="cuda")
    with swj.Context.from_spec(SPEC, F, EPS, opts=_opts()) as ctx:
        ctx.precond_setup()
        assert ctx.sweep_clusters() >= 2, "the apply must run on several clusters here"
        ref = _reference(ctx, b)
        # helpers withheld, polls bounded at 256 reads
        ctx.set_opts(_opts(wait_limit=256))
        ctx.set_test_hooks(swj.TEST_WITHHOLD_HELPERS)
        r = ctx.vector()
        t0 = time.perf_counter()
        ctx.precond_apply(b, r)
        with pytest.raises(swj.SwjError) as e:
            ctx.sync()
        assert e.value.status == swj.ETIMEOUT
        assert time.perf_counter() - t0 < 30.0        # the kernel returned on its own
        # the status stays until the next set-up
        with pytest.raises(swj.SwjError):
            ctx.sync()
        # normal launches again: a new set-up clears it, P^-1 b is what it was
        ctx.set_test_hooks(0)
        ctx.set_opts(_opts())
        ctx.precond_setup()
        again = _reference(ctx, b)
        assert torch.equal(again, ref)


def test_setup_wait_timeout_is_reported_and_the_context_recovers():
    b = torch.tensor(np.random.default_rng(8).normal(size=SPEC.n_unknowns), device="cuda")
    with swj.Context.from_spec(SPEC, F, EPS, opts=_opts()) as ctx:
        ctx.precond_setup()
        ref = _reference(ctx, b)
        ctx.set_opts(_opts(wait_limit=1))
        t0 = time.perf_counter()
        with pytest.raises(swj.SwjError) as e:
            ctx.precond_setup()
        assert e.value.status == swj.ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        ctx.set_opts(_opts())
        ctx.precond_setup()
        again = _reference(ctx, b)
        assert torch.equal(again, ref)


def test_test_hooks_reject_unknown_flags():
    with swj.Context.from_spec(SPEC, F, EPS, opts=_opts()) as ctx:
        with pytest.raises(swj.SwjError) as e:
            ctx.set_test_hooks(2)
        assert e.value.status == swj.EINVAL
