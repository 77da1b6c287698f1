"""swj_residual_noalloc, the residual entry point for callers that cannot
allocate device memory (a serving loop whose latency budget cannot absorb the
device-wide synchronisation of cudaMalloc/cudaFree, or a host framework that
owns the whole device-memory budget).  It must give what swj_residual gives,
through the C ABI, on consecutive calls that reuse its static scratch.

This file is collected last on purpose: it also runs after every other test
has used the library in the same process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1403_5044_b300 import swj
from paper_1403_5044_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {swj.FP64: 1e-12, swj.FP32: 2e-6}   # the residual parity tolerances of the other tests


def noalloc_fn():
    f = swj.lib().swj_residual_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(swj.Mesh), ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return f


def oracle_scale(spec, F, eps, u):
    m = O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    return np.maximum(1.0, O.residual_scale(m, F, eps, u))


# 41x21 and 181x61 keep the context's launch plan; at 361x121 (the largest
# serving mesh) and 494x85 the partial sums of that plan do not fit and fewer
# source chunks are used, filling the scratch; 361x187 is the largest mesh
# with N = 361 that fits at all (one chunk).
@pytest.mark.parametrize("spec,F,eps", [W.SOLVE_41x21, W.SOLVE_181x61, (W.domain_mesh(361, 121), 0.7, 0.3),
                                        (W.domain_mesh(494, 85), 0.8, 0.2),
                                        (W.domain_mesh(361, 187), 0.6, 0.25)])
def test_noalloc_residual_matches_swj_residual_on_two_calls(spec, F, eps):
    f = noalloc_fn()
    u = W.random_state(spec, seed=17, amp=0.06)
    scale = oracle_scale(spec, F, eps, u)
    mesh = swj.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    stream = torch.cuda.current_stream()
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    with swj.Context.from_spec(spec, F, eps) as ctx:
        for prec in (swj.FP64, swj.FP32):
            ref = ctx.residual(ud, ctx.vector(), prec)
            ctx.sync()
            for call in range(2):
                E = torch.full_like(ud, float("nan"))
                rc = f(ctypes.byref(mesh), F, eps, ctypes.c_void_p(ud.data_ptr()),
                       ctypes.c_void_p(E.data_ptr()), prec, ctypes.c_void_p(stream.cuda_stream))
                assert rc == swj.OK, swj.strerror(rc)
                torch.cuda.synchronize()
                err = ((E - ref).abs().cpu().numpy() / scale).max()
                assert err <= TOL[prec], (prec, call, err)


@pytest.mark.parametrize("spec", [W.domain_mesh(361, 188), W.MESH_721x241])
def test_noalloc_rejects_a_mesh_larger_than_its_scratch(spec):
    f = noalloc_fn()
    mesh = swj.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    u = torch.zeros(spec.n_unknowns, dtype=torch.float64, device="cuda")
    E = torch.zeros_like(u)
    rc = f(ctypes.byref(mesh), 0.7, 0.1, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(E.data_ptr()),
           swj.FP32, None)
    assert rc == swj.ESIZE
    assert swj.strerror(rc) == "mesh exceeds the no-allocation scratch"
