"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/swj.h declares; argument validation needs no GPU."""
import ctypes

import pytest

from paper_1403_5044_b300 import build, swj


@pytest.fixture(scope="module")
def lib():
    build.build()
    return swj.lib()


def test_every_declared_function_is_exported(lib):
    names = swj.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(lib):
    assert swj.strerror(swj.OK) == "ok"
    assert swj.strerror(swj.ENAN).startswith("NaN")
    assert "sm_103a" in swj.version()


def test_default_opts(lib):
    o = swj.default_opts()
    assert o.solve_mode == swj.SOLVE_MIXED and o.gmres_restart == 30 and o.ftol_inf == 1e-10
    assert o.block_bw == -1 and o.autotune == 1 and o.refine_precision == swj.FF
    assert o.jvp == swj.JVP_FD and o.forcing == swj.FORCING_SOURCE and o.lu_products == swj.LU_SLICED
    assert o.lu_order == swj.LU_TWO_SIDED and o.wait_limit == 0 and o.sm_partition == 1


@pytest.mark.parametrize("N,M,dx,dy", [(3, 5, 0.5, 0.5), (10, 2, 0.5, 0.5), (10, 5, 0.0, 0.5), (10, 5, 0.5, -1.0)])
def test_create_rejects_bad_mesh_without_touching_the_gpu(lib, N, M, dx, dy):
    h = ctypes.c_void_p()
    mesh = swj.Mesh(N, M, -1.0, dx, dy, 0.05)
    rc = lib.swj_create(ctypes.byref(h), ctypes.byref(mesh), 0.7, 0.1, None, None)
    assert rc == swj.EINVAL and not h.value


@pytest.mark.parametrize("field,value", [("block_bw", 2), ("block_bw", -2), ("gmres_restart", 0),
                                         ("gmres_restart", 61), ("eta_max", 1.5), ("solve_mode", 7),
                                         ("autotune", 2), ("refine_precision", 1),
                                         ("jvp", 2), ("jvp", -1),
                                         ("forcing", 2), ("forcing", -1),
                                         ("lu_products", 2), ("lu_products", -1),
                                         ("lu_order", 2), ("lu_order", -1),
                                         ("wait_limit", -1), ("sm_partition", 2), ("sm_partition", -1)])
def test_create_rejects_bad_options(lib, field, value):
    h = ctypes.c_void_p()
    mesh = swj.Mesh(9, 5, -2.0, 0.5, 0.4, 0.05)
    o = swj.default_opts()
    setattr(o, field, value)
    rc = lib.swj_create(ctypes.byref(h), ctypes.byref(mesh), 0.7, 0.1, ctypes.byref(o), None)
    assert rc == swj.EINVAL


def test_create_rejects_bad_parameters(lib):
    h = ctypes.c_void_p()
    mesh = swj.Mesh(9, 5, -2.0, 0.5, 0.4, 0.05)
    assert lib.swj_create(ctypes.byref(h), ctypes.byref(mesh), 0.0, 0.1, None, None) == swj.EINVAL
    assert lib.swj_create(ctypes.byref(h), ctypes.byref(mesh), 0.7, -0.1, None, None) == swj.EINVAL
