"""Thin ctypes binding of libswj (include/swj.h).

Argument marshalling only: every step of the residual, JVP, preconditioner
and solve runs in the CUDA library.  Device buffers are torch CUDA float64
tensors (torch is used for device memory and streams).  If the library is
missing the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libswj.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "swj.h")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ELINESEARCH, EGMRES, ENAN, ETIMEOUT, ESINGULAR, ESIZE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10
PENDING = 1
FP64, FP32, FF = 0, 1, 2
JVP_FD, JVP_EXACT = 0, 1
FORCING_SOURCE, FORCING_PRESSURE = 0, 1
LU_FP64, LU_SLICED = 0, 1
LU_TOP_DOWN, LU_TWO_SIDED = 0, 1
SOLVE_FP64, SOLVE_MIXED = 0, 1
TEST_WITHHOLD_HELPERS = 1


class SwjError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, strerror(status), status))


class Mesh(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("x1", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("n_rad", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("solve_mode", ctypes.c_int), ("block_bw", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("max_newton", ctypes.c_int),
                ("max_krylov", ctypes.c_int), ("ftol_inf", ctypes.c_double),
                ("eta_max", ctypes.c_double), ("eta_min", ctypes.c_double),
                ("fd_h", ctypes.c_double), ("refine_max", ctypes.c_int),
                ("mixed_tol_inf", ctypes.c_double), ("refine_tol_inf", ctypes.c_double),
                ("verbose", ctypes.c_int), ("autotune", ctypes.c_int), ("refine_precision", ctypes.c_int),
                ("jvp", ctypes.c_int), ("forcing", ctypes.c_int),
                ("lu_products", ctypes.c_int), ("lu_order", ctypes.c_int), ("wait_limit", ctypes.c_int),
                ("sm_partition", ctypes.c_int)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("max_group", ctypes.c_int), ("keep_contexts", ctypes.c_int), ("opts", Opts)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("queued", ctypes.c_int), ("active", ctypes.c_int),
                ("peak_active", ctypes.c_int), ("bytes_held", ctypes.c_size_t),
                ("peak_bytes_held", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("contexts_created", ctypes.c_longlong), ("contexts_reused", ctypes.c_longlong),
                ("contexts_evicted", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestTimes(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("group_size", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("residual_evals", ctypes.c_int),
                ("residual_evals_fp64", ctypes.c_int), ("krylov_iters", ctypes.c_int),
                ("precond_applies", ctypes.c_int), ("line_search_cuts", ctypes.c_int),
                ("final_norm_inf", ctypes.c_double), ("final_norm_inf_fp64", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("pairs_per_residual_hi", ctypes.c_int), ("pairs_per_residual_lo", ctypes.c_int),
                ("residual_evals_ff", ctypes.c_int), ("exact_jvps", ctypes.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["pairs_per_residual"] = (d.pop("pairs_per_residual_hi") << 31) | d.pop("pairs_per_residual_lo")
        return d


_LIB = None
_vp = ctypes.c_void_p


def lib():
    """Load libswj.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libswj.so not built: run `python -m paper_1403_5044_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        sig = {
            "swj_default_opts": (None, [P(Opts)]),
            "swj_create": (ctypes.c_int, [P(_vp), P(Mesh), ctypes.c_double, ctypes.c_double, P(Opts), _vp]),
            "swj_batch_create": (ctypes.c_int, [P(_vp), P(Mesh), ctypes.c_int, P(ctypes.c_double),
                                                 P(ctypes.c_double), P(Opts), _vp]),
            "swj_batch_count": (ctypes.c_int, [_vp]),
            "swj_batch_set_params": (ctypes.c_int, [_vp, P(ctypes.c_double), P(ctypes.c_double)]),
            "swj_destroy": (None, [_vp]),
            "swj_pair_variants": (ctypes.c_int, [ctypes.c_int]),
            "swj_pair_variant_name": (ctypes.c_char_p, [ctypes.c_int, ctypes.c_int]),
            "swj_pair_config": (ctypes.c_int, [_vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                               P(ctypes.c_int), P(ctypes.c_int)]),
            "swj_set_pair_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
            "swj_footprint_bytes": (ctypes.c_size_t, [P(Mesh), ctypes.c_int, P(Opts)]),
            "swj_server_default_opts": (None, [P(ServerOpts)]),
            "swj_server_create": (ctypes.c_int, [P(_vp), P(ServerOpts)]),
            "swj_server_submit": (ctypes.c_int, [_vp, P(Mesh), ctypes.c_double, ctypes.c_double,
                                                 P(ctypes.c_longlong)]),
            "swj_server_poll": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_int, P(Stats), _vp,
                                               P(RequestTimes)]),
            "swj_server_get_info": (ctypes.c_int, [_vp, P(ServerInfo)]),
            "swj_server_drain": (ctypes.c_int, [_vp]),
            "swj_server_destroy": (None, [_vp]),
            "swj_set_params": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
            "swj_set_opts": (ctypes.c_int, [_vp, P(Opts)]),
            "swj_solve_host": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp, _vp, P(Stats)]),
            "swj_set_test_hooks": (ctypes.c_int, [_vp, ctypes.c_int]),
            "swj_workspace_bytes": (ctypes.c_size_t, [_vp]),
            "swj_initial_guess_flat": (ctypes.c_int, [_vp, _vp]),
            "swj_residual": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
            "swj_jvp": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
            "swj_precond_setup": (ctypes.c_int, [_vp]),
            "swj_precond_apply": (ctypes.c_int, [_vp, _vp, _vp]),
            "swj_jvp_exact": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
            "swj_initial_guess_linear": (ctypes.c_int, [_vp, _vp]),
            "swj_solve_continuation": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
            "swj_resample": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "swj_preconditioned_jacobian": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
            "swj_precond_sweep_clusters": (ctypes.c_int, [_vp]),
            "swj_precond_chain_sms": (ctypes.c_int, [_vp]),
            "swj_solve": (ctypes.c_int, [_vp, _vp, _vp]),
            "swj_unpack": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "swj_surface": (ctypes.c_int, [_vp, _vp, _vp]),
            "swj_sync": (ctypes.c_int, [_vp]),
            "swj_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "swj_version": (ctypes.c_char_p, []),
            "swj_kernel_launches": (ctypes.c_ulonglong, []),
            "swj_set_kernel_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
            "swj_pair_timing": (ctypes.c_int, [_vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int)]),
            "swj_reset_pair_timing": (ctypes.c_int, [_vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def header_functions(path: str = HEADER):
    """Names of every function the public header declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(swj_[a-z0-9_]+)\s*\(", txt)))


def strerror(status: int) -> str:
    return lib().swj_strerror(int(status)).decode()


def version() -> str:
    return lib().swj_version().decode()


def pair_variants(precision) -> int:
    return int(lib().swj_pair_variants(int(precision)))


def pair_variant_name(precision, variant) -> str:
    return lib().swj_pair_variant_name(int(precision), int(variant)).decode()


def kernel_launches() -> int:
    """Kernel launches issued by the library since it was loaded."""
    return int(lib().swj_kernel_launches())


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().swj_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "solve_mode" and isinstance(v, str):
            v = {"fp64": SOLVE_FP64, "mixed": SOLVE_MIXED}[v]
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a):
    """Address of a contiguous float64 host buffer (numpy array or CPU torch tensor), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise ValueError("expected a contiguous float64 CPU tensor")
        return _vp(a.data_ptr())
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("expected a contiguous float64 numpy array")
    return _vp(a.ctypes.data)


def _check(rc, what):
    if rc != OK:
        raise SwjError(rc, what)
    return rc


class Context:
    """One mesh, one (F, eps), one CUDA stream (torch's current stream by
    default).  Mirrors swj_create / swj_destroy."""

    def __init__(self, N, M, x1, dx, dy, F, eps, n_rad=0.05, opts: Opts | None = None, stream=None, **kw):
        import torch
        self.mesh = Mesh(int(N), int(M), float(x1), float(dx), float(dy), float(n_rad))
        self.opts = opts if opts is not None else default_opts(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = getattr(stream, "cuda_stream", stream)
        self._h = _vp()
        _check(lib().swj_create(ctypes.byref(self._h), ctypes.byref(self.mesh), float(F), float(eps),
                                ctypes.byref(self.opts), _vp(handle)), "swj_create")
        self.N, self.M, self.F, self.eps = int(N), int(M), float(F), float(eps)
        self.n_unknowns = 2 * (self.N + 1) * self.M

    @classmethod
    def from_spec(cls, spec, F, eps, **kw):
        return cls(spec.N, spec.M, spec.x1, spec.dx, spec.dy, F, eps, n_rad=spec.n_rad, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().swj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- thin wrappers -------------------------------------------------------
    def vector(self):
        import torch
        return torch.empty(self.n_unknowns, dtype=torch.float64, device="cuda")

    def set_params(self, F, eps):
        _check(lib().swj_set_params(self._h, float(F), float(eps)), "swj_set_params")
        self.F, self.eps = float(F), float(eps)

    def set_opts(self, opts: Opts):
        _check(lib().swj_set_opts(self._h, ctypes.byref(opts)), "swj_set_opts")
        self.opts = opts

    def workspace_bytes(self):
        return int(lib().swj_workspace_bytes(self._h))

    def initial_guess_flat(self, u):
        _check(lib().swj_initial_guess_flat(self._h, _ptr(u)), "swj_initial_guess_flat")
        return u

    def initial_guess_linear(self, u):
        _check(lib().swj_initial_guess_linear(self._h, _ptr(u)), "swj_initial_guess_linear")
        return u

    def resample_from(self, src, u_src, u):
        """u (on this mesh) <- u_src, a solution on src's mesh (swj_resample)."""
        _check(lib().swj_resample(src._h, _ptr(u_src), self._h, _ptr(u)), "swj_resample")
        return u

    def solve_continuation(self, u, steps, check=True):
        st = Stats()
        rc = lib().swj_solve_continuation(self._h, _ptr(u), int(steps), ctypes.cast(ctypes.byref(st), _vp))
        if check:
            _check(rc, "swj_solve_continuation")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def preconditioned_jacobian(self, u, out, col0=0, ncols=None, precision=FP64):
        """Columns of J(u) P^-1 into `out` (a CUDA float64 tensor of
        n_unknowns * ncols, column-major)."""
        ncols = self.n_unknowns - col0 if ncols is None else ncols
        _check(lib().swj_preconditioned_jacobian(self._h, _ptr(u), int(col0), int(ncols), _ptr(out), int(precision)),
               "swj_preconditioned_jacobian")
        return out

    def residual(self, u, E, precision=FP64):
        _check(lib().swj_residual(self._h, _ptr(u), _ptr(E), int(precision)), "swj_residual")
        return E

    def jvp(self, u, Eu, v, Jv, precision=FP64):
        _check(lib().swj_jvp(self._h, _ptr(u), _ptr(Eu), _ptr(v), _ptr(Jv), int(precision)), "swj_jvp")
        return Jv

    def jvp_exact(self, u, v, Jv, precision=FP64):
        _check(lib().swj_jvp_exact(self._h, _ptr(u), _ptr(v), _ptr(Jv), int(precision)), "swj_jvp_exact")
        return Jv

    def precond_setup(self):
        _check(lib().swj_precond_setup(self._h), "swj_precond_setup")

    def precond_apply(self, b, r):
        _check(lib().swj_precond_apply(self._h, _ptr(b), _ptr(r)), "swj_precond_apply")
        return r

    def sweep_clusters(self):
        return int(lib().swj_precond_sweep_clusters(self._h))

    def chain_sms(self):
        return int(lib().swj_precond_chain_sms(self._h))

    def set_test_hooks(self, hooks):
        """swj_set_test_hooks: TEST_WITHHOLD_HELPERS makes the multi-cluster
        apply's bounded polls run out (for testing the timeout path)."""
        _check(lib().swj_set_test_hooks(self._h, int(hooks)), "swj_set_test_hooks")

    def solve(self, u, check=True):
        st = Stats()
        rc = lib().swj_solve(self._h, _ptr(u), ctypes.cast(ctypes.byref(st), _vp))
        if check:
            _check(rc, "swj_solve")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def solve_host(self, u0_host, setup=True, u_host=None, zeta_host=None, phi_host=None, check=True):
        """swj_solve_host: the solve from and to host buffers (contiguous
        float64 numpy arrays or CPU torch tensors, pinned or not)."""
        st = Stats()
        rc = lib().swj_solve_host(self._h, _host_ptr(u0_host), int(bool(setup)), _host_ptr(u_host),
                                  _host_ptr(zeta_host), _host_ptr(phi_host), ctypes.byref(st))
        if check:
            _check(rc, "swj_solve_host")
        d = st.as_dict()
        d["rc"] = rc
        return d

    def unpack(self, u, zeta=None, phi=None):
        _check(lib().swj_unpack(self._h, _ptr(u), _ptr(zeta), _ptr(phi)), "swj_unpack")

    def surface(self, u, out):
        _check(lib().swj_surface(self._h, _ptr(u), _ptr(out)), "swj_surface")
        return out

    def sync(self):
        _check(lib().swj_sync(self._h), "swj_sync")

    def pair_config(self, precision):
        """(variant, threads per block, targets per thread, packed) of the all-pairs kernel."""
        v, t, r, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().swj_pair_config(self._h, int(precision), ctypes.byref(v), ctypes.byref(t),
                                     ctypes.byref(r), ctypes.byref(p)), "swj_pair_config")
        return v.value, t.value, r.value, bool(p.value)

    def set_pair_config(self, precision, variant):
        _check(lib().swj_set_pair_config(self._h, int(precision), int(variant)), "swj_set_pair_config")

    def set_kernel_timing(self, enable=True):
        _check(lib().swj_set_kernel_timing(self._h, int(bool(enable))), "swj_set_kernel_timing")

    def reset_pair_timing(self):
        _check(lib().swj_reset_pair_timing(self._h), "swj_reset_pair_timing")

    def pair_timing(self, precision):
        """(total device ms, launches) of the timed all-pairs launches."""
        ms, n = ctypes.c_double(), ctypes.c_int()
        _check(lib().swj_pair_timing(self._h, int(precision), ctypes.byref(ms), ctypes.byref(n)),
               "swj_pair_timing")
        return ms.value, n.value


class BatchContext(Context):
    """`count` instances on one mesh, instance i with (F[i], eps[i]); mirrors
    swj_batch_create.  Vectors hold the instances back to back: a vector()
    is count * n_unknowns doubles, and `view(x)` shows it as [count, n]."""

    def __init__(self, N, M, x1, dx, dy, F, eps, n_rad=0.05, opts: Opts | None = None, stream=None, **kw):
        import torch
        F = [float(f) for f in F]
        eps = [float(e) for e in eps]
        if len(F) != len(eps) or not F:
            raise ValueError("F and eps must be non-empty and of equal length")
        self.mesh = Mesh(int(N), int(M), float(x1), float(dx), float(dy), float(n_rad))
        self.opts = opts if opts is not None else default_opts(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = getattr(stream, "cuda_stream", stream)
        self.count = len(F)
        Fa = (ctypes.c_double * self.count)(*F)
        ea = (ctypes.c_double * self.count)(*eps)
        self._h = _vp()
        _check(lib().swj_batch_create(ctypes.byref(self._h), ctypes.byref(self.mesh), self.count, Fa, ea,
                                      ctypes.byref(self.opts), _vp(handle)), "swj_batch_create")
        self.N, self.M, self.F, self.eps = int(N), int(M), F, eps
        self.n_unknowns = 2 * (self.N + 1) * self.M

    @classmethod
    def from_spec(cls, spec, F, eps, **kw):
        return cls(spec.N, spec.M, spec.x1, spec.dx, spec.dy, F, eps, n_rad=spec.n_rad, **kw)

    def vector(self):
        import torch
        return torch.empty(self.count * self.n_unknowns, dtype=torch.float64, device="cuda")

    def view(self, x):
        return x.view(self.count, -1)

    def set_params(self, F, eps):
        F = [float(f) for f in F]
        eps = [float(e) for e in eps]
        _check(lib().swj_batch_set_params(self._h, (ctypes.c_double * self.count)(*F),
                                          (ctypes.c_double * self.count)(*eps)), "swj_batch_set_params")
        self.F, self.eps = F, eps

    def solve(self, u, check=True):
        """Solve every instance; returns (rc, [stats dict per instance])."""
        st = (Stats * self.count)()
        rc = lib().swj_solve(self._h, _ptr(u), ctypes.cast(st, _vp))
        if check:
            _check(rc, "swj_solve")
        out = []
        for i in range(self.count):
            d = st[i].as_dict()
            d["rc"] = st[i].status
            out.append(d)
        return rc, out


def footprint_bytes(spec, count=1, opts: Opts | None = None, **kw):
    """Device bytes a context of `count` instances of mesh `spec` holds once its
    preconditioner is built (swj_footprint_bytes)."""
    m = Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    o = opts if opts is not None else default_opts(**kw)
    return int(lib().swj_footprint_bytes(ctypes.byref(m), int(count), ctypes.byref(o)))


class Server:
    """The serving loop of swj_server_*: submit() queues a solve and returns
    its id; poll(id, wait) returns None while it is pending, else a dict with
    the status, solver counters, zeta ([M, N] numpy array) and times."""

    def __init__(self, hbm_budget_bytes=0, max_active=4, max_group=8, keep_contexts=True,
                 opts: Opts | None = None, **kw):
        so = ServerOpts()
        lib().swj_server_default_opts(ctypes.byref(so))
        so.hbm_budget_bytes = int(hbm_budget_bytes)
        so.max_active = int(max_active)
        so.max_group = int(max_group)
        so.keep_contexts = int(bool(keep_contexts))
        so.opts = opts if opts is not None else default_opts(**kw)
        self._h = _vp()
        _check(lib().swj_server_create(ctypes.byref(self._h), ctypes.byref(so)), "swj_server_create")
        self._shape = {}

    def submit(self, spec, F, eps):
        m = Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
        rid = ctypes.c_longlong()
        _check(lib().swj_server_submit(self._h, ctypes.byref(m), float(F), float(eps), ctypes.byref(rid)),
               "swj_server_submit")
        self._shape[rid.value] = (spec.M, spec.N)
        return rid.value

    def poll(self, rid, wait=False):
        import numpy as np
        M, N = self._shape[rid]
        z = np.empty((M, N), dtype=np.float64)
        st, tm = Stats(), RequestTimes()
        rc = lib().swj_server_poll(self._h, int(rid), int(bool(wait)), ctypes.byref(st),
                                   z.ctypes.data_as(_vp), ctypes.byref(tm))
        if rc == PENDING:
            return None
        del self._shape[rid]
        if rc == EINVAL:
            raise SwjError(rc, "swj_server_poll")
        d = st.as_dict()
        d.update(rc=rc, zeta=z, queue_ms=tm.queue_ms, run_ms=tm.run_ms, latency_ms=tm.latency_ms,
                 group_size=tm.group_size)
        return d

    def info(self):
        i = ServerInfo()
        _check(lib().swj_server_get_info(self._h, ctypes.byref(i)), "swj_server_get_info")
        return i.as_dict()

    def drain(self):
        _check(lib().swj_server_drain(self._h), "swj_server_drain")

    def close(self):
        if getattr(self, "_h", None):
            lib().swj_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
