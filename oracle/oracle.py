"""
Plain FP64 CPU oracle for the nonlinear ship-wave residual E(u) and its root.

TEST INFRASTRUCTURE ONLY.  This module is the independent reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it.  It shares no
code with the product library: every step below is written out from the
paper (Pethiyagoda, McCue, Moroney & Back, "Jacobian-free Newton-Krylov
methods with GPU acceleration for computing nonlinear ship wave patterns",
arXiv 1403.5044), and the one heavy loop (the all-pairs boundary-integral sum)
is plain C in ``pairsum.c``.

Contents, in the paper's order:
  * mesh and unknown vector                      (Section 3, Eq. unknowns)
  * trapezoidal integration of zeta, phi along x (Section 3, Eq. zetaapprox)
  * cubic-spline slopes zeta_y, phi_y along y    (Section 3, after Eq. zetaapprox)
  * half-mesh (two-point) interpolation          (Section 3)
  * free-surface condition E1                    (Eq. freeSurfCond)
  * boundary-integral equation E2 with the
    singularity subtraction and the closed-form
    integral I of S2                              (Eq. IntegroEqn, Eq. S2, Eq. IS2)
  * radiation conditions E3..E6                   (Eq. numUpRadiation, Appendix A)
  * equation ordering                             (Appendix A)
  * linear Jacobian used by the preconditioner    (Appendix B, Eqs. PreA-PreD)
  * finite-difference Jacobian-vector product     (Eq. JvApprox)
  * the exact Jacobian-vector product, by the
    complex-step derivative of E                  (the derivative Eq. JvApprox approximates)
  * the linear-problem initial guess and mesh
    bootstrapping by resampling                   (Section 4.1, Section 2.3)
  * reference root-finders (dense FD-Newton for tiny meshes, Newton-GMRES
    with the linear-Jacobian preconditioner)      (Section 4)

Readings where the paper is silent or garbled (each one is also listed in the
design notes of the repository):
  R1 the image part of K1 has (y + y*)^2 in its denominator;
  R2 zeta_x, zeta_y inside K1 are evaluated at the integration point;
  R3 x0 in the flat initial guess is the first mesh abscissa x1;
  R4 y1 = 0;
  R5 the spline along y is clamped with zero slope at y1 = 0 (even
     extension) and uses the not-a-knot condition at y_M;
  R6 w(i,j) is the product trapezoidal weight (half weights on the edges);
  R7 the last term of the linear E2 multiplies I by the target's zeta_x*;
  R8 in the case lists of PreB and PreC the first matching case applies;
  R9 block bandwidth b keeps the blocks of D with |l - m| <= (b - 1)/2;
 R10 the FD step is h = sqrt(eps_mach) max(1, ||u||_2) / ||v||_2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np
from scipy.interpolate import CubicSpline

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


# --------------------------------------------------------------------------
# the C all-pairs sum
# --------------------------------------------------------------------------
def build_c(force: bool = False) -> str:
    """Compile ``pairsum.c`` into ``_pairsum.so`` next to it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "pairsum.c")
    out = os.path.join(_HERE, "_pairsum.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_c())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_pairsum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double] + [dp] * 10
        lib.oracle_pairsum.restype = None
        lib.oracle_pair_kernels.argtypes = [ctypes.c_double] * 9 + [dp]
        lib.oracle_pair_kernels.restype = None
        lib.oracle_pairsum_targets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double] + [dp] * 8 + \
            [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp]
        lib.oracle_pairsum_targets.restype = None
        lib.oracle_pairsum_cs.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 9 + [dp]
        lib.oracle_pairsum_cs.restype = None
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pair_kernels(dx, dy, dyp, dz, zx_s, zy_s, A, B, C):
    """K1, K2, S2 of one (source, target) pair (Eq. IntegroEqn kernels, Eq. S2)."""
    out = np.zeros(3)
    _lib().oracle_pair_kernels(dx, dy, dyp, dz, zx_s, zy_s, A, B, C, _p(out))
    return out


# --------------------------------------------------------------------------
# mesh and unknowns
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Mesh:
    """N x M mesh with spacings dx, dy, first abscissa x1, y1 = 0 (R4), and
    the decay rate n of the upstream radiation condition (n = 0.05 in the
    paper, Section 3)."""
    N: int
    M: int
    x1: float
    dx: float
    dy: float
    n_rad: float = 0.05

    @property
    def n_unknowns(self) -> int:
        return 2 * (self.N + 1) * self.M

    def x(self):
        return self.x1 + self.dx * np.arange(self.N)

    def y(self):
        return self.dy * np.arange(self.M)

    def x_star(self):
        """Half-mesh abscissae x_{k+1/2}, k = 1..N-1."""
        return self.x1 + self.dx * (np.arange(self.N - 1) + 0.5)


def unpack(mesh: Mesh, u):
    """Split u per Eq. unknowns into phi_1[l], phi_x[l, k], zeta_1[l], zeta_x[l, k]."""
    N, M = mesh.N, mesh.M
    half = (N + 1) * M
    dt = np.complex128 if np.iscomplexobj(u) else np.float64   # complex: jvp_exact's step
    P = np.asarray(u[:half], dtype=dt).reshape(M, N + 1)
    Z = np.asarray(u[half:], dtype=dt).reshape(M, N + 1)
    return P[:, 0].copy(), P[:, 1:].copy(), Z[:, 0].copy(), Z[:, 1:].copy()


def pack(mesh: Mesh, phi1, phix, zeta1, zetax):
    """Inverse of :func:`unpack`."""
    P = np.concatenate([np.asarray(phi1)[:, None], np.asarray(phix)], axis=1)
    Z = np.concatenate([np.asarray(zeta1)[:, None], np.asarray(zetax)], axis=1)
    return np.concatenate([P.ravel(), Z.ravel()])


def flat_guess(mesh: Mesh):
    """Flat-surface initial guess of Section 4.1: phi_1 = x0 (= x1, R3),
    phi_x = 1, zeta_1 = 0, zeta_x = 0."""
    N, M = mesh.N, mesh.M
    return pack(mesh, np.full(M, mesh.x1), np.ones((M, N)), np.zeros(M), np.zeros((M, N)))


# --------------------------------------------------------------------------
# mesh step: integration along x, spline along y, half-mesh values
# --------------------------------------------------------------------------
def trapezoid_x(mesh: Mesh, f1, fx):
    """Eq. zetaapprox: f_{k+1,l} = f_{k,l} + dx/2 (fx_{k,l} + fx_{k+1,l})."""
    f = np.empty_like(fx)
    f[:, 0] = f1
    for k in range(mesh.N - 1):
        f[:, k + 1] = f[:, k] + 0.5 * mesh.dx * (fx[:, k] + fx[:, k + 1])
    return f


def spline_slope_y(mesh: Mesh, f):
    """d f / d y at the mesh nodes from the cubic spline through f[:, k] in y
    for every k (Section 3).  End conditions (R5): zero slope at y1 = 0, the
    even extension of the symmetric flow, and not-a-knot at y_M."""
    f = np.asarray(f)
    f = f if np.iscomplexobj(f) else f.astype(np.float64)   # complex for the complex step only
    cs = CubicSpline(mesh.y(), f, axis=0,
                     bc_type=((1, np.zeros(f.shape[1:])), "not-a-knot"))
    return cs(mesh.y(), 1)


def half_mesh(q):
    """Two-point interpolation to (x_{k+1/2}, y_l): (q_k + q_{k+1}) / 2."""
    return 0.5 * (q[:, :-1] + q[:, 1:])


def surface(mesh: Mesh, u):
    """All per-node and per-target quantities of the mesh step, as a dict.

    Node arrays have shape [M, N], target arrays [M, N-1]."""
    phi1, phix, zeta1, zetax = unpack(mesh, u)
    zeta = trapezoid_x(mesh, zeta1, zetax)
    # Eq. zetaapprox applied to g = phi - x: the trapezoidal rule integrates
    # the constant slope 1 of x exactly, so integrating phi_x - 1 from
    # phi_1 - x1 gives phi - x at every node.  E(u) depends on phi only
    # through phi - x (Eq. IntegroEqn: phi - phi* - x + x*, phi* - x*) and
    # through phi_x, phi_y, so g avoids carrying the O(|x|) part of phi
    # through the sums and the spline.
    g = trapezoid_x(mesh, phi1 - mesh.x1, phix - 1.0)
    phi = g + mesh.x()[None, :]
    phiy = spline_slope_y(mesh, g)
    zetay = spline_slope_y(mesh, zeta)
    st = {
        "phi1": phi1, "phix": phix, "zeta1": zeta1, "zetax": zetax,
        "phi": phi, "zeta": zeta, "phiy": phiy, "zetay": zetay, "g": g,
    }
    for name in ("g", "zeta", "phix", "phiy", "zetax", "zetay"):
        st[name + "_t"] = half_mesh(st[name])
    st["phi_t"] = st["g_t"] + mesh.x_star()[None, :]
    return st


# --------------------------------------------------------------------------
# closed form of I = int int S2 dx dy (Eq. IS2)
# --------------------------------------------------------------------------
def _G(A, B, C, s, t):
    """A function whose mixed derivative d^2 G / ds dt is (A s^2 + B s t + C t^2)^(-1/2):
        G = s/sqrt(C) asinh((B s + 2 C t)/(sqrt(D)|s|)) + t/sqrt(A) asinh((2 A s + B t)/(sqrt(D)|t|)),
    D = 4AC - B^2 > 0.  Each term is zero where its prefactor s or t is zero
    (its limit there).  The asinh form is the logarithm form of the paper
    with one-variable terms dropped; they cancel in the four-corner sum."""
    # (A, B, C are complex only under the complex step of jvp_exact; s, t are geometry)
    dt = np.result_type(np.asarray(A), np.asarray(B), np.asarray(C), np.float64)
    A, B, C = (np.asarray(v, dtype=dt) for v in (A, B, C))
    s, t = (np.asarray(v, dtype=np.float64) for v in (s, t))
    A, B, C, s, t = np.broadcast_arrays(A, B, C, s, t)
    sD = np.sqrt(4.0 * A * C - B * B)
    out = np.zeros(s.shape, dtype=dt)
    ns, nt = s != 0.0, t != 0.0
    out[ns] += s[ns] / np.sqrt(C[ns]) * np.arcsinh((B[ns] * s[ns] + 2.0 * C[ns] * t[ns]) / (sD[ns] * np.abs(s[ns])))
    out[nt] += t[nt] / np.sqrt(A[nt]) * np.arcsinh((2.0 * A[nt] * s[nt] + B[nt] * t[nt]) / (sD[nt] * np.abs(t[nt])))
    return out


def rect_integral(A, B, C, s1, s2, t1, t2):
    """int_{s1}^{s2} int_{t1}^{t2} (A s^2 + B s t + C t^2)^(-1/2) dt ds."""
    return _G(A, B, C, s2, t2) - _G(A, B, C, s1, t2) - _G(A, B, C, s2, t1) + _G(A, B, C, s1, t1)


def I_S2(mesh: Mesh, A, B, C, xt, yt):
    """Eq. IS2: the integral of S2 over [x1, xN] x [y1, yM] for targets at
    (xt, yt) with coefficients A, B, C.  The image part of S2 has -B and
    y + y* (Eq. S2), so it is the same rectangle integral with t = y + y*."""
    xN = mesh.x1 + (mesh.N - 1) * mesh.dx
    yM = (mesh.M - 1) * mesh.dy
    s1, s2 = mesh.x1 - xt, xN - xt
    direct = rect_integral(A, B, C, s1, s2, 0.0 - yt, yM - yt)
    image = rect_integral(A, -B, C, s1, s2, 0.0 + yt, yM + yt)
    return direct + image


# --------------------------------------------------------------------------
# the residual
# --------------------------------------------------------------------------
def pressure(x, y):
    """Applied surface pressure of the pressure-forcing variant (the
    hovercraft-like forcing the Discussion names as the next configuration;
    the paper gives no formula): the smooth bump with compact support
    p = exp(2 + 1/(x^2 - 1) + 1/(y^2 - 1)) for |x| < 1 and |y| < 1, else 0,
    equal to 1 at the centre."""
    x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    out = np.zeros(x.shape)
    inside = (np.abs(x) < 1.0) & (np.abs(y) < 1.0)
    xi, yi = x[inside], y[inside]
    out[inside] = np.exp(2.0 + 1.0 / (xi * xi - 1.0) + 1.0 / (yi * yi - 1.0))
    return out


def free_surface_E1(F, phix, phiy, zetax, zetay, zeta):
    """Eq. freeSurfCond written as E1 = 0."""
    num = (1 + zetax ** 2) * phiy ** 2 + (1 + zetay ** 2) * phix ** 2 - 2 * zetax * zetay * phix * phiy
    return 0.5 * num / (1 + zetax ** 2 + zetay ** 2) + zeta / F ** 2 - 0.5


def integral_sum(mesh: Mesh, st):
    """The trapezoidal all-pairs sum of E2 (C, ``pairsum.c``); returns the
    sum and the per-target sum of absolute term values, both [M, N-1].
    With complex mesh values (the complex step of jvp_exact) the sum is
    complex and the second array sums |Im| of the terms."""
    N, M = mesh.N, mesh.M
    if any(np.iscomplexobj(st[k]) for k in ("zeta", "zetax", "zetay", "g", "zeta_t", "zetax_t", "zetay_t", "g_t")):
        cc = lambda a: np.ascontiguousarray(a, dtype=np.complex128)
        arrs = [cc(st[k]) for k in ("zeta", "zetax", "zetay", "g", "zeta_t", "zetax_t", "zetay_t", "g_t")]
        s = np.zeros((M, N - 1), dtype=np.complex128)
        a = np.zeros((M, N - 1))
        _lib().oracle_pairsum_cs(N, M, mesh.x1, mesh.dx, mesh.dy,
                                 *[ctypes.c_void_p(x.ctypes.data) for x in arrs],
                                 ctypes.c_void_p(s.ctypes.data), _p(a))
        return s, a
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    zeta, zetax, zetay, g = c(st["zeta"]), c(st["zetax"]), c(st["zetay"]), c(st["g"])
    zt, zxt, zyt, gt = c(st["zeta_t"]), c(st["zetax_t"]), c(st["zetay_t"]), c(st["g_t"])
    s = np.zeros((M, N - 1))
    a = np.zeros((M, N - 1))
    _lib().oracle_pairsum(N, M, mesh.x1, mesh.dx, mesh.dy,
                          _p(zeta), _p(zetax), _p(zetay), _p(g),
                          _p(zt), _p(zxt), _p(zyt), _p(gt), _p(s), _p(a))
    return s, a


def residual_E2_at(mesh: Mesh, F: float, eps: float, u, targets):
    """E2 and its tolerance scale at the listed targets only (flat indices
    t = l (N-1) + k into the [M, N-1] target array); for sampled checks on
    meshes too large for a full evaluation."""
    st = surface(mesh, u)
    tidx = np.ascontiguousarray(np.asarray(targets, dtype=np.int32))
    k, l = tidx % (mesh.N - 1), tidx // (mesh.N - 1)
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    s = np.zeros(tidx.size)
    a = np.zeros(tidx.size)
    _lib().oracle_pairsum_targets(mesh.N, mesh.M, mesh.x1, mesh.dx, mesh.dy,
                                  _p(c(st["zeta"])), _p(c(st["zetax"])), _p(c(st["zetay"])), _p(c(st["g"])),
                                  _p(c(st["zeta_t"])), _p(c(st["zetax_t"])), _p(c(st["zetay_t"])),
                                  _p(c(st["g_t"])), int(tidx.size),
                                  tidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(s), _p(a))
    xt = mesh.x_star()[k]
    yt = mesh.y()[l]
    zxt, zyt = st["zetax_t"][l, k], st["zetay_t"][l, k]
    I = I_S2(mesh, 1 + zxt ** 2, 2 * zxt * zyt, 1 + zyt ** 2, xt, yt)
    src = eps / np.sqrt(xt ** 2 + yt ** 2 + (st["zeta_t"][l, k] + 1) ** 2)
    gt = st["g_t"][l, k]
    E2 = 2 * math.pi * gt + src - s - zxt * I
    scale = a + np.abs(2 * math.pi * gt) + np.abs(src) + np.abs(zxt * I)
    return E2, scale


def residual_parts(mesh: Mesh, F: float, eps: float, u, pairs: bool = True, forcing: str = "source"):
    """Every row family of E(u) before ordering, plus the tolerance scale of
    each E2 row (sum of absolute values of its terms).  With pairs=False the
    all-pairs sum is skipped and E2 / scale2 are left as NaN (for sampled
    checks on large meshes, see residual_E2_at)."""
    st = surface(mesh, u)
    xt = mesh.x_star()[None, :]
    yt = mesh.y()[:, None]
    zxt, zyt = st["zetax_t"], st["zetay_t"]
    A = 1 + zxt ** 2
    B = 2 * zxt * zyt
    C = 1 + zyt ** 2
    I = I_S2(mesh, A, B, C, xt, yt)
    if forcing == "source":
        src = eps / np.sqrt(xt ** 2 + yt ** 2 + (st["zeta_t"] + 1) ** 2)
    elif forcing == "pressure":
        src = np.zeros(st["zeta_t"].shape)
    else:
        raise ValueError(forcing)
    if pairs:
        S, Sabs = integral_sum(mesh, st)
    else:
        S = Sabs = np.full(st["g_t"].shape, np.nan)
    E1 = free_surface_E1(F, st["phix_t"], st["phiy_t"], zxt, zyt, st["zeta_t"])
    if forcing == "pressure":
        # Bernoulli's equation with the applied pressure eps p on the surface
        E1 = E1 + eps * pressure(xt, yt)
    # Eq. IntegroEqn with every term moved to one side, the second integral
    # split per the singularity subtraction (Section 3):
    E2 = 2 * math.pi * st["g_t"] + src - S - zxt * I
    n, x1, dx = mesh.n_rad, mesh.x1, mesh.dx
    phi1, phix, zeta1, zetax = st["phi1"], st["phix"], st["zeta1"], st["zetax"]
    E3 = x1 * (phix[:, 0] - 1) + n * (phi1 - x1)
    E4 = x1 * (phix[:, 1] - phix[:, 0]) / dx + n * (phix[:, 0] - 1)
    E5 = x1 * zetax[:, 0] + n * zeta1
    E6 = x1 * (zetax[:, 1] - zetax[:, 0]) / dx + n * zetax[:, 0]
    scale2 = Sabs + np.abs(2 * math.pi * st["g_t"]) + np.abs(src) + np.abs(zxt * I)
    return dict(E1=E1, E2=E2, E3=E3, E4=E4, E5=E5, E6=E6, I=I, src=src, S=S,
                scale2=scale2, st=st, Sabs=Sabs)


def order(mesh: Mesh, E1, E2, E3, E4, E5, E6):
    """Appendix A ordering: per l [E3, E4, E1_{1..N-1}], then per l [E5, E6, E2_{1..N-1}]."""
    top = np.concatenate([E3[:, None], E4[:, None], E1], axis=1)
    bot = np.concatenate([E5[:, None], E6[:, None], E2], axis=1)
    return np.concatenate([top.ravel(), bot.ravel()])


def residual(mesh: Mesh, F: float, eps: float, u, forcing: str = "source"):
    """E(u) of Eq. nonlinearsys, length 2(N+1)M, Appendix A order."""
    p = residual_parts(mesh, F, eps, u, forcing=forcing)
    return order(mesh, p["E1"], p["E2"], p["E3"], p["E4"], p["E5"], p["E6"])


def residual_scale(mesh: Mesh, F: float, eps: float, u, forcing: str = "source"):
    """Per-row magnitude that parity tolerances are relative to: for E2 rows
    the sum of absolute values of every term, for the other rows 1."""
    p = residual_parts(mesh, F, eps, u, forcing=forcing)
    one = np.ones_like(p["E1"])
    r = np.ones(mesh.M)
    return order(mesh, one, p["scale2"], r, r, r, r)


# --------------------------------------------------------------------------
# linear Jacobian (Appendix B), dense, optionally truncated to block bandwidth b
# --------------------------------------------------------------------------
def jacobian_linear(mesh: Mesh, F: float, b: int | None = None):
    """Dense Jacobian of the linearised discrete system, entries from
    Eqs. PreA-PreD plus the (linear) radiation rows E3..E6, in Appendix A
    order.  With b given, the entries of the zeta_x columns of the E2 rows are
    kept only for |l - m| <= (b - 1)/2 (Section 4.2, R9)."""
    N, M, dx, x1, n = mesh.N, mesh.M, mesh.dx, mesh.x1, mesh.n_rad
    H = (N + 1) * M
    J = np.zeros((2 * H, 2 * H))
    half_bw = None if b is None else (b - 1) // 2
    x, y, xs = mesh.x(), mesh.y(), mesh.x_star()
    cx = np.ones(N); cx[0] = cx[-1] = 0.5
    cy = np.ones(M); cy[0] = cy[-1] = 0.5
    w = dx * mesh.dy * cy[:, None] * cx[None, :]           # w[m, n] (0-based)
    col_phi1 = lambda l: l * (N + 1)
    col_phix = lambda nn, l: l * (N + 1) + nn               # nn = 1..N
    col_zeta1 = lambda l: H + l * (N + 1)
    col_zetax = lambda nn, l: H + l * (N + 1) + nn
    row_E3 = lambda l: l * (N + 1)
    row_E4 = lambda l: l * (N + 1) + 1
    row_E1 = lambda k, l: l * (N + 1) + 1 + k               # k = 1..N-1
    row_E5 = lambda l: H + l * (N + 1)
    row_E6 = lambda l: H + l * (N + 1) + 1
    row_E2 = lambda k, l: H + l * (N + 1) + 1 + k

    def preB(nn, k):   # d zeta*_k / d zeta_x_n  times F^2 (first matching case, R8)
        if nn == 1 and k == 1:
            return dx / 4
        if nn == 1 and k > 1:
            return dx / 2
        if nn < k:
            return dx
        if nn == k:
            return 3 * dx / 4
        if nn == k + 1:
            return dx / 4
        return 0.0

    I_lin = None
    for l in range(M):
        # radiation rows
        J[row_E3(l), col_phi1(l)] = n
        J[row_E3(l), col_phix(1, l)] = x1
        J[row_E4(l), col_phix(1, l)] = n - x1 / dx
        J[row_E4(l), col_phix(2, l)] = x1 / dx
        J[row_E5(l), col_zeta1(l)] = n
        J[row_E5(l), col_zetax(1, l)] = x1
        J[row_E6(l), col_zetax(1, l)] = n - x1 / dx
        J[row_E6(l), col_zetax(2, l)] = x1 / dx
        for k in range(1, N):
            # PreA
            J[row_E1(k, l), col_phix(k, l)] += 0.5
            J[row_E1(k, l), col_phix(k + 1, l)] += 0.5
            # d E1 / d zeta_1 and PreB
            J[row_E1(k, l), col_zeta1(l)] = 1 / F ** 2
            for nn in range(1, N + 1):
                v = preB(nn, k)
                if v:
                    J[row_E1(k, l), col_zetax(nn, l)] = v / F ** 2
            # d E2 / d phi_1 and PreC (= 2 pi F^2 times PreB)
            J[row_E2(k, l), col_phi1(l)] = 2 * math.pi
            for nn in range(1, N + 1):
                v = preB(nn, k)
                if v:
                    J[row_E2(k, l), col_phix(nn, l)] = 2 * math.pi * v
            # PreD
            xt, yt = xs[k - 1], y[l]
            K3 = 1 / np.sqrt((x[None, :] - xt) ** 2 + (y[:, None] - yt) ** 2) \
                + 1 / np.sqrt((x[None, :] - xt) ** 2 + (y[:, None] + yt) ** 2)
            I_lin = I_S2(mesh, 1.0, 0.0, 1.0, xt, yt)
            diag = 0.5 * np.sum(w * K3) - 0.5 * float(I_lin)
            nn = np.arange(1, N + 1)
            for m in range(M):
                if half_bw is not None and abs(l - m) > half_bw:
                    continue
                # "otherwise" case of PreD for every n of column block m
                J[row_E2(k, l), col_zetax(nn, m)] = -w[m, :] * K3[m, :]
            # first case of PreD: n = k, k+1 and m = l
            J[row_E2(k, l), col_zetax(k, l)] += diag
            J[row_E2(k, l), col_zetax(k + 1, l)] += diag
    return J


# --------------------------------------------------------------------------
# Jacobian-vector products and reference solvers
# --------------------------------------------------------------------------
def fd_step(u, v, eps_mach=np.finfo(np.float64).eps):
    """R10: h = sqrt(eps_mach) max(1, ||u||_2) / ||v||_2."""
    nv = np.linalg.norm(v)
    return 0.0 if nv == 0 else math.sqrt(eps_mach) * max(1.0, np.linalg.norm(u)) / nv


def jvp_fd(mesh, F, eps, u, v, Eu=None, h=None, forcing="source"):
    """Eq. JvApprox (with P^{-1} v already applied by the caller):
    J v ~ (E(u + h v) - E(u)) / h."""
    if Eu is None:
        Eu = residual(mesh, F, eps, u, forcing=forcing)
    if h is None:
        h = fd_step(u, v)
    return (residual(mesh, F, eps, u + h * v, forcing=forcing) - Eu) / h


def jvp_exact(mesh, F, eps, u, v, h=1e-30, forcing="source"):
    """J(u) v of the discrete residual, exactly (to rounding): the directional
    derivative d E(u + t v) / dt at t = 0, computed by the complex step
    Im E(u + i h v) / h.  Every operation of E is analytic in u (the
    trapezoid and spline are linear, the kernels and the closed form of I are
    compositions of products, quotients, square roots and asinh), so no
    difference is taken and h only needs to be tiny.  Returns (Jv, scale):
    scale is, per E2 row, the sum of |d/dt| of the terms of the row (the
    tolerance scale of the row), and |Jv| elsewhere."""
    uc = np.asarray(u, dtype=np.float64) + 1j * h * np.asarray(v, dtype=np.float64)
    p = residual_parts(mesh, F, eps, uc, forcing=forcing)
    Jv = order(mesh, p["E1"], p["E2"], p["E3"], p["E4"], p["E5"], p["E6"]).imag / h
    st = p["st"]
    s2 = (p["Sabs"] + np.abs((2 * math.pi * st["g_t"]).imag) + np.abs(p["src"].imag)
          + np.abs((st["zetax_t"] * p["I"]).imag)) / h
    z = lambda e: np.zeros(e.shape)
    scale = order(mesh, z(p["E1"]), s2, z(p["E3"]), z(p["E4"]), z(p["E5"]), z(p["E6"]))
    scale = np.where(scale > 0, scale, np.abs(Jv))
    return Jv, scale


def linear_solution(mesh, F, eps, b=None, forcing="source"):
    """The solution of the linearised problem (Section 2.3, the weak-source
    limit), offered as an initial guess in Section 4.1: one Newton step from
    the flat state with the linear Jacobian of Appendix B,
        u_L = u0 - J_lin^{-1} E(u0),
    exact for the discretised linear problem when b is None (untruncated);
    with a block bandwidth b the same step with the truncated matrix."""
    u0 = flat_guess(mesh)
    return u0 - np.linalg.solve(jacobian_linear(mesh, F, b), residual(mesh, F, eps, u0, forcing=forcing))


def resample(src: Mesh, u_src, dst: Mesh):
    """Mesh bootstrapping (Section 4.1 bootstraps in eps; the same idea across
    meshes): the unknowns of ``dst`` from a solution on ``src`` by bilinear
    interpolation of the source's node fields, coordinates clamped to the
    source mesh.  phi_1 and zeta_1 come from g = phi - x and zeta at
    (x1 of dst, y); phi_x and zeta_x from their node values."""
    st = surface(src, u_src)
    def bilinear(f, x, y):
        fi = np.clip((x - src.x1) / src.dx, 0.0, src.N - 1)
        fj = np.clip(y / src.dy, 0.0, src.M - 1)
        i0 = np.minimum(np.floor(fi).astype(int), src.N - 2)
        j0 = np.minimum(np.floor(fj).astype(int), src.M - 2)
        a, b = fi - i0, fj - j0
        return ((1 - a) * (1 - b) * f[j0, i0] + a * (1 - b) * f[j0, i0 + 1]
                + (1 - a) * b * f[j0 + 1, i0] + a * b * f[j0 + 1, i0 + 1])
    X, Y = np.meshgrid(dst.x(), dst.y())
    x1 = np.full(dst.M, dst.x1)
    phi1 = bilinear(st["g"], x1, dst.y()) + dst.x1
    zeta1 = bilinear(st["zeta"], x1, dst.y())
    return pack(dst, phi1, bilinear(st["phix"], X, Y), zeta1, bilinear(st["zetax"], X, Y))


def preconditioned_jacobian(mesh, F, eps, u, b=None):
    """J(u) P_b^-1 (Section 4.2), J exact column by column (jvp_exact) and
    P_b the Appendix B Jacobian truncated to block bandwidth b."""
    n = mesh.n_unknowns
    J = np.column_stack([jvp_exact(mesh, F, eps, u, e)[0] for e in np.eye(n)])
    return J @ np.linalg.inv(jacobian_linear(mesh, F, b))


def jacobian_fd(mesh, F, eps, u, h=1e-6, forcing="source"):
    """Dense Jacobian by central differences (tiny meshes only)."""
    n = u.size
    J = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        J[:, j] = (residual(mesh, F, eps, u + e, forcing=forcing) - residual(mesh, F, eps, u - e, forcing=forcing)) / (2 * h)
    return J


def newton_dense(mesh, F, eps, u0, tol=1e-10, max_iter=50, forcing="source"):
    """Damped Newton (Eqs. newtonstep0, newtonstep) with a dense central-
    difference Jacobian and a halving line search on ||E||_2."""
    u = np.array(u0, dtype=np.float64)
    E = residual(mesh, F, eps, u, forcing=forcing)
    for it in range(max_iter):
        if np.max(np.abs(E)) < tol:
            return u, it
        du = np.linalg.solve(jacobian_fd(mesh, F, eps, u, forcing=forcing), -E)
        lam = 1.0
        while True:
            un = u + lam * du
            En = residual(mesh, F, eps, un, forcing=forcing)
            if np.linalg.norm(En) <= (1 - 1e-4 * lam) * np.linalg.norm(E) or lam < 2 ** -10:
                break
            lam *= 0.5
        u, E = un, En
    raise RuntimeError("oracle dense Newton did not converge")


def gmres_right(apply_J, apply_Pinv, rhs, rtol, restart=30, max_iter=600):
    """Right-preconditioned restarted GMRES (Saad & Schultz), textbook form:
    Arnoldi with modified Gram-Schmidt on K_m(J P^{-1}, r), least squares for
    the small Hessenberg problem solved directly each step."""
    x = np.zeros_like(rhs)
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0:
        return x, 0
    total = 0
    r = rhs.copy()
    while total < max_iter:
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            break
        V = [r / beta]
        Z = []
        Hm = np.zeros((restart + 1, restart))
        y = None
        for j in range(restart):
            z = apply_Pinv(V[j])
            Z.append(z)
            wv = apply_J(z)
            for i in range(j + 1):
                Hm[i, j] = np.dot(wv, V[i])
                wv = wv - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(wv)
            total += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(Hm[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - Hm[:j + 2, :j + 1] @ y)
            if res <= rtol * bnorm or Hm[j + 1, j] == 0 or total >= max_iter:
                break
            V.append(wv / Hm[j + 1, j])
        x = x + np.array(Z[:len(y)]).T @ y
        r = rhs - apply_J(x)
        if res <= rtol * bnorm:
            break
    return x, total


def newton_gmres(mesh, F, eps, u0, tol=1e-10, max_newton=50, b=None, eta=1e-4, restart=30, forcing="source"):
    """Damped inexact Newton with right-preconditioned GMRES and the linear-
    Jacobian preconditioner of Section 4.2 (dense LU of ``jacobian_linear``;
    small and mid-size meshes).  Returns (u, newton_iterations)."""
    import scipy.linalg as sla
    P = jacobian_linear(mesh, F, b)
    lu = sla.lu_factor(P)
    u = np.array(u0, dtype=np.float64)
    E = residual(mesh, F, eps, u, forcing=forcing)
    for it in range(max_newton):
        if np.max(np.abs(E)) < tol:
            return u, it
        Eu = E
        du, _ = gmres_right(lambda z: jvp_fd(mesh, F, eps, u, z, Eu, forcing=forcing),
                            lambda v: sla.lu_solve(lu, v), -E, eta, restart=restart)
        lam = 1.0
        while True:
            un = u + lam * du
            En = residual(mesh, F, eps, un, forcing=forcing)
            if np.linalg.norm(En) <= (1 - 1e-4 * lam) * np.linalg.norm(E) or lam < 2 ** -10:
                break
            lam *= 0.5
        u, E = un, En
    if np.max(np.abs(E)) < tol:
        return u, max_newton
    raise RuntimeError("oracle Newton-GMRES did not converge")


def zeta_phi(mesh: Mesh, u):
    """zeta and phi on the N x M mesh (arrays [M, N]) rebuilt from u."""
    phi1, phix, zeta1, zetax = unpack(mesh, u)
    return trapezoid_x(mesh, zeta1, zetax), trapezoid_x(mesh, phi1, phix)
