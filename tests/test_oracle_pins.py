"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an independent quadrature, a geometric definition, a special state with
a known residual, the linear Jacobian printed in Appendix B, or a symmetry.
No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import CubicSpline

import oracle as O
from paper_1403_5044_b300 import workloads as W


def _mesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


TINY = W.MeshSpec(9, 5, -2.0, 0.5, 0.4)
SMALL = W.MeshSpec(7, 4, -1.5, 0.5, 0.3)


# ---------------------------------------------------------------- Eq. IS2
def _corner_polar(A, B, C, a, b):
    """Unsigned int over the rectangle with corners (0, 0) and (a, b) of
    (A s^2 + B s t + C t^2)^(-1/2), by polar coordinates about the singular
    corner: with Q = r^2 q(theta) the radial integral is exact and the
    remaining angular integrand is smooth on each side of the diagonal."""
    if a == 0.0 or b == 0.0:
        return 0.0
    ta = 0.0 if a > 0 else (math.pi if b > 0 else -math.pi)
    tb = math.pi / 2 if b > 0 else -math.pi / 2
    lo, hi = min(ta, tb), max(ta, tb)
    tc = math.atan2(b, a)
    q = lambda th: A * math.cos(th) ** 2 + B * math.cos(th) * math.sin(th) + C * math.sin(th) ** 2
    R = lambda th: min(abs(a) / max(abs(math.cos(th)), 1e-300), abs(b) / max(abs(math.sin(th)), 1e-300))
    f = lambda th: R(th) / math.sqrt(q(th))
    v1 = integrate.quad(f, lo, tc, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    v2 = integrate.quad(f, tc, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return v1 + v2


def _rect_polar(A, B, C, s1, s2, t1, t2):
    W_ = lambda a, b: math.copysign(1.0, a) * math.copysign(1.0, b) * _corner_polar(A, B, C, a, b)
    return W_(s2, t2) - W_(s1, t2) - W_(s2, t1) + W_(s1, t1)


@pytest.mark.parametrize("A,B,C", [(1.0, 0.0, 1.0), (1.3, 0.4, 1.1), (1.02, -0.3, 1.6), (2.5, 1.9, 1.7)])
@pytest.mark.parametrize("box", [(-3.0, 4.0, -2.0, 5.0), (-0.25, 7.75, 0.0, 2.4), (-5.1, -0.1, 0.3, 2.0),
                                 (0.5, 3.0, -4.0, -1.0), (-1.0, 1.0, -1.0, 1.0)])
def test_I_closed_form_matches_polar_quadrature(A, B, C, box):
    s1, s2, t1, t2 = box
    got = float(O.rect_integral(A, B, C, s1, s2, t1, t2))
    ref = _rect_polar(A, B, C, s1, s2, t1, t2)
    assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (got, ref)


def test_I_closed_form_matches_2d_quadrature_off_singularity():
    A, B, C = 1.4, 0.7, 1.2
    s1, s2, t1, t2 = 0.5, 2.0, -1.0, 1.5
    ref = integrate.dblquad(lambda t, s: (A * s * s + B * s * t + C * t * t) ** -0.5, s1, s2, t1, t2,
                            epsabs=1e-13, epsrel=1e-13)[0]
    assert abs(float(O.rect_integral(A, B, C, s1, s2, t1, t2)) - ref) < 1e-10


def test_I_image_part_is_mirror_of_direct():
    """I over the half domain with the image term equals the direct term alone
    over the mirrored full domain [x1, xN] x [-yM, yM] (Eq. S2, Eq. IS2)."""
    mesh = _mesh(TINY)
    yM = (mesh.M - 1) * mesh.dy
    xN = mesh.x1 + (mesh.N - 1) * mesh.dx
    rng = np.random.default_rng(3)
    for _ in range(10):
        A, C = 1 + rng.uniform(0, 0.5, 2)
        B = rng.uniform(-0.5, 0.5)
        xt = mesh.x1 + mesh.dx * (rng.integers(0, mesh.N - 1) + 0.5)
        yt = mesh.dy * rng.integers(0, mesh.M)
        half = float(O.I_S2(mesh, A, B, C, xt, yt))
        full = float(O.rect_integral(A, B, C, mesh.x1 - xt, xN - xt, -yM - yt, yM - yt))
        assert abs(half - full) < 1e-12 * abs(full)


# ---------------------------------------------------------------- kernels
def _grad_inv_r(P, Q, h=1e-5):
    """Central-difference gradient of 1/|P - Q| with respect to P."""
    g = np.zeros(3)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g[d] = (1 / np.linalg.norm(P + e - Q) - 1 / np.linalg.norm(P - e - Q)) / (2 * h)
    return g


def test_K1_is_normal_derivative_of_green_function_with_image():
    """K1 dA is the derivative of 1/r along the (unnormalised) upward normal
    N = (-zeta_x, -zeta_y, 1) of the integration surface, with sign such
    that K1 = -N . grad_P (1/|P - P*|); the image point is the source mirrored
    in y = 0, whose surface slope in y flips (R1, R2)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        xs, ys, zs, zx, zy = rng.uniform(-2, 2), rng.uniform(0, 2), rng.uniform(-.3, .3), rng.uniform(-.5, .5), rng.uniform(-.5, .5)
        xt, yt, zt = rng.uniform(-2, 2), rng.uniform(0, 2), rng.uniform(-.3, .3)
        P, Pm, T = np.array([xs, ys, zs]), np.array([xs, -ys, zs]), np.array([xt, yt, zt])
        N1, Nm = np.array([-zx, -zy, 1.0]), np.array([-zx, zy, 1.0])
        K1_ref = -N1 @ _grad_inv_r(P, T) - Nm @ _grad_inv_r(Pm, T)
        K2_ref = 1 / np.linalg.norm(P - T) + 1 / np.linalg.norm(Pm - T)
        K1, K2, _ = O.pair_kernels(xs - xt, ys - yt, ys + yt, zs - zt, zx, zy, 1.0, 0.0, 1.0)
        assert abs(K1 - K1_ref) < 1e-7 * max(1, abs(K1_ref))
        assert abs(K2 - K2_ref) < 1e-13 * K2_ref


def test_S2_equals_K2_on_the_tangent_plane():
    """S2 is K2 with the surface replaced by the target's tangent plane
    (Eq. S2 with A, B, C of the target).  For a source on y = 0 the direct and
    the image point both lie on that plane when dz = zx* dx - zy* y*, and
    then S2 = K2 exactly."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        zxt, zyt = rng.uniform(-.6, .6, 2)
        A, B, C = 1 + zxt ** 2, 2 * zxt * zyt, 1 + zyt ** 2
        dx, yt = rng.uniform(-3, 3), rng.uniform(0.1, 2)
        dz = zxt * dx - zyt * yt
        K1, K2, S2 = O.pair_kernels(dx, -yt, yt, dz, 0.0, 0.0, A, B, C)
        assert abs(S2 - K2) < 1e-13 * K2


# ---------------------------------------------------------------- mesh step
def test_trapezoid_exact_for_linear_slope():
    mesh = _mesh(TINY)
    x = mesh.x()
    a, b = 0.3, -0.7
    fx = np.tile(a + b * x, (mesh.M, 1))
    f1 = np.full(mesh.M, 0.25)
    f = O.trapezoid_x(mesh, f1, fx)
    exact = 0.25 + a * (x - x[0]) + 0.5 * b * (x ** 2 - x[0] ** 2)
    assert np.allclose(f, exact[None, :], rtol=0, atol=1e-14)


def test_spline_reproduces_even_cubics_and_is_clamped():
    mesh = _mesh(W.MeshSpec(9, 7, -2.0, 0.5, 0.35))
    y = mesh.y()
    c0, c2, c3 = 0.4, -1.3, 0.8
    f = np.tile((c0 + c2 * y ** 2 + c3 * y ** 3)[:, None], (1, mesh.N))
    fy = O.spline_slope_y(mesh, f)
    assert np.allclose(fy, (2 * c2 * y + 3 * c3 * y ** 2)[:, None], rtol=0, atol=1e-12)
    lin = np.tile(y[:, None], (1, mesh.N))
    assert np.all(O.spline_slope_y(mesh, lin)[0] == 0.0)


def test_spline_equals_full_domain_spline_of_even_extension():
    """R5: the half-domain spline with zero slope at y = 0 and not-a-knot at
    y_M is the full mirrored-domain not-a-knot spline of the even data."""
    mesh = _mesh(W.MeshSpec(5, 8, -1.0, 0.5, 0.25))
    rng = np.random.default_rng(2)
    f = rng.normal(size=(mesh.M, mesh.N))
    y = mesh.y()
    yf = np.concatenate([-y[:0:-1], y])
    ff = np.concatenate([f[:0:-1], f], axis=0)
    full = CubicSpline(yf, ff, axis=0, bc_type="not-a-knot")(yf, 1)[mesh.M - 1:]
    assert np.allclose(O.spline_slope_y(mesh, f), full, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- residual
def test_E1_is_bernoulli_with_kinematic_condition():
    """Eq. freeSurfCond is Eq. NondimDyn after eliminating Phi_z with
    Eq. NondimKin: rebuild (Phi_x, Phi_y, Phi_z) from phi_x = Phi_x + Phi_z zeta_x,
    phi_y = Phi_y + Phi_z zeta_y and the kinematic condition."""
    rng = np.random.default_rng(7)
    F = 0.8
    for _ in range(20):
        px, py, zx, zy, z = rng.uniform(-1, 2), rng.uniform(-1, 1), rng.uniform(-.7, .7), rng.uniform(-.7, .7), rng.uniform(-.3, .3)
        Mx = np.array([[1, 0, zx], [0, 1, zy], [zx, zy, -1.0]])
        V = np.linalg.solve(Mx, [px, py, 0.0])
        ref = 0.5 * V @ V + z / F ** 2 - 0.5
        assert abs(O.free_surface_E1(F, px, py, zx, zy, z) - ref) < 1e-13


@pytest.mark.parametrize("spec", [TINY, SMALL])
def test_flat_state_residual_is_source_term_only(spec):
    """At the flat state (Section 4.1) zeta = 0 and phi = x, so every row
    vanishes except E2 = eps / sqrt(x*^2 + y*^2 + 1) (Eq. IntegroEqn)."""
    mesh = _mesh(spec)
    u0 = O.flat_guess(mesh)
    assert np.all(O.residual(mesh, 0.7, 0.0, u0) == 0.0)
    eps = 0.37
    p = O.residual_parts(mesh, 0.7, eps, u0)
    src = eps / np.sqrt(mesh.x_star()[None, :] ** 2 + mesh.y()[:, None] ** 2 + 1)
    assert np.abs(p["E2"] - src).max() < 1e-15
    for k in ("E1", "E3", "E4", "E5", "E6"):
        assert np.all(p[k] == 0.0)


@pytest.mark.parametrize("spec", [TINY, SMALL])
def test_linear_jacobian_of_appendix_B_equals_fd_jacobian_at_flat_state(spec):
    """At u0 with eps = 0 the nonlinear Jacobian is the linear one: K1
    multiplies g - g* = 0, K2 = S2 = K3 on z = 0, and only the source term
    depends on eps.  The dense matrix built from Eqs. PreA-PreD (Appendix B)
    must therefore equal the central-difference Jacobian of the oracle."""
    mesh = _mesh(spec)
    J_lin = O.jacobian_linear(mesh, 0.7)
    J_fd = O.jacobian_fd(mesh, 0.7, 0.0, O.flat_guess(mesh), h=1e-5)
    assert np.abs(J_lin - J_fd).max() < 1e-8 * np.abs(J_lin).max()


def test_banded_linear_jacobian_keeps_only_block_band():
    mesh = _mesh(TINY)
    full = O.jacobian_linear(mesh, 0.7)
    b3 = O.jacobian_linear(mesh, 0.7, b=3)
    H, N1 = (mesh.N + 1) * mesh.M, mesh.N + 1
    for l in range(mesh.M):
        for m in range(mesh.M):
            blk = (slice(H + l * N1, H + (l + 1) * N1), slice(H + m * N1, H + (m + 1) * N1))
            if abs(l - m) <= 1:
                assert np.array_equal(b3[blk], full[blk])
            else:
                assert np.all(b3[blk] == 0.0)
    assert np.array_equal(b3[:H], full[:H]) and np.array_equal(b3[H:, :H], full[H:, :H])


def test_integral_sum_with_images_equals_full_mirrored_mesh():
    """The y-symmetry construction (R1, R2, R6): the half-domain sum with
    image terms equals the sum over the explicit mirrored mesh j = -(M-1)..M-1
    with direct terms only, zeta_y odd and trapezoid weights on the full
    domain."""
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=4, amp=0.15)
    st = O.surface(mesh, u)
    S_half, _ = O.integral_sum(mesh, st)
    N, M = mesh.N, mesh.M
    x, y = mesh.x(), mesh.y()
    jj = np.arange(-(M - 1), M)
    cx = np.ones(N); cx[[0, -1]] = 0.5
    cyf = np.ones(jj.size); cyf[[0, -1]] = 0.5
    far = 1e30   # pushes the image point of the oracle's kernel to infinity
    S_full = np.zeros((M, N - 1))
    for l in range(M):
        for k in range(N - 1):
            xt, yt = mesh.x_star()[k], y[l]
            zt, zxt, zyt, gt = st["zeta_t"][l, k], st["zetax_t"][l, k], st["zetay_t"][l, k], st["g_t"][l, k]
            A, B, C = 1 + zxt ** 2, 2 * zxt * zyt, 1 + zyt ** 2
            acc = 0.0
            for a, j in enumerate(jj):
                r = abs(j)
                sgn = -1.0 if j < 0 else 1.0
                for i in range(N):
                    K1, K2, S2 = O.pair_kernels(x[i] - xt, sgn * y[r] - yt, far, st["zeta"][r, i] - zt,
                                                st["zetax"][r, i], sgn * st["zetay"][r, i], A, B, C)
                    w = mesh.dx * mesh.dy * cx[i] * cyf[a]
                    acc += w * ((st["g"][r, i] - gt) * K1 + st["zetax"][r, i] * K2 - zxt * S2)
            S_full[l, k] = acc
    assert np.abs(S_half - S_full).max() < 1e-12 * np.abs(S_full).max()


# ---------------------------------------------------------------- JVP, solves
def test_fd_jvp_is_first_order():
    """Eq. JvApprox is a first-order difference quotient: halving h halves
    its error against a fourth-order central difference."""
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=8, amp=0.1)
    v = np.random.default_rng(9).normal(size=u.size)
    F, eps = 0.7, 0.3
    E = lambda w: O.residual(mesh, F, eps, w)
    h = 1e-3
    ref = (8 * (E(u + h * v) - E(u - h * v)) - (E(u + 2 * h * v) - E(u - 2 * h * v))) / (12 * h)
    Eu = E(u)
    e1 = np.abs(O.jvp_fd(mesh, F, eps, u, v, Eu, h=2e-4) - ref).max()
    e2 = np.abs(O.jvp_fd(mesh, F, eps, u, v, Eu, h=1e-4) - ref).max()
    assert 1.8 < e1 / e2 < 2.2


def test_exact_jvp_is_the_limit_of_fourth_order_differences():
    """The complex-step J v against fourth-order central differences of the
    real residual: the gap shrinks like h^4 (a factor ~10^4 per decade of h)
    until the differences' own rounding (~eps_mach |E| / h) takes over, so it
    is the derivative, not an approximation with an error of its own."""
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=10, amp=0.1)
    v = np.random.default_rng(11).normal(size=u.size)
    F, eps = 0.7, 0.3
    Jv, scale = O.jvp_exact(mesh, F, eps, u, v)
    E = lambda w: O.residual(mesh, F, eps, w)
    gaps = []
    for h in (1e-2, 1e-3, 1e-4):
        ref = (8 * (E(u + h * v) - E(u - h * v)) - (E(u + 2 * h * v) - E(u - 2 * h * v))) / (12 * h)
        gaps.append(np.abs(Jv - ref).max() / np.abs(Jv).max())
    assert 3e3 < gaps[0] / gaps[1] < 3e4
    assert gaps[2] < gaps[1] / 5 and gaps[2] < 1e-9
    assert np.all(scale >= np.abs(Jv) * (1 - 1e-12))


def test_exact_jvp_at_the_flat_state_is_the_appendix_B_jacobian():
    """At the flat state with eps = 0 the exact Jacobian of E is the linear
    Jacobian written case by case from Eqs. PreA-PreD (Appendix B)."""
    for spec in (TINY, W.MeshSpec(12, 6, -3.0, 0.5, 0.45)):
        mesh = _mesh(spec)
        u0 = O.flat_guess(mesh)
        P = O.jacobian_linear(mesh, 0.8)
        for seed in (12, 13):
            v = np.random.default_rng(seed).normal(size=u0.size)
            Jv, _ = O.jvp_exact(mesh, 0.8, 0.0, u0, v)
            assert np.abs(Jv - P @ v).max() <= 1e-13 * np.abs(P @ v).max()


def test_exact_jvp_is_linear_in_v():
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=14, amp=0.1)
    rng = np.random.default_rng(15)
    v1, v2 = rng.normal(size=u.size), rng.normal(size=u.size)
    J = lambda v: O.jvp_exact(mesh, 0.7, 0.3, u, v)[0]
    a, b = J(v1), J(v2)
    assert np.abs(J(2 * v1 - 3 * v2) - (2 * a - 3 * b)).max() <= 1e-13 * np.abs(a).max()


def test_complex_step_leaves_the_real_residual_unchanged():
    """The oracle's complex path (used only by jvp_exact) evaluated at a real
    point gives the real residual."""
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=16, amp=0.1)
    p = O.residual_parts(mesh, 0.7, 0.3, u.astype(np.complex128))
    Ec = O.order(mesh, p["E1"], p["E2"], p["E3"], p["E4"], p["E5"], p["E6"])
    Er = O.residual(mesh, 0.7, 0.3, u)
    assert np.abs(Ec.imag).max() == 0.0
    assert np.abs(Ec.real - Er).max() <= 1e-13 * max(1.0, np.abs(Er).max())


def test_linear_solution_is_the_weak_source_limit_and_solves_the_linear_system():
    spec = W.MeshSpec(11, 5, -2.5, 0.5, 0.5)
    mesh = _mesh(spec)
    F, eps = 0.7, 0.02
    uL = O.linear_solution(mesh, F, eps)
    u0 = O.flat_guess(mesh)
    J = O.jacobian_linear(mesh, F)
    # the affine model of E about u0 with the linear Jacobian vanishes at u_L
    assert np.abs(O.residual(mesh, F, eps, u0) + J @ (uL - u0)).max() < 1e-13
    # and the nonlinear root is O(eps^2) away from it
    u, _ = O.newton_dense(mesh, F, eps, u0, tol=1e-13)
    assert np.abs(u - uL).max() < 5 * eps ** 2 * max(1.0, np.abs(uL - u0).max() / eps)


def test_resample_onto_the_same_mesh_is_the_identity():
    spec = W.MeshSpec(13, 7, -3.0, 0.5, 0.4)
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=21, amp=0.1)
    assert np.abs(O.resample(mesh, u, mesh) - u).max() <= 1e-14 * np.abs(u).max()


def test_resample_onto_a_sub_mesh_picks_the_node_values():
    """A mesh whose nodes are every other node of the source (same x1) gets
    the source's node values: the trapezoid integral is not resampled, the
    unknowns phi_x, zeta_x are the node values, phi_1, zeta_1 the first column."""
    fine = W.MeshSpec(21, 9, -4.0, 0.25, 0.3)
    coarse = W.MeshSpec(11, 5, -4.0, 0.5, 0.6)
    u = W.random_state(fine, seed=22, amp=0.1)
    mf, mc = _mesh(fine), _mesh(coarse)
    got = O.resample(mf, u, mc)
    p1, px, z1, zx = O.unpack(mf, u)
    ref = O.pack(mc, p1[::2], px[::2, ::2], z1[::2], zx[::2, ::2])
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def test_preconditioned_jacobian_is_the_identity_at_the_linear_limit():
    """At the flat state with eps = 0 the exact Jacobian is the untruncated
    preconditioner, so J P^-1 = I and every eigenvalue is 1."""
    mesh = _mesh(TINY)
    A = O.preconditioned_jacobian(mesh, 0.7, 0.0, O.flat_guess(mesh))
    assert np.abs(A - np.eye(A.shape[0])).max() < 1e-12


def test_truncation_moves_the_spectrum_away_from_1():
    """Block-banded P (b = 1) against the untruncated one at a nonlinear
    state: the eigenvalues of J P^-1 spread further from 1."""
    spec = W.MeshSpec(9, 7, -2.0, 0.5, 0.4)
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=23, amp=0.05)
    full = np.abs(np.linalg.eigvals(O.preconditioned_jacobian(mesh, 0.7, 0.2, u)) - 1).max()
    band = np.abs(np.linalg.eigvals(O.preconditioned_jacobian(mesh, 0.7, 0.2, u, 1)) - 1).max()
    assert band > full


def test_pressure_forcing_flat_state_residual_is_the_pressure_only():
    """Pressure forcing: at the flat state every row vanishes except E1, which
    is eps p(x*, y*) (the source term is absent from E2)."""
    spec = W.MeshSpec(15, 7, -2.0, 0.3, 0.3)
    mesh = _mesh(spec)
    eps = 0.3
    p = O.residual_parts(mesh, 0.7, eps, O.flat_guess(mesh), forcing="pressure")
    xt, yt = mesh.x_star()[None, :], mesh.y()[:, None]
    assert np.abs(p["E1"] - eps * O.pressure(xt, yt)).max() < 1e-15
    assert np.abs(p["E2"]).max() < 1e-15
    for k in ("E3", "E4", "E5", "E6"):
        assert np.abs(p[k]).max() < 1e-15
    # the bump is nonzero only inside the unit square around the origin
    assert np.count_nonzero(p["E1"]) == np.count_nonzero((np.abs(xt) < 1) & (np.abs(yt) < 1) & (p["E1"] == p["E1"]))


def test_pressure_forcing_weak_limit_is_the_linear_solution():
    """As eps -> 0 the root under an applied pressure approaches the linear
    one, u_L = u0 - J_lin^-1 E(u0): the difference is O(eps^2)."""
    spec = W.MeshSpec(13, 5, -2.5, 0.4, 0.4)
    mesh = _mesh(spec)
    u0 = O.flat_guess(mesh)
    errs = []
    for eps in (0.04, 0.02, 0.01):
        u, _ = O.newton_dense(mesh, 0.7, eps, u0, tol=1e-13, forcing="pressure")
        uL = O.linear_solution(mesh, 0.7, eps, forcing="pressure")
        errs.append(np.abs(u - uL).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_pressure_forcing_jacobian_differs_from_source_only_by_the_source_term():
    """The two forcings give the same Jacobian up to the derivative of the
    source term eps / r with respect to zeta* (complex step, exact)."""
    spec = TINY
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=24, amp=0.1)
    v = np.random.default_rng(25).normal(size=u.size)
    Js, _ = O.jvp_exact(mesh, 0.7, 0.3, u, v)
    Jp, _ = O.jvp_exact(mesh, 0.7, 0.3, u, v, forcing="pressure")
    st = O.surface(mesh, u)
    dst = O.surface(mesh, v + 0 * u)     # the tangent of zeta* is the surface map of v without constants
    xt, yt = mesh.x_star()[None, :], mesh.y()[:, None]
    r2 = xt ** 2 + yt ** 2 + (st["zeta_t"] + 1) ** 2
    # zeta is linear in u with no constant, so surface(v)["zeta_t"] is the tangent of zeta*
    dsrc = -0.3 * (st["zeta_t"] + 1) * dst["zeta_t"] / r2 ** 1.5
    z = np.zeros_like(dsrc)
    diff = O.order(mesh, z, dsrc, z[:, 0], z[:, 0], z[:, 0], z[:, 0])
    assert np.abs((Js - Jp) - diff).max() <= 1e-13 * np.abs(Js).max()


def test_dense_newton_and_newton_gmres_reach_the_same_root():
    spec = TINY
    mesh = _mesh(spec)
    u0 = O.flat_guess(mesh)
    ua, _ = O.newton_dense(mesh, 0.7, 0.1, u0, tol=1e-11)
    ub, _ = O.newton_gmres(mesh, 0.7, 0.1, u0, tol=1e-11, eta=1e-8)
    assert np.abs(ua - ub).max() < 1e-8
    assert np.abs(O.residual(mesh, 0.7, 0.1, ub)).max() < 1e-11


def test_weak_source_limit_is_the_linear_solution():
    """Section 2.3: as eps -> 0 the nonlinear root approaches the linear one,
    u_L = u0 - J_lin^{-1} E(u0), with an O(eps^2) difference."""
    spec = W.MeshSpec(11, 5, -2.5, 0.5, 0.5)
    mesh = _mesh(spec)
    F = 0.7
    u0 = O.flat_guess(mesh)
    J = O.jacobian_linear(mesh, F)
    errs = []
    for eps in (0.04, 0.02, 0.01):
        u, _ = O.newton_dense(mesh, F, eps, u0, tol=1e-13)
        uL = u0 - np.linalg.solve(J, O.residual(mesh, F, eps, u0))
        errs.append(np.abs(u - uL).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_converged_crest_below_limiting_height():
    """The highest crest stays below the limiting height F^2/2 (Section 6)."""
    spec = TINY
    mesh = _mesh(spec)
    F = 0.7
    u, _ = O.newton_gmres(mesh, F, 0.3, O.flat_guess(mesh), tol=1e-10, eta=1e-6)
    zeta, _ = O.zeta_phi(mesh, u)
    assert zeta.max() < F ** 2 / 2


def test_oracle_matches_its_stored_regression_values():
    """Guards the oracle against unintended change: the stored values were
    written by tests/golden/make_golden.py from the oracle alone."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_residual_9x5.txt")
    ref = np.loadtxt(path)
    mesh = _mesh(TINY)
    E = O.residual(mesh, 0.7, 0.3, W.random_state(TINY, seed=4, amp=0.15))
    assert np.abs(E - ref).max() < 1e-13 * max(1.0, np.abs(ref).max())


def test_integrating_phi_minus_x_equals_integrating_phi():
    """Eq. zetaapprox integrates the constant 1 exactly, so the oracle's g =
    phi - x (integrated from phi_x - 1) equals trapezoid(phi_x) - x up to
    rounding of the O(|x|) values."""
    spec = W.MeshSpec(61, 7, -16.0, 0.6, 0.5)
    mesh = _mesh(spec)
    u = W.random_state(spec, seed=13, amp=0.2)
    st = O.surface(mesh, u)
    phi1, phix, _, _ = O.unpack(mesh, u)
    phi = O.trapezoid_x(mesh, phi1, phix)
    assert np.abs((phi - mesh.x()[None, :]) - st["g"]).max() < 64 * np.finfo(float).eps * 20.0 * spec.N
