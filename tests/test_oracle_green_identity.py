"""Pin of the double-layer term of E2 by Green's second identity.

The term in question is the integral of (phi - phi* - x + x*) K1 in
Eq. IntegroEqn (Section 2.2), discretised in Section 3 as the trapezoidal sum
of w (g - g*) K1 with g = phi - x.  Its sign and its coefficient are fixed
here by a theorem rather than by the oracle's own formula:

For a function Psi harmonic in the fluid z < zeta(x, y), even in y and
decaying at infinity, and a point P* on the surface, Green's second identity
over the fluid (the hemisphere at infinity contributes -2 pi Psi(P*) through
the subtracted Psi*) gives

    2 pi Psi(P*) = int_plane [ (Psi - Psi*) N.(Q - P*) / |Q - P*|^3
                               + (N . grad Psi) / |Q - P*| ] dx dy,

with Q = (x, y, zeta) and N = (-zeta_x, -zeta_y, 1) the unnormalised upward
normal (N dx dy = n dS).  The paper's equation is this identity for
Psi = Phi - x with the kinematic condition N . grad Psi = zeta_x substituted
and the source singularity added.

The test builds a state that is NOT a solution: a smooth non-flat surface
(a Gaussian bump) and Psi from a point singularity above it.  It feeds
phi = x + Psi(x, y, zeta) and zeta through the oracle's E2 with eps = 0,
then adds, computed here by adaptive polar quadrature, what the kinematic
condition would have removed (the integral of (zeta_x - N . grad Psi) / r over
the mirrored rectangle) and subtracts the identity's integrand over the plane
outside the rectangle.  What is left is the discretisation error of the
oracle alone, so it must fall at the trapezoidal rate O(dx^2) under
refinement.  A sign error in the double-layer term, or phi - phi* read for
g - g*, leaves an O(0.1) remainder that does not converge.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

# the manufactured surface (even in y) and the exterior singularity above it
_A, _XC, _SX, _SY = 0.25, 0.3, 1.0, 0.8
_Q, _X0, _Z0 = 0.6, -0.5, 1.2


def _zeta(x, y):
    return _A * np.exp(-((x - _XC) / _SX) ** 2 - (y / _SY) ** 2)


def _zeta_x(x, y):
    return _zeta(x, y) * (-2.0 * (x - _XC) / _SX ** 2)


def _zeta_y(x, y):
    return _zeta(x, y) * (-2.0 * y / _SY ** 2)


def _psi(x, y, z):
    """Potential of a point singularity at (x0, 0, z0), z0 > max zeta:
    harmonic everywhere in the fluid, even in y, O(1/R) at infinity."""
    return _Q / np.sqrt((x - _X0) ** 2 + y ** 2 + (z - _Z0) ** 2)


def _grad_psi(x, y, z):
    R3 = ((x - _X0) ** 2 + y ** 2 + (z - _Z0) ** 2) ** 1.5
    return -_Q * (x - _X0) / R3, -_Q * y / R3, -_Q * (z - _Z0) / R3


def _psi_s(x, y):
    """Psi on the surface, i.e. g = phi - x of the manufactured state."""
    return _psi(x, y, _zeta(x, y))


def _phi_x(x, y):
    """d/dx of phi(x, y) = x + Psi(x, y, zeta(x, y))."""
    px, _, pz = _grad_psi(x, y, _zeta(x, y))
    return 1.0 + px + pz * _zeta_x(x, y)


def _psi_n(x, y):
    """N . grad Psi on the surface, N = (-zeta_x, -zeta_y, 1)."""
    px, py, pz = _grad_psi(x, y, _zeta(x, y))
    return pz - px * _zeta_x(x, y) - py * _zeta_y(x, y)


def _state(mesh):
    """The unknowns of Eq. unknowns for the manufactured surface and phi."""
    X, Y = np.meshgrid(mesh.x(), mesh.y())
    y = mesh.y()
    return O.pack(mesh, mesh.x1 + _psi_s(mesh.x1, y), _phi_x(X, Y), _zeta(mesh.x1, y), _zeta_x(X, Y))


def _polar(f, xt, yt, box, inside):
    """Integral of f(x, y) over the rectangle box = (X1, X2, Y1, Y2)
    (inside=True) or over the plane outside it (inside=False), in polar
    coordinates about (xt, yt), which lies inside the box: the area element
    r dr cancels an integrable 1/r at the centre, and the angular
    integral is split at the corner directions."""
    X1, X2, Y1, Y2 = box
    corners = [(X2, Y2), (X1, Y2), (X1, Y1), (X2, Y1)]
    angs = sorted(math.atan2(cy - yt, cx - xt) % (2 * math.pi) for cx, cy in corners)

    def edge(th):
        c, s = math.cos(th), math.sin(th)
        r = math.inf
        if c > 0:
            r = min(r, (X2 - xt) / c)
        if c < 0:
            r = min(r, (X1 - xt) / c)
        if s > 0:
            r = min(r, (Y2 - yt) / s)
        if s < 0:
            r = min(r, (Y1 - yt) / s)
        return r

    def radial(th):
        c, s = math.cos(th), math.sin(th)
        h = lambda r: f(xt + r * c, yt + r * s) * r
        lo, hi = (0.0, edge(th)) if inside else (edge(th), math.inf)
        return integrate.quad(h, lo, hi, epsabs=1e-13, epsrel=1e-12, limit=200)[0]

    bps = angs + [angs[0] + 2 * math.pi]
    return sum(integrate.quad(radial, lo, hi, epsabs=1e-12, epsrel=1e-11, limit=200)[0]
               for lo, hi in zip(bps[:-1], bps[1:]))


def _identity_pieces(xt, yt, box):
    """For a surface point above (xt, yt): the kinematic correction
    int_box (zeta_x - N . grad Psi) / r, the identity's integrand over the
    plane outside the box, and the double-layer part inside the box alone
    (its size, to show the test is sensitive to it).  box is the mirrored
    rectangle [x1, xN] x [-yM, yM]: with Psi and zeta even in y, the image
    terms of the half domain are the mirrored half."""
    zt = _zeta(xt, yt)
    pt = _psi(xt, yt, zt)

    def double_layer(x, y):
        dx, dy, dz = x - xt, y - yt, _zeta(x, y) - zt
        n_dot = -_zeta_x(x, y) * dx - _zeta_y(x, y) * dy + dz
        return (_psi_s(x, y) - pt) * n_dot / (dx * dx + dy * dy + dz * dz) ** 1.5

    def inv_r(x, y):
        dx, dy, dz = x - xt, y - yt, _zeta(x, y) - zt
        return 1.0 / math.sqrt(dx * dx + dy * dy + dz * dz)

    kin = _polar(lambda x, y: (_zeta_x(x, y) - _psi_n(x, y)) * inv_r(x, y), xt, yt, box, True)
    out = _polar(lambda x, y: double_layer(x, y) + _psi_n(x, y) * inv_r(x, y), xt, yt, box, False)
    dl_in = _polar(double_layer, xt, yt, box, True)
    return kin, out, dl_in


X1, X2, YM = -4.0, 4.0, 4.0
D0 = 0.4
# half-mesh targets of the coarsest mesh; refining by 3 keeps every one of
# them a half-mesh target (x1 + (k + 1/2) dx -> index 3k + 1)
TARGETS = [(0.2, 0.4), (1.0, 0.0), (-1.0, 0.8), (0.6, 1.2), (-2.2, 2.0)]


def _mesh(d):
    return O.Mesh(int(round((X2 - X1) / d)) + 1, int(round(YM / d)) + 1, X1, d, d)


def _target_index(mesh, xt, yt):
    k = int(round((xt - mesh.x1) / mesh.dx - 0.5))
    l = int(round(yt / mesh.dy))
    assert abs(mesh.x1 + (k + 0.5) * mesh.dx - xt) < 1e-12 and abs(l * mesh.dy - yt) < 1e-12
    return l * (mesh.N - 1) + k


@pytest.fixture(scope="module")
def pieces():
    box = (X1, X2, -YM, YM)
    return [_identity_pieces(xt, yt, box) for xt, yt in TARGETS]


@pytest.fixture(scope="module")
def remainders(pieces):
    """Green's-identity remainder per target on meshes dx = 0.4, 0.4/3, 0.4/9."""
    rows = []
    for d in (D0, D0 / 3, D0 / 9):
        mesh = _mesh(d)
        idx = [_target_index(mesh, xt, yt) for xt, yt in TARGETS]
        E2, _ = O.residual_E2_at(mesh, 0.7, 0.0, _state(mesh), idx)
        rows.append([E2[i] + kin - out for i, (kin, out, _) in enumerate(pieces)])
    return np.array(rows)


def test_green_identity_remainder_falls_at_the_trapezoid_rate(remainders):
    """E2 of the oracle plus the kinematic correction minus the outside part
    is the identity's discretisation error: it falls ~9x per 3x refinement
    (O(dx^2)), and its Richardson extrapolation is ~0."""
    r0, r1, r2 = np.abs(remainders)
    assert np.all(r1 <= r0 / 6) and np.all(r2 <= r1 / 6), remainders
    assert np.all(r2 < 1e-3), remainders
    extrap = remainders[2] - (remainders[1] - remainders[2]) / 8.0
    assert np.all(np.abs(extrap) < 1e-4), extrap


def test_green_identity_is_sensitive_to_the_double_layer_term(pieces, remainders):
    """The double-layer part at the targets on the bump is two to three
    orders larger than the finest remainder, so a sign error or a missing
    -x + x* in its coefficient cannot pass the test above."""
    dl = np.array([p[2] for p in pieces])
    strong = np.abs(dl) > 0.03
    assert strong.sum() >= 3, dl
    assert np.all(np.abs(remainders[2][strong]) < 0.01 * np.abs(dl[strong])), (remainders[2], dl)


def test_sampled_E2_equals_the_full_residual_rows():
    """The sampled E2 used above is the E2 block of the full residual
    (Appendix A order), so the identity pins the full residual too."""
    for d in (D0, D0 / 3):
        mesh = _mesh(d)
        u = _state(mesh)
        idx = [_target_index(mesh, xt, yt) for xt, yt in TARGETS]
        E2s, _ = O.residual_E2_at(mesh, 0.7, 0.0, u, idx)
        E = O.residual(mesh, 0.7, 0.0, u)
        H = (mesh.N + 1) * mesh.M
        rows = [H + (t // (mesh.N - 1)) * (mesh.N + 1) + 2 + t % (mesh.N - 1) for t in idx]
        assert np.allclose(E[rows], E2s, rtol=0, atol=1e-13), (E[rows], E2s)
