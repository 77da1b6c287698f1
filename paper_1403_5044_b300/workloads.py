"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module holds no arithmetic of the method: it only names the meshes and
parameters of the workloads and draws seeded random states in the layout of
the unknown vector u (Section 3, Eq. unknowns:
u = [phi_1, (phi_x)_1..N] per y-row, then [zeta_1, (zeta_x)_1..N] per y-row).

Mesh recipe.  The paper's meshes are regular with dx = dy and y1 = 0.  The
workloads below place them on the domains x in [x1, xN], y in [0, yM]:
  41x21   on [-10, 10] x [0, 8]   (dx = 0.5, dy = 0.4)
  181x61  on [-16, 20] x [0, 12]  (dx = dy = 0.2)
  721x241 on [-16, 20] x [0, 12]  (dx = dy = 0.05)
  121x41, 61x21, 361x121 on the same [-16, 20] x [0, 12] (dx = 0.3, 0.6, 0.1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class MeshSpec:
    N: int
    M: int
    x1: float
    dx: float
    dy: float
    n_rad: float = 0.05

    @property
    def n_unknowns(self) -> int:
        return 2 * (self.N + 1) * self.M

    @property
    def pairs(self) -> int:
        """(source, target) pairs of one boundary-integral sum: (N-1)M * NM."""
        return (self.N - 1) * self.M * self.N * self.M


def domain_mesh(N: int, M: int, x1: float = -16.0, xN: float = 20.0, yM: float = 12.0) -> MeshSpec:
    return MeshSpec(N, M, x1, (xN - x1) / (N - 1), yM / (M - 1))


MESH_41x21 = MeshSpec(41, 21, -10.0, 0.5, 0.4)
MESH_181x61 = domain_mesh(181, 61)
MESH_721x241 = domain_mesh(721, 241)
MESH_121x41 = domain_mesh(121, 41)
SERVE_MESHES = [domain_mesh(61, 21), domain_mesh(121, 41), domain_mesh(181, 61), domain_mesh(361, 121)]

# (mesh, F, eps) of the single-instance workloads
SOLVE_41x21 = (MESH_41x21, 0.7, 0.1)
SOLVE_181x61 = (MESH_181x61, 0.7, 0.4)
SOLVE_721x241 = (MESH_721x241, 0.7, 0.8)


def batch_params(count: int = 64, seed: int = 1403_5044, F_range=(0.5, 1.0), eps_range=(0.05, 0.6)):
    """(F, eps) per instance of the batched workload: drawn in the order F then
    eps for each instance from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        F = rng.uniform(*F_range)
        eps = rng.uniform(*eps_range)
        out.append((float(F), float(eps)))
    return out


def serve_requests(count: int = 2000, seed: int = 1403_5045, rate: float = 1.0,
                   F_range=(0.5, 1.0), eps_range=(0.05, 0.5), meshes=None):
    """Poisson arrival stream: list of (arrival_time_s, mesh, F, eps)."""
    rng = np.random.default_rng(seed)
    meshes = SERVE_MESHES if meshes is None else meshes
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        m = meshes[int(rng.integers(len(meshes)))]
        F = float(rng.uniform(*F_range))
        eps = float(rng.uniform(*eps_range))
        out.append((t, m, F, eps))
    return out


def flat_state(mesh: MeshSpec) -> np.ndarray:
    """u of a flat surface with the uniform stream: phi_1 = x1, phi_x = 1,
    zeta_1 = 0, zeta_x = 0 (the input values named in Section 4.1)."""
    N, M = mesh.N, mesh.M
    P = np.zeros((M, N + 1))
    P[:, 0] = mesh.x1
    P[:, 1:] = 1.0
    Z = np.zeros((M, N + 1))
    return np.concatenate([P.ravel(), Z.ravel()])


def random_state(mesh: MeshSpec, seed: int, amp: float = 0.05, modes: int = 6) -> np.ndarray:
    """A seeded smooth random state near the flat one: phi_1, phi_x, zeta_1,
    zeta_x each get a sum of `modes` random plane waves (wavelengths 2..12
    length units, like the transverse and divergent waves of the paper's
    figures) of amplitude ~amp, damped upstream."""
    rng = np.random.default_rng(seed)
    N, M = mesh.N, mesh.M
    x = mesh.x1 + mesh.dx * np.arange(N)
    y = mesh.dy * np.arange(M)
    X, Y = np.meshgrid(x, y)                      # [M, N]

    def field():
        f = np.zeros((M, N))
        for _ in range(modes):
            lam = rng.uniform(2.0, 12.0)
            th = rng.uniform(-np.pi / 2, np.pi / 2)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.normal() * amp / np.sqrt(modes)
            kx, ky = 2 * np.pi / lam * np.cos(th), 2 * np.pi / lam * np.sin(th)
            f += a * np.cos(kx * X + ky * Y + ph)
        return f * (0.5 + 0.5 * np.tanh((X - x[0]) / 3.0 - 1.0))

    P = np.zeros((M, N + 1))
    Z = np.zeros((M, N + 1))
    P[:, 0] = mesh.x1 + field()[:, 0]
    P[:, 1:] = 1.0 + field()
    Z[:, 0] = field()[:, 0]
    Z[:, 1:] = field()
    return np.concatenate([P.ravel(), Z.ravel()])
