"""Writes the oracle's converged roots under tests/golden/.  Calls only the
oracle and the seeded input generators; run from the repository root:

    python tests/golden/make_roots.py [181x61] [121x41]

Each root is the oracle's damped inexact Newton iteration with
right-preconditioned GMRES (Section 4.1; the preconditioner is the
untruncated linear Jacobian of Appendix B, factored densely) from the flat
initial guess, stopped at ||E||_inf < 1e-11.  The files hold zeta (and phi)
at every mesh node (Eq. zetaapprox applied to the root's unknowns), row by
row in y, x fastest, to 13 significant digits: the values the GPU solves are
compared with.

  oracle_root_181x61.txt       the 181x61 workload: x in [-16, 20], y in [0, 12],
                               F = 0.7, eps = 0.4; zeta and phi
  oracle_root_121x41_batch.txt instances 0 and 63 of the 64-instance 121x41
                               batch (F, eps from workloads.batch_params); zeta
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1403_5044_b300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-11
BATCH_SAMPLE = (0, 63)


def _mesh(spec):
    return O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)


def root(spec, F, eps):
    mesh = _mesh(spec)
    t0 = time.time()
    u, its = O.newton_gmres(mesh, F, eps, O.flat_guess(mesh), tol=TOL, eta=1e-8, b=None)
    E = O.residual(mesh, F, eps, u)
    zeta, phi = O.zeta_phi(mesh, u)
    return zeta, phi, its, float(np.abs(E).max()), time.time() - t0


def _write_block(f, spec, F, eps, zeta, phi, its, einf, secs, label):
    """phi=None writes zeta alone."""
    f.write("# instance %s: mesh %dx%d x1=%r dx=%r dy=%r n=%r F=%r eps=%r\n"
            % (label, spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad, F, eps))
    f.write("# newton_iterations=%d final_norm_inf=%.3e oracle_seconds=%.1f\n" % (its, einf, secs))
    if phi is None:
        for z in zeta.ravel():
            f.write("%.12e\n" % z)
    else:
        for z, p in zip(zeta.ravel(), phi.ravel()):
            f.write("%.12e %.12e\n" % (z, p))


def make_181x61():
    spec, F, eps = W.SOLVE_181x61
    zeta, phi, its, einf, secs = root(spec, F, eps)
    with open(os.path.join(HERE, "oracle_root_181x61.txt"), "w") as f:
        f.write("# oracle root (zeta phi per node, [M][N] row-major) of the 181x61 solve, flat start\n")
        f.write("# written by tests/golden/make_roots.py from the oracle only; stop ||E||_inf < %.0e\n" % TOL)
        _write_block(f, spec, F, eps, zeta, phi, its, einf, secs, "0")
    print("181x61: %d Newton steps, ||E||_inf %.2e, %.0f s" % (its, einf, secs))


def make_121x41_batch():
    spec = W.MESH_121x41
    params = W.batch_params()
    with open(os.path.join(HERE, "oracle_root_121x41_batch.txt"), "w") as f:
        f.write("# oracle roots (zeta per node, [M][N] row-major) of sampled instances of the\n")
        f.write("# 64 x 121x41 batch (workloads.batch_params()), flat start\n")
        f.write("# written by tests/golden/make_roots.py from the oracle only; stop ||E||_inf < %.0e\n" % TOL)
        for i in BATCH_SAMPLE:
            F, eps = params[i]
            zeta, phi, its, einf, secs = root(spec, F, eps)
            _write_block(f, spec, F, eps, zeta, None, its, einf, secs, str(i))
            print("121x41 #%d: %d Newton steps, ||E||_inf %.2e, %.0f s" % (i, its, einf, secs))


def load(path):
    """Blocks of a root file: list of (header dict, zeta [M][N], phi [M][N]
    or None)."""
    blocks, cur = [], None
    with open(path) as f:
        for line in f:
            if line.startswith("# instance"):
                kv = dict(t.split("=") for t in line.split(":", 1)[1].split()[2:])
                nm = line.split(":", 1)[1].split()[1]
                N, M = (int(v) for v in nm.split("x"))
                cur = {"label": line.split()[2].rstrip(":"), "N": N, "M": M,
                       **{k: float(v) for k, v in kv.items()}, "rows": []}
                blocks.append(cur)
            elif line.startswith("# newton_iterations") and cur is not None:
                cur.update({k: float(v) for k, v in (t.split("=") for t in line[2:].split())})
            elif line.startswith("#"):
                continue
            else:
                cur["rows"].append([float(v) for v in line.split()])
    out = []
    for b in blocks:
        a = np.array(b.pop("rows"))
        a = a.reshape(b["M"] * b["N"], -1)
        out.append((b, a[:, 0].reshape(b["M"], b["N"]),
                    a[:, 1].reshape(b["M"], b["N"]) if a.shape[1] > 1 else None))
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["181x61", "121x41"]
    if "121x41" in which:
        make_121x41_batch()
    if "181x61" in which:
        make_181x61()
