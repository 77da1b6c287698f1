"""Spectral diagnostics of the preconditioned Jacobian J P^-1 (Section 4.2:
the preconditioner should cluster its eigenvalues; the paper's Figs. 2-3
show them for several block bandwidths b).

The library forms J(u) P^-1 on the GPU column by column
(swj_preconditioned_jacobian: a preconditioner apply of e_j, then the exact
Jacobian-vector product); this module only takes its eigenvalues on the host
(numpy) and summarises how tightly they cluster around 1.  Meant for small
meshes: the matrix is (2(N+1)M)^2 doubles."""
import numpy as np

from . import swj


def preconditioned_jacobian(ctx, u, precision=swj.FP64):
    """The dense J(u) P^-1 of a single-instance context, as a numpy array."""
    import torch
    n = ctx.n_unknowns
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    ctx.preconditioned_jacobian(u, out, 0, n, precision)
    # column-major on the device: row r, column c at c * n + r
    return out.view(n, n).t().cpu().numpy()


def clustering(eigs, radius=0.5):
    """Summary of a spectrum against the ideal J P^-1 = I: the largest
    distance from 1, the fraction within `radius` of 1, and the ratio of the
    largest to the smallest modulus."""
    eigs = np.asarray(eigs)
    d = np.abs(eigs - 1.0)
    mod = np.abs(eigs)
    return {"n": int(eigs.size), "max_dist_from_1": float(d.max()), "median_dist_from_1": float(np.median(d)),
            "frac_within_%g" % radius: float(np.mean(d < radius)),
            "modulus_ratio": float(mod.max() / mod.min()) if mod.min() > 0 else float("inf")}


def spectrum(ctx, u, precision=swj.FP64):
    """Eigenvalues of J(u) P^-1 and their clustering summary."""
    eigs = np.linalg.eigvals(preconditioned_jacobian(ctx, u, precision))
    return eigs, clustering(eigs)
