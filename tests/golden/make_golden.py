"""Writes the stored oracle values under tests/golden/.  Calls only the
oracle and the seeded input generators; run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1403_5044_b300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    spec = W.MeshSpec(9, 5, -2.0, 0.5, 0.4)
    F, eps, seed, amp = 0.7, 0.3, 4, 0.15
    mesh = O.Mesh(spec.N, spec.M, spec.x1, spec.dx, spec.dy, spec.n_rad)
    u = W.random_state(spec, seed=seed, amp=amp)
    E = O.residual(mesh, F, eps, u)
    with open(os.path.join(HERE, "oracle_residual_9x5.txt"), "w") as f:
        f.write("# oracle E(u) (Appendix A order) on a 9x5 mesh, x1=-2, dx=0.5, dy=0.4, n=0.05\n")
        f.write("# F=%r eps=%r; u = workloads.random_state(seed=%d, amp=%r)\n" % (F, eps, seed, amp))
        f.write("# written by tests/golden/make_golden.py from the oracle only (regression fixture)\n")
        for v in E:
            f.write("%.17e\n" % v)


if __name__ == "__main__":
    main()
