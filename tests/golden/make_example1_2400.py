"""Writes example1_2400_oracle.txt: the oracle's GMRES(10) residual histories
for the paper's Example 1 at its first grid, N = 2400 (Section 5.1: circular
inclusion, delta = 1, eta = 1/800, a = 20, M = 8, PPW = 12), for 100
iterations: the paper's left-preconditioned form with the finite-difference
symbol (the preconditioned residual ||Q_M (f - P_N u)|| / ||Q_M f||), and
GMRES(10) without a preconditioner (||f - P_N u|| / ||f||).  It calls only
the oracle and the seeded input generator; the GPU tests compare the GPU
histories with these values.  Runs for several minutes on a CPU:

    python tests/golden/make_example1_2400.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2409_16172_gb300 import synth as S  # noqa: E402


def main():
    N, its = 2400, 100
    p = S.example1(N)
    med = O.make_medium(p.c, p.zeta, p.a, p.omega, p.M, 0, 1.0, None, 0.0, p.meta["a_node"], 1)
    workers = os.cpu_count() or 1
    A = lambda u: O.apply_operator(med, u)
    Q = lambda v: O.apply_preconditioner(med, v, workers=workers)
    _, left = O.gmres(A, p.f[0], Q, restart=10, tol=1e-14, maxit=its, side="left",
                      record_history=True)
    _, none = O.gmres(A, p.f[0], None, restart=10, tol=1e-14, maxit=its, record_history=True)
    out = os.path.join(HERE, "example1_2400_oracle.txt")
    with open(out, "w") as fh:
        fh.write("# The oracle's GMRES(10) histories for Example 1 (Section 5.1) at N = 2400,\n"
                 "# omega = 400 pi, delta = 1, eta = 1/800, a = 20, M = 8, PPW = 12, written by\n"
                 "# make_example1_2400.py.  columns: iteration  left form with the\n"
                 "# finite-difference symbol (preconditioned residual)  no preconditioner\n")
        for i in range(its):
            fh.write(f"{i + 1} {left['history'][i]:.17e} {none['history'][i]:.17e}\n")
    print(out, np.log10(none["history"][-1] / left["history"][-1]))


if __name__ == "__main__":
    main()
