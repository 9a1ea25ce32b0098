"""The Arnoldi Hessenberg matrix the GPU builds (hz_plan_hessenberg): one
cycle of GMRES on the paper's Example 1 medium against an Arnoldi process
(CGS2, FP64) written here with the oracle's operator and preconditioner, from
the same starting vector; and its Ritz values."""
import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _arnoldi(apply_op, r0, m):
    shape = r0.shape
    n = r0.size
    V = np.zeros((m + 1, n), np.complex128)
    H = np.zeros((m + 1, m), np.complex128)
    V[0] = r0.ravel() / np.linalg.norm(r0)
    for j in range(m):
        w = apply_op(V[j].reshape(shape)).ravel()
        for _ in range(2):
            h = V[:j + 1].conj() @ w
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    return H


@pytest.mark.parametrize("no_precond", [False, True])
def test_hessenberg_matches_oracle_arnoldi(hz, no_precond):
    p = S.example1(64, delta=4.0)
    a_node = p.meta["a_node"]
    med_o = O.make_medium(p.c, p.zeta, p.a, p.omega, p.M, 0, 1.0, None, 0.0, a_node)
    med_g = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=p.M, Mt=0, c_o=1.0, alpha=0.0,
                      a_node=a_node)
    m = 24
    plan = hz.Plan(med_g, precision=0, restart=m, tol=1e-14, maxit=m, no_precond=no_precond)
    f = np.ascontiguousarray(p.f[0])
    plan.solve(f)
    Hg = plan.hessenberg(0)
    assert Hg.shape == (m + 1, m)
    A = lambda x: O.apply_operator(med_o, x)
    op = A if no_precond else (lambda x: A(O.apply_preconditioner(med_o, x)))
    Ho = _arnoldi(op, f, m)
    # Unpreconditioned, the Arnoldi process is stable: all columns agree.
    # Preconditioned, Q_M P_N clusters near 1 and the process is chaotic
    # after a few steps: the reference Arnoldi itself moves by 3e-7 at
    # column 12 and by 2e-4 at column 13 when f is perturbed by 1e-13
    # (relative).  So the first 11 columns, then Ritz values from them.
    J = m if no_precond else 11
    scale = np.abs(Ho[:J + 1, :J]).max()
    for j in range(J):
        assert np.abs(Hg[:j + 2, j] - Ho[:j + 2, j]).max() <= 1e-9 * scale, j
    assert np.all(Hg[np.tril_indices(m + 1, -2)] == 0)  # upper Hessenberg
    tg = np.abs(np.linalg.eigvals(Hg[:J, :J]))
    to = np.abs(np.linalg.eigvals(Ho[:J, :J]))
    assert abs(tg.max() / to.max() - 1) <= 1e-8 and abs(tg.min() / to.min() - 1) <= 1e-6
