"""Axis lengths with a factor 5 (radix-5 butterflies and the composite radices
6 and 10 of the transform engine): the grids of the paper's Section 5
(Example 1's N = 2400 / 3600 / 4800, Table 2's N = 120 ... 1920, Table 1's
N = 180 ... 2880).  Parity against the oracle element by element at small
and ragged shapes in 2D and 3D, every launch shape, the full 2400^2 Example 1
apply, 4800-long rows and 1920-long columns, and Example 1's GMRES(10)
residual history at N = 240 against the oracle's GMRES step by step."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel, within

pytestmark = pytest.mark.gpu

SHAPES = [(20, 40), (60, 120), (40, 180), (240, 60), (16, 360), (12, 480), (24, 720), (8, 960),
          (8, 1440), (1920, 8), (8, 2400), (8, 2880), (3600, 8), (12, 4800), (20, 40, 60),
          (40, 24, 120), (60, 20, 16)]


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("shape", SHAPES)
def test_apply_both_precisions(hz, shape):
    p = S.small_problem(shape, 71, M=5, Mt=3, width=2)
    med_g, med_o = media(hz, p)
    v = S.random_field(np.random.Generator(np.random.PCG64(72)), shape, 2)
    ref = np.stack([O.apply_preconditioner(med_o, v[b]) for b in range(2)])
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, max_nrhs=2)
        got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
        e = rel(got, ref)
        assert within(e, prec, "radix5"), (shape, prec, e)
        if prec == 0:  # element by element as well
            assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(60, 120), (40, 24, 120), (24, 720)])
def test_every_launch_shape(hz, shape):
    p = S.small_problem(shape, 73, M=6, Mt=3, width=2)
    med_g, med_o = media(hz, p)
    v = S.random_field(np.random.Generator(np.random.PCG64(74)), shape, 2)
    ref = np.stack([O.apply_preconditioner(med_o, v[b]) for b in range(2)])
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, max_nrhs=2)
        for kpb, mode, pair in ((1, 1, 1), (1, 2, 0), (2, 2, 1), (4, 1, 0), (4, 2, 2),
                                (1, 0, 0), (1, 3, 1), (2, 3, 2), (4, 3, 0)):
            plan.set_tune(syminv_kpb=kpb, rowinv_mode=mode, col_pair=pair)
            got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
            e = rel(got, ref)
            assert within(e, prec, "radix5"), (prec, kpb, mode, pair, e)


def test_operator_and_small_solve(hz):
    """The operator on a factor-5 grid, and an FGMRES solve whose true
    residual the oracle's operator confirms."""
    p = S.small_problem((60, 120), 75, M=5, Mt=3, width=3)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1, restart=30, tol=1e-8, maxit=3000)
    v = S.random_field(np.random.Generator(np.random.PCG64(76)), p.shape)
    assert rel(plan.apply_operator(_dev(v)).cpu().numpy(), O.apply_operator(med_o, v)) <= 1e-12
    u, st = plan.solve(_dev(p.f[0]))
    r = rel(O.apply_operator(med_o, u.cpu().numpy()), p.f[0])
    assert st[0]["converged"] and r <= 1e-8, (st, r)


def test_example1_2400_apply_full_size(hz):
    """Example 1 at the paper's N = 2400 (M = 8, a = 20, PPW 12): the whole
    apply against the oracle in FP64 (element by element) and complex64,
    through autotuned plans."""
    p = S.example1(2400)
    med_o = O.make_medium(p.c, p.zeta, p.a, p.omega, p.M, 0, 1.0, None, 0.0, p.meta["a_node"])
    med_g = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=p.M, Mt=0, c_o=1.0, alpha=0.0,
                      a_node=p.meta["a_node"])
    v = S.random_field(np.random.Generator(np.random.PCG64(77)), p.shape)
    ref = O.apply_preconditioner(med_o, v, workers=8)
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, restart=10)
        plan.autotune()
        got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
        e = rel(got, ref)
        assert within(e, prec, "radix5"), (prec, e)
        if prec == 0:
            assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("no_precond", [False, True])
def test_example1_history_at_240(hz, no_precond):
    """Example 1's GMRES(10) at N = 240 (2^4 3 5, one of Table 2's grids):
    the per-step residual history against the oracle's GMRES."""
    p = S.example1(240)
    med_o = O.make_medium(p.c, p.zeta, p.a, p.omega, p.M, 0, 1.0, None, 0.0, p.meta["a_node"])
    med_g = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=p.M, Mt=0, c_o=1.0, alpha=0.0,
                      a_node=p.meta["a_node"])
    plan = hz.Plan(med_g, precision=0, restart=10, tol=1e-14, maxit=30, no_precond=no_precond)
    u, st, H = plan.solve(np.ascontiguousarray(p.f[0]), history=30)
    A = lambda x: O.apply_operator(med_o, x)
    Q = None if no_precond else (lambda x: O.apply_preconditioner(med_o, x))
    _, so = O.gmres(A, p.f[0], Q, restart=10, tol=1e-14, maxit=30, record_history=True)
    ho = np.asarray(so["history"])
    # the first two cycles step by step (rounding is amplified after that,
    # as at the power-of-two sizes)
    np.testing.assert_allclose(H[0][:20], ho[:20], rtol=1e-6)
    if not no_precond:
        assert math.log10(ho[0] / ho[29]) > 1.0
