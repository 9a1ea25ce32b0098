"""Edge and degenerate cases through the C ABI: empty input, the smallest
and the longest axes, a constant medium (one node: the Fourier multiplier
Q_1 of Eqn. OneInterpPoint), the case where Q_M is exactly P_N^{-1}
(discrete symbol, a > 0, no regularisation: one GMRES step), and media that
take node values only."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel, within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _apply_both(hz, med_g, med_o, shape, seed):
    v = S.random_field(np.random.Generator(np.random.PCG64(seed)), shape)
    ref = O.apply_preconditioner(med_o, v)
    plan = hz.Plan(med_g, precision=1)
    for prec in (0, 1):
        got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
        assert within(rel(got, ref), prec, "small"), (shape, prec, rel(got, ref))


def test_empty_input_is_refused(hz):
    import torch
    p = S.small_problem((16, 16), 3, M=4, Mt=2, width=2)
    med, _ = media(hz, p, oracle=False)
    plan = hz.Plan(med, precision=1)
    x = _dev(np.zeros((1, 16, 16), complex))
    y = torch.zeros_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for fn in (hz.lib.hz_apply_preconditioner,):
        st = fn(plan._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 0, 1, s)
        assert st == 1  # HZ_ERR_INVALID_ARG, nothing launched
    for prec in (0, 1):
        assert hz.lib.hz_apply_operator(plan._h, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), 0, prec, s) == 1
    torch.cuda.synchronize()
    assert torch.count_nonzero(y) == 0


@pytest.mark.parametrize("shape", [(8, 8), (8, 8, 8), (1024, 8, 8), (8, 1024), (2048, 8)])
def test_smallest_and_longest_axes(hz, shape):
    p = S.small_problem(shape, 41, M=3, Mt=0, width=0)
    med_g, med_o = media(hz, p)
    _apply_both(hz, med_g, med_o, shape, 42)


def test_constant_medium_is_one_node_fourier_multiplier(hz):
    """c constant, no layer: every requested node collapses to one and Q_M is
    the multiplier 1 / (w^2 + i w a_1 - c^2 |xi|^2) of Eqn. 021."""
    shape = (32, 48)
    c = np.full(shape, 1.3)
    omega = 2 * np.pi * 32 / (6 * 1.3)
    med_g = hz.Medium(c, None, None, omega=omega, M=6, Mt=0, c_o=1.3, alpha=0.2)
    med_o = O.make_medium(c, None, None, omega, 6, 0, 1.3, None, 0.2)
    assert med_g.info()["K"] == 1 == med_o.nodes.K
    v = S.random_field(np.random.Generator(np.random.PCG64(5)), shape)
    xi2 = O.xi2_grid(shape, 1.0)
    closed = np.fft.ifftn(np.fft.fftn(v) / (omega ** 2 + 1j * omega * 0.2 * omega - 1.69 * xi2))
    plan = hz.Plan(med_g, precision=1)
    for prec in (0, 1):
        got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
        assert within(rel(got, closed), prec, "closed_const"), (prec, rel(got, closed))


def test_exact_inverse_converges_in_one_step(hz):
    """Constant c, constant a > 0, the finite-difference symbol and alpha = 0:
    Q_M = P_N^{-1} exactly, so (F)GMRES stops after one Arnoldi step."""
    shape = (64, 64)
    c = np.full(shape, 1.0)
    a = np.full(shape, 7.0)
    omega = 2 * np.pi * 64 / 8
    med_g = hz.Medium(c, None, a, omega=omega, M=4, Mt=0, c_o=1.0, alpha=0.0, a_node=7.0,
                      symbol_kind=1)
    med_o = O.make_medium(c, None, a, omega, 4, 0, 1.0, None, 0.0, 7.0, 1)
    f = S.random_field(np.random.Generator(np.random.PCG64(6)), shape)
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, restart=10, tol=1e-6)
        u, st = plan.solve(np.ascontiguousarray(f))
        assert st[0]["converged"] and st[0]["iters"] == 1, st
        assert rel(O.apply_operator(med_o, u), f) <= 1e-6


def test_medium_at_node_values_only(hz):
    """c takes node values only (hat weights 0/1): the apply still matches the
    oracle, which there equals the un-interpolated Op(q) pointwise."""
    shape = (24, 32)
    r = np.random.Generator(np.random.PCG64(7))
    c = r.choice([1.0, 1.25, 1.5, 1.75, 2.0], size=shape)
    c[0, 0], c[0, 1] = 1.0, 2.0
    omega = 2 * np.pi * 24 / 8
    med_g = hz.Medium(c, None, None, omega=omega, M=5, Mt=0, c_o=1.0, alpha=0.15)
    med_o = O.make_medium(c, None, None, omega, 5, 0, 1.0, None, 0.15)
    _apply_both(hz, med_g, med_o, shape, 8)
