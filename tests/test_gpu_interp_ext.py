"""GPU parity of the interpolation extensions the paper names in Section 6 —
bivariate interpolation in (c, a) for damping that does not follow the wave
speed, and the quadratic Lagrange and cubic Hermite bases in c — against the
oracle, through the C ABI: node tables, the apply in both precisions with
every x-inverse form, at ragged 2D/3D shapes with a layer, a full-size apply
on sampled points through the plane-wave closed form, and solves checked
with the oracle's own operator."""
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


FORMS = {
    # (problem options, medium options)
    "bivariate": (dict(M=4, Mt=2, damping=(0.05, 0.4)), dict(Ma=3)),
    "bivariate-Ma2": (dict(M=3, Mt=3, damping=(0.0, 0.3)), dict(Ma=2)),
    "lagrange": (dict(M=5, Mt=2), dict(basis=1)),
    "lagrange-M7": (dict(M=7, Mt=3, contrast=0.9), dict(basis=1)),
    "hermite": (dict(M=4, Mt=2), dict(basis=2)),
    "hermite-M6": (dict(M=6, Mt=3, contrast=0.9), dict(basis=2)),
}


@pytest.mark.parametrize("shape", [(64, 32), (48, 192), (64, 64), (12, 48, 8), (24, 16, 32)])
@pytest.mark.parametrize("form", sorted(FORMS))
def test_apply_matches_oracle(hz, shape, form):
    popt, mopt = FORMS[form]
    p = S.small_problem(shape, 21, width=2, **popt)
    med_g, med_o = media(hz, p, alpha=0.1, **mopt)
    info = med_g.info()
    assert info["K"] == med_o.nodes.K
    np.testing.assert_allclose(info["gamma"], med_o.nodes.gamma, rtol=1e-15, atol=0)
    np.testing.assert_allclose(info["a"], med_o.nodes.a, rtol=1e-15, atol=0)
    v = S.random_field(np.random.Generator(np.random.PCG64(22)), shape, 2)
    ref = np.stack([O.apply_preconditioner(med_o, v[b]) for b in range(2)])
    # (64, 64): the default launch shape (one node per block, column pairs) of
    # a square grid is the symbol pass compiled with its line stride
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, max_nrhs=2)
        for mode in (0, 1, 3):
            plan.set_tune(rowinv_mode=mode)
            got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
            assert within(rel(got, ref), prec, "interp_small"), (form, prec, mode, rel(got, ref))


def test_bad_extension_options_are_refused(hz):
    p = S.small_problem((16, 16), 3, M=4, Mt=2, width=2, damping=(0.0, 0.2))
    for kw in (dict(basis=1), dict(M=5, Ma=3, basis=1), dict(M=5, basis=3), dict(M=5, Ma=2, basis=2),
               dict(M=12, Mt=4, Ma=5), dict(M=30, Mt=6, basis=2)):
        kw = dict(kw)
        M = kw.pop("M", 4)
        with pytest.raises(hz.HzError):
            media(hz, p, M=M, oracle=False, **kw)


def _plane_wave(shape, kvec):
    idx = np.indices(shape, dtype=np.float64)
    return np.exp(1j * sum(2.0 * np.pi * k * idx[a] / shape[a] for a, k in enumerate(kvec)))


def _plane_wave_expected(med_o, shape, kvec, pts):
    """sum_k w_k(x) q_k(|xi|^2) at flat points pts: Q_M of a plane wave is
    the plane wave times the interpolated symbol, for any weights."""
    xi2 = sum(O.xi2_axis(shape[a], 1.0)[k % shape[a]] for a, k in enumerate(kvec))
    W = med_o.W.reshape(med_o.nodes.K, -1)
    qk = np.array([O.symbol_of(med_o.nodes, k, med_o.omega, np.array([xi2]))[0]
                   for k in range(med_o.nodes.K)])
    return (W[:, pts] * qk[:, None]).sum(axis=0)


@pytest.mark.parametrize("form", ["bivariate", "lagrange", "hermite"])
def test_full_size_apply_plane_wave(hz, form):
    """512^2 bivariate (K = 16 x 3 = 48 planes), 1024^2 quadratic (K = 11 + 4)
    and 1024^2 cubic Hermite (K = 8 + 4 + 8) applies through autotuned
    plans, on 4096 sampled points."""
    if form == "bivariate":
        p = S.damping_problem(N=512, Ma=3)
        med_g, med_o = media(hz, p, alpha=0.1, Ma=3)
        assert med_o.nodes.K == 48
    elif form == "hermite":
        p = S.config2()
        med_g, med_o = media(hz, p, alpha=0.1, M=8, basis=2)
        assert med_o.nodes.K == 20 and med_g.info()["K"] == 20
    else:
        p = S.config2()
        med_g, med_o = media(hz, p, alpha=0.1, M=11, basis=1)
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol)
    plan.autotune()
    kv = (37, -101)
    w = _plane_wave(p.shape, kv)
    pts = np.random.Generator(np.random.PCG64(32)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    for prec in (1, 0):
        got = plan.apply_preconditioner(_dev(w), precision=prec).cpu().numpy().ravel()
        assert within(rel(got[pts], exp), prec, "interp_full"), (form, prec, rel(got[pts], exp))


@pytest.mark.parametrize("mopt", [dict(Ma=3), dict(M=7, basis=1), dict(M=6, basis=2)])
def test_solve_with_extension_converges(hz, mopt):
    """FGMRES with the bivariate or quadratic preconditioner reaches the
    tolerance by the oracle's operator on a 128^2 damping medium."""
    p = S.damping_problem(N=128, Ma=3, width=16, M=6, Mt=2)
    mopt = dict(mopt)
    M = mopt.pop("M", p.M)
    med_g, med_o = media(hz, p, alpha=0.1, M=M, **mopt)
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol)
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)


def test_noalloc_apply_on_bivariate_medium(hz):
    """The allocation-free apply takes the per-point (node, weight) records too."""
    import torch
    p = S.small_problem((64, 96), 5, M=4, Mt=2, width=2, damping=(0.05, 0.3))
    med, _ = media(hz, p, oracle=False, Ma=3)
    plan = hz.Plan(med, precision=1)
    x = _dev(S.random_field(np.random.Generator(np.random.PCG64(6)), p.shape, 1))
    for prec in (0, 1):
        y = torch.zeros_like(x)
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = hz.lib.hz_apply_preconditioner_noalloc(med.handle, ctypes.c_void_p(x.data_ptr()),
                                                    ctypes.c_void_p(y.data_ptr()), 1, prec, s)
        assert st == 0
        ref = plan.apply_preconditioner(x, precision=prec)
        torch.cuda.synchronize()
        assert within(rel(y.cpu().numpy(), ref.cpu().numpy()), prec, "same_path")
