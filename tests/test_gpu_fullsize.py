"""Parity at the benchmark workloads' full sizes, with the launch shapes the
benchmark uses (autotuned plans): the 1024^2 apply element by element
against the oracle, the 512^2 x 64 batched apply on two of its right-hand
sides, the 256^3 apply on sampled points through the plane-wave closed form
(Q_M e^{i xi.x} = sum_k w_k(x) q_k(xi) e^{i xi.x}, exact for the discrete
pair), and full solves checked with the oracle's own operator."""
import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _plane_wave(shape, kvec):
    """exp(2 pi i sum_a k_a j_a / N_a) on the grid (index form of e^{i xi.x})."""
    idx = np.indices(shape, dtype=np.float64)
    ph = sum(2.0 * np.pi * k * idx[a] / shape[a] for a, k in enumerate(kvec))
    return np.exp(1j * ph)


def _plane_wave_expected(med_o, shape, kvec, pts):
    """sum_k w_k(x) q_k(|xi|^2) at the flat points pts (Eqn. 105/405 with the
    per-node symbols of Eqn. 021)."""
    xi2 = 0.0
    for a, k in enumerate(kvec):
        xi2 += O.xi2_axis(shape[a], 1.0)[k % shape[a]]
    W = med_o.W.reshape(med_o.nodes.K, -1)
    qk = np.array([O.node_symbol(med_o.nodes.gamma[k], med_o.nodes.a[k], med_o.omega,
                                 np.array([xi2]))[0] for k in range(med_o.nodes.K)])
    return (W[:, pts] * qk[:, None]).sum(axis=0)


def test_config2_apply_and_solve_full_size(hz):
    p = S.config2()
    med_g, med_o = media(hz, p, alpha=0.1)
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol, graphs=True)
    plan.autotune()
    v = S.random_field(np.random.Generator(np.random.PCG64(31)), p.shape)
    ref = O.apply_preconditioner(med_o, v)
    got = plan.apply_preconditioner(_dev(v), precision=1).cpu().numpy()
    assert rel(got, ref) <= 5e-5, rel(got, ref)
    # plane wave through the same plan
    kv = (37, -101)
    w = _plane_wave(p.shape, kv)
    got = plan.apply_preconditioner(_dev(w), precision=1).cpu().numpy().ravel()
    pts = np.random.Generator(np.random.PCG64(32)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    assert rel(got[pts], exp) <= 5e-5
    # the solve the benchmark times; residual by the oracle's operator
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)
    assert abs(r - st[0]["rel_true_resid"]) <= 1e-9


def test_config4_batched_apply_sampled_rhs(hz):
    p = S.config4()
    med_g, med_o = media(hz, p, alpha=0.15)
    nrhs = p.f.shape[0]
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol, max_nrhs=nrhs, graphs=True)
    plan.autotune()
    v = S.random_field(np.random.Generator(np.random.PCG64(33)), p.shape, nrhs)
    got = plan.apply_preconditioner(_dev(v), precision=1).cpu().numpy()
    for b in (0, nrhs // 2, nrhs - 1):
        assert rel(got[b], O.apply_preconditioner(med_o, v[b])) <= 5e-5


def test_config3_plane_wave_and_solve_full_size(hz):
    p = S.config3()
    med_g, med_o = media(hz, p, alpha=0.15)
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol)
    plan.autotune()
    kv = (5, -17, 64)
    w = _plane_wave(p.shape, kv)
    got = plan.apply_preconditioner(_dev(w), precision=1).cpu().numpy().ravel()
    pts = np.random.Generator(np.random.PCG64(34)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    assert rel(got[pts], exp) <= 5e-5
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)
