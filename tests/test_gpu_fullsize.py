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
    assert within(rel(got, ref), 1, "cfg2"), rel(got, ref)
    # plane wave through the same plan
    kv = (37, -101)
    w = _plane_wave(p.shape, kv)
    got = plan.apply_preconditioner(_dev(w), precision=1).cpu().numpy().ravel()
    pts = np.random.Generator(np.random.PCG64(32)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    assert within(rel(got[pts], exp), 1, "cfg2"), rel(got[pts], exp)
    # the solve the benchmark times; residual by the oracle's operator
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)
    assert abs(r - st[0]["rel_true_resid"]) <= 1e-9


def test_config4_batched_apply_sampled_rhs(hz):
    p = S.config4()
    med_g, med_o = media(hz, p, alpha=0.1)
    nrhs = p.f.shape[0]
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol, max_nrhs=nrhs, graphs=True)
    plan.autotune()
    v = S.random_field(np.random.Generator(np.random.PCG64(33)), p.shape, nrhs)
    got = plan.apply_preconditioner(_dev(v), precision=1).cpu().numpy()
    for b in (0, nrhs // 2, nrhs - 1):
        e = rel(got[b], O.apply_preconditioner(med_o, v[b]))
        assert within(e, 1, "cfg4"), (b, e)


def test_config4_batched_solve_every_rhs(hz):
    """The 512^2 x 64 batched FGMRES(40) solve the benchmark times (autotuned
    plan, captured cycle graphs, all 64 right-hand sides in lock step):
    every right-hand side's true residual, computed by the oracle's own
    operator from the returned solution, meets the tolerance and agrees with
    the residual the library reports."""
    p = S.config4()
    med_g, med_o = media(hz, p, alpha=0.1)
    nrhs = p.f.shape[0]
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol, max_nrhs=nrhs, graphs=True)
    plan.autotune()
    f = _dev(p.f)
    u, st = plan.solve(f)
    u = u.cpu().numpy()
    assert len(st) == nrhs
    for b in range(nrhs):
        r = rel(O.apply_operator(med_o, u[b]), p.f[b])
        assert st[b]["converged"] and r <= p.tol, (b, st[b], r)
        assert abs(r - st[b]["rel_true_resid"]) <= 1e-9, (b, r, st[b]["rel_true_resid"])


def test_config3_plane_wave_and_solve_full_size(hz):
    p = S.config3()
    med_g, med_o = media(hz, p, alpha=0.3)
    plan = hz.Plan(med_g, precision=1, restart=p.restart, tol=p.tol)
    plan.autotune()
    kv = (5, -17, 64)
    w = _plane_wave(p.shape, kv)
    got = plan.apply_preconditioner(_dev(w), precision=1).cpu().numpy().ravel()
    pts = np.random.Generator(np.random.PCG64(34)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    assert within(rel(got[pts], exp), 1, "cfg3"), rel(got[pts], exp)
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)


@pytest.mark.parametrize("N,d,K", [(2048, 2, (12, 4)), (192, 3, (9, 3))])
def test_largest_and_radix3_serving_grids_plane_wave(hz, N, d, K):
    """The serving recipe's largest 2D grid (2048^2, 3 radix-16/8 stages per
    axis) and its radix-3 3D grid (192^3 = 3 * 64 per axis): the apply of a
    plane wave through an autotuned plan against the per-point closed form,
    in both precisions, on 4096 sampled points; then the solve, checked with
    the oracle's operator."""
    p = S.bump_problem(N, 61 + d, d=d, n_bumps=6, amp=0.8, width=24 if d == 2 else 16,
                       ppw=8.0, M=K[0], Mt=K[1])
    med_g, med_o = media(hz, p, alpha=0.15)
    plan = hz.Plan(med_g, precision=1, restart=40, tol=1e-6)
    plan.autotune()
    kv = (37, -101) if d == 2 else (17, -29, 41)
    w = _plane_wave(p.shape, kv)
    pts = np.random.Generator(np.random.PCG64(63)).integers(0, p.n, 4096)
    exp = _plane_wave_expected(med_o, p.shape, kv, pts) * w.ravel()[pts]
    for prec in (1, 0):
        got = plan.apply_preconditioner(_dev(w), precision=prec).cpu().numpy().ravel()
        assert within(rel(got[pts], exp), prec, f"grid{N}"), (N, d, prec, rel(got[pts], exp))
    # and the solve, by the oracle's own operator
    u, st = plan.solve(np.ascontiguousarray(p.f[0]))
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)
    assert abs(r - st[0]["rel_true_resid"]) <= 1e-9
