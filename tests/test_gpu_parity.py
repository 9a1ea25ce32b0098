"""Parity of the CUDA path against the CPU oracle, element by element, on
seeded synthetic media (several tiles, ragged tails, 2D and 3D), through the
C ABI.  Tolerances: 1e-10 relative (2-norm) for the FP64 apply, operator and
solve pieces; for the complex64 preconditioner apply the stated per-family
bound of gpu_util.C64_BOUND (FP32 rounding, ~eps32 log2(n), amplified near
|xi| = omega / c_k by at most 1/alpha)."""
import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel, within

pytestmark = pytest.mark.gpu

SHAPES_2D = [(16, 16), (24, 48), (96, 12), (64, 32), (128, 128), (48, 192), (8, 2048)]
SHAPES_3D = [(8, 12, 16), (16, 16, 16), (24, 16, 32), (12, 48, 8)]


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_node_table_matches_oracle(hz):
    for p in (S.small_problem((32, 24), 3, M=5, Mt=3, width=3), S.config1()):
        med_g, med_o = media(hz, p)
        info = med_g.info()
        assert info["K"] == med_o.nodes.K and info["M"] == med_o.nodes.M
        np.testing.assert_allclose(info["gamma"], med_o.nodes.gamma, rtol=1e-15, atol=1e-15)
        np.testing.assert_allclose(info["a"], med_o.nodes.a, rtol=1e-15)
    # c_o strictly inside the speed range: two equispaced segments
    p = S.small_problem((16, 16), 4, M=6, Mt=2, width=2, contrast=0.5)
    c = p.c.copy()
    c[c == 1.0] = 1.0
    c[6:10, 6:10] = 0.8
    p.c = c
    med_g, med_o = media(hz, p)
    np.testing.assert_allclose(med_g.info()["gamma"], med_o.nodes.gamma, rtol=1e-15)


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_apply_preconditioner_fp64(hz, shape):
    p = S.small_problem(shape, 11, M=5, Mt=3, width=2)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=0, max_nrhs=2)
    v = S.random_field(np.random.Generator(np.random.PCG64(5)), shape, 2)
    ref = np.stack([O.apply_preconditioner(med_o, v[b]) for b in range(2)])
    got = plan.apply_preconditioner(_dev(v), precision=0).cpu().numpy()
    assert rel(got, ref) <= 1e-10, rel(got, ref)
    # element-wise as well: every point within 1e-10 of the largest value
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_apply_preconditioner_c64(hz, shape):
    p = S.small_problem(shape, 12, M=5, Mt=3, width=2)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1)
    v = S.random_field(np.random.Generator(np.random.PCG64(6)), shape)
    ref = O.apply_preconditioner(med_o, v)
    got = plan.apply_preconditioner(_dev(v), precision=1).cpu().numpy()
    assert within(rel(got, ref), 1, "small"), rel(got, ref)


@pytest.mark.parametrize("shape", [(16, 16), (24, 48), (8, 12, 16)])
def test_apply_preconditioner_variants(hz, shape):
    """No layer; single node (Q_1); finite-difference symbol; damping in the
    operator and the symbol."""
    p = S.small_problem(shape, 13, M=4, Mt=0, width=0, a_const=2.0)
    for kw in (dict(), dict(M=1), dict(symbol_kind=1), dict(a_node=2.0, alpha=0.0)):
        med_g, med_o = media(hz, p, **kw)
        plan = hz.Plan(med_g, precision=0)
        v = S.random_field(np.random.Generator(np.random.PCG64(7)), shape)
        ref = O.apply_preconditioner(med_o, v)
        got = plan.apply_preconditioner(_dev(v), precision=0).cpu().numpy()
        assert rel(got, ref) <= 1e-10, (kw, rel(got, ref))


@pytest.mark.parametrize("shape", SHAPES_2D[:4] + SHAPES_3D[:3])
def test_apply_operator(hz, shape):
    p = S.small_problem(shape, 14, M=4, Mt=2, width=2, a_const=1.5)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=0, max_nrhs=3)
    v = S.random_field(np.random.Generator(np.random.PCG64(8)), shape, 3)
    ref = np.stack([O.apply_operator(med_o, v[b]) for b in range(3)])
    got = plan.apply_operator(_dev(v)).cpu().numpy()
    assert rel(got, ref) <= 1e-12, rel(got, ref)
    # precision 1: complex64 input (as flexible GMRES stores Z), FP64
    # arithmetic; the reference is the oracle's operator on the same
    # complex64-rounded values, so only FP64 rounding separates them
    v32 = v.astype(np.complex64)
    ref32 = np.stack([O.apply_operator(med_o, v32[b].astype(np.complex128)) for b in range(3)])
    got32 = plan.apply_operator(_dev(v32)).cpu().numpy()
    assert got32.dtype == np.complex128
    assert rel(got32, ref32) <= 1e-12, rel(got32, ref32)


@pytest.mark.parametrize("prec", [0, 1])
def test_gmres_small_matches_dense_and_oracle(hz, prec):
    p = S.small_problem((24, 32), 15, M=5, Mt=3, width=3)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=prec, restart=20, tol=1e-10, maxit=2000)
    u, st = plan.solve(_dev(p.f[0]))
    u = u.cpu().numpy()
    assert st[0]["converged"], st
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert r <= 1e-10, r
    A = O.assemble_dense(lambda x: O.apply_operator(med_o, x), p.shape)
    x_lu = np.linalg.solve(A, p.f[0].ravel()).reshape(p.shape)
    assert rel(u, x_lu) <= 1e-7


def test_solve_stats_phase_times(hz):
    """hz_solve_stats carries the solve's own phase times and the
    preconditioner's algorithmic bytes while profiling is on (step by step),
    and zeros otherwise; the phases fit inside the solve's wall time."""
    p = S.small_problem((64, 96), 16, M=5, Mt=3, width=3)
    med, _ = media(hz, p, oracle=False)
    K = med.info()["K"]
    n = p.n
    plan = hz.Plan(med, precision=1, restart=20, tol=1e-8, maxit=2000)
    u, st = plan.solve(_dev(p.f[0]))
    assert st[0]["converged"]
    assert st[0]["ms_precond"] == 0 and st[0]["ms_arnoldi"] == 0
    assert st[0]["model_bytes_precond"] == 0
    hz.profile_enable(True)
    try:
        u, st = plan.solve(_dev(p.f[0]))
    finally:
        hz.profile_enable(False)
        hz.profile_read(reset=True)
    s = st[0]
    assert s["converged"]
    assert s["ms_precond"] > 0 and s["ms_stencil"] > 0 and s["ms_arnoldi"] > 0
    assert s["ms_precond"] + s["ms_stencil"] + s["ms_arnoldi"] <= s["ms_total"] * 1.01
    # one complex64 apply per Arnoldi step: between the input and output
    # alone (24 B/pt) and the fixed model with every plane (plus the output
    # cleared by the scattering form)
    per_apply = s["model_bytes_precond"] / s["iters"]
    assert 24 * n <= per_apply <= n * ((4 + 2 * K) * 8 + 4 + 32), (per_apply, n, K)


def test_gmres_config1_fp64(hz):
    """2D 128^2, K = 8, GMRES(30), FP64 throughout, tol 1e-6: the true residual
    computed by the oracle's own operator meets the tolerance and the
    iteration count is close to the oracle's GMRES."""
    p = S.config1()
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=0, restart=30, tol=1e-6, maxit=4000)
    u, st = plan.solve(_dev(p.f[0]))
    u = u.cpu().numpy()
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-6, (st, r)
    uo, sto = O.gmres(lambda x: O.apply_operator(med_o, x), p.f[0],
                      lambda v: O.apply_preconditioner(med_o, v), restart=30, tol=1e-6)
    assert abs(st[0]["iters"] - sto["iters"]) <= 2, (st, sto["iters"])
    assert rel(u, uo) <= 1e-4


def test_gmres_multi_rhs_and_host_buffers(hz):
    p = S.bump_problem(64, 21, width=8, ppw=8.0, M=4, Mt=2, nrhs=3)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1, restart=25, tol=1e-6, maxit=2000, max_nrhs=3)
    f = np.ascontiguousarray(p.f)
    u, st = plan.solve(f)  # host numpy buffers, staged by the library
    for b in range(3):
        r = rel(O.apply_operator(med_o, u[b]), f[b])
        assert st[b]["converged"] and r <= 1e-6, (b, st[b], r)
    # each right-hand side alone gives the same answer as in the batch
    plan1 = hz.Plan(med_g, precision=1, restart=25, tol=1e-6, maxit=2000, max_nrhs=1)
    u1, st1 = plan1.solve(np.ascontiguousarray(f[1:2]))
    assert st1[0]["iters"] == st[1]["iters"]
    assert rel(u1[0], u[1]) <= 1e-12


def test_edge_cases(hz):
    p = S.small_problem((16, 16), 16, M=4, Mt=2, width=2)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1, restart=10, tol=1e-6, maxit=3)
    # zero right-hand side: zero solution, converged at once
    u, st = plan.solve(np.zeros((1, 16, 16), complex))
    assert st[0]["converged"] and np.all(u == 0) and st[0]["iters"] == 0
    # maxit reached: NOT_CONVERGED with the iterate and its stats
    u, st = plan.solve(_dev(p.f[0]))
    assert not st[0]["converged"] and st[0]["iters"] == 3 and st[0]["status"] == 4
    with pytest.raises(hz.HzError) as e:
        plan.solve(_dev(p.f[0]), raise_on_fail=True)
    assert e.value.status == 4
    # invalid media and grids are rejected on the host
    bad = p.c.copy()
    bad[3, 3] = -1.0
    with pytest.raises(hz.HzError) as e:
        hz.Medium(bad, p.zeta, omega=p.omega, M=4, Mt=2)
    assert e.value.status == 8
    bad = p.c.copy()
    bad[0, 0] = 1.3  # inside the layer, c != c_o
    with pytest.raises(hz.HzError) as e:
        hz.Medium(bad, p.zeta, omega=p.omega, M=4, Mt=2)
    assert e.value.status == 8
    with pytest.raises(hz.HzError) as e:
        hz.Medium(np.ones((22, 16)), omega=3.0, M=2)
    assert e.value.status == 1
    with pytest.raises(hz.HzError):
        plan.apply_operator(_dev(np.zeros((2, 16, 16), complex)))  # nrhs > max_nrhs


def test_graph_replay_matches_stepwise(hz):
    """The captured-cycle mode (opts.graphs) launches the same kernels in the
    same order: identical iterates and counts, also for several right-hand
    sides that retire at different steps."""
    p = S.bump_problem(64, 41, width=8, ppw=8.0, M=4, Mt=2, nrhs=3)
    med_g, _ = media(hz, p, oracle=False)
    out = []
    for graphs in (False, True):
        plan = hz.Plan(med_g, precision=1, restart=15, tol=1e-7, maxit=3000, max_nrhs=3,
                       graphs=graphs)
        u, st = plan.solve(np.ascontiguousarray(p.f))
        out.append((u, [s["iters"] for s in st], [s["converged"] for s in st]))
        u, st = plan.solve(np.ascontiguousarray(p.f))  # replay of the captured graph
        assert np.array_equal(u, out[-1][0])
    assert out[0][1] == out[1][1] and all(out[1][2])
    assert np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 48, 24)])
def test_gmres_3d_matches_oracle(hz, shape):
    p = S.small_problem(shape, 42, M=5, Mt=2, width=3)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1, restart=20, tol=1e-8, maxit=3000)
    u, st = plan.solve(_dev(p.f[0]))
    u = u.cpu().numpy()
    r = rel(O.apply_operator(med_o, u), p.f[0])
    assert st[0]["converged"] and r <= 1e-8, (st, r)
    uo, sto = O.gmres(lambda x: O.apply_operator(med_o, x), p.f[0],
                      lambda v: O.apply_preconditioner(med_o, v), restart=20, tol=1e-8)
    assert abs(st[0]["iters"] - sto["iters"]) <= 3, (st[0]["iters"], sto["iters"])


@pytest.mark.parametrize("shape", [(64, 32), (128, 128), (48, 192), (8, 2048), (12, 48, 8),
                                   (24, 16, 32), (1024, 24), (512, 48)])
def test_apply_every_launch_shape(hz, shape):
    """Every symbol-pass node grouping, one or two columns per thread (full or
    half-size blocks), and every x-inverse form (fused weighted sum; in place
    + gather; one line per (row, node) added into the cleared output) give
    the oracle's apply, in both precisions and with two right-hand sides."""
    p = S.small_problem(shape, 14, M=6, Mt=3, width=2)
    med_g, med_o = media(hz, p)
    v = S.random_field(np.random.Generator(np.random.PCG64(15)), shape, 2)
    ref = np.stack([O.apply_preconditioner(med_o, v[b]) for b in range(2)])
    for prec in (0, 1):
        plan = hz.Plan(med_g, precision=prec, max_nrhs=2)
        for kpb, mode, pair in ((1, 1, 1), (1, 2, 0), (2, 2, 1), (4, 1, 0), (4, 2, 1), (2, 0, 1),
                                (1, 0, 0), (1, 2, 2), (2, 1, 2), (4, 0, 2), (1, 3, 1), (2, 3, 0),
                                (4, 3, 2)):
            plan.set_tune(syminv_kpb=kpb, rowinv_mode=mode, col_pair=pair)
            got = plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy()
            assert within(rel(got, ref), prec, "small"), (prec, kpb, mode, pair, rel(got, ref))


def test_set_tune_rejects_out_of_range(hz):
    p = S.small_problem((16, 16), 3, M=4, Mt=2, width=2)
    med_g, _ = media(hz, p)
    plan = hz.Plan(med_g, precision=1)
    for bad in (dict(syminv_kpb=3), dict(rowinv_mode=4), dict(dots_vc=5), dict(upd_bps=0),
                dict(dots_bps=5), dict(upd_bps=9), dict(col_pair=3)):
        with pytest.raises(hz.HzError):
            plan.set_tune(**bad)


def test_autotune_choices_are_valid_and_cached(hz):
    p = S.bump_problem(128, 43, width=8, ppw=8.0, M=5, Mt=2, nrhs=2)
    med_g, med_o = media(hz, p)
    plan = hz.Plan(med_g, precision=1, restart=20, tol=1e-8, maxit=2000, max_nrhs=2)
    r = plan.autotune()
    assert r["cached"] == 0
    assert r["dots_bps"] in (1, 2, 3, 4) and r["dots_vc"] in (2, 4, 8)
    assert r["upd_bps"] in (2, 4, 6, 8) and r["syminv_kpb"] in (1, 2, 4)
    assert r["rowinv_mode"] in (0, 1, 2, 3) and r["col_pair"] in (0, 1, 2)
    assert 0 < r["dots_us"] <= r["dots_us_default"] * 1.0001
    u, st = plan.solve(np.ascontiguousarray(p.f))
    for b in range(2):
        assert st[b]["converged"]
        assert rel(O.apply_operator(med_o, u[b]), p.f[b]) <= 1e-8
    plan2 = hz.Plan(med_g, precision=1, restart=20, tol=1e-8, maxit=2000, max_nrhs=2)
    r2 = plan2.autotune()
    assert r2["cached"] == 1 and r2["syminv_kpb"] == r["syminv_kpb"]
    # the tuned preconditioner apply still matches the oracle
    v = S.random_field(np.random.Generator(np.random.PCG64(9)), p.shape)
    ref = O.apply_preconditioner(med_o, v)
    got = plan2.apply_preconditioner(_dev(v), precision=0).cpu().numpy()
    assert rel(got, ref) <= 1e-10


def test_scattering_x_inverse_is_bitwise_reproducible(hz):
    """The one-line-per-(row, node) x-inverse adds into its output with
    atomics; with the (segment, t) records a point receives at most two
    additions onto an exact zero, so repeated applies agree bit for bit (and
    with two right-hand sides in one batch as alone)."""
    p = S.small_problem((96, 128), 17, M=6, Mt=3, width=3)
    med_g, med_o = media(hz, p)
    v = S.random_field(np.random.Generator(np.random.PCG64(18)), p.shape, 2)
    for prec in (1, 0):
        plan = hz.Plan(med_g, precision=prec, max_nrhs=2)
        plan.set_tune(rowinv_mode=3)
        outs = [plan.apply_preconditioner(_dev(v), precision=prec).cpu().numpy() for _ in range(4)]
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        alone = plan.apply_preconditioner(_dev(v[1:2]), precision=prec).cpu().numpy()
        assert np.array_equal(alone[0], outs[0][1])
        ref = O.apply_preconditioner(med_o, v[0])
        assert within(rel(outs[0][0], ref), prec, "small")
