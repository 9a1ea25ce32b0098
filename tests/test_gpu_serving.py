"""Serving layer (hz_submit / hz_poll): mixed requests overlap on the GPU,
each result equals the same request solved alone, admission respects the
HBM budget, and malformed or oversized requests are refused."""
import numpy as np
import pytest

import oracle as O
from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _requests():
    out = []
    for shape, seed, M, Mt, nrhs in [((64, 64), 1, 5, 2, 2), ((96, 128), 2, 6, 2, 1),
                                     ((16, 24, 32), 3, 4, 2, 1), ((256, 256), 4, 6, 2, 1),
                                     ((48, 48), 5, 3, 1, 3), ((32, 32, 32), 6, 6, 2, 1)]:
        p = S.small_problem(shape, seed, M=M, Mt=Mt, width=3)
        f = S.random_field(np.random.Generator(np.random.PCG64(seed)), shape, nrhs)
        out.append((p, f))
    return out


def _submit(srv, p, f, **kw):
    return srv.submit(p.c, f, omega=p.omega, M=p.M, Mt=p.Mt, zeta=p.zeta, alpha=0.15,
                      restart=30, tol=1e-8, **kw)


def test_mixed_requests_match_solo_solves_and_oracle(hz):
    reqs = _requests()
    # default launch shapes, as the standalone plans below use
    srv = hz.Server(max_slots=3, autotune=-1)
    tickets = [_submit(srv, p, f) for p, f in reqs]
    results = [srv.result(t) for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_active"] >= 2, st  # requests really overlapped
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (p, f), (done, u, stats, status) in zip(reqs, results):
        assert done and status == 0
        med_o = O.make_medium(p.c, p.zeta, None, p.omega, p.M, p.Mt, 1.0, None, 0.15)
        for b in range(f.shape[0]):
            assert stats[b]["converged"]
            assert rel(O.apply_operator(med_o, u[b]), f[b]) <= 1e-8
        # the same request through a plan on its own
        med = hz.Medium(p.c, p.zeta, omega=p.omega, M=p.M, Mt=p.Mt, alpha=0.15)
        plan = hz.Plan(med, precision=1, restart=30, tol=1e-8, max_nrhs=f.shape[0])
        u1, st1 = plan.solve(np.ascontiguousarray(f))
        assert np.array_equal(u1, u), rel(u1, u)
        assert [s["iters"] for s in st1] == [s["iters"] for s in stats]
    srv.close()


def test_result_same_alone_and_in_mix(hz):
    reqs = _requests()
    p, f = reqs[1]
    solo = hz.Server(max_slots=1)
    ua = solo.result(_submit(solo, p, f))[1]
    solo.close()
    mix = hz.Server(max_slots=4)
    ts = [_submit(mix, q, g) for q, g in reqs[3:]] + [_submit(mix, p, f)] + \
         [_submit(mix, q, g) for q, g in reqs[:3]]
    out = {t: mix.result(t) for t in ts}
    assert np.array_equal(out[ts[len(reqs) - 3]][1], ua)
    assert mix.stats()["max_active"] >= 2
    mix.close()


def test_admission_by_hbm_budget(hz):
    reqs = _requests()[:4]
    fps = [hz.request_footprint(p.shape, p.M, p.Mt, 1, 30, f.shape[0]) for p, f in reqs]
    budget = int(max(fps) * 1.2)  # room for the largest alone, never two of the big ones
    srv = hz.Server(max_slots=4, hbm_budget=budget)
    ts = [_submit(srv, p, f) for p, f in reqs]
    for t in ts:
        done, u, stats, status = srv.result(t)
        assert done and status == 0
    st = srv.stats()
    assert st["completed"] == 4 and st["hbm_in_use"] == 0
    srv.close()
    # a request larger than the whole budget is refused at submit
    small = hz.Server(max_slots=1, hbm_budget=1 << 20)
    p, f = reqs[0]
    with pytest.raises(hz.HzError) as e:
        _submit(small, p, f)
    assert e.value.status == 7
    small.close()


def test_queue_limit_and_bad_request(hz):
    reqs = _requests()
    srv = hz.Server(max_slots=1, max_queue=1)
    p, f = reqs[3]
    t0 = _submit(srv, p, f)
    refused = 0
    for _ in range(4):
        try:
            _submit(srv, p, f)
        except hz.HzError as e:
            assert e.status == 7
            refused += 1
    assert refused >= 2
    srv.result(t0)
    with pytest.raises(hz.HzError) as e:
        srv.submit(np.ones((22, 16)), np.zeros((1, 22, 16), complex), omega=3.0, M=2)
    assert e.value.status == 1
    srv.close()


@pytest.mark.parametrize("order", [0, 1])
def test_admission_order(hz, order):
    """One slot, a large request running, then a large and a small request
    queued: in arrival order (0) the large one goes first; smallest footprint
    first (1) lets the small one overtake it.  The results do not depend on
    the order."""
    import time
    big = S.small_problem((512, 512), 41, M=6, Mt=2, width=8)
    small = S.small_problem((64, 64), 42, M=5, Mt=2, width=3)
    fb = S.random_field(np.random.Generator(np.random.PCG64(43)), big.shape, 2)
    fs = S.random_field(np.random.Generator(np.random.PCG64(44)), small.shape, 1)
    srv = hz.Server(max_slots=1, order=order)
    t_run = _submit(srv, big, fb)
    t0 = time.time()
    while srv.stats()["active"] < 1 and time.time() - t0 < 10:
        time.sleep(0.001)
    t_big = _submit(srv, big, fb)
    t_small = _submit(srv, small, fs)
    srv.wait(t_small, timeout=600)
    pb = srv.poll(t_big)  # consumes the ticket when done
    big_done_first = pb[0]
    res = {t_small: srv.poll(t_small), t_run: srv.result(t_run, timeout=600),
           t_big: pb if big_done_first else srv.result(t_big, timeout=600)}
    srv.close()
    assert big_done_first == (order == 0)
    assert np.array_equal(res[t_run][1], res[t_big][1])
    for t in (t_run, t_big, t_small):
        assert res[t][0] and res[t][3] == 0


def test_extension_requests_are_served(hz):
    """Bivariate (c, a) and quadratic-basis requests go through the server and
    give the result of the same request solved on its own plan."""
    p = S.small_problem((64, 96), 8, M=5, Mt=2, width=3, damping=(0.05, 0.3))
    f = S.random_field(np.random.Generator(np.random.PCG64(8)), p.shape, 2)
    srv = hz.Server(max_slots=2)
    cases = [dict(Ma=3), dict(basis=1)]
    tickets = [srv.submit(p.c, f, omega=p.omega, M=p.M, Mt=p.Mt, zeta=p.zeta, a=p.a, alpha=0.15,
                          restart=30, tol=1e-8, **kw) for kw in cases]
    for kw, t in zip(cases, tickets):
        done, u, stats, status = srv.result(t)
        assert done and status == 0 and all(s["converged"] for s in stats)
        med_o = O.make_medium(p.c, p.zeta, p.a, p.omega, p.M, p.Mt, 1.0, None, 0.15,
                              Ma=max(kw.get("Ma", 1), 1), basis=kw.get("basis", 0))
        for b in range(f.shape[0]):
            assert rel(O.apply_operator(med_o, u[b]), f[b]) <= 1e-8
        med = hz.Medium(p.c, p.zeta, p.a, omega=p.omega, M=p.M, Mt=p.Mt, alpha=0.15, **kw)
        plan = hz.Plan(med, precision=1, restart=30, tol=1e-8, max_nrhs=f.shape[0])
        u1, _ = plan.solve(np.ascontiguousarray(f))
        assert np.array_equal(u1, u), rel(u1, u)
    srv.close()


def _batch_problem():
    p = S.small_problem((512, 512), 9, M=6, Mt=2, width=8)
    fs = [S.random_field(np.random.Generator(np.random.PCG64(90 + i)), p.shape, k)
          for i, k in enumerate((2, 1, 1))]
    return p, fs


def _submit_b(srv, p, f):
    return srv.submit(p.c, f, omega=p.omega, M=p.M, Mt=p.Mt, zeta=p.zeta, alpha=0.15,
                      restart=10, tol=1e-10, maxit=3000)


def test_batched_requests_join_at_restart_boundaries(hz):
    """Continuous batching (batch_slots): requests on the same medium share
    one batched solve.  b, submitted right after a, joins a's batch at a
    restart boundary instead of starting its own; c joins later if the batch
    is still iterating; each leaves when its right-hand sides are done.
    Every request's solution is bit for bit the one it gets alone in a
    batch, every right-hand side meets the tolerance by the oracle's
    operator, and a request on another medium runs beside the batch."""
    import time
    p, (fa, fb, fc) = _batch_problem()
    q = S.small_problem((64, 64), 8, M=5, Mt=2, width=3)
    fq = S.random_field(np.random.Generator(np.random.PCG64(99)), q.shape, 1)
    alone = {}
    for name, f in (("a", fa), ("b", fb), ("c", fc)):
        srv = hz.Server(max_slots=1, batch_slots=4)
        done, u, st, status = srv.result(_submit_b(srv, p, f))
        assert done and status == 0
        alone[name] = (u, st)
        srv.close()
    srv = hz.Server(max_slots=2, batch_slots=4)
    ta = _submit_b(srv, p, fa)
    tb = _submit_b(srv, p, fb)
    tq = srv.submit(q.c, fq, omega=q.omega, M=q.M, Mt=q.Mt, zeta=q.zeta, alpha=0.15,
                    restart=10, tol=1e-10, maxit=3000)
    time.sleep(0.02)
    tc = _submit_b(srv, p, fc)
    res = {k: srv.result(t, timeout=600) for k, t in (("a", ta), ("b", tb), ("c", tc), ("q", tq))}
    stats = srv.stats()
    srv.close()
    assert stats["batch_joins"] >= 1, stats
    assert stats["completed"] == 4 and stats["failed"] == 0
    for k in ("a", "b", "c"):
        assert np.array_equal(res[k][1], alone[k][0]), k
        assert [s["iters"] for s in res[k][2]] == [s["iters"] for s in alone[k][1]]
    med_o = O.make_medium(p.c, p.zeta, None, p.omega, p.M, p.Mt, 1.0, None, 0.15)
    for k, f in (("a", fa), ("b", fb), ("c", fc)):
        done, u, st, status = res[k]
        assert done and status == 0
        for b in range(f.shape[0]):
            assert st[b]["converged"]
            assert rel(O.apply_operator(med_o, u[b]), f[b]) <= 1e-10
    medq = O.make_medium(q.c, q.zeta, None, q.omega, q.M, q.Mt, 1.0, None, 0.15)
    assert rel(O.apply_operator(medq, res["q"][1][0]), fq[0]) <= 1e-10
