"""Failure detection without a GPU fault: host-side injection only.
An allocator that fails, a NaN right-hand side and a server wait that runs
out all come back as status codes; the device stays usable afterwards."""
import ctypes as C

import numpy as np
import pytest

from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel

pytestmark = pytest.mark.gpu

ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def test_failing_allocator_reports_oom(hz):
    p = S.small_problem((32, 32), 51, M=4, Mt=2, width=2)
    calls = []

    def fail_alloc(nbytes, ctx):
        calls.append(nbytes)
        return None

    def no_free(ptr, ctx):
        pass

    a, f = ALLOC(fail_alloc), FREE(no_free)
    assert hz.lib.hz_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None) == 0
    try:
        with pytest.raises(hz.HzError) as e:
            hz.Medium(p.c, p.zeta, omega=p.omega, M=4, Mt=2)
        assert e.value.status == 2 and calls
    finally:
        assert hz.lib.hz_set_allocator(None, None, None) == 0
    # the device is fine afterwards
    med, med_o = media(hz, p)
    plan = hz.Plan(med, precision=1, restart=20, tol=1e-8)
    u, st = plan.solve(np.ascontiguousarray(p.f))
    assert st[0]["converged"]


def test_nan_rhs_is_a_breakdown_status(hz):
    p = S.small_problem((32, 32), 52, M=4, Mt=2, width=2)
    med, _ = media(hz, p, oracle=False)
    plan = hz.Plan(med, precision=1, restart=20, tol=1e-8)
    f = np.ascontiguousarray(p.f.copy())
    f[0, 3, 4] = np.nan
    u, st = plan.solve(f)
    assert st[0]["status"] == 5 and not st[0]["converged"]
    with pytest.raises(hz.HzError) as e:
        plan.solve(f, raise_on_fail=True)
    assert e.value.status == 5
    # a clean solve on the same plan still works
    u, st = plan.solve(np.ascontiguousarray(p.f))
    assert st[0]["converged"]


def test_server_wait_times_out_then_completes(hz):
    p = S.config2()
    srv = hz.Server(max_slots=1)
    t = srv.submit(p.c, p.f, omega=p.omega, M=p.M, Mt=p.Mt, zeta=p.zeta, alpha=0.1)
    with pytest.raises(hz.HzError) as e:
        srv.wait(t, timeout=1e-3)
    assert e.value.status == 6
    done, u, stats, status = srv.result(t, timeout=600)
    assert done and status == 0 and stats[0]["converged"]
    srv.close()
