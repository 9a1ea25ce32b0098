"""The allocation-free preconditioner entry point, called through the C ABI,
gives the same result as the plan-based hz_apply_preconditioner, on two
calls in a row (the shared scratch keeps the previous call's contents), in
both precisions, and refuses work that does not fit its fixed scratch."""
import ctypes

import numpy as np
import pytest

from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel, within

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    import torch
    assert torch.cuda.is_available()
    return hz_module()


def _noalloc(hz, med, x, y, nrhs, prec):
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return hz.lib.hz_apply_preconditioner_noalloc(med.handle, ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr()), nrhs, prec, s)


@pytest.mark.parametrize("shape,nrhs", [((64, 96), 2), ((24, 16, 32), 1), ((256, 256), 1)])
def test_noalloc_matches_plan_apply(hz, shape, nrhs):
    import torch
    p = S.small_problem(shape, 31, M=5, Mt=3, width=2)
    med, _ = media(hz, p, oracle=False)
    plan = hz.Plan(med, precision=1, max_nrhs=nrhs)
    rng = np.random.Generator(np.random.PCG64(3))
    for prec in (0, 1):
        # two different inputs in a row, so that the second call starts from
        # the first call's scratch contents
        for call in range(2):
            v = S.random_field(rng, shape, nrhs)
            x = torch.from_numpy(v).cuda()
            ref = plan.apply_preconditioner(x, precision=prec).cpu().numpy()
            y = torch.full_like(x, complex(np.nan, np.nan))
            st = _noalloc(hz, med, x, y, nrhs, prec)
            assert st == 0, hz.last_error()
            got = y.cpu().numpy()
            assert within(rel(got, ref), prec, "same_path"), (prec, call, rel(got, ref))


ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def test_noalloc_allocates_nothing(hz):
    """With an allocator that refuses every request installed, a warm call
    still succeeds, asks the library allocator for nothing, and leaves the
    device's free memory and torch's allocated bytes unchanged."""
    import torch
    shape, nrhs = (128, 96), 2
    p = S.small_problem(shape, 33, M=5, Mt=3, width=2)
    med, _ = media(hz, p, oracle=False)
    plan = hz.Plan(med, precision=1, max_nrhs=nrhs)
    v = S.random_field(np.random.Generator(np.random.PCG64(5)), shape, nrhs)
    x = torch.from_numpy(v).cuda()
    ref = plan.apply_preconditioner(x, precision=1).cpu().numpy()
    y = torch.empty_like(x)
    assert _noalloc(hz, med, x, y, nrhs, 1) == 0, hz.last_error()  # first call: set-up
    torch.cuda.synchronize()
    calls = []

    def refuse(nbytes, ctx):
        calls.append(nbytes)
        return None

    a, f = ALLOC(refuse), FREE(lambda ptr, ctx: None)
    assert hz.lib.hz_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p),
                                   None) == 0
    try:
        free0, _ = torch.cuda.mem_get_info()
        used0 = torch.cuda.memory_allocated()
        y.fill_(complex(np.nan, np.nan))
        torch.cuda.synchronize()
        st = _noalloc(hz, med, x, y, nrhs, 1)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used1 = torch.cuda.memory_allocated()
    finally:
        assert hz.lib.hz_set_allocator(None, None, None) == 0
    assert st == 0, hz.last_error()
    assert calls == []
    assert free1 == free0 and used1 == used0, (free0, free1, used0, used1)
    assert within(rel(y.cpu().numpy(), ref), 1, "same_path")


def test_noalloc_rejects_oversized_work(hz):
    import torch
    p = S.small_problem((512, 512), 32, M=12, Mt=4, width=2)
    med, _ = media(hz, p, oracle=False)
    x = torch.zeros((1, 512, 512), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    st = _noalloc(hz, med, x, y, 1, 0)  # 512^2 * 17 * 16 B > 32 MiB
    assert st == 1
    assert "static limit" in hz.last_error()
