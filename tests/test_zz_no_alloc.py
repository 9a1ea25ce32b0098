"""The allocation-free preconditioner entry point, called through the C ABI,
gives the same result as the plan-based hz_apply_preconditioner, on two
calls in a row (the shared scratch keeps the previous call's contents), in
both precisions, and refuses work that does not fit its fixed scratch."""
import ctypes

import numpy as np
import pytest

from paper_2409_16172_gb300 import synth as S

from gpu_util import hz_module, media, rel

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
    for prec, tol in ((0, 1e-10), (1, 5e-5)):
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
            assert rel(got, ref) <= tol, (prec, call, rel(got, ref))


def test_noalloc_rejects_oversized_work(hz):
    import torch
    p = S.small_problem((512, 512), 32, M=12, Mt=4, width=2)
    med, _ = media(hz, p, oracle=False)
    x = torch.zeros((1, 512, 512), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    st = _noalloc(hz, med, x, y, 1, 0)  # 512^2 * 17 * 16 B > 32 MiB
    assert st == 1
    assert "static limit" in hz.last_error()
