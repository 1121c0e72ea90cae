"""The allocation-free FP64 forward entry point (favest_fwd_fp64_noalloc), for callers
that cannot allocate device memory at the call site.  It must reproduce favest_fwd of
an FP64 plan to the FP64 tolerance on consecutive calls that share its static scratch
array, allocate no device memory, and refuse requests that do not fit the array.  This
file is collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def test_noalloc_matches_planned_fwd_on_consecutive_calls():
    # (511, 1) is the largest request the 32 MB array holds: the device-side grid and
    # table kernels at their largest size
    cases = [(16, 2), (100, 1), (255, 3), (511, 1), (16, 2)]
    for L, B in cases:
        tt, tp = synthetic.grid_field(L, B, seed=500 + L)
        dtt = torch.as_tensor(tt).cuda()
        dtp = torch.as_tensor(tp).cuda()
        plan = api.Plan(L, B)
        ra, rb = plan.fwd(dtt, dtp)
        torch.cuda.synchronize()
        ra, rb = ra.cpu().numpy(), rb.cpu().numpy()
        for _ in range(2):
            a = torch.full((B, L * L + 2 * L), float("nan"), dtype=torch.complex128, device="cuda")
            b = torch.full_like(a, float("nan"))
            api.favest_fwd_fp64_noalloc(L, B, dtt, dtp, a, b)
            torch.cuda.synchronize()
            assert normwise_err(a.cpu().numpy(), ra) < 1e-12
            assert normwise_err(b.cpu().numpy(), rb) < 1e-12
        plan.close()


def test_noalloc_allocates_no_device_memory():
    """After one call, further calls leave the device's free memory unchanged (inputs and
    outputs allocated beforehand)."""
    L, B = 127, 2
    tt, tp = synthetic.grid_field(L, B, seed=77)
    dtt = torch.as_tensor(tt).cuda()
    dtp = torch.as_tensor(tp).cuda()
    a = torch.empty((B, L * L + 2 * L), dtype=torch.complex128, device="cuda")
    b = torch.empty_like(a)
    api.favest_fwd_fp64_noalloc(L, B, dtt, dtp, a, b)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        api.favest_fwd_fp64_noalloc(L, B, dtt, dtp, a, b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_requests_beyond_its_scratch():
    """Through the C ABI directly: sizes beyond the array are refused before any launch
    (the small buffer is never touched)."""
    assert api.favest_noalloc_scratch_bytes() == 32 << 20
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = api.lib()
    for L, B in [(1023, 32), (1023, 1), (511, 2), (2047, 1), (16, 5000), (16, 0), (0, 1)]:
        assert lib.favest_fwd_fp64_noalloc(L, B, p, p, p, p, s) == api.FAVEST_EINVAL, (L, B)
    torch.cuda.synchronize()


def test_noalloc_binding_checks_tensors():
    """The Python binding refuses tensors the C entry point would misread."""
    L, B = 16, 1
    good = torch.zeros((B, L + 1, 2 * (L + 1)), dtype=torch.complex128, device="cuda")
    coef = torch.zeros((B, L * L + 2 * L), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        api.favest_fwd_fp64_noalloc(L, B, good.to(torch.complex64), good, coef, coef)
    with pytest.raises(ValueError):
        api.favest_fwd_fp64_noalloc(L, B, good, good.cpu(), coef, coef)
    with pytest.raises(ValueError):
        api.favest_fwd_fp64_noalloc(L, B, good, good, coef[:, :-1], coef)
    with pytest.raises(ValueError):
        api.favest_fwd_fp64_noalloc(L, B, good, good.transpose(1, 2), coef, coef)
