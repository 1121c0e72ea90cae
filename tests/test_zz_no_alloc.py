"""The allocation-free FP64 forward entry point (favest_fwd_fp64_noalloc), for callers
that cannot allocate device memory at the call site.  It must reproduce favest_fwd of
an FP64 plan to the FP64 tolerance on consecutive calls that share its static scratch
array, and refuse requests that do not fit the array.  This file is collected last so
that a failure here comes after every other test has run."""
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
    cases = [(16, 2), (100, 1), (255, 3), (16, 2)]
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


def test_noalloc_rejects_requests_beyond_its_scratch():
    assert api.favest_noalloc_scratch_bytes() == 32 << 20
    t = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(api.FavestError) as err:
        api.favest_fwd_fp64_noalloc(1023, 32, t, t, t, t)
    assert err.value.status == api.FAVEST_EINVAL
    with pytest.raises(api.FavestError):
        api.favest_fwd_fp64_noalloc(511, 2, t, t, t, t)
