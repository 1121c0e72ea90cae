"""Failure detection on the GPU without a fault: every device-side wait of the tensor-core
GEMM is bounded; when one runs out the kernel records FAVEST_ETIMEOUT in the plan's
status word, releases its tensor memory and returns, and the context stays usable.  The
self-test entry point launches the GEMM with its operand loads switched off (a barrier
that nothing completes) and a small poll bound."""
import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402


def test_wait_timeout_reports_status_and_context_survives(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)
    L, B = 63, 2
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    for limit in (1 << 12, 1 << 16):
        st, ms = plan.selftest_wait_timeout(limit)
        assert st == api.FAVEST_ETIMEOUT, (st, api.favest_strerror(st))
        assert ms > 0.0
    assert plan.status() == 0          # the status word was read and cleared
    # the same plan and context still compute correctly
    a, b = synthetic.coefficients(L, B, seed=77)
    a = a.astype(np.complex64)
    b = b.astype(np.complex64)
    tt, tp = plan.adj(torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, theta, phi = orc.grid(L)
    rt, rp = orc.adj_sep(L, x, a[1].astype(np.complex128), b[1].astype(np.complex128), len(phi))
    assert normwise_err(tt[1].cpu().numpy().astype(np.complex128).ravel(), rt.ravel()) < 1e-6
    assert normwise_err(tp[1].cpu().numpy().astype(np.complex128).ravel(), rp.ravel()) < 1e-6


def test_selftest_rejects_fp64_plans():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    plan = api.Plan(16, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    st, _ = plan.selftest_wait_timeout(1 << 10)
    assert st == api.FAVEST_EUNSUPPORTED
