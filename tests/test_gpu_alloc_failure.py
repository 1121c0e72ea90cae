"""Device allocation failure during creation (the hook favest_debug_fail_alloc): every
allocation of every kind of plan is failed in turn; creation must return FAVEST_ENOMEM and
leave the device's free memory exactly as it found it (nothing leaked on any error path), and
the next creation must succeed and compute correct results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)
    yield
    api.lib().favest_debug_fail_alloc(-1)


def _makers():
    X = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.6, 0.0, 0.8]])
    return {
        "fp64": lambda: api.Plan(40, 2, api.FAVEST_FP64, api.FAVEST_IO_C128),
        "split": lambda: api.Plan(63, 4, api.FAVEST_BF16X6, api.FAVEST_IO_C64),
        "split_real": lambda: api.Plan(95, 3, api.FAVEST_BF16X6, api.FAVEST_IO_R32),
        "split_bluestein": lambda: api.Plan(150, 1, api.FAVEST_BF16X6, api.FAVEST_IO_C64),
        "cg": lambda: api.CgPlan(20, 2),
        "scatter": lambda: api.ScatterPlan(12, X, None, batch=1),
        "batch": lambda: api.BatchPlan([15, 31, 31], graph=False),
    }


@pytest.mark.parametrize("kind", list(_makers()))
def test_every_allocation_failure_is_clean(kind):
    lib = api.lib()
    make = _makers()[kind]
    lib.favest_debug_fail_alloc(-1)
    obj = make()
    n = lib.favest_debug_alloc_count()
    obj.close()
    torch.cuda.synchronize()
    assert n >= 3
    for k in range(n):
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        lib.favest_debug_fail_alloc(k)
        with pytest.raises(api.FavestError) as e:
            make()
        lib.favest_debug_fail_alloc(-1)
        assert e.value.status == api.FAVEST_ENOMEM, (kind, k)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (kind, k, free0 - free1)
    # and the device is fine afterwards
    if kind == "split":
        p = make()
        a, b = synthetic.coefficients(63, 4, seed=1)
        da = torch.as_tensor(a).to(torch.complex64).cuda()
        db = torch.as_tensor(b).to(torch.complex64).cuda()
        tt, tp = p.adj(da, db)
        a2, b2 = p.fwd(tt, tp)
        torch.cuda.synchronize()
        assert p.status() == 0
        assert float((a2 - da).abs().max() / da.abs().max()) < 1e-6
        p.close()
