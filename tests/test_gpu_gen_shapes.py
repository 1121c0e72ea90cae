"""Every generator shape the tuner offers, applied with favest_plan_set_gen_shape, in both
directions of a real split-precision plan: results bit-identical to the untuned shape; the
setter's checks on real plans (unknown shapes rejected, FP64 plans accept and ignore)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

SHAPES = [(lt, mb, nj) for nj in (2, 1) for lt, mb in ((128, 1), (64, 1), (32, 1), (128, 2), (64, 2), (32, 2),
                                                        (32, 4))]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


@pytest.mark.parametrize("L,B", [(63, 2), (300, 1)])
def test_every_shape_both_directions_bit_identical(L, B):
    a, b = synthetic.coefficients(L, B, seed=4100 + L, decay=1.0)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    ca = torch.as_tensor(a).to(torch.complex64).cuda()
    cb = torch.as_tensor(b).to(torch.complex64).cuda()
    t0, p0 = plan.adj(ca, cb)
    f0, g0 = plan.fwd(t0, p0)
    for sh in SHAPES:
        plan.set_gen_shape(*sh)
        assert plan.gen_shape() == sh[:2] and plan.gen_chains() == sh[2]
        t1, p1 = plan.adj(ca, cb)
        f1, g1 = plan.fwd(t0, p0)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert torch.equal(t0, t1) and torch.equal(p0, p1), sh
        assert torch.equal(f0, f1) and torch.equal(g0, g1), sh
    with pytest.raises(api.FavestError):
        plan.set_gen_shape(96, 1, 2)
    plan.close()
    p64 = api.Plan(16, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    p64.set_gen_shape(32, 4, 1)
    with pytest.raises(api.FavestError):
        p64.set_gen_shape(32, 4, 3)
    p64.close()
