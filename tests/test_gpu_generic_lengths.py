"""GPU parity of the split-precision path at longitude counts n = 2(L+1) that are not powers
of two: the FP32 DFT then runs its generic mixed-radix stages (radix-4/2 butterflies, register
butterflies for the odd primes 3..13, warp-parallel butterflies for larger primes).  Each
degree below puts a different set of radices on those stages.  Checked against the FP64 path
on the same complex64 input (adjoint and forward), bar 1e-6 normwise, and for the roundtrip
of bandlimited coefficients."""
import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL = 1e-6

# L -> n = 2(L+1): 34 = 2*17, 110 = 2*5*11, 140 = 4*5*7, 156 = 4*3*13, 186 = 2*3*31,
# 250 = 2*5^3, 294 = 2*3*7^2, 2002 = 2*7*11*13
CASES = [(16, 2), (54, 3), (69, 2), (77, 2), (92, 1), (124, 2), (146, 1), (1000, 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _c64(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex64).cuda().contiguous()


def _h(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("L,B", CASES)
def test_split_vs_fp64_generic_lengths(L, B):
    a, b = synthetic.coefficients(L, B, seed=2100 + L, decay=1.0)
    ps = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
    ca, cb = _c64(a), _c64(b)
    st, sp = ps.adj(ca, cb)
    rt, rp = p64.adj(ca, cb)
    torch.cuda.synchronize()
    assert ps.status() == 0 and p64.status() == 0
    assert normwise_err(_h(st), _h(rt)) < TOL
    assert normwise_err(_h(sp), _h(rp)) < TOL
    # forward on the same (complex64) field
    fa, fb = ps.fwd(rt, rp)
    ga, gb = p64.fwd(rt, rp)
    torch.cuda.synchronize()
    assert ps.status() == 0
    assert normwise_err(_h(fa), _h(ga)) < TOL
    assert normwise_err(_h(fb), _h(gb)) < TOL
    # bandlimited roundtrip through the split path alone
    assert normwise_err(_h(fa), a) < 2 * TOL
    assert normwise_err(_h(fb), b) < 2 * TOL
