"""Tangent Field A of Sec. 5.2 (T = L s1 + grad* v1, eq. RosbyHaurwitz; band-limited to
degree 6): the paper's Gauss-Legendre experiments on the GPU paths.

  Table 1 (GL row): relative L2 reconstruction error |T - T^rec|_2 / |T|_2 with
      T^rec = AdjVSHT(FwdVSHT(T)), L = 10, 30, 50, 100, 120, 150;
  Table 2 (GL row, L = 40): T0 -> coefficients c0 -> T1 -> c1 -> T2 with sup norms
      |T1 - T0|, |T2 - T0|, |T2 - T1| and max |c1 - c0|.

T0 is sampled on each grid by the oracle from the field's exact coefficients (an FP64
evaluation independent of the CUDA path); the L2 norm is the grid's quadrature norm.
The paper's values (MATLAB + NFFT) are the bar for the FP64 path: the GL rule
reproduces a field of degree 6 exactly, so what remains is rounding, and ours must
not exceed theirs.  The split form is held to its own 1e-6 bar."""
import math

import numpy as np
import pytest

from helpers import cidx, read_field_a

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _exact(L, coefs):
    K = L * L + 2 * L
    a = np.zeros(K, complex)
    b = np.zeros(K, complex)
    for fam, l, m, v in coefs:
        (a if fam == "a" else b)[cidx(l, m)] = v
    return a, b


def _field(orc, L, coefs):
    x, W, theta, phi = orc.grid(L)
    a, b = _exact(L, coefs)
    tt, tp = orc.adj_sep(L, x, a, b, len(phi))
    w = np.repeat(W, len(phi)) * (2 * math.pi / len(phi))
    return tt, tp, w


def _l2_rel(tt, tp, rt, rp, w):
    num = np.sum(w * (np.abs(rt - tt) ** 2 + np.abs(rp - tp) ** 2).ravel())
    den = np.sum(w * (np.abs(tt) ** 2 + np.abs(tp) ** 2).ravel())
    return math.sqrt(num / den)


def _dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda().view(1, *x.shape).contiguous()


def _host(t):
    return t.detach().cpu().numpy()[0].astype(np.complex128)


@pytest.mark.parametrize("L", [10, 30, 50, 100, 120, 150])
def test_table1_gl_row(orc, L):
    coefs, t1, _ = read_field_a()
    tt, tp, w = _field(orc, L, coefs)
    p64 = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    a, b = p64.fwd(_dev(tt, torch.complex128), _dev(tp, torch.complex128))
    rt, rp = p64.adj(a, b)
    torch.cuda.synchronize()
    err64 = _l2_rel(tt, tp, _host(rt), _host(rp), w)
    assert err64 <= t1[L], (L, err64, t1[L])
    # the coefficients themselves are the exact ones
    ea, eb = _exact(L, coefs)
    assert max(np.max(np.abs(_host(a) - ea)), np.max(np.abs(_host(b) - eb))) < 1e-13
    # split precision (complex64 fields); nphi with a prime factor above 128 (L = 150:
    # 2 151) runs that stage through the Bluestein convolution
    p16 = api.Plan(L, 1, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    a16, b16 = p16.fwd(_dev(tt, torch.complex64), _dev(tp, torch.complex64))
    r16t, r16p = p16.adj(a16, b16)
    torch.cuda.synchronize()
    assert _l2_rel(tt, tp, _host(r16t), _host(r16p), w) < 1e-6


def test_table2_gl_row(orc):
    coefs, _, t2 = read_field_a()
    L = 40
    tt, tp, _ = _field(orc, L, coefs)
    p64 = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    T0 = (_dev(tt, torch.complex128), _dev(tp, torch.complex128))
    c0 = p64.fwd(*T0)
    T1 = p64.adj(*c0)
    c1 = p64.fwd(*T1)
    T2 = p64.adj(*c1)
    torch.cuda.synchronize()

    def sup(u, v):
        return max(np.max(np.abs(_host(u[0]) - _host(v[0]))), np.max(np.abs(_host(u[1]) - _host(v[1]))))
    got = [sup(T1, T0), sup(T2, T0), sup(T2, T1), sup(c1, c0)]
    for g, bound in zip(got, t2):
        assert g <= bound, (got, t2)
