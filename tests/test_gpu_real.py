"""Real-field mode of the split-precision path (FAVEST_IO_R32): real float32 field
components, half-spectrum complex64 coefficients (orders m >= 0; real fields have
a_{l,-m} = (-1)^m conj(a_lm), Sec. 3 takes T_k in R^3).  Bar: normwise max relative
error <= 1e-6 per field and family against the FP64 complex path (GPU) and the oracle
on the same float32-rounded input, as for the complex form."""
import numpy as np
import pytest

from helpers import full_of_half, half_of_full, hidx, normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _f32(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.float32).cuda().contiguous()


def _c64(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex64).cuda().contiguous()


def _h(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _real_input(L, B, seed):
    tt, tp = synthetic.real_grid_field(L, B, seed)
    return tt.astype(np.float32).astype(np.float64), tp.astype(np.float32).astype(np.float64)


def _half_input(L, B, seed, decay=1.0):
    a, b = synthetic.half_coefficients(L, B, seed, decay=decay)
    return a.astype(np.complex64).astype(np.complex128), b.astype(np.complex64).astype(np.complex128)


# L = 16: nphi = 34 (mixed-radix FFT, rows 8-byte aligned, an equator ring);
# odd batches leave the last field pair half empty
CASES = [(1, 1), (2, 3), (16, 1), (16, 5), (31, 2), (63, 3), (100, 2), (127, 17), (255, 4), (511, 1)]


@pytest.mark.parametrize("L,B", CASES)
def test_real_fwd_vs_fp64_complex(L, B):
    tt, tp = _real_input(L, B, 500 + L)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C128)
    ra, rb = pr.fwd(_f32(tt), _f32(tp))
    ca, cb = p64.fwd(torch.as_tensor(tt + 0j).cuda(), torch.as_tensor(tp + 0j).cuda())
    torch.cuda.synchronize()
    assert pr.status() == 0 and p64.status() == 0
    ea, eb = half_of_full(_h(ca), L), half_of_full(_h(cb), L)
    assert normwise_err(_h(ra), ea) < TOL
    assert normwise_err(_h(rb), eb) < TOL
    # a_l0 and b_l0 of a real field are real
    m0 = [hidx(l, 0) for l in range(1, L + 1)]
    assert np.all(_h(ra)[:, m0].imag == 0) and np.all(_h(rb)[:, m0].imag == 0)


@pytest.mark.parametrize("L,B", CASES)
def test_real_adj_vs_fp64_complex(L, B):
    a, b = _half_input(L, B, 600 + L)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C128)
    tt, tp = pr.adj(_c64(a), _c64(b))
    fa, fb = full_of_half(a, L), full_of_half(b, L)
    ct, cp = p64.adj(torch.as_tensor(fa).cuda(), torch.as_tensor(fb).cuda())
    torch.cuda.synchronize()
    assert pr.status() == 0 and p64.status() == 0
    ct, cp = _h(ct), _h(cp)
    # the Hermitian extension synthesises a real field
    assert np.max(np.abs(ct.imag)) < 1e-12 * np.max(np.abs(ct))
    got_t = tt.cpu().numpy().astype(np.float64).reshape(B, -1)
    got_p = tp.cpu().numpy().astype(np.float64).reshape(B, -1)
    assert normwise_err(got_t, ct.real.reshape(B, -1)) < TOL
    assert normwise_err(got_p, cp.real.reshape(B, -1)) < TOL


def test_real_vs_oracle(orc):
    L, B = 31, 3
    x, W, theta, phi = orc.grid(L)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    tt, tp = _real_input(L, B, 701)
    ra, rb = pr.fwd(_f32(tt), _f32(tp))
    a, b = _half_input(L, B, 702)
    st, sp = pr.adj(_c64(a), _c64(b))
    torch.cuda.synchronize()
    for f in range(B):
        oa, ob = orc.fwd_sep(L, x, W, tt[f] + 0j, tp[f] + 0j)
        assert normwise_err(_h(ra)[f], half_of_full(oa, L)) < TOL
        assert normwise_err(_h(rb)[f], half_of_full(ob, L)) < TOL
        ot, op = orc.adj_sep(L, x, full_of_half(a[f], L), full_of_half(b[f], L), len(phi))
        assert normwise_err(st.cpu().numpy()[f].ravel().astype(np.float64), ot.real.ravel()) < TOL
        assert normwise_err(sp.cpu().numpy()[f].ravel().astype(np.float64), op.real.ravel()) < TOL


def test_real_imaginary_part_of_order_zero_is_ignored():
    """The adjoint of the Hermitian extension uses Re a_l0, Re b_l0 only."""
    L, B = 63, 2
    a, b = _half_input(L, B, 711)
    a2, b2 = a.copy(), b.copy()
    m0 = [hidx(l, 0) for l in range(1, L + 1)]
    rng = np.random.default_rng(712)
    a2[:, m0] += 1j * rng.standard_normal((B, L))
    b2[:, m0] += 1j * rng.standard_normal((B, L))
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    t1, p1 = pr.adj(_c64(a), _c64(b))
    t2, p2 = pr.adj(_c64(a2), _c64(b2))
    torch.cuda.synchronize()
    assert torch.equal(t1, t2) and torch.equal(p1, p2)


def test_real_roundtrip_and_pair_independence():
    """fwd(adj(c)) = c, and a field's result does not depend on its pair partner."""
    L, B = 255, 5
    a, b = _half_input(L, B, 721)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    tt, tp = pr.adj(_c64(a), _c64(b))
    ra, rb = pr.fwd(tt, tp)
    torch.cuda.synchronize()
    assert normwise_err(_h(ra), a) < 2 * TOL
    assert normwise_err(_h(rb), b) < 2 * TOL
    # field 2 alone (its partner, field 3, zero)
    p1 = api.Plan(L, 1, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    st, sp = p1.adj(_c64(a[2:3]), _c64(b[2:3]))
    sa, sb = p1.fwd(tt[2:3].contiguous(), tp[2:3].contiguous())
    torch.cuda.synchronize()
    # a leak between the two fields of a pair would be O(1); allow rounding-order noise
    for x, y in ((st[0], tt[2]), (sp[0], tp[2]), (sa[0], ra[2]), (sb[0], rb[2])):
        assert normwise_err(_h(x).ravel(), _h(y).ravel()) < 1e-7


@pytest.mark.parametrize("decay", [1.5, 0.5])
def test_real_l1023_vs_fp64_complex(decay):
    """L = 1023, 32 real fields (the precision workload's size): adjoint and forward of
    the split real form against the FP64 complex path on the same input, 4 sampled
    fields (including the last, which pairs with field 30)."""
    L, B = 1023, 32
    a, b = _half_input(L, B, 731, decay=decay)
    pr = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    tt, tp = pr.adj(_c64(a), _c64(b))
    ra, rb = pr.fwd(tt, tp)
    torch.cuda.synchronize()
    assert pr.status() == 0
    pick = [0, 7, 30, 31]
    p64 = api.Plan(L, len(pick), api.FAVEST_FP64, api.FAVEST_IO_C128)
    fa = torch.as_tensor(full_of_half(a[pick], L)).cuda()
    fb = torch.as_tensor(full_of_half(b[pick], L)).cuda()
    ct, cp = p64.adj(fa, fb)
    xt = tt[pick].to(torch.float64).to(torch.complex128).contiguous()
    xp = tp[pick].to(torch.float64).to(torch.complex128).contiguous()
    ca, cb = p64.fwd(xt, xp)
    torch.cuda.synchronize()
    got_t = tt[pick].cpu().numpy().astype(np.float64).reshape(len(pick), -1)
    got_p = tp[pick].cpu().numpy().astype(np.float64).reshape(len(pick), -1)
    assert normwise_err(got_t, _h(ct).real.reshape(len(pick), -1)) < TOL
    assert normwise_err(got_p, _h(cp).real.reshape(len(pick), -1)) < TOL
    assert normwise_err(_h(ra)[pick], half_of_full(_h(ca), L)) < TOL
    assert normwise_err(_h(rb)[pick], half_of_full(_h(cb), L)) < TOL


# ---------------------------------------------------------------------------
# FP64 path on real fields (FAVEST_IO_R64 and FAVEST_IO_R32): bar 1e-12 against the FP64
# complex path on the same input
# ---------------------------------------------------------------------------
def _f64(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.float64).cuda().contiguous()


def _c128(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex128).cuda().contiguous()


@pytest.mark.parametrize("L,B", [(1, 1), (2, 3), (16, 5), (31, 2), (100, 3), (255, 4)])
def test_fp64_real_vs_complex(L, B):
    tt, tp = synthetic.real_grid_field(L, B, 1300 + L)
    a, b = synthetic.half_coefficients(L, B, 1400 + L)
    pr = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_R64)
    pc = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C128)
    ra, rb = pr.fwd(_f64(tt), _f64(tp))
    ca, cb = pc.fwd(_c128(tt + 0j), _c128(tp + 0j))
    st, sp = pr.adj(_c128(a), _c128(b))
    ct, cp = pc.adj(_c128(full_of_half(a, L)), _c128(full_of_half(b, L)))
    torch.cuda.synchronize()
    assert pr.status() == 0 and pc.status() == 0
    assert normwise_err(_h(ra), half_of_full(_h(ca), L)) < 1e-12
    assert normwise_err(_h(rb), half_of_full(_h(cb), L)) < 1e-12
    assert normwise_err(st.cpu().numpy().reshape(B, -1), _h(ct).real.reshape(B, -1)) < 1e-12
    assert normwise_err(sp.cpu().numpy().reshape(B, -1), _h(cp).real.reshape(B, -1)) < 1e-12
    # roundtrip on the exact grid, and R32 I/O (float fields, complex64 coefficients)
    a2, b2 = pr.fwd(st, sp)
    p32 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_R32)
    t32, q32 = p32.adj(_c64(a), _c64(b))
    torch.cuda.synchronize()
    assert normwise_err(_h(a2), a) < 1e-12 and normwise_err(_h(b2), b) < 1e-12
    assert normwise_err(t32.cpu().numpy().astype(np.float64).reshape(B, -1), st.cpu().numpy().reshape(B, -1)) < 1e-6


def test_fp64_real_vs_oracle(orc):
    L, B = 24, 2
    x, W, theta, phi = orc.grid(L)
    tt, tp = synthetic.real_grid_field(L, B, 1500)
    pr = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_R64)
    ra, rb = pr.fwd(_f64(tt), _f64(tp))
    a, b = synthetic.half_coefficients(L, B, 1501)
    st, sp = pr.adj(_c128(a), _c128(b))
    torch.cuda.synchronize()
    for f in range(B):
        oa, ob = orc.fwd_sep(L, x, W, tt[f] + 0j, tp[f] + 0j)
        assert normwise_err(_h(ra)[f], half_of_full(oa, L)) < 1e-12
        assert normwise_err(_h(rb)[f], half_of_full(ob, L)) < 1e-12
        ot, op = orc.adj_sep(L, x, full_of_half(a[f], L), full_of_half(b[f], L), len(phi))
        assert normwise_err(st.cpu().numpy()[f].ravel(), ot.real.ravel()) < 1e-12
        assert normwise_err(sp.cpu().numpy()[f].ravel(), op.real.ravel()) < 1e-12
