"""Degrees above 1023 and longitude lengths with prime factors above 128 (the paper's timing
degrees, Table 3: nphi = 2(L+1) = 502 = 2 251, 1002 = 2 3 167, 1502 = 2 751, 4502 = 2 2251),
against the FP64 oracle (Def. FwdVSHT eq. fwdvsht2, Def. AdjVSHT eq. SLvec).

At L >= 2047 the oracle is run on a strided subset of the orders: coefficients are drawn only
on the orders m = mstart - L + k mstep, so the oracle's synthesis restricted to those orders
is the whole field, and its analysis of any field restricted to those orders gives exactly
those coefficients (the partition is pinned on the CPU by
test_strided_order_subsets_partition_the_transforms).  Bars: 1e-12 normwise for the FP64
path, 1e-6 for the split path; sampled coefficients also against the literal form O1."""
import numpy as np
import pytest

from helpers import cidx, full_of_half, half_of_full, normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL64 = 1e-12
TOL_SPLIT = 1e-6
MSTEP = 16


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _subset_coefficients(L, B, seed, mstart, decay=1.0):
    """Drawn coefficients with every order outside m = mstart - L + k MSTEP set to zero."""
    a, b = synthetic.coefficients(L, B, seed=seed, decay=decay)
    ms = synthetic.orders(L)
    off = ((ms + L - mstart) % MSTEP) != 0
    a[:, off] = 0.0
    b[:, off] = 0.0
    return a, b, ~off


@pytest.mark.parametrize("L,io", [(2047, api.FAVEST_IO_C128), (2250, api.FAVEST_IO_C128)])
def test_fp64_above_1023_vs_oracle_subset(orc, L, io):
    """FP64 path, one field, L = 2047 (nphi = 4096) and L = 2250 (nphi = 4502 = 2 2251, a
    prime radix in the FP64 Stockham DFT): every grid value against the oracle, the forward
    of that field on the drawn orders against the oracle, the roundtrip, and sampled
    coefficients against O1."""
    mstart = 5
    a, b, on = _subset_coefficients(L, 1, seed=L, mstart=mstart)
    plan = api.Plan(L, 1, api.FAVEST_FP64, io)
    tt, tp = plan.adj(_dev(a, torch.complex128), _dev(b, torch.complex128))
    ga, gb = plan.fwd(tt, tp)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    rt, rp = orc.adj_sep_orders(L, x, a[0], b[0], len(phi), mstart, MSTEP)
    ht, hp = _host(tt)[0], _host(tp)[0]
    assert normwise_err(ht.ravel(), rt.ravel()) < TOL64
    assert normwise_err(hp.ravel(), rp.ravel()) < TOL64
    ra, rb = orc.fwd_sep_orders(L, x, W, ht, hp, mstart, MSTEP)
    ha, hb = _host(ga)[0], _host(gb)[0]
    assert normwise_err(ha[on], ra[on]) < TOL64 and normwise_err(hb[on], rb[on]) < TOL64
    assert normwise_err(ha, a[0]) < TOL64 and normwise_err(hb, b[0]) < TOL64
    ls = np.array([L, L, L - 1, 1000, 3 * L // 4], dtype=np.int32)
    ms = np.array([mstart - L, mstart - L + 16 * 100, mstart - L + 16 * 120, mstart - L + 16 * 80,
                   mstart - L + 16 * 60], dtype=np.int32)
    sa, sb = orc.fwd_literal_grid_coefs(L, x, W, ht, hp, ls, ms)
    idx = cidx(ls, ms)
    assert np.max(np.abs(ha[idx] - sa)) < TOL64 * np.max(np.abs(ra))
    assert np.max(np.abs(hb[idx] - sb)) < TOL64 * np.max(np.abs(rb))
    plan.close()


@pytest.mark.parametrize("L,B", [(2047, 8), (2250, 4)])
def test_split_above_1023_vs_oracle_subset(orc, L, B):
    """Split path at L = 2047 (power-of-two DFT of 4096 points through the generic engine) and
    L = 2250 (Bluestein stage for the radix 2251): field 0 of the batch against the oracle
    in both directions."""
    mstart = 11
    a, b, on = _subset_coefficients(L, B, seed=L + 1, mstart=mstart, decay=1.5)
    a = a.astype(np.complex64).astype(np.complex128)
    b = b.astype(np.complex64).astype(np.complex128)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    tt, tp = plan.adj(_dev(a, torch.complex64), _dev(b, torch.complex64), share_lambda=True)
    ga, gb = plan.fwd(tt, tp, share_lambda=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    rt, rp = orc.adj_sep_orders(L, x, a[0], b[0], len(phi), mstart, MSTEP)
    ht, hp = _host(tt)[0], _host(tp)[0]
    assert normwise_err(ht.ravel(), rt.ravel()) < TOL_SPLIT
    assert normwise_err(hp.ravel(), rp.ravel()) < TOL_SPLIT
    ra, rb = orc.fwd_sep_orders(L, x, W, ht, hp, mstart, MSTEP)
    ha, hb = _host(ga)[0], _host(gb)[0]
    assert normwise_err(ha[on], ra[on]) < TOL_SPLIT and normwise_err(hb[on], rb[on]) < TOL_SPLIT
    assert normwise_err(ha, a[0]) < TOL_SPLIT and normwise_err(hb, b[0]) < TOL_SPLIT
    plan.close()


@pytest.mark.parametrize("L", [150, 250, 500, 750])
def test_split_bluestein_lengths_vs_oracle(orc, L):
    """Split path at degrees whose nphi has a prime factor above 128 (151, 251, 167, 751):
    the whole transform of two fields against the oracle, both directions."""
    B = 2
    a, b = synthetic.coefficients(L, B, seed=3 * L, decay=1.0)
    a = a.astype(np.complex64).astype(np.complex128)
    b = b.astype(np.complex64).astype(np.complex128)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    tt, tp = plan.adj(_dev(a, torch.complex64), _dev(b, torch.complex64))
    ga, gb = plan.fwd(tt, tp)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    for f in range(B):
        rt, rp = orc.adj_sep(L, x, a[f], b[f], len(phi))
        ht, hp = _host(tt)[f], _host(tp)[f]
        assert normwise_err(ht.ravel(), rt.ravel()) < TOL_SPLIT
        assert normwise_err(hp.ravel(), rp.ravel()) < TOL_SPLIT
        ra, rb = orc.fwd_sep(L, x, W, ht, hp)
        assert normwise_err(_host(ga)[f], ra) < TOL_SPLIT
        assert normwise_err(_host(gb)[f], rb) < TOL_SPLIT
    plan.close()


def test_split_bluestein_real_fields_vs_oracle(orc):
    """Real-field split plan at L = 250 (nphi = 502 = 2 251): the real DFTs through the
    Bluestein stage, field 1 of 3 against the oracle."""
    L, B = 250, 3
    ah, bh = synthetic.half_coefficients(L, B, seed=77)
    ah = ah.astype(np.complex64)
    bh = bh.astype(np.complex64)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    tt, tp = plan.adj(_dev(ah, torch.complex64), _dev(bh, torch.complex64))
    ga, gb = plan.fwd(tt, tp)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    f = 1
    rt, rp = orc.adj_sep(L, x, full_of_half(ah[f].astype(np.complex128), L),
                         full_of_half(bh[f].astype(np.complex128), L), len(phi))
    ht = tt[f].cpu().numpy().astype(np.float64)
    hp = tp[f].cpu().numpy().astype(np.float64)
    assert normwise_err(ht.ravel(), rt.real.ravel()) < TOL_SPLIT
    assert normwise_err(hp.ravel(), rp.real.ravel()) < TOL_SPLIT
    ra, rb = orc.fwd_sep(L, x, W, ht.astype(np.complex128), hp.astype(np.complex128))
    assert normwise_err(_host(ga)[f], half_of_full(ra, L)) < TOL_SPLIT
    assert normwise_err(_host(gb)[f], half_of_full(rb, L)) < TOL_SPLIT
    plan.close()


def test_degree_limit():
    with pytest.raises(api.FavestError) as e:
        api.Plan(2560, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    assert e.value.status == api.FAVEST_EUNSUPPORTED
