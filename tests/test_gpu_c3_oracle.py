"""Parity at the full precision-form size: L = 1023 on the 1024 x 2048 Gauss-Legendre grid,
coefficients N(0,1)(l+1)^-1.5 from seed 2, every coefficient and every grid value of one
field against the FP64 oracle (separable form O3, Def. FwdVSHT eq. fwdvsht2 and
Def. AdjVSHT eq. SLvec), and O3 itself against the literal Clebsch-Gordan form O1 at the
polar rings and at the highest orders, where the recurrence's scaling and the polar patch
of the split adjoint do their work.

  * FP64 path (complex128 I/O, one field): adjoint and forward within 1e-12 normwise.
  * Split path (complex64 I/O, the bench's batch of 32, field 0 checked): adjoint within
    1e-6 of the oracle's synthesis of the same (complex64) coefficients, forward within
    1e-6 of the oracle's analysis of the same complex64 field.
  * Real-field split plan (batch 32) and the generic-length split plan at L = 1000
    (nphi = 2002 = 2 7 11 13), field 0 each, same bars.

Normwise error: max |got - ref| / max |ref| per family (the reading of "max relative
coefficient error" this library uses throughout)."""
import numpy as np
import pytest

from helpers import cidx, full_of_half, half_of_full, normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL64 = 1e-12
TOL_SPLIT = 1e-6
L3, B3 = 1023, 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def c3(orc):
    """The bench's coefficient batch (rounded to complex64, so that both paths and the oracle
    see identical values) and the oracle's synthesis of field 0 and analysis of it."""
    a, b = synthetic.coefficients(L3, B3, seed=2, decay=1.5)
    a = a.astype(np.complex64).astype(np.complex128)
    b = b.astype(np.complex64).astype(np.complex128)
    x, W, _, phi = orc.grid(L3)
    rt, rp = orc.adj_sep(L3, x, a[0], b[0], len(phi))
    ra, rb = orc.fwd_sep(L3, x, W, rt, rp)
    return {"a": a, "b": b, "x": x, "W": W, "rt": rt, "rp": rp, "ra": ra, "rb": rb}


def test_fp64_path_full_size_vs_oracle(orc, c3):
    """FP64 path, complex128, one field: the adjoint's every grid value and the forward's
    every coefficient (of the oracle's own field) within 1e-12."""
    a, b = c3["a"][:1], c3["b"][:1]
    plan = api.Plan(L3, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    tt, tp = plan.adj(_dev(a, torch.complex128), _dev(b, torch.complex128))
    ga, gb = plan.fwd(_dev(c3["rt"][None], torch.complex128), _dev(c3["rp"][None], torch.complex128))
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert normwise_err(_host(tt)[0].ravel(), c3["rt"].ravel()) < TOL64
    assert normwise_err(_host(tp)[0].ravel(), c3["rp"].ravel()) < TOL64
    ra, rb = c3["ra"], c3["rb"]
    assert normwise_err(_host(ga)[0], ra) < TOL64
    assert normwise_err(_host(gb)[0], rb) < TOL64
    # the oracle's analysis of its own synthesis recovers the drawn coefficients
    assert normwise_err(ra, a[0]) < TOL64 and normwise_err(rb, b[0]) < TOL64
    plan.close()


def test_oracle_o3_vs_literal_at_poles_and_high_orders(orc, c3):
    """O3 against O1 at L = 1023 where the work is hardest: the rings nearest the poles
    (j = 0, 1, L-1, L) and coefficients of orders |m| >= 1000 (the sectoral start far below
    the FP64 range at the polar rings), so that the full-size reference is pinned by an
    independent evaluation, not only by its small-L pins."""
    x = c3["x"]
    nphi = 2 * (L3 + 1)
    js = np.array([0, 0, 1, 1, L3 - 1, L3 - 1, L3, L3], dtype=np.int32)
    ks = np.array([0, 777, 5, 2000, 1024, 3, 11, 2047], dtype=np.int32)
    lt, lp, nr = orc.adj_literal_grid_points(L3, L3 + 1, nphi, x, c3["a"][0], c3["b"][0], js, ks)
    scale = max(np.max(np.abs(c3["rt"])), np.max(np.abs(c3["rp"])))
    # measured 4.3e-14 on x86-64; the FP64 bar leaves room for other rounding orders
    assert np.max(np.abs(c3["rt"][js, ks] - lt)) < TOL64 * scale
    assert np.max(np.abs(c3["rp"][js, ks] - lp)) < TOL64 * scale
    assert np.max(np.abs(nr)) < 1e-13 * scale          # tangent field: no normal component
    ls = np.array([1000, 1001, 1010, 1023, 1023, 1023, 1022, 1005], dtype=np.int32)
    ms = np.array([1000, -1000, 1004, 1023, -1023, 1001, -1017, 1005], dtype=np.int32)
    ra, rb = c3["ra"], c3["rb"]
    sa, sb = orc.fwd_literal_grid_coefs(L3, x, c3["W"], c3["rt"], c3["rp"], ls, ms)
    idx = cidx(ls, ms)
    assert np.max(np.abs(ra[idx] - sa)) < 1e-13 * np.max(np.abs(ra))
    assert np.max(np.abs(rb[idx] - sb)) < 1e-13 * np.max(np.abs(rb))


def test_split_path_full_size_vs_oracle(orc, c3):
    """Split path in the bench's launch configuration (batch 32, complex64, the λ operand
    shared by the adjoint and forward calls of the step): field 0's adjoint against the
    oracle's synthesis, and the forward of that complex64 field against the oracle's
    analysis of the same complex64 values."""
    plan = api.Plan(L3, B3, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    plan.tune()
    da, db = _dev(c3["a"], torch.complex64), _dev(c3["b"], torch.complex64)
    tt, tp = plan.adj(da, db, share_lambda=True)
    ga, gb = plan.fwd(tt, tp, share_lambda=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ht, hp = _host(tt)[0], _host(tp)[0]
    assert normwise_err(ht.ravel(), c3["rt"].ravel()) < TOL_SPLIT
    assert normwise_err(hp.ravel(), c3["rp"].ravel()) < TOL_SPLIT
    ra, rb = orc.fwd_sep(L3, c3["x"], c3["W"], ht, hp)
    assert normwise_err(_host(ga)[0], ra) < TOL_SPLIT
    assert normwise_err(_host(gb)[0], rb) < TOL_SPLIT
    plan.close()


def test_split_real_fields_full_size_vs_oracle(orc):
    """Real-field split plan at L = 1023, batch 32: field 0's real synthesis against the
    oracle's synthesis of the Hermitian extension (whose imaginary part is zero to
    rounding), and the half spectrum of its forward against the oracle's analysis."""
    L = L3
    ah, bh = synthetic.half_coefficients(L, B3, seed=2, decay=1.5)
    ah = ah.astype(np.complex64)
    bh = bh.astype(np.complex64)
    plan = api.Plan(L, B3, api.FAVEST_BF16X6, api.FAVEST_IO_R32)
    tt, tp = plan.adj(_dev(ah, torch.complex64), _dev(bh, torch.complex64), share_lambda=True)
    ga, gb = plan.fwd(tt, tp, share_lambda=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    fa = full_of_half(ah[0].astype(np.complex128), L)
    fb = full_of_half(bh[0].astype(np.complex128), L)
    rt, rp = orc.adj_sep(L, x, fa, fb, len(phi))
    assert np.max(np.abs(rt.imag)) < 1e-13 * np.max(np.abs(rt.real))
    ht = tt[0].cpu().numpy().astype(np.float64)
    hp = tp[0].cpu().numpy().astype(np.float64)
    assert normwise_err(ht.ravel(), rt.real.ravel()) < TOL_SPLIT
    assert normwise_err(hp.ravel(), rp.real.ravel()) < TOL_SPLIT
    ra, rb = orc.fwd_sep(L, x, W, ht.astype(np.complex128), hp.astype(np.complex128))
    assert normwise_err(_host(ga)[0], half_of_full(ra, L)) < TOL_SPLIT
    assert normwise_err(_host(gb)[0], half_of_full(rb, L)) < TOL_SPLIT
    plan.close()


def test_split_generic_length_L1000_vs_oracle(orc):
    """The paper's nearest timing degree, L = 1000 (nphi = 2002 = 2 7 11 13: the generic
    mixed-radix DFT stages), batch 32: field 0 against the oracle, both directions."""
    L, B = 1000, 32
    a, b = synthetic.coefficients(L, B, seed=2, decay=1.5)
    a = a.astype(np.complex64).astype(np.complex128)
    b = b.astype(np.complex64).astype(np.complex128)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    tt, tp = plan.adj(_dev(a, torch.complex64), _dev(b, torch.complex64), share_lambda=True)
    ga, gb = plan.fwd(tt, tp, share_lambda=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    x, W, _, phi = orc.grid(L)
    rt, rp = orc.adj_sep(L, x, a[0], b[0], len(phi))
    ht, hp = _host(tt)[0], _host(tp)[0]
    assert normwise_err(ht.ravel(), rt.ravel()) < TOL_SPLIT
    assert normwise_err(hp.ravel(), rp.ravel()) < TOL_SPLIT
    ra, rb = orc.fwd_sep(L, x, W, ht, hp)
    assert normwise_err(_host(ga)[0], ra) < TOL_SPLIT
    assert normwise_err(_host(gb)[0], rb) < TOL_SPLIT
    plan.close()
