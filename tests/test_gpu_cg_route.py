"""GPU parity of the paper's Clebsch-Gordan route (Thm. 1, Thm. 2) on the FP64 path:
fields as Cartesian components [batch][3][nlat][nphi].  Checked against the oracle's
statement of both theorems, against the theta/phi FP64 path on the same fields (an
independent GPU computation of the same transforms), for tangency of the synthesised
fields and for the roundtrip.  Bar: 1e-12 normwise (FP64 path)."""
import ctypes

import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cg_route  # noqa: E402
from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _mesh(orc, L):
    x, W, theta, phi = orc.grid(L)
    TH, PH = np.meshgrid(theta, phi, indexing="ij")
    w = np.repeat(W, len(phi)) * (2 * np.pi / len(phi))
    return x, W, theta, phi, TH.ravel(), PH.ravel(), w


def _cart_planes(orc, th, ph, tt, tp):
    """[3][nlat][nphi] Cartesian planes of the tangent field (T_theta, T_phi)."""
    c = orc.sph_to_cart(th, ph, tt.ravel(), tp.ravel())       # npts x 3
    return np.ascontiguousarray(c.T.reshape(3, *tt.shape))


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex128).cuda().contiguous()


@pytest.mark.parametrize("L,B", [(1, 1), (2, 2), (8, 3), (16, 1), (31, 2)])
def test_cg_route_vs_oracle_theorems(orc, L, B):
    x, W, theta, phi, th, ph, w = _mesh(orc, L)
    rng = np.random.default_rng(800 + L)
    shape = (B, 3, len(theta), len(phi))
    T = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)     # any vectors, not only tangent
    cp = api.CgPlan(L, B)
    a, b = cp.fwd(_dev(T))
    ca, cb = synthetic.coefficients(L, B, seed=900 + L)
    Tr = cp.adj(_dev(ca), _dev(cb))
    torch.cuda.synchronize()
    assert cp.status() == 0
    for f in range(B):
        Tf = T[f].reshape(3, -1).T
        oa, ob = cg_route.fwd_cg(L, th, ph, w, Tf)
        assert normwise_err(a[f].cpu().numpy(), oa) < TOL
        assert normwise_err(b[f].cpu().numpy(), ob) < TOL
        oT = cg_route.adj_cg(L, ca[f], cb[f], th, ph)              # npts x 3
        assert normwise_err(Tr[f].cpu().numpy().reshape(3, -1).T.ravel(), oT.ravel()) < TOL


@pytest.mark.parametrize("L,B", [(16, 2), (63, 3), (255, 2)])
def test_cg_route_equals_theta_phi_path(orc, L, B):
    """The CG route on Cartesian components and the theta/phi path on the same tangent
    fields give the same coefficients; the CG adjoint is the theta/phi adjoint in
    Cartesian components and is tangent."""
    x, W, theta, phi, th, ph, w = _mesh(orc, L)
    tt, tp = synthetic.grid_field(L, B, seed=1000 + L)
    Tc = np.stack([_cart_planes(orc, th, ph, tt[f], tp[f]) for f in range(B)])
    cp = api.CgPlan(L, B)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C128)
    a1, b1 = cp.fwd(_dev(Tc))
    a2, b2 = p64.fwd(_dev(tt), _dev(tp))
    ca, cb = synthetic.coefficients(L, B, seed=1100 + L)
    Tcg = cp.adj(_dev(ca), _dev(cb))
    st, sp = p64.adj(_dev(ca), _dev(cb))
    torch.cuda.synchronize()
    assert normwise_err(a1.cpu().numpy(), a2.cpu().numpy()) < TOL
    assert normwise_err(b1.cpu().numpy(), b2.cpu().numpy()) < TOL
    for f in range(B):
        ref = _cart_planes(orc, th, ph, st[f].cpu().numpy(), sp[f].cpu().numpy())
        got = Tcg[f].cpu().numpy()
        assert normwise_err(got.ravel(), ref.ravel()) < TOL
        # normal component x . T of the synthesised field vanishes
        xr = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        normal = np.sum(xr * got.reshape(3, -1), axis=0)
        assert np.max(np.abs(normal)) < TOL * np.max(np.abs(got))


def test_cg_route_normal_fields_and_roundtrip(orc):
    """A purely normal field g(x) x has no tangent coefficients (Y^div, Y^curl are
    tangent), and fwd_cart(adj_cart(c)) = c on the exact grid."""
    L, B = 40, 2
    x, W, theta, phi, th, ph, w = _mesh(orc, L)
    rng = np.random.default_rng(77)
    g = rng.standard_normal((B, len(theta) * len(phi))) + 1j * rng.standard_normal((B, len(theta) * len(phi)))
    xr = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    Tn = np.stack([(xr * g[f]).reshape(3, len(theta), len(phi)) for f in range(B)])
    cp = api.CgPlan(L, B)
    a, b = cp.fwd(_dev(Tn))
    ca, cb = synthetic.coefficients(L, B, seed=78)
    ra, rb = cp.fwd(cp.adj(_dev(ca), _dev(cb)))
    torch.cuda.synchronize()
    # coefficients of a random tangent field of this amplitude are ~ |g| sqrt(4 pi / N) ~ 0.03 |g|
    assert np.max(np.abs(a.cpu().numpy())) < 1e-12 * np.max(np.abs(g))
    assert np.max(np.abs(b.cpu().numpy())) < 1e-12 * np.max(np.abs(g))
    assert normwise_err(ra.cpu().numpy(), ca) < TOL
    assert normwise_err(rb.cpu().numpy(), cb) < TOL


def test_cg_plan_rejects_other_calls():
    """A CG plan serves only the Cartesian calls, and those only CG plans."""
    cp = api.CgPlan(8, 1)
    p = api.Plan(8, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
    t = torch.zeros((1, 9, 18), dtype=torch.complex128, device="cuda")
    T = torch.zeros((1, 3, 9, 18), dtype=torch.complex128, device="cuda")
    c = torch.zeros((1, 80), dtype=torch.complex128, device="cuda")
    with pytest.raises(api.FavestError) as e1:
        api.favest_fwd(cp.handle, t, t, c, c)
    st = api.lib().favest_fwd_cart(ctypes.c_void_p(p.handle), api._ptr(T), api._ptr(c), api._ptr(c),
                                   api._stream(None))
    assert e1.value.status == api.FAVEST_EINVAL and st == api.FAVEST_EINVAL


def _rdev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.float64).cuda().contiguous()


@pytest.mark.parametrize("L,B", [(1, 1), (2, 3), (8, 2), (16, 3), (31, 1)])
def test_cg_route_real_fields_vs_oracle_theorems(orc, L, B):
    """Real fields (the paper's, Sec. 3) on the CG route: the half spectra (m >= 0) of the
    forward against the oracle's Thm. 1 on the same real field, whose full spectrum must be
    Hermitian (a_{l,-m} = (-1)^m conj a_lm, the relation the pair packing rests on); the
    adjoint of half-spectrum coefficients against the oracle's Thm. 2 of their Hermitian
    extension, which is real.  Odd batches leave the second field of the last pair empty."""
    from helpers import full_of_half, half_of_full
    x, W, theta, phi, th, ph, w = _mesh(orc, L)
    rng = np.random.default_rng(1300 + L)
    T = rng.standard_normal((B, 3, len(theta), len(phi)))
    cp = api.CgPlan(L, B, real=True)
    a, b = cp.fwd(_rdev(T))
    ha, hb = synthetic.half_coefficients(L, B, seed=1400 + L)
    Tr = cp.adj(_dev(ha), _dev(hb))
    torch.cuda.synchronize()
    assert cp.status() == 0 and Tr.dtype == torch.float64
    for f in range(B):
        oa, ob = cg_route.fwd_cg(L, th, ph, w, T[f].reshape(3, -1).T.astype(np.complex128))
        assert normwise_err(full_of_half(half_of_full(oa, L), L), oa) < TOL
        assert normwise_err(a[f].cpu().numpy(), half_of_full(oa, L)) < TOL
        assert normwise_err(b[f].cpu().numpy(), half_of_full(ob, L)) < TOL
        oT = cg_route.adj_cg(L, full_of_half(ha[f], L), full_of_half(hb[f], L), th, ph)   # npts x 3
        assert np.max(np.abs(oT.imag)) < TOL * np.max(np.abs(oT.real))
        assert normwise_err(Tr[f].cpu().numpy().reshape(3, -1).T.ravel(), oT.real.ravel()) < TOL


@pytest.mark.parametrize("L,B", [(63, 3), (255, 2)])
def test_cg_route_real_equals_complex_route_and_theta_phi(orc, L, B):
    """Real CG plans against the complex CG route on the same (real-valued) fields and
    against the real theta/phi FP64 path (FAVEST_IO_R64) on tangent fields; roundtrip."""
    from helpers import full_of_half, half_of_full
    x, W, theta, phi, th, ph, w = _mesh(orc, L)
    tt, tp = synthetic.grid_field(L, B, seed=1500 + L)
    tt, tp = tt.real.copy(), tp.real.copy()
    Tc = np.stack([_cart_planes(orc, th, ph, tt[f], tp[f]).real for f in range(B)])
    cr = api.CgPlan(L, B, real=True)
    cc = api.CgPlan(L, B)
    pr = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_R64)
    ar, br = cr.fwd(_rdev(Tc))
    ac, bc = cc.fwd(_dev(Tc))
    at, bt = pr.fwd(_rdev(tt), _rdev(tp))
    torch.cuda.synchronize()
    assert normwise_err(ar.cpu().numpy(), half_of_full(ac.cpu().numpy(), L)) < TOL
    assert normwise_err(br.cpu().numpy(), half_of_full(bc.cpu().numpy(), L)) < TOL
    assert normwise_err(ar.cpu().numpy(), at.cpu().numpy()) < TOL
    assert normwise_err(br.cpu().numpy(), bt.cpu().numpy()) < TOL
    ha, hb = synthetic.half_coefficients(L, B, seed=1600 + L)
    Tr = cr.adj(_dev(ha), _dev(hb))
    Tx = cc.adj(_dev(full_of_half(ha, L)), _dev(full_of_half(hb, L)))
    ra, rb = cr.fwd(Tr)
    torch.cuda.synchronize()
    assert normwise_err(Tr.cpu().numpy().ravel(), Tx.cpu().numpy().real.ravel()) < TOL
    assert normwise_err(ra.cpu().numpy(), ha) < TOL
    assert normwise_err(rb.cpu().numpy(), hb) < TOL


def test_cg_real_plan_arguments():
    with pytest.raises(api.FavestError) as e:
        api.CgPlan(8, 0, real=True)
    assert e.value.status == api.FAVEST_EINVAL
    h = ctypes.c_void_p()
    assert api.lib().favest_cg_plan_create_ex(8, 1, api.FAVEST_IO_C64, None, None, ctypes.byref(h)) == api.FAVEST_EINVAL
    cp = api.CgPlan(8, 5, real=True)
    assert api.lib().favest_plan_batch(ctypes.c_void_p(cp.handle)) == 5
    with pytest.raises(ValueError):
        cp.fwd(torch.zeros((5, 3, 9, 18), dtype=torch.complex128, device="cuda"))
