"""Transforms at arbitrary points (the paper's FaVeST_fwd(T, L, X, w) / FaVeST_adj(a, b, X),
Sec. 4.4) against the oracle's literal form O1 at the same points (Def. FwdVSHT eq. fwdvsht2,
Def. AdjVSHT eq. SLvec, built from eqs. Blm1, Blm2, vsh2 and the Clebsch-Gordan values of
eq. ninecoeff): FP64 bar, normwise max relative error <= 1e-12 per family and field.

Point sets: area-uniform random points (z ~ U[-1, 1], phi ~ U[0, 2 pi)) standing in for
the spherical designs of Sec. 5.1, which are not available here; the exact poles and points
within 1e-9 of them; and the Gauss-Legendre grid, where the result must equal the grid
transforms of the same field."""
import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _points(n, seed, poles=False):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    if poles:
        z[:4] = [1.0, -1.0, np.cos(1e-9), -np.cos(2e-9)]
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    X = np.stack([r * np.cos(ph), r * np.sin(ph), z], -1)
    if poles:
        X[:2, :2] = 0.0
        X[2:4, 0] = np.sin([1e-9, 2e-9])
        X[2:4, 1] = 0.0
    return X


def _angles(X):
    return np.arctan2(np.hypot(X[:, 0], X[:, 1]), X[:, 2]), np.arctan2(X[:, 1], X[:, 0])


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128).contiguous()


@pytest.mark.parametrize("L,B,n,seed,poles", [(1, 1, 7, 1, False), (4, 2, 60, 2, True), (16, 2, 900, 3, True),
                                              (31, 1, 3000, 4, False), (16, 2, 20000, 5, False),
                                              (64, 1, 5000, 6, True)])
def test_scatter_vs_literal_oracle(orc, L, B, n, seed, poles):
    """Forward with random positive weights and the adjoint of drawn coefficients against O1,
    including the chunked forward and the order-split adjoint (large n) and the poles."""
    X = _points(n, seed, poles)
    rng = np.random.default_rng(100 + seed)
    w = rng.uniform(0.5, 1.5, n) * 4 * np.pi / n
    T = rng.standard_normal((B, n, 3)) + 1j * rng.standard_normal((B, n, 3))
    a, b = synthetic.coefficients(L, B, seed=200 + seed)
    plan = api.ScatterPlan(L, X, w, batch=B)
    ga, gb = plan.fwd(_dev(T))
    gT = plan.adj(_dev(a), _dev(b))
    torch.cuda.synchronize()
    ga, gb, gT = ga.cpu().numpy(), gb.cpu().numpy(), gT.cpu().numpy()
    th, ph = _angles(X)
    for f in range(B):
        ra, rb = orc.fwd_literal(L, th, ph, w, T[f])
        assert normwise_err(ga[f], ra) < TOL64
        assert normwise_err(gb[f], rb) < TOL64
        rT = orc.adj_literal(L, a[f], b[f], th, ph)
        assert normwise_err(gT[f].ravel(), rT.ravel()) < TOL64
        # the synthesis is tangent: T . x = 0 to rounding
        assert np.max(np.abs(np.sum(gT[f] * X, -1))) < 1e-12 * np.max(np.abs(gT[f]))
    plan.close()


def test_scatter_on_gauss_legendre_grid_equals_grid_transforms(orc):
    """On the Gauss-Legendre points with their weights the scattered transforms are the grid
    transforms: the Clebsch-Gordan plan's favest_fwd_cart / favest_adj_cart of the same
    Cartesian field, and the roundtrip recovers band-limited coefficients."""
    L, B = 24, 2
    x, W, theta, phi = orc.grid(L)
    nlat, nphi = L + 1, 2 * (L + 1)
    th = np.repeat(theta, nphi)
    ph = np.tile(phi, nlat)
    X = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    w = np.repeat(W, nphi) * (2 * np.pi / nphi)
    a, b = synthetic.coefficients(L, B, seed=9)
    sp = api.ScatterPlan(L, X, w, batch=B)
    T = sp.adj(_dev(a), _dev(b))
    a2, b2 = sp.fwd(T)
    cg = api.CgPlan(L, B)
    Tg = cg.adj(_dev(a), _dev(b))                      # [B, 3, nlat, nphi]
    torch.cuda.synchronize()
    Ts = T.cpu().numpy()
    Tc = Tg.cpu().numpy().reshape(B, 3, nlat * nphi).transpose(0, 2, 1)
    assert normwise_err(Ts.reshape(B, -1), Tc.reshape(B, -1)) < TOL64
    assert normwise_err(a2.cpu().numpy(), a) < TOL64
    assert normwise_err(b2.cpu().numpy(), b) < TOL64
    ca, cb = cg.fwd(torch.as_tensor(np.ascontiguousarray(Tc.transpose(0, 2, 1).reshape(B, 3, nlat, nphi))).cuda())
    torch.cuda.synchronize()
    assert normwise_err(a2.cpu().numpy(), ca.cpu().numpy()) < TOL64
    sp.close()
    cg.close()


def test_scatter_unit_weights_is_exact_adjoint():
    """With unit weights the forward is A^H: <A c, T> = <c, A^H T> at arbitrary points."""
    L, B, n = 20, 2, 777
    X = _points(n, 11)
    rng = np.random.default_rng(12)
    T = rng.standard_normal((B, n, 3)) + 1j * rng.standard_normal((B, n, 3))
    a, b = synthetic.coefficients(L, B, seed=13)
    plan = api.ScatterPlan(L, X, None, batch=B)
    AT = plan.adj(_dev(a), _dev(b)).cpu().numpy()
    ha, hb = plan.fwd(_dev(T))
    lhs = np.vdot(AT, T)
    rhs = np.vdot(a, ha.cpu().numpy()) + np.vdot(b, hb.cpu().numpy())
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    plan.close()


def test_scatter_argument_errors():
    X = _points(10, 1)
    for L, B, pts in [(0, 1, X), (2048, 1, X), (4, 0, X), (4, 1, X * 1.001)]:
        with pytest.raises(api.FavestError) as e:
            api.ScatterPlan(L, pts, None, batch=B)
        assert e.value.status == api.FAVEST_EINVAL
    with pytest.raises(ValueError):
        api.ScatterPlan(4, X[:, :2])
