"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs.  FP64 path bar: normwise max relative error <= 1e-12 per family and
field (max |diff| / max |ref|)."""
import numpy as np
import pytest

from helpers import cidx, normwise_err, rms_err, sample_coefs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _dev(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _gpu_adj(L, a, b, io=api.FAVEST_IO_C128):
    B = a.shape[0]
    dt = torch.complex128 if io == api.FAVEST_IO_C128 else torch.complex64
    plan = api.Plan(L, B, api.FAVEST_FP64, io)
    tt, tp = plan.adj(_dev(a, dt), _dev(b, dt))
    torch.cuda.synchronize()
    assert plan.status() == 0
    return _host(tt), _host(tp)


def _gpu_fwd(L, tt, tp, io=api.FAVEST_IO_C128, unit=False):
    B = tt.shape[0]
    dt = torch.complex128 if io == api.FAVEST_IO_C128 else torch.complex64
    plan = api.Plan(L, B, api.FAVEST_FP64, io)
    a, b = plan.fwd(_dev(tt, dt), _dev(tp, dt), unit_weights=unit)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return _host(a), _host(b)


@pytest.mark.parametrize("L", [1, 2, 7, 8, 16])
def test_fp64_small_vs_literal_oracle(orc, L):
    """Full transforms against the literal Clebsch-Gordan oracle (O1)."""
    B = 2
    a, b = synthetic.coefficients(L, B, seed=L)
    tt, tp = _gpu_adj(L, a, b)
    x, W, theta, phi = orc.grid(L)
    t = np.repeat(theta, len(phi))
    p = np.tile(phi, len(theta))
    for f in range(B):
        S = orc.adj_literal(L, a[f], b[f], t, p)
        et = np.stack([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)], -1)
        ep = np.stack([-np.sin(p), np.cos(p), np.zeros_like(p)], -1)
        rt = np.sum(S * et, -1).reshape(L + 1, -1)
        rp = np.sum(S * ep, -1).reshape(L + 1, -1)
        assert normwise_err(tt[f].ravel(), rt.ravel()) < TOL64
        assert normwise_err(tp[f].ravel(), rp.ravel()) < TOL64
    # forward on random (not band-limited) fields
    gt, gp = synthetic.grid_field(L, B, seed=100 + L)
    ga, gb = _gpu_fwd(L, gt, gp)
    w = np.repeat(W, len(phi)) * (2 * np.pi / len(phi))
    for f in range(B):
        T = orc.sph_to_cart(t, p, gt[f].ravel(), gp[f].ravel())
        ra, rb = orc.fwd_literal(L, t, p, w, T)
        assert normwise_err(ga[f], ra) < TOL64
        assert normwise_err(gb[f], rb) < TOL64


@pytest.mark.parametrize("L,B", [(16, 1), (31, 3), (50, 2), (63, 4), (100, 1)])
def test_fp64_mid_vs_separable_oracle(orc, L, B):
    """Full transforms against the separable oracle (O3); odd/even latitude counts,
    non-power-of-two longitude lengths (2(L+1) = 102, 202) and both column groupings."""
    a, b = synthetic.coefficients(L, B, seed=1000 + L)
    tt, tp = _gpu_adj(L, a, b)
    x, W, theta, phi = orc.grid(L)
    for f in range(B):
        rt, rp = orc.adj_sep(L, x, a[f], b[f], len(phi))
        assert normwise_err(tt[f].ravel(), rt.ravel()) < TOL64
        assert normwise_err(tp[f].ravel(), rp.ravel()) < TOL64
    gt, gp = synthetic.grid_field(L, B, seed=2000 + L)
    ga, gb = _gpu_fwd(L, gt, gp)
    for f in range(B):
        ra, rb = orc.fwd_sep(L, x, W, gt[f], gp[f])
        assert normwise_err(ga[f], ra) < TOL64
        assert normwise_err(gb[f], rb) < TOL64


def test_fp64_roundtrip_exact(orc):
    """fwd(adj(c)) = c on the exact grid (Sec. 4.3 error discussion; Table 2 analogue)."""
    for L, B in [(16, 1), (127, 2), (255, 3)]:
        a, b = synthetic.coefficients(L, B, seed=5 + L)
        plan = api.Plan(L, B)
        da, db = _dev(a), _dev(b)
        tt, tp = plan.adj(da, db)
        a2, b2 = plan.fwd(tt, tp)
        torch.cuda.synchronize()
        assert normwise_err(_host(a2), a) < TOL64
        assert normwise_err(_host(b2), b) < TOL64


def test_fp64_c2_full_size(orc):
    """L = 511, 512 x 1024 grid, one field, seed 1: every coefficient against O3 and
    sampled coefficients / points against the literal form O1."""
    L = 511
    a, b = synthetic.coefficients(L, 1, seed=1)
    tt, tp = _gpu_adj(L, a, b)
    x, W, theta, phi = orc.grid(L)
    rng = np.random.default_rng(11)
    js = rng.integers(0, L + 1, 24)
    ks = rng.integers(0, 2 * (L + 1), 24)
    js[:2] = [0, L]
    rt, rp, _ = orc.adj_literal_grid_points(L, L + 1, 2 * (L + 1), x, a[0], b[0], js, ks)
    scale = max(np.max(np.abs(tt)), np.max(np.abs(tp)))
    assert np.max(np.abs(tt[0][js, ks] - rt)) < TOL64 * scale
    assert np.max(np.abs(tp[0][js, ks] - rp)) < TOL64 * scale
    ga, gb = _gpu_fwd(L, tt, tp)
    ra, rb = orc.fwd_sep(L, x, W, tt[0], tp[0])
    assert normwise_err(ga[0], ra) < TOL64
    assert normwise_err(gb[0], rb) < TOL64
    ls, ms = sample_coefs(L, 24, rng)
    sa, sb = orc.fwd_literal_grid_coefs(L, x, W, tt[0], tp[0], ls, ms)
    idx = cidx(ls, ms)
    sc = np.max(np.abs(ra))
    assert np.max(np.abs(ga[0][idx] - sa)) < TOL64 * sc
    assert np.max(np.abs(gb[0][idx] - sb)) < TOL64 * np.max(np.abs(rb))
    # and the roundtrip recovers the drawn coefficients
    assert normwise_err(ga[0], a[0]) < TOL64


def test_fp64_c3_shape_c64_io_sampled(orc):
    """L = 1023, 1024 x 2048 grid, batch 32, complex64 fields (the precision-form
    workload run through the FP64 path): sampled coefficients against O1."""
    L, B = 1023, 32
    a, b = synthetic.coefficients(L, B, seed=2, decay=1.5)
    tt, tp = _gpu_adj(L, a, b, io=api.FAVEST_IO_C64)
    ga, gb = _gpu_fwd(L, tt, tp, io=api.FAVEST_IO_C64)
    x, W, theta, phi = orc.grid(L)
    rng = np.random.default_rng(22)
    for f in [0, 17, 31]:
        ls, ms = sample_coefs(L, 12, rng)
        sa, sb = orc.fwd_literal_grid_coefs(L, x, W, tt[f].astype(np.complex128),
                                            tp[f].astype(np.complex128), ls, ms)
        idx = cidx(ls, ms)
        # complex64 outputs: compare against the FP64 oracle at fp32 resolution
        sc = max(np.max(np.abs(a[f])), np.max(np.abs(b[f])))
        assert np.max(np.abs(ga[f][idx] - sa)) < 2e-6 * sc
        assert np.max(np.abs(gb[f][idx] - sb)) < 2e-6 * sc


def test_fp64_unit_weights_is_exact_adjoint(orc):
    """With unit weights the forward map is A^H: <A c, T> = <c, A^H T>."""
    L, B = 40, 2
    a, b = synthetic.coefficients(L, B, seed=3)
    gt, gp = synthetic.grid_field(L, B, seed=4)
    tt, tp = _gpu_adj(L, a, b)
    ha, hb = _gpu_fwd(L, gt, gp, unit=True)
    lhs = np.vdot(tt, gt) + np.vdot(tp, gp)
    rhs = np.vdot(a, ha) + np.vdot(b, hb)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_single_mode_closed_form(orc):
    """grad* Y_{l0 m0} -> a = sqrt(l0(l0+1)) delta: build the field with the GPU adjoint
    of a unit coefficient, check it against the oracle and recover the coefficient."""
    L = 64
    for (l0, m0) in [(1, 0), (64, -64), (33, 5)]:
        a = np.zeros((1, L * L + 2 * L), complex)
        b = np.zeros_like(a)
        a[0, cidx(l0, m0)] = 1.0
        tt, tp = _gpu_adj(L, a, b)
        ga, gb = _gpu_fwd(L, tt, tp)
        assert np.max(np.abs(ga - a)) < 1e-12 and np.max(np.abs(gb)) < 1e-12
        b2, a2 = a.copy(), np.zeros_like(a)
        tt, tp = _gpu_adj(L, a2, b2)
        ga, gb = _gpu_fwd(L, tt, tp)
        assert np.max(np.abs(gb - b2)) < 1e-12 and np.max(np.abs(ga)) < 1e-12
