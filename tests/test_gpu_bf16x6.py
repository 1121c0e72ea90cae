"""GPU parity of the split-precision tensor-core path (FAVEST_BF16X6): complex64
fields and coefficients, FP64 recurrence, Legendre contraction on tcgen05 with three
bf16 pieces per operand.  Bar: normwise max relative error <= 1e-6 against the FP64
path (GPU or oracle) on the same complex64 input."""
import numpy as np
import pytest

from helpers import cidx, normwise_err, rms_err, sample_coefs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _c64(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex64).cuda().contiguous()


def _h(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _run(L, B, prec, fn, *args):
    plan = api.Plan(L, B, prec, api.FAVEST_IO_C64)
    out = getattr(plan, fn)(*args)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return [_h(o) for o in out]


@pytest.mark.parametrize(
    "L,B", [(1, 1), (2, 1), (8, 1), (16, 1), (31, 3), (63, 2), (100, 1), (127, 17), (255, 2), (511, 1)]
)
def test_bf16x6_vs_oracle(orc, L, B):
    a, b = synthetic.coefficients(L, B, seed=300 + L)
    a = a.astype(np.complex64).astype(np.complex128)
    b = b.astype(np.complex64).astype(np.complex128)
    tt, tp = _run(L, B, api.FAVEST_BF16X6, "adj", _c64(a), _c64(b))
    x, W, theta, phi = orc.grid(L)
    for f in range(min(B, 3)):
        rt, rp = orc.adj_sep(L, x, a[f], b[f], len(phi))
        assert normwise_err(tt[f].ravel(), rt.ravel()) < TOL
        assert normwise_err(tp[f].ravel(), rp.ravel()) < TOL
    gt, gp = synthetic.grid_field(L, B, seed=400 + L)
    gt = gt.astype(np.complex64).astype(np.complex128)
    gp = gp.astype(np.complex64).astype(np.complex128)
    ga, gb = _run(L, B, api.FAVEST_BF16X6, "fwd", _c64(gt), _c64(gp))
    for f in range(min(B, 3)):
        ra, rb = orc.fwd_sep(L, x, W, gt[f], gp[f])
        assert normwise_err(ga[f], ra) < TOL
        assert normwise_err(gb[f], rb) < TOL


def test_bf16x6_c3_vs_fp64_path(orc):
    """L = 1023, batch 32, complex64 fields, spectrum (l+1)^-1.5 (seed 2): the split
    form against the FP64 path on the same complex64 input, forward and adjoint."""
    L, B = 1023, 32
    a, b = synthetic.coefficients(L, B, seed=2, decay=1.5)
    da, db = _c64(a), _c64(b)
    p16 = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
    t16, q16 = p16.adj(da, db)
    t64, q64 = p64.adj(da, db)
    torch.cuda.synchronize()
    assert p16.status() == 0 and p64.status() == 0
    assert normwise_err(_h(t16).reshape(B, -1), _h(t64).reshape(B, -1)) < TOL
    assert normwise_err(_h(q16).reshape(B, -1), _h(q64).reshape(B, -1)) < TOL
    # forward on the same complex64 field (the FP64-path synthesis)
    a16, b16 = p16.fwd(t64, q64)
    a64, b64 = p64.fwd(t64, q64)
    torch.cuda.synchronize()
    e_a = normwise_err(_h(a16), _h(a64))
    e_b = normwise_err(_h(b16), _h(b64))
    assert max(e_a, e_b) < TOL, (e_a, e_b)
    assert rms_err(_h(a16), _h(a64)) < TOL
    # the FP64 path itself agrees with the oracle on sampled coefficients
    x, W, theta, phi = orc.grid(L)
    rng = np.random.default_rng(9)
    ls, ms = sample_coefs(L, 10, rng)
    sa, sb = orc.fwd_literal_grid_coefs(L, x, W, _h(t64)[5], _h(q64)[5], ls, ms)
    idx = cidx(ls, ms)
    sc = max(np.max(np.abs(a[5])), np.max(np.abs(b[5])))
    assert np.max(np.abs(_h(a64)[5][idx] - sa)) < 2e-6 * sc


def test_bf16x6_roundtrip():
    for L, B in [(255, 16), (511, 4)]:
        a, b = synthetic.coefficients(L, B, seed=17)
        plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
        da, db = _c64(a), _c64(b)
        tt, tp = plan.adj(da, db)
        a2, b2 = plan.fwd(tt, tp)
        torch.cuda.synchronize()
        ref_a = a.astype(np.complex64).astype(np.complex128)
        ref_b = b.astype(np.complex64).astype(np.complex128)
        assert normwise_err(_h(a2), ref_a) < 2 * TOL
        assert normwise_err(_h(b2), ref_b) < 2 * TOL


@pytest.mark.parametrize("decay", [1.0, 0.5])
def test_bf16x6_polar_rings_flat_spectrum(decay):
    """Flatter spectra than (l+1)^-1.5 put more weight on the polar rings, where the
    adjoint divides the scalar sums by sin(theta_j); the split form must stay within
    the bar against the FP64 path there too (L = 1023, 4 fields)."""
    L, B = 1023, 4
    a, b = synthetic.coefficients(L, B, seed=71, decay=decay)
    da, db = _c64(a), _c64(b)
    p16 = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
    t16, q16 = p16.adj(da, db)
    t64, q64 = p64.adj(da, db)
    torch.cuda.synchronize()
    assert p16.status() == 0 and p64.status() == 0
    for g, r in ((t16, t64), (q16, q64)):
        g, r = _h(g), _h(r)
        assert normwise_err(g.reshape(B, -1), r.reshape(B, -1)) < TOL
        # the polar rings themselves, relative to the field's maximum
        pole = np.concatenate([g[:, :3] - r[:, :3], g[:, -3:] - r[:, -3:]], axis=1)
        assert np.abs(pole).max() < TOL * np.abs(r).max()


@pytest.mark.parametrize("L,B", [(63, 2), (255, 3), (767, 1)])
def test_generator_shape_does_not_change_results(L, B):
    """The autotuner may pick another generator shape (latitudes per block, order groups,
    one or two latitude recurrences per thread): the transforms stay bit-identical.  Untuned
    plans start with two recurrences per thread from 384 folded latitudes (L >= 766) up."""
    a, b = synthetic.coefficients(L, B, seed=3000 + L, decay=1.0)
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    assert plan.gen_chains() == (2 if L >= 766 else 1)
    ca, cb = _c64(a), _c64(b)
    t0, p0 = plan.adj(ca, cb)
    f0, g0 = plan.fwd(t0, p0)
    torch.cuda.synchronize()
    plan.tune()
    assert plan.gen_chains() in (1, 2) and plan.gen_shape()[0] in (32, 64, 128)
    t1, p1 = plan.adj(ca, cb)
    f1, g1 = plan.fwd(t0, p0)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(t0, t1) and torch.equal(p0, p1)
    assert torch.equal(f0, f1) and torch.equal(g0, g1)
