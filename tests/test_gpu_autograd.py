"""Differentiation form: L = 255 on the 256 x 512 Gauss-Legendre grid, 16 fields,
seed 4.  Losses
    L_c(a, b) = sum |FwdVSHT(AdjVSHT(a, b) * g)|^2      (gradients w.r.t. a, b)
    L_T(T)    = sum |FwdVSHT(T * g)|^2                   (gradient w.r.t. the grid field)
with g a fixed positive mask ~ U[0.5, 1.5] on the grid.  The autograd gradients (the
library's weighted-adjoint and unit-weight forward kernels) are checked against
FP64 central differences along 64 random directions and against the analytic
gradient evaluated with the CPU oracle.  PyTorch's complex gradient of a real loss is
2 dL/d(conj z), so the directional derivative along d is Re sum conj(grad) d.

Both losses are exactly quadratic, so a central difference has no truncation error at
any step; what limits it is the rounding of the two loss values (~1e-14 relative for
the FP64 path) divided by the step.  At the configured step h = 1e-6 that noise is about
1e-7 of |grad| |d|, so the check there is scaled by |grad| |d| (tolerance 1e-6); a
second difference at h = 1e-2 is checked against the directional derivative itself
(tolerance 1e-7)."""
import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402
from paper_1908_00041_gb300.autograd import adj_vsht, fwd_vsht  # noqa: E402

L, B, SEED = 255, 16, 4
H = 1e-6
H_WIDE = 1e-2
NDIR = 64


def _fd_errors(loss_at, grads, dirs):
    """Worst errors over directions: |fd(h=1e-6) - an| / (|grad| |d|) and
    |fd(h=1e-2) - an| / max(|an|, 1e-3 |grad| |d|)."""
    gnorm = np.sqrt(sum(np.sum(np.abs(g) ** 2) for g in grads))
    e_small = e_wide = 0.0
    for d in dirs:
        dn = np.sqrt(sum(np.sum(np.abs(x) ** 2) for x in d))
        an = float(np.real(sum(np.sum(np.conj(g) * x) for g, x in zip(grads, d))))
        fd6 = (loss_at(d, H) - loss_at(d, -H)) / (2 * H)
        fd2 = (loss_at(d, H_WIDE) - loss_at(d, -H_WIDE)) / (2 * H_WIDE)
        e_small = max(e_small, abs(fd6 - an) / (gnorm * dn))
        e_wide = max(e_wide, abs(fd2 - an) / max(abs(an), 1e-3 * gnorm * dn))
    return e_small, e_wide


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)
    rng = np.random.default_rng(SEED)
    a, b = synthetic.coefficients(L, B, seed=None, decay=1.0, rng=rng)
    g = synthetic.mask(L, rng)
    dirs = []
    for _ in range(NDIR):
        da = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
        db = rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)
        nrm = np.sqrt(np.sum(np.abs(da) ** 2) + np.sum(np.abs(db) ** 2))
        dirs.append((da / nrm, db / nrm))
    plan = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C128)
    return plan, a, b, g, dirs


def _cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(torch.complex128).cuda()


def _loss_c(plan, a, b, g):
    tt, tp = adj_vsht(plan, a, b)
    ra, rb = fwd_vsht(plan, tt * g, tp * g)
    return (ra.abs() ** 2).sum() + (rb.abs() ** 2).sum()


def _loss_T(plan, tt, tp, g):
    ra, rb = fwd_vsht(plan, tt * g, tp * g)
    return (ra.abs() ** 2).sum() + (rb.abs() ** 2).sum()


def test_grad_coefficients_fd(setup):
    plan, a, b, g, dirs = setup
    gg = torch.as_tensor(g).cuda()
    ta = _cuda(a).requires_grad_(True)
    tb = _cuda(b).requires_grad_(True)
    loss = _loss_c(plan, ta, tb, gg)
    loss.backward()
    ga, gb = ta.grad.detach().cpu().numpy(), tb.grad.detach().cpu().numpy()

    def loss_at(d, h):
        with torch.no_grad():
            return _loss_c(plan, _cuda(a + h * d[0]), _cuda(b + h * d[1]), gg).item()

    e_small, e_wide = _fd_errors(loss_at, (ga, gb), dirs)
    assert e_small < 1e-6, e_small
    assert e_wide < 1e-7, e_wide


def test_grad_field_fd(setup):
    plan, a, b, g, dirs = setup
    gg = torch.as_tensor(g).cuda()
    rng = np.random.default_rng(SEED + 1)
    tt, tp = synthetic.grid_field(L, B, seed=SEED + 2)
    xt = _cuda(tt).requires_grad_(True)
    xp = _cuda(tp).requires_grad_(True)
    _loss_T(plan, xt, xp, gg).backward()
    gt, gp = xt.grad.detach().cpu().numpy(), xp.grad.detach().cpu().numpy()
    fdirs = []
    for _ in range(NDIR):
        dt = rng.standard_normal(tt.shape) + 1j * rng.standard_normal(tt.shape)
        dp = rng.standard_normal(tp.shape) + 1j * rng.standard_normal(tp.shape)
        nrm = np.sqrt(np.sum(np.abs(dt) ** 2) + np.sum(np.abs(dp) ** 2))
        fdirs.append((dt / nrm, dp / nrm))

    def loss_at(d, h):
        with torch.no_grad():
            return _loss_T(plan, _cuda(tt + h * d[0]), _cuda(tp + h * d[1]), gg).item()

    e_small, e_wide = _fd_errors(loss_at, (gt, gp), fdirs)
    assert e_small < 1e-6, e_small
    assert e_wide < 1e-7, e_wide


def test_grad_field_analytic(setup, orc):
    """grad_T = g W A (2 r), r = A^H W (g T) (W the point weights W_j 2 pi / nphi): the
    oracle's synthesis of 2 r times the mask and the weights (2 fields)."""
    plan, a, b, g, dirs = setup
    gg = torch.as_tensor(g).cuda()
    tt, tp = synthetic.grid_field(L, B, seed=SEED + 2)
    xt = _cuda(tt).requires_grad_(True)
    xp = _cuda(tp).requires_grad_(True)
    _loss_T(plan, xt, xp, gg).backward()
    gt, gp = xt.grad.detach().cpu().numpy(), xp.grad.detach().cpu().numpy()
    x, W, theta, phi = orc.grid(L)
    nphi = len(phi)
    wpt = (W * (2 * np.pi / nphi))[:, None]
    for f in (0, B - 1):
        ra, rb = orc.fwd_sep(L, x, W, g * tt[f], g * tp[f])
        t2, p2 = orc.adj_sep(L, x, 2 * ra, 2 * rb, nphi)
        assert normwise_err(gt[f].ravel(), (g * wpt * t2).ravel()) < 1e-11
        assert normwise_err(gp[f].ravel(), (g * wpt * p2).ravel()) < 1e-11


def test_grad_coefficients_analytic(setup, orc):
    """grad = A^H (g W A (2 r)), r = A^H W (g A c), evaluated by the oracle (2 fields)."""
    plan, a, b, g, dirs = setup
    gg = torch.as_tensor(g).cuda()
    ta = _cuda(a).requires_grad_(True)
    tb = _cuda(b).requires_grad_(True)
    _loss_c(plan, ta, tb, gg).backward()
    ga, gb = ta.grad.detach().cpu().numpy(), tb.grad.detach().cpu().numpy()
    x, W, theta, phi = orc.grid(L)
    nphi = len(phi)
    for f in (0, B - 1):
        tt, tp = orc.adj_sep(L, x, a[f], b[f], nphi)
        ra, rb = orc.fwd_sep(L, x, W, g * tt, g * tp)
        t2, p2 = orc.adj_sep(L, x, 2 * ra, 2 * rb, nphi)
        ea, eb = orc.fwd_sep(L, x, W, g * t2, g * p2)
        assert normwise_err(ga[f], ea) < 1e-11
        assert normwise_err(gb[f], eb) < 1e-11


@pytest.mark.parametrize("prec,io,tol", [(api.FAVEST_FP64, api.FAVEST_IO_C128, 1e-13),
                                         (api.FAVEST_BF16X6, api.FAVEST_IO_C64, 2e-6)])
def test_weighted_adjoint_and_unit_forward_identities(prec, io, tol):
    """<W A c, T> = <c, A^H W T> and <A c, T> = <c, A^H T> (dot-product tests of the
    two backward operators against the two forward operators)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Ls, Bs = 63, 3
    plan = api.Plan(Ls, Bs, prec, io)
    dt = plan.cdtype
    a, b = synthetic.coefficients(Ls, Bs, seed=11)
    tt, tp = synthetic.grid_field(Ls, Bs, seed=12)
    ca, cb = (torch.as_tensor(v).to(dt).cuda().contiguous() for v in (a, b))
    xt, xp = (torch.as_tensor(v).to(dt).cuda().contiguous() for v in (tt, tp))
    wt, wp = plan.adj(ca, cb, weighted=True)
    fa, fb = plan.fwd(xt, xp)
    ut, up = plan.adj(ca, cb)
    ua, ub = plan.fwd(xt, xp, unit_weights=True)
    torch.cuda.synchronize()
    assert plan.status() == 0

    def dot(u, v):
        return complex(torch.sum(torch.conj(u.to(torch.complex128)) * v.to(torch.complex128)).item())

    lhs = dot(wt, xt) + dot(wp, xp)
    rhs = dot(ca, fa) + dot(cb, fb)
    assert abs(lhs - rhs) <= tol * abs(rhs)
    lhs = dot(ut, xt) + dot(up, xp)
    rhs = dot(ca, ua) + dot(cb, ub)
    assert abs(lhs - rhs) <= tol * abs(rhs)


def test_bf16x6_backward_matches_fp64():
    """The split-precision plan back-propagates through the same operators: its
    gradient of L_c agrees with the FP64 plan's within the split form's bar."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Ls, Bs = 127, 2
    a, b = synthetic.coefficients(Ls, Bs, seed=21)
    g = synthetic.mask(Ls, np.random.default_rng(22))
    grads = []
    for prec, io, dt in ((api.FAVEST_FP64, api.FAVEST_IO_C128, torch.complex128),
                         (api.FAVEST_BF16X6, api.FAVEST_IO_C64, torch.complex64)):
        plan = api.Plan(Ls, Bs, prec, io)
        gg = torch.as_tensor(g).to(torch.float64 if dt == torch.complex128 else torch.float32).cuda()
        ta = torch.as_tensor(a).to(torch.complex64).to(dt).cuda().requires_grad_(True)
        tb = torch.as_tensor(b).to(torch.complex64).to(dt).cuda().requires_grad_(True)
        _loss_c(plan, ta, tb, gg).backward()
        grads.append((ta.grad.cpu().numpy().astype(np.complex128), tb.grad.cpu().numpy().astype(np.complex128)))
    assert normwise_err(grads[1][0], grads[0][0]) < 2e-6
    assert normwise_err(grads[1][1], grads[0][1]) < 2e-6


# ---------------------------------------------------------------------------
# Real fields: the backward operators are the transposes for the real inner products
# ---------------------------------------------------------------------------
def _rdot(u, v):
    """Re sum conj(u) v (the real inner product of complex or real tensors)."""
    return float(torch.sum(torch.conj(u.to(torch.complex128)) * v.to(torch.complex128)).real.item())


@pytest.mark.parametrize("prec,io,tol", [(api.FAVEST_FP64, api.FAVEST_IO_R64, 1e-13),
                                         (api.FAVEST_BF16X6, api.FAVEST_IO_R32, 2e-6)])
def test_real_transposes(prec, io, tol):
    """<F(T), g> = <T, F^T g> and <S(c), h> = <c, S^T h> for the real FwdVSHT F and the
    real AdjVSHT S, with F^T, S^T computed by the FAVEST_FLAG_REAL_TRANSPOSE calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Ls, Bs = 63, 3
    plan = api.Plan(Ls, Bs, prec, io)
    tt, tp = synthetic.real_grid_field(Ls, Bs, seed=31)
    ga, gb = synthetic.half_coefficients(Ls, Bs, seed=32)
    T = [torch.as_tensor(v).to(plan.fdtype).cuda().contiguous() for v in (tt, tp)]
    g = [torch.as_tensor(v).to(plan.cdtype).cuda().contiguous() for v in (ga, gb)]
    Fa, Fb = plan.fwd(*T)
    Ft, Fp = plan.adj(*g, weighted=True, real_transpose=True)
    Sa, Sb = plan.adj(*g)
    St = plan.fwd(*T, unit_weights=True, real_transpose=True)
    torch.cuda.synchronize()
    lhs, rhs = _rdot(Fa, g[0]) + _rdot(Fb, g[1]), _rdot(T[0], Ft) + _rdot(T[1], Fp)
    assert abs(lhs - rhs) <= tol * abs(rhs)
    lhs, rhs = _rdot(Sa, T[0]) + _rdot(Sb, T[1]), _rdot(g[0], St[0]) + _rdot(g[1], St[1])
    assert abs(lhs - rhs) <= tol * abs(rhs)


def test_real_grad_fd():
    """Autograd through real-field FP64 plans: L(c) = sum |F(S(c) g)|^2 and
    L(T) = sum |F(T g)|^2 against central differences (h = 1e-2; the losses are
    quadratic) along random directions."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Ls, Bs = 47, 2
    plan = api.Plan(Ls, Bs, api.FAVEST_FP64, api.FAVEST_IO_R64)
    rng = np.random.default_rng(41)
    a, b = synthetic.half_coefficients(Ls, Bs, seed=None, rng=rng)
    gmask = torch.as_tensor(synthetic.mask(Ls, rng)).cuda()
    tt, tp = synthetic.real_grid_field(Ls, Bs, seed=42)

    def loss_c(ca, cb):
        xt, xp = adj_vsht(plan, ca, cb)
        ra, rb = fwd_vsht(plan, xt * gmask, xp * gmask)
        return (ra.abs() ** 2).sum() + (rb.abs() ** 2).sum()

    def loss_t(xt, xp):
        ra, rb = fwd_vsht(plan, xt * gmask, xp * gmask)
        return (ra.abs() ** 2).sum() + (rb.abs() ** 2).sum()

    ca = torch.as_tensor(a).cuda().requires_grad_(True)
    cb = torch.as_tensor(b).cuda().requires_grad_(True)
    loss_c(ca, cb).backward()
    xt = torch.as_tensor(tt).cuda().requires_grad_(True)
    xp = torch.as_tensor(tp).cuda().requires_grad_(True)
    loss_t(xt, xp).backward()
    h = 1e-2
    for _ in range(8):
        da = torch.as_tensor(rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)).cuda()
        db = torch.as_tensor(rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)).cuda()
        with torch.no_grad():
            fd = (loss_c(ca + h * da, cb + h * db) - loss_c(ca - h * da, cb - h * db)).item() / (2 * h)
        an = _rdot(ca.grad, da) + _rdot(cb.grad, db)
        assert abs(fd - an) <= 1e-9 * max(abs(an), 1e-3 * (ca.grad.norm() * da.norm()).item())
        dt = torch.as_tensor(rng.standard_normal(tt.shape)).cuda()
        dp = torch.as_tensor(rng.standard_normal(tp.shape)).cuda()
        with torch.no_grad():
            fd = (loss_t(xt + h * dt, xp + h * dp) - loss_t(xt - h * dt, xp - h * dp)).item() / (2 * h)
        an = _rdot(xt.grad, dt) + _rdot(xp.grad, dp)
        assert abs(fd - an) <= 1e-9 * max(abs(an), 1e-3 * (xt.grad.norm() * dt.norm()).item())
