"""Ragged batches (the batching form): fields of mixed degree in one call, grouped by
degree, with one persistent tensor-core Legendre launch over a merged work queue, an
optional CUDA-graph replay and the generator autotuner.  Checked against single-field
plans, the FP64 path and the oracle."""
import numpy as np
import pytest

from helpers import normwise_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _pack_coefs(bp, coefs, dtype):
    a = torch.zeros(bp.coef_elems, dtype=dtype, device="cuda")
    b = torch.zeros(bp.coef_elems, dtype=dtype, device="cuda")
    for i, (ca, cb) in enumerate(coefs):
        bp.coef(a, i).copy_(torch.as_tensor(ca).to(dtype))
        bp.coef(b, i).copy_(torch.as_tensor(cb).to(dtype))
    return a, b


def _coefs(Ls, seed, decay=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for L in Ls:
        a, b = synthetic.coefficients(L, 1, seed=None, decay=decay, rng=rng)
        out.append((a[0].astype(np.complex64), b[0].astype(np.complex64)))
    return out


def _h(t):
    return t.detach().cpu().numpy().astype(np.complex128)


LS = [63, 31, 127, 63, 255, 31, 127, 63]


def test_batch_matches_single_plans():
    coefs = _coefs(LS, 31)
    bp = api.BatchPlan(LS, api.FAVEST_BF16X6, api.FAVEST_IO_C64, graph=False)
    a, b = _pack_coefs(bp, coefs, torch.complex64)
    tt, tp = bp.adj(a, b)
    ra, rb = bp.fwd(tt, tp)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for i, L in enumerate(LS):
        p = api.Plan(L, 1, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
        ca = torch.as_tensor(coefs[i][0]).cuda().view(1, -1).contiguous()
        cb = torch.as_tensor(coefs[i][1]).cuda().view(1, -1).contiguous()
        st, sp = p.adj(ca, cb)
        sa, sb = p.fwd(st, sp)
        torch.cuda.synchronize()
        assert normwise_err(_h(bp.field(tt, i)).ravel(), _h(st[0]).ravel()) < TOL
        assert normwise_err(_h(bp.field(tp, i)).ravel(), _h(sp[0]).ravel()) < TOL
        assert normwise_err(_h(bp.coef(ra, i)), _h(sa[0])) < TOL
        assert normwise_err(_h(bp.coef(rb, i)), _h(sb[0])) < TOL


def test_batch_vs_oracle(orc):
    coefs = _coefs(LS, 32)
    bp = api.BatchPlan(LS, api.FAVEST_BF16X6, api.FAVEST_IO_C64, graph=False)
    a, b = _pack_coefs(bp, coefs, torch.complex64)
    tt, tp = bp.adj(a, b)
    torch.cuda.synchronize()
    for i in (1, 4):
        L = LS[i]
        x, W, theta, phi = orc.grid(L)
        ca, cb = (c.astype(np.complex128) for c in coefs[i])
        rt, rp = orc.adj_sep(L, x, ca, cb, len(phi))
        assert normwise_err(_h(bp.field(tt, i)).ravel(), rt.ravel()) < TOL
        assert normwise_err(_h(bp.field(tp, i)).ravel(), rp.ravel()) < TOL
        fa, fb = orc.fwd_sep(L, x, W, _h(bp.field(tt, i)), _h(bp.field(tp, i)))
        ra, rb = bp.fwd(tt, tp)
        torch.cuda.synchronize()
        assert normwise_err(_h(bp.coef(ra, i)), fa) < TOL
        assert normwise_err(_h(bp.coef(rb, i)), fb) < TOL


def test_batch_fp64_matches_single_plans():
    Ls = [16, 40, 16, 33]
    coefs = _coefs(Ls, 33)
    bp = api.BatchPlan(Ls, api.FAVEST_FP64, api.FAVEST_IO_C128, graph=False)
    a, b = _pack_coefs(bp, [(x.astype(np.complex128), y.astype(np.complex128)) for x, y in coefs],
                       torch.complex128)
    tt, tp = bp.adj(a, b)
    ra, rb = bp.fwd(tt, tp)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for i, L in enumerate(Ls):
        p = api.Plan(L, 1, api.FAVEST_FP64, api.FAVEST_IO_C128)
        ca = torch.as_tensor(coefs[i][0]).to(torch.complex128).cuda().view(1, -1).contiguous()
        cb = torch.as_tensor(coefs[i][1]).to(torch.complex128).cuda().view(1, -1).contiguous()
        st, sp = p.adj(ca, cb)
        torch.cuda.synchronize()
        assert normwise_err(_h(bp.field(tt, i)).ravel(), _h(st[0]).ravel()) < 1e-13
        assert normwise_err(_h(bp.field(tp, i)).ravel(), _h(sp[0]).ravel()) < 1e-13
        # the roundtrip recovers the (complex64-valued) coefficients
        assert normwise_err(_h(bp.coef(ra, i)), coefs[i][0].astype(np.complex128)) < 1e-12


def test_batch_graph_replay_and_autotune():
    coefs = _coefs(LS, 34)
    ref = api.BatchPlan(LS, api.FAVEST_BF16X6, api.FAVEST_IO_C64, graph=False)
    a, b = _pack_coefs(ref, coefs, torch.complex64)
    t0, p0 = ref.adj(a, b)
    f0a, f0b = ref.fwd(t0, p0)
    bp = api.BatchPlan(LS, api.FAVEST_BF16X6, api.FAVEST_IO_C64, autotune=True, graph=True)
    for g in bp.groups():
        assert g["gen_lt"] in (32, 64, 128) and g["gen_mb"] in (1, 2, 4)
    tt = torch.empty_like(t0)
    tp = torch.empty_like(p0)
    fa = torch.empty_like(f0a)
    fb = torch.empty_like(f0b)
    for _ in range(4):          # eager, capture, replay, replay
        tt.zero_()
        fa.zero_()
        bp.adj(a, b, tt, tp)
        bp.fwd(tt, tp, fa, fb)
        torch.cuda.synchronize()
        assert bp.status() == 0
        # the generator's shape does not change what it computes
        assert torch.equal(tt, t0) and torch.equal(tp, p0)
        assert torch.equal(fa, f0a) and torch.equal(fb, f0b)
    # new buffers: runs (and later captures) again
    tt2, tp2 = bp.adj(a, b)
    torch.cuda.synchronize()
    assert torch.equal(tt2, t0)


def test_batching_form_config_vs_fp64():
    """256 fields, degrees drawn uniformly from {31, 63, 127, 255, 511} (seed 3),
    coefficients N(0,1)(l+1)^-1, complex64: the split form against the FP64 path on the
    same input, sampled fields."""
    Ls, rng = synthetic.ragged_degrees(256, [31, 63, 127, 255, 511], seed=3)
    Ls = [int(x) for x in Ls]
    coefs = []
    for L in Ls:
        ca, cb = synthetic.coefficients(L, 1, seed=None, decay=1.0, rng=rng)
        coefs.append((ca[0].astype(np.complex64), cb[0].astype(np.complex64)))
    bp = api.BatchPlan(Ls, api.FAVEST_BF16X6, api.FAVEST_IO_C64, graph=True)
    a, b = _pack_coefs(bp, coefs, torch.complex64)
    tt, tp = bp.adj(a, b)
    ra, rb = bp.fwd(tt, tp)
    torch.cuda.synchronize()
    assert bp.status() == 0
    pick = [int(i) for i in np.random.default_rng(5).choice(len(Ls), 12, replace=False)]
    for L in sorted({Ls[i] for i in pick}):
        idx = [i for i in pick if Ls[i] == L]
        p64 = api.Plan(L, len(idx), api.FAVEST_FP64, api.FAVEST_IO_C64)
        ca = torch.stack([torch.as_tensor(coefs[i][0]) for i in idx]).cuda().contiguous()
        cb = torch.stack([torch.as_tensor(coefs[i][1]) for i in idx]).cuda().contiguous()
        st, sp = p64.adj(ca, cb)
        xt = torch.stack([bp.field(tt, i) for i in idx]).contiguous()
        xp = torch.stack([bp.field(tp, i) for i in idx]).contiguous()
        fa, fb = p64.fwd(xt, xp)
        torch.cuda.synchronize()
        for k, i in enumerate(idx):
            assert normwise_err(_h(bp.field(tt, i)).ravel(), _h(st[k]).ravel()) < TOL
            assert normwise_err(_h(bp.field(tp, i)).ravel(), _h(sp[k]).ravel()) < TOL
            assert normwise_err(_h(bp.coef(ra, i)), _h(fa[k])) < TOL
            assert normwise_err(_h(bp.coef(rb, i)), _h(fb[k])) < TOL


# ---------------------------------------------------------------------------
# Real fields in ragged batches (half-spectrum coefficients, real planes)
# ---------------------------------------------------------------------------
LS_REAL = [63, 31, 127, 63, 16, 31, 63]        # L = 16: mixed-radix DFT, odd plane lengths


def _half_coefs(Ls, seed):
    rng = np.random.default_rng(seed)
    out = []
    for L in Ls:
        a, b = synthetic.half_coefficients(L, 1, seed=None, rng=rng)
        out.append((a[0], b[0]))
    return out


@pytest.mark.parametrize("prec,io,tol", [(api.FAVEST_BF16X6, api.FAVEST_IO_R32, 1e-6),
                                         (api.FAVEST_FP64, api.FAVEST_IO_R64, 1e-13)])
def test_real_batch_matches_single_plans(prec, io, tol):
    coefs = _half_coefs(LS_REAL, 61)
    bp = api.BatchPlan(LS_REAL, prec, io, graph=(prec == api.FAVEST_BF16X6))
    a, b = _pack_coefs(bp, coefs, bp.cdtype)
    for _ in range(3 if prec == api.FAVEST_BF16X6 else 1):   # eager, capture, replay
        tt, tp = bp.adj(a, b)
        ra, rb = bp.fwd(tt, tp)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for i, L in enumerate(LS_REAL):
        p = api.Plan(L, 1, prec, io)
        ca = torch.as_tensor(coefs[i][0]).to(bp.cdtype).cuda().view(1, -1).contiguous()
        cb = torch.as_tensor(coefs[i][1]).to(bp.cdtype).cuda().view(1, -1).contiguous()
        st, sp = p.adj(ca, cb)
        sa, sb = p.fwd(st, sp)
        torch.cuda.synchronize()
        ft = bp.field(tt, i).cpu().numpy().astype(np.float64).ravel()
        fp = bp.field(tp, i).cpu().numpy().astype(np.float64).ravel()
        assert normwise_err(ft, st[0].cpu().numpy().astype(np.float64).ravel()) < tol
        assert normwise_err(fp, sp[0].cpu().numpy().astype(np.float64).ravel()) < tol
        assert normwise_err(_h(bp.coef(ra, i)), _h(sa[0])) < tol
        assert normwise_err(_h(bp.coef(rb, i)), _h(sb[0])) < tol
        # and the roundtrip recovers the coefficients
        assert normwise_err(_h(bp.coef(ra, i)), coefs[i][0]) < 2e-6


def test_batching_form_one_field_per_degree_vs_oracle(orc):
    """The C4 batch (256 fields, degrees 31 .. 511 drawn as in the bench form): the first
    field of every degree against the oracle's separable transforms (Def. AdjVSHT eq. SLvec,
    Def. FwdVSHT eq. fwdvsht2) on the same complex64-rounded coefficients, and the forward of
    the batch's grid field against the oracle's forward of that field, bar 1e-6."""
    Ls, rng = synthetic.ragged_degrees(256, [31, 63, 127, 255, 511], seed=3)
    Ls = [int(x) for x in Ls]
    coefs = []
    for L in Ls:
        ca, cb = synthetic.coefficients(L, 1, seed=None, decay=1.0, rng=rng)
        coefs.append((ca[0].astype(np.complex64), cb[0].astype(np.complex64)))
    bp = api.BatchPlan(Ls, api.FAVEST_BF16X6, api.FAVEST_IO_C64, graph=True)
    a, b = _pack_coefs(bp, coefs, torch.complex64)
    tt, tp = bp.adj(a, b)
    ra, rb = bp.fwd(tt, tp)
    tt, tp = bp.adj(a, b)        # a second call of each replays the captured graph
    ra, rb = bp.fwd(tt, tp)
    torch.cuda.synchronize()
    assert bp.status() == 0
    for L in sorted(set(Ls)):
        i = Ls.index(L)
        x, W, _, phi = orc.grid(L)
        ca, cb = (c.astype(np.complex128) for c in coefs[i])
        ot, op = orc.adj_sep(L, x, ca, cb, len(phi))
        ht, hp = _h(bp.field(tt, i)), _h(bp.field(tp, i))
        assert normwise_err(ht.ravel(), ot.ravel()) < TOL, L
        assert normwise_err(hp.ravel(), op.ravel()) < TOL, L
        oa, ob = orc.fwd_sep(L, x, W, ht, hp)
        assert normwise_err(_h(bp.coef(ra, i)), oa) < TOL, L
        assert normwise_err(_h(bp.coef(rb, i)), ob) < TOL, L
