"""FAVEST_FLAG_SHARE_LAMBDA: one recurrence pass of the split path serves an adjoint and the
forward call after it (or the reverse).  The Legendre values lambda_l^m(theta_j) (Sec. 3,
definition of Y_lm) do not depend on the direction, so the shared pass must give results
bitwise identical to two separate passes, and launch exactly one generator per pair."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api, synthetic  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _dev(a, dtype=torch.complex64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _gens(prof):
    return {k: v[1] for k, v in prof.items() if k.startswith("gen_lambda")}


@pytest.mark.parametrize("L,B,io", [(63, 4, api.FAVEST_IO_C64), (300, 8, api.FAVEST_IO_C64),
                                    (511, 32, api.FAVEST_IO_C64), (127, 6, api.FAVEST_IO_R32)])
def test_shared_pair_bitwise_equal(L, B, io):
    plan = api.Plan(L, B, api.FAVEST_BF16X6, io)
    if io == api.FAVEST_IO_R32:
        a, b = synthetic.half_coefficients(L, B, seed=L)
    else:
        a, b = synthetic.coefficients(L, B, seed=L)
    da, db = _dev(a), _dev(b)
    # reference: each call generates its own layout
    t0, p0 = plan.adj(da, db)
    a0, b0 = plan.fwd(t0, p0)
    # adjoint then forward sharing one pass
    plan.profile(True)
    plan.profile_read()
    t1, p1 = plan.adj(da, db, share_lambda=True)
    a1, b1 = plan.fwd(t1, p1, share_lambda=True)
    prof = plan.profile_read()
    assert _gens(prof) == {"gen_lambda_both": 1}
    # forward then adjoint sharing one pass (the order of a backward pass)
    a2, b2 = plan.fwd(t0, p0, share_lambda=True)
    t2, p2 = plan.adj(da, db, share_lambda=True)
    prof = plan.profile_read()
    plan.profile(False)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert _gens(prof) == {"gen_lambda_both": 1}
    for x, y in [(t0, t1), (p0, p1), (a0, a1), (b0, b1), (a0, a2), (b0, b2), (t0, t2), (p0, p2)]:
        assert torch.equal(x, y)
    plan.close()


def test_pairing_rules():
    """A flagged call reuses the operand only right after a flagged call of the other
    direction; two flagged calls of the same direction each generate; an unflagged call in
    between ends the pairing; FP64 plans accept the flag and launch no generator."""
    L, B = 95, 4
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    a, b = synthetic.coefficients(L, B, seed=5)
    da, db = _dev(a), _dev(b)
    t, p = plan.adj(da, db)
    ref_a, ref_b = plan.fwd(t, p)
    plan.profile(True)
    plan.profile_read()
    plan.adj(da, db, t, p, share_lambda=True)
    plan.adj(da, db, t, p, share_lambda=True)
    assert _gens(plan.profile_read()) == {"gen_lambda_both": 2}
    plan.adj(da, db, t, p, share_lambda=True)
    plan.adj(da, db, t, p)                               # ends the pairing
    ga, gb = plan.fwd(t, p, share_lambda=True)           # so this one generates again
    assert _gens(plan.profile_read()) == {"gen_lambda_both": 2, "gen_lambda_adj": 1}
    plan.fwd(t, p, ga, gb, share_lambda=True)
    plan.profile(False)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(ga, ref_a) and torch.equal(gb, ref_b)
    plan.close()
    p64 = api.Plan(L, B, api.FAVEST_FP64, api.FAVEST_IO_C64)
    p64.profile(True)
    t64, q64 = p64.adj(da, db, share_lambda=True)
    x64, y64 = p64.fwd(t64, q64, share_lambda=True)
    prof = p64.profile_read()
    torch.cuda.synchronize()
    assert not _gens(prof) and p64.status() == 0
    p64.close()


def test_pair_captured_in_a_cuda_graph():
    """An adjoint and forward pair sharing one generator pass, with the polar patch on the
    plan's side stream, captured into a CUDA graph by the caller and replayed: bitwise the
    eager results, and again after new coefficients are copied into the captured buffers."""
    L, B = 255, 8
    plan = api.Plan(L, B, api.FAVEST_BF16X6, api.FAVEST_IO_C64)
    a0, b0 = synthetic.coefficients(L, B, seed=41, decay=1.0)
    a1, b1 = synthetic.coefficients(L, B, seed=42, decay=1.0)
    a = torch.as_tensor(a0).to(torch.complex64).cuda()
    b = torch.as_tensor(b0).to(torch.complex64).cuda()
    tt = torch.empty(plan.field_shape(), dtype=torch.complex64, device="cuda")
    tp = torch.empty_like(tt)
    ra = torch.empty_like(a)
    rb = torch.empty_like(b)

    def step():
        plan.adj(a, b, tt, tp, share_lambda=True)
        plan.fwd(tt, tp, ra, rb, share_lambda=True)

    eager = []
    for ca, cb in ((a0, b0), (a1, b1)):
        a.copy_(torch.as_tensor(ca).to(torch.complex64))
        b.copy_(torch.as_tensor(cb).to(torch.complex64))
        step()
        torch.cuda.synchronize()
        eager.append((tt.clone(), tp.clone(), ra.clone(), rb.clone()))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                                   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        step()
    for k, (ca, cb) in enumerate(((a0, b0), (a1, b1))):
        a.copy_(torch.as_tensor(ca).to(torch.complex64))
        b.copy_(torch.as_tensor(cb).to(torch.complex64))
        g.replay()
        torch.cuda.synchronize()
        assert plan.status() == 0
        for got, ref in zip((tt, tp, ra, rb), eager[k]):
            assert torch.equal(got, ref)
    plan.close()
