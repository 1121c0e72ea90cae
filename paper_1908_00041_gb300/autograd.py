"""Reverse-mode differentiation of FwdVSHT and AdjVSHT (torch.autograd.Function).

Writing A for AdjVSHT (coefficients (a, b) -> tangent field (T_theta, T_phi) on the
grid, Def. AdjVSHT, eq. SLvec) and W for the diagonal of point weights W_j 2 pi / nphi,
FwdVSHT (Def. FwdVSHT, eq. fwdvsht2) is A^H W.  Both maps are complex-linear, so the
vector-Jacobian product of each is its Hermitian transpose applied to the incoming
gradient (PyTorch's complex gradients are conjugate Wirtinger derivatives, for which a
linear map M back-propagates by M^H):

    FwdVSHT backward:  grad_T = W A grad_(a,b)       weighted adjoint kernel path
    AdjVSHT backward:  grad_(a,b) = A^H grad_T       forward kernel path, unit weights

Both backward passes run the library's own kernels (favest_adj_ex with
FAVEST_FLAG_WEIGHTED, favest_fwd_ex with FAVEST_FLAG_UNIT_WEIGHTS); the Legendre
values are regenerated by the recurrence inside those kernels, nothing is stored
between the forward and the backward pass.

Real-field plans map real fields to half spectra (orders m >= 0).  Their vector-Jacobian
products are the transposes for the real inner products, which add per-order factors
(FAVEST_FLAG_REAL_TRANSPOSE): FwdVSHT back-propagates by W Re sum_{m>=0} g_lm Y_lm (the
weighted real adjoint with orders m > 0 halved), AdjVSHT by the unit-weight real forward
with orders m > 0 doubled.
"""
import torch

from . import api


def _contig(t, dtype):
    """t as a contiguous tensor of the plan's dtype (None stays None)."""
    if t is None:
        return None
    return t.to(dtype).contiguous()


class _FwdVSHT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Tth, Tph, plan):
        ctx.plan = plan
        fd = getattr(plan, "fdtype", plan.cdtype)
        a, b = plan.fwd(_contig(Tth, fd), _contig(Tph, fd), stream=torch.cuda.current_stream().cuda_stream)
        return a, b

    @staticmethod
    def backward(ctx, ga, gb):
        plan = ctx.plan
        if ga is None:
            ga = torch.zeros(plan.coef_shape(), dtype=plan.cdtype, device="cuda")
        if gb is None:
            gb = torch.zeros(plan.coef_shape(), dtype=plan.cdtype, device="cuda")
        gt, gp = plan.adj(_contig(ga, plan.cdtype), _contig(gb, plan.cdtype), weighted=True,
                          real_transpose=getattr(plan, "real", False),
                          stream=torch.cuda.current_stream().cuda_stream)
        return gt, gp, None


class _AdjVSHT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, plan):
        ctx.plan = plan
        Tth, Tph = plan.adj(_contig(a, plan.cdtype), _contig(b, plan.cdtype),
                            stream=torch.cuda.current_stream().cuda_stream)
        return Tth, Tph

    @staticmethod
    def backward(ctx, gt, gp):
        plan = ctx.plan
        fd = getattr(plan, "fdtype", plan.cdtype)
        if gt is None:
            gt = torch.zeros(plan.field_shape(), dtype=fd, device="cuda")
        if gp is None:
            gp = torch.zeros(plan.field_shape(), dtype=fd, device="cuda")
        ga, gb = plan.fwd(_contig(gt, fd), _contig(gp, fd), unit_weights=True,
                          real_transpose=getattr(plan, "real", False),
                          stream=torch.cuda.current_stream().cuda_stream)
        return ga, gb, None


def fwd_vsht(plan, Tth, Tph):
    """Differentiable FwdVSHT: (Tth, Tph) [batch, L+1, 2(L+1)] -> (a, b) [batch, K]
    (K = L^2+2L, or L(L+3)/2 for a real-field plan)."""
    return _FwdVSHT.apply(Tth, Tph, plan)


def adj_vsht(plan, a, b):
    """Differentiable AdjVSHT: (a, b) [batch, K] -> (Tth, Tph) [batch, L+1, 2(L+1)]."""
    return _AdjVSHT.apply(a, b, plan)
