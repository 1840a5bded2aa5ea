"""Differentiation through the truncated block product (hand-written adjoint).

The LNV method minimises Omega(L) = 2 Tr[(3LSL - 2LSLSL)(H - mu S)]
(Sec. 2.3.2, Eq. 8) using its gradient with respect to L; forces and
stresses need the derivative with respect to H (Sec. 3.1).  Both follow
from the adjoints of the two operations Omega is built from:

  C = (A.B)|pat(C):   dA = (dC . B^T)|pat(A),   dB = (A^T . dC)|pat(B)
  t = Tr[X Y]:        dX = t_bar (Y^T)|pat(X),  dY = t_bar (X^T)|pat(Y)

Each adjoint is itself a truncated product or a masked transpose and runs
in the library's kernels (lsq_block_matmul with transpose flags,
lsq_transpose); this module only wires them into torch.autograd.
"""
import torch
from torch.utils.checkpoint import checkpoint

from . import F64, block_matmul, trace, transpose


def _prec(t):
    return F64 if t.dtype == torch.float64 else 1


class BlockMatmulFn(torch.autograd.Function):
    """C = A.B on pattern range_c (A on range_a, B on range_b)."""

    @staticmethod
    def forward(ctx, A, B, geom, b, ra, rb, rc):
        prec = _prec(A)
        C = torch.empty((geom.nnzb(rc), b, b), dtype=A.dtype, device=A.device)
        block_matmul(geom, b, A.contiguous(), ra, B.contiguous(), rb, C, rc, precision=prec)
        ctx.save_for_backward(A, B)
        ctx.meta = (geom, b, ra, rb, rc, prec)
        return C

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        geom, b, ra, rb, rc, prec = ctx.meta
        dC = dC.contiguous()
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = torch.empty_like(A)
            block_matmul(geom, b, dC, rc, B, rb, dA, ra, precision=prec, trans_b=True)
        if ctx.needs_input_grad[1]:
            dB = torch.empty_like(B)
            block_matmul(geom, b, A, ra, dC, rc, dB, rb, precision=prec, trans_a=True)
        return dA, dB, None, None, None, None, None


class TraceFn(torch.autograd.Function):
    """t = Tr[X Y] (X on range_x, Y on range_y), accumulated in float64."""

    @staticmethod
    def forward(ctx, X, Y, geom, b, rx, ry):
        prec = _prec(X)
        t = trace(geom, b, X.contiguous(), rx, Y.contiguous(), ry, precision=prec)
        ctx.save_for_backward(X, Y)
        ctx.meta = (geom, b, rx, ry, prec)
        return torch.tensor(t, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, g):
        # dX = g (Y^T)|pat(X): the masked transpose runs with alpha = 1 and the scaling by the
        # incoming gradient stays on the device (no host synchronisation)
        X, Y = ctx.saved_tensors
        geom, b, rx, ry, prec = ctx.meta
        dX = dY = None
        if ctx.needs_input_grad[0]:
            dX = torch.empty_like(X)
            transpose(geom, b, Y.contiguous(), ry, dX, rx, precision=prec)
            dX.mul_(g.to(dX.dtype))
        if ctx.needs_input_grad[1]:
            dY = torch.empty_like(Y)
            transpose(geom, b, X.contiguous(), rx, dY, ry, precision=prec)
            dY.mul_(g.to(dY.dtype))
        return dX, dY, None, None, None, None


def block_matmul_ad(geom, b, A, ra, B, rb, rc):
    """Differentiable truncated product C = (A.B)|range_c."""
    return BlockMatmulFn.apply(A, B, geom, b, ra, rb, rc)


def trace_ad(geom, b, X, rx, Y, ry):
    return TraceFn.apply(X, Y, geom, b, rx, ry)


def lnv_omega(geom, b, L, S, H, mu, ranges, spin=2.0, recompute=True):
    """Differentiable Omega(L, S, H) (eV), general (not necessarily symmetric) L.

    ranges = (R_S, R_H, R_L, R_LS, R3) range ids of geom: S, H, L, L+S and
    H+L+S.  Omega = spin [3 (Tr[LSL H] - mu Tr[LSL S]) - 2 (Tr[LSLSL H] -
    mu Tr[LSLSL S])], with LSL kept on R3 and LSLSL on H's range, so H - mu S
    is never formed.  With recompute=True the intermediates LS, SL, LSL and
    LSLSL are not stored for backward; they are recomputed from L, S, H.
    """
    rS, rH, rL, r1, r3 = ranges

    def body(L, S, H):
        LS = block_matmul_ad(geom, b, L, rL, S, rS, r1)
        SL = block_matmul_ad(geom, b, S, rS, L, rL, r1)
        LSL = block_matmul_ad(geom, b, LS, r1, L, rL, r3)
        LSLSL = block_matmul_ad(geom, b, LSL, r3, SL, r1, rH)
        t_lsl = trace_ad(geom, b, H, rH, LSL, r3) - mu * trace_ad(geom, b, S, rS, LSL, r3)
        t_5 = trace_ad(geom, b, H, rH, LSLSL, rH) - mu * trace_ad(geom, b, S, rS, LSLSL, rH)
        return spin * (3.0 * t_lsl - 2.0 * t_5)

    if recompute and torch.is_grad_enabled():
        return checkpoint(body, L, S, H, use_reentrant=False)
    return body(L, S, H)
