"""torch.autograd wrapper of the truncated factorization (Q1, [R11 R12]) with the permutation
held fixed.  Forward: rqrcp_factor / rqrcp_factor_mixed + rqrcp_lowrank(_f32) for Q1; backward:
rqrcp_backward(_f32).  Argument marshalling only: every step runs in librqrcp's kernels."""
from __future__ import annotations

import torch

from . import binding


def _check(code, where):
    if code != binding.RQRCP_OK:
        raise binding.RQRCPError(code, where)


def truncated_factor(A, k: int, b: int = 64, p: int = 8, seed: int = 0):
    """(Q1, R, jpvt) with A[:, jpvt] ~= Q1 @ R: Q1 is m x k, R = [R11 R12] is k x n (pivoted
    column order, R11 upper triangular).  FP64 input runs the plain form, FP32 the mixed form."""
    if A.dtype == torch.float64:
        f = binding.factor(A, k, b, p, seed)
    elif A.dtype == torch.float32:
        f = binding.factor_mixed(A, k, b, p, seed)
    else:
        raise TypeError("truncated_factor expects float64 or float32")
    m, n = A.shape
    Q1 = torch.empty((k, m), dtype=A.dtype, device=A.device).t()
    work = binding.workspace(binding.rqrcp_lowrank_workspace_size(m, n, k), A.device)
    _check(binding.rqrcp_lowrank(f.A, k, f.tau, f.jpvt, None, Q1, work), "rqrcp_lowrank")
    code, _ = binding.rqrcp_read_status(work)
    _check(code, "device status")
    R = binding.colmajor(torch.triu(f.A[:k, :]))
    return Q1, R, f.jpvt


class RQRCPFunction(torch.autograd.Function):
    """apply(A, k, b, p, seed) -> (Q1, R, jpvt); gradients flow to A through Q1 and R."""

    @staticmethod
    def forward(ctx, A, k, b, p, seed):
        Acm = binding.colmajor(A.detach())
        Q1, R, jpvt = truncated_factor(Acm, k, b, p, seed)
        ctx.save_for_backward(Acm, jpvt, Q1, R)
        ctx.mark_non_differentiable(jpvt)
        return Q1, R, jpvt

    @staticmethod
    def backward(ctx, dQ1, dR, _djpvt):
        Acm, jpvt, Q1, R = ctx.saved_tensors
        m, n = Acm.shape
        k = Q1.shape[1]
        dt = Acm.dtype
        dQ1 = torch.zeros_like(Q1) if dQ1 is None else binding.colmajor(dQ1.to(dt))
        dR = torch.zeros_like(R) if dR is None else binding.colmajor(dR.to(dt))
        dA = torch.empty((n, m), dtype=dt, device=Acm.device).t()
        prec = binding.RQRCP_PREC_FP64 if dt == torch.float64 else binding.RQRCP_PREC_MIXED
        work = binding.workspace(binding.rqrcp_backward_workspace_size(m, n, k, prec), Acm.device)
        _check(binding.rqrcp_backward(Acm, jpvt, Q1, R, dQ1, dR, dA, work), "rqrcp_backward")
        code, _ = binding.rqrcp_read_status(work)
        _check(code, "device status")
        return dA, None, None, None, None


def rqrcp_truncated(A, k: int, b: int = 64, p: int = 8, seed: int = 0):
    return RQRCPFunction.apply(A, k, b, p, seed)
