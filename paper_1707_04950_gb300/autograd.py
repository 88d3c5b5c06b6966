"""torch.autograd.Function over the C ABI: an efficiency e_n of the surface given by its Fourier
coefficients, differentiable in those coefficients through sgf_gradient (the discrete adjoint of the
accelerated system). Marshalling only: the solve and the gradient run in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sgf


class Efficiency(torch.autograd.Function):
    """e = Efficiency.apply(a, b, par, n, precision, tol): a, b float64 tensors of the cosine and sine
    coefficients (a[0] the mean height, b[0] ignored), par the remaining problem parameters (a
    workload dictionary of paper_1707_04950_gb300.inputs), n the Rayleigh mode. The forward pass
    builds the operator and solves; the backward pass runs the adjoint solve and returns
    de_n/da, de_n/db (the operator keeps the cell assignment of the forward build)."""

    @staticmethod
    def forward(ctx, a, b, par, n=0, precision=64, tol=1e-12):
        p = dict(par, a=a.detach().cpu().numpy().astype(np.float64), b=b.detach().cpu().numpy().astype(np.float64))
        op = sgf.Operator(p, precision=precision)
        mu = torch.zeros(p["N"], dtype=torch.complex128, device="cuda")
        st, its, rr = sgf.sgf_solve(op.ctx, tol, 4000, mu.data_ptr())
        if st != 0:
            op.close()
            raise sgf.SgfError(st, f"forward solve stopped at relative residual {rr:g} after {its} applications")
        _, eff, _ = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), n, n)
        ctx.op, ctx.mu, ctx.n, ctx.tol, ctx.M = op, mu, n, tol, len(p["a"]) - 1
        ctx.dtype, ctx.device = a.dtype, a.device
        return torch.tensor(float(eff[0]), dtype=a.dtype, device=a.device)

    @staticmethod
    def backward(ctx, grad_out):
        ga, gb, _, _, _ = sgf.sgf_gradient(ctx.op.ctx, ctx.mu.data_ptr(), ctx.n, ctx.M, ctx.tol)
        ctx.op.close()
        ga = torch.from_numpy(ga).to(dtype=ctx.dtype, device=ctx.device)
        gb = torch.from_numpy(gb).to(dtype=ctx.dtype, device=ctx.device)
        return grad_out * ga, grad_out * gb, None, None, None, None


def efficiency(a, b, par, n=0, precision=64, tol=1e-12):
    return Efficiency.apply(a, b, par, n, precision, tol)
