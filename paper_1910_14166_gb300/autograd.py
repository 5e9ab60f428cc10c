"""torch.autograd binding of the ridge / OLS solve and its hand-written
adjoint (not in the paper).

    x = ihs_ridge(A, b, lam)          # forward: IHS to convergence on the GPU
    loss(x).backward()                # backward: ihs_adjoint through the C ABI

Forward runs the library's IHS iteration (Eq. 2 with the ridge term kept
exact).  Backward solves (A^T A + lam I) v = dL/dx by conjugate gradients
preconditioned with the last sketched Cholesky factor and returns
dL/db = A v and dL/dA = r v^T - (A v) x^T with r = b - A x.
"""
from __future__ import annotations

import torch

from . import IHS


class IHSRidge(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, b, lam, m, s, seed, precision, iters):
        A_ = A.detach().contiguous()
        b_ = b.detach().contiguous().to(torch.float64)
        solver = IHS(A_, b_, kind="ridge", param=float(lam), m=m, s=s, seed=seed,
                     precision=precision)
        x, _ = solver.solve(iters=int(iters))
        ctx.solver = solver
        ctx.save_for_backward(x)
        return x.clone()

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        dLdb, dLdA, _ = ctx.solver.adjoint(x, gx.detach().contiguous().to(torch.float64),
                                           want_A=ctx.needs_input_grad[0])
        return dLdA, dLdb, None, None, None, None, None, None


def ihs_ridge(A, b, lam=1e-3, m=None, s=1, seed=0, precision="tf32", iters=40):
    """Ridge solution x = (A^T A + lam I)^{-1} A^T b by IHS, differentiable in A and b."""
    if m is None:
        m = 10 * A.shape[1]
    return IHSRidge.apply(A, b, lam, m, s, seed, precision, iters)
