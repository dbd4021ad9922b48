"""Differentiable posterior-mean solve: ``SylvSolve`` (torch.autograd.Function).

forward(Yobs, tau, kappa, beta) -> X = G(tau, kappa, beta)^{-1} b(beta, Yobs)   (eq. mu*)
backward: one adjoint solve G lambda = dl/dX with the same operator (G is symmetric), then the
library's gradient reduction gives dl/dtau, dl/dkappa, dl/dbeta (see ``sylv_backward``).
tau, kappa, beta are CPU float64 tensors of length k; Yobs is a CUDA float64 tensor
(R, m, ld).  The graph, noise maps and frequencies are fixed inputs held by ``SylvProblem``,
which keeps ONE solver handle for them: the first forward creates it (``sylv_create``), and
every later forward or backward at other parameter values updates it in place
(``sylv_set_params``: the pixel blocks are recomputed, the graph and noise maps kept), the
repeated solves across parameter values that Sec. 5 describes.
"""

import numpy as np
import torch

from .operator import Operator


class SylvProblem:
    """Fixed parts of the system: Laplacian CSR, noise maps D, frequencies nu, mass w, and
    the one handle built on them."""

    def __init__(self, *, rowptr, col, val, D, nu, w=None, ld=None, nu0=0.0, device="cuda"):
        self.rowptr, self.col, self.val, self.D, self.nu, self.w = rowptr, col, val, D, nu, w
        self.ld, self.nu0, self.device = ld, nu0, device
        self._op = None
        self._theta = None

    def operator(self, tau, kappa, beta):
        """The handle with prior scalars tau, kappa and spectral indices beta (host arrays):
        created on the first call, updated in place when the values differ from the last."""
        theta = tuple(np.asarray(v, dtype=np.float64).reshape(-1).tobytes()
                      for v in (tau, kappa, beta))
        if self._op is None:
            self._op = Operator(rowptr=self.rowptr, col=self.col, val=self.val, D=self.D,
                                tau=tau, kappa=kappa, nu=self.nu, beta=beta, w=self.w,
                                ld=self.ld, nu0=self.nu0, device=self.device)
        elif theta != self._theta:
            self._op.set_params(tau, kappa, beta=beta)
        self._theta = theta
        return self._op

    def close(self):
        if self._op is not None:
            self._op.close()
            self._op = None
            self._theta = None


class SylvSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Yobs, tau, kappa, beta, problem, solve_kw):
        theta = tuple(t.detach().cpu().numpy().copy() for t in (tau, kappa, beta))
        op = problem.operator(*theta)
        Y = Yobs if Yobs.dim() == 3 else Yobs.unsqueeze(0)
        X, info = op.solve(op.rhs(Y), **solve_kw)
        ctx.problem = problem
        ctx.theta = theta
        ctx.solve_kw = solve_kw
        ctx.squeeze = Yobs.dim() == 2
        ctx.save_for_backward(Y, X)
        ctx.info = info
        return X[0] if ctx.squeeze else X

    @staticmethod
    def backward(ctx, grad_X):
        Y, X = ctx.saved_tensors
        g = grad_X.unsqueeze(0) if ctx.squeeze else grad_X
        # the handle may have moved to another forward's parameters since: back to this one's
        op = ctx.problem.operator(*ctx.theta)
        gt, gk, gb, _, _ = op.backward(X, g.contiguous().to(torch.float64), Y, **ctx.solve_kw)
        as_t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64)  # noqa: E731
        return None, as_t(gt), as_t(gk), as_t(gb), None, None


def sylv_solve_differentiable(Yobs, tau, kappa, beta, problem, **solve_kw):
    return SylvSolve.apply(Yobs, tau, kappa, beta, problem, solve_kw)
