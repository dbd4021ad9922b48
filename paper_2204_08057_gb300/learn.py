"""Learning the prior and mixing parameters by repeated solves (Sec. 5: the parameters of A and
Q are learned by solving the system for many of their values).

``HyperLearner`` runs gradient descent on a loss of the posterior mean over theta =
(log tau, log kappa, beta): per step the handle's parameters are replaced in place
(``sylv_set_params``: only the per-pixel blocks are rebuilt), the right-hand side is formed for
the new mixing, the forward solve starts from the previous step's posterior mean and the
adjoint solve from the previous adjoint (warm starts, the simplest recycling of earlier solves
across theta), and ``sylv_backward`` gives the gradient.  Every solve and reduction runs in the
library's kernels; this driver only holds theta and the step rule.
"""

import numpy as np


class HyperLearner:
    """loss_grad(X) -> (loss, dl/dX) for the (R, k, ld) posterior mean X, as float, tensor."""

    def __init__(self, op, Yobs, loss_grad, tau, kappa, beta, *, lr=0.05,
                 learn=("tau", "kappa", "beta"), warm=True, normalize=False, **solve_kw):
        self.op = op
        self.Y = Yobs
        self.loss_grad = loss_grad
        self.log_tau = np.log(np.asarray(tau, np.float64))
        self.log_kappa = np.log(np.asarray(kappa, np.float64))
        self.beta = np.asarray(beta, np.float64).copy()
        self.lr = float(lr)
        self.learn = tuple(learn)
        self.warm = bool(warm)
        self.normalize = bool(normalize)   # steps of length lr along -gradient
        self.solve_kw = dict(solve_kw)
        self.X = None
        self.lam = None
        self.history = []

    @property
    def theta(self):
        return np.exp(self.log_tau), np.exp(self.log_kappa), self.beta.copy()

    def step(self):
        tau, kappa, beta = self.theta
        self.op.set_params(tau, kappa, beta=beta)
        Bv = self.op.rhs(self.Y)
        X0 = self.X if (self.warm and self.X is not None) else None
        X, info = self.op.solve(Bv, X0, **self.solve_kw)
        loss, g = self.loss_grad(X)
        lam0 = self.lam if (self.warm and self.lam is not None) else None
        gt, gk, gb, lam, info_b = self.op.backward(X, g, self.Y, lam0=lam0, **self.solve_kw)
        # chain rule to log tau, log kappa: dl/dlog(t) = t dl/dt
        d_tau = tau * gt if "tau" in self.learn else 0.0 * gt
        d_kappa = kappa * gk if "kappa" in self.learn else 0.0 * gk
        d_beta = gb if "beta" in self.learn else 0.0 * gb
        scale = self.lr
        if self.normalize:
            norm = np.sqrt(np.sum(d_tau ** 2) + np.sum(d_kappa ** 2) + np.sum(d_beta ** 2))
            scale = self.lr / norm if norm > 0 else 0.0
        self.log_tau -= scale * d_tau
        self.log_kappa -= scale * d_kappa
        self.beta -= scale * d_beta
        self.X, self.lam = X, lam
        rec = {"loss": float(loss), "forward_iterations": info["iterations"],
               "adjoint_iterations": info_b["iterations"], "tau": tau.tolist(),
               "kappa": kappa.tolist(), "beta": beta.tolist()}
        self.history.append(rec)
        return rec
