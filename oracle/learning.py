"""The learning loop of ``paper_2204_08057_gb300.learn`` on the oracle (TEST INFRASTRUCTURE
ONLY): gradient descent over (log tau, log kappa, beta) on a loss of the posterior mean, with
the direct solve and the adjoint gradient formulas of ``gradient``."""

import numpy as np

from . import gradient


def learn(L, D, nu, Y, loss_grad, tau, kappa, beta, steps, lr, learn=("tau", "kappa", "beta"),
          w=None):
    """loss_grad(X (k, n) or (R, k, n)) -> (loss, dl/dX).  Returns the list of per-step records
    (loss and the theta at which it was evaluated)."""
    log_tau = np.log(np.asarray(tau, np.float64))
    log_kappa = np.log(np.asarray(kappa, np.float64))
    beta = np.asarray(beta, np.float64).copy()
    out = []
    for _ in range(steps):
        t, kp = np.exp(log_tau), np.exp(log_kappa)
        X, _, _ = gradient.posterior_mean(L, D, t, kp, nu, beta, Y, w)
        Xs = X[0] if np.ndim(Y) == 2 else X
        loss, g = loss_grad(Xs)
        gt, gk, gb, _ = gradient.adjoint_gradient(L, D, t, kp, nu, beta, Y, Xs, g, w)
        out.append({"loss": float(loss), "tau": t.copy(), "kappa": kp.copy(), "beta": beta.copy()})
        if "tau" in learn:
            log_tau -= lr * t * gt
        if "kappa" in learn:
            log_kappa -= lr * kp * gk
        if "beta" in learn:
            beta -= lr * gb
    return out
