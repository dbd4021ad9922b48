"""Pins of the oracle's learning loop (Sec. 5: parameters learned by repeated solves), no GPU:
its update uses the gradient reached by a route that does not go through the adjoint formulas
(assembled sensitivities), and small steps decrease the loss."""

import numpy as np

import synth
from oracle import gradient, learning, model


def _setup():
    g = synth.latlong_sphere(5, 6)
    nu = synth.PLANCK_NU[[0, 3, 5, 7, 8]]
    p = synth.make_problem("learn", g, 3, nu, [-2.0, 0.5, 1.5], [0.2, 0.5, 1.0],
                           [1.0, 2.0, 0.5], 31, noise="lognormal")
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)
    Xt = p.X_true

    def loss_grad(X):
        d = X - Xt
        return float(np.sum(d * d)), 2.0 * d
    return p, L, loss_grad


def test_update_uses_the_sensitivity_gradient():
    p, L, lg = _setup()
    tau0, kappa0, beta0 = np.array([0.8, 1.5, 0.7]), np.array([0.3, 0.4, 0.9]), p.beta + 0.1
    recs = learning.learn(L, p.D, p.nu, p.Yobs[0], lg, tau0, kappa0, beta0, steps=2, lr=1e-3)
    X, _, _ = gradient.posterior_mean(L, p.D, tau0, kappa0, p.nu, beta0, p.Yobs[0])
    gs = gradient.sensitivity_gradient(L, p.D, tau0, kappa0, p.nu, beta0, p.Yobs[0],
                                       lg(X[0])[1])
    exp_tau = np.exp(np.log(tau0) - 1e-3 * tau0 * gs[0])
    exp_kappa = np.exp(np.log(kappa0) - 1e-3 * kappa0 * gs[1])
    exp_beta = beta0 - 1e-3 * gs[2]
    assert np.allclose(recs[1]["tau"], exp_tau, rtol=1e-10)
    assert np.allclose(recs[1]["kappa"], exp_kappa, rtol=1e-10)
    assert np.allclose(recs[1]["beta"], exp_beta, rtol=1e-10, atol=1e-12)


def test_small_steps_decrease_the_loss():
    p, L, lg = _setup()
    recs = learning.learn(L, p.D, p.nu, p.Yobs[0], lg, [0.5, 3.0, 2.0], [0.5, 0.2, 0.3],
                          p.beta + 0.2, steps=6, lr=2e-3)
    losses = [r["loss"] for r in recs]
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
