"""Pins of the oracle's learning loop (Sec. 5: parameters learned by repeated solves), no GPU:
its update uses the gradient reached by a route that does not go through the adjoint formulas
(assembled sensitivities); small steps decrease the loss; on one pixel, one source and one
channel, where the posterior mean is a scalar fraction, the whole trajectory equals gradient
descent written out by hand, and the loop finds the tau that produced its target."""

import numpy as np
import scipy.sparse as sp

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


# One pixel (no neighbours, L = 0), one source, one channel: G = tau kappa^2 + a^2 d and
# x = a d y / G with a = (nu / 100)^beta (eq. mu*), so every derivative is a fraction.
_NU, _D, _Y = 217.0, 2.5, 0.7
_STAR = (1.7, 0.9, -0.6)   # tau, kappa, beta that produce the target


def _scalar_x(t, k, b):
    a = (_NU / 100.0) ** b
    return a * _D * _Y / (t * k * k + a * a * _D)


def _scalar_loss_grad(X):
    r = X - _scalar_x(*_STAR)
    return float(np.sum(r * r)), 2.0 * r


def _scalar_learn(tau, kappa, beta, steps, lr, learn):
    return learning.learn(sp.csr_matrix((1, 1)), np.array([[_D]]), np.array([_NU]),
                          np.array([[_Y]]), _scalar_loss_grad, [tau], [kappa], [beta],
                          steps=steps, lr=lr, learn=learn)


def test_scalar_trajectory_is_hand_written_gradient_descent():
    steps, lr = 5, 0.5
    recs = _scalar_learn(2.4, 0.5, -0.2, steps, lr, ("tau", "kappa", "beta"))
    xs = _scalar_x(*_STAR)
    lt, lk, b = np.log(2.4), np.log(0.5), -0.2
    for rec in recs:
        t, k = np.exp(lt), np.exp(lk)
        a = (_NU / 100.0) ** b
        S = t * k * k + a * a * _D
        x = a * _D * _Y / S
        dl = 2.0 * (x - xs)
        g_tau = dl * (-x * k * k / S)
        g_kappa = dl * (-x * 2.0 * t * k / S)
        g_beta = dl * np.log(_NU / 100.0) * a * (_D * _Y / S) * (1.0 - 2.0 * a * a * _D / S)
        assert np.isclose(rec["tau"][0], t, rtol=1e-13)
        assert np.isclose(rec["kappa"][0], k, rtol=1e-13)
        assert np.isclose(rec["beta"][0], b, rtol=1e-13, atol=1e-15)
        assert np.isclose(rec["loss"], (x - xs) ** 2, rtol=1e-10)
        lt -= lr * t * g_tau
        lk -= lr * k * g_kappa
        b -= lr * g_beta


def test_scalar_loop_recovers_the_generating_tau():
    recs = _scalar_learn(2.0 * _STAR[0], _STAR[1], _STAR[2], 200, 5.0, ("tau",))
    assert abs(recs[-1]["tau"][0] - _STAR[0]) < 1e-9 * _STAR[0]
    assert recs[-1]["loss"] < 1e-20
