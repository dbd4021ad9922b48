"""Derivatives of a loss on the posterior mean (TEST INFRASTRUCTURE ONLY).

The posterior mean X(theta) solves G(theta) x = b(theta) (eq. mu*), with theta the prior
hyperparameters tau_j, kappa_j and the spectral indices beta_j of the power-law mixing matrix
a_cj = (nu_c/100)^beta_j.  The paper fixes these (Sec. 5 notes they must be learned by repeated
solves); differentiating the solve is the derived step used here:

    dl = <g, dX>,  G dX = db - dG X   =>   dl/dtheta = lambda^T (db/dtheta - dG/dtheta X),
    with G lambda = g = dl/dX  (G symmetric, so the adjoint solve uses the same operator).

Three routes, used to pin each other:
* ``adjoint_gradient``: the closed formulas below, one adjoint solve.
* ``sensitivity_gradient``: dG/dtheta and db/dtheta assembled as sparse matrices and one
  forward sensitivity solve per parameter.
* ``fd_gradient``: central finite differences of the direct solve.

Formulas (per source j; W the mass diagonal, L the Laplacian):
    dl/dtau_j   = -lambda_j^T (kappa_j^2 W + L) x_j
    dl/dkappa_j = -2 tau_j kappa_j lambda_j^T W x_j
    dl/dbeta_j  = sum_c ln(nu_c/100) a_cj [ lambda_j^T D_c y_c - (lambda a_c)^T D_c x_j
                                           - lambda_j^T D_c (X a_c) ]
summed over right-hand sides when several are given.
"""

import numpy as np
import scipy.sparse as sp

from . import model, solve


def _as_batch(Z):
    Z = np.asarray(Z, np.float64)
    return Z[None] if Z.ndim == 2 else Z


def posterior_mean(L, D, tau, kappa, nu, beta, Y, w=None):
    A = model.powerlaw_mixing(nu, beta)
    G = model.assemble_G(L, D, tau, kappa, A, w)
    Yb = _as_batch(Y)
    b = np.stack([model.rhs(D, y, A) for y in Yb])
    return solve.solve_direct(G, b), G, A


def adjoint_gradient(L, D, tau, kappa, nu, beta, Y, X, g, w=None):
    """Returns (g_tau, g_kappa, g_beta, lambda) for loss gradient g = dl/dX."""
    A = model.powerlaw_mixing(nu, beta)
    G = model.assemble_G(L, D, tau, kappa, A, w)
    lam = solve.solve_direct(G, _as_batch(g))
    gt, gk, gb = gradient_from_adjoint(L, D, tau, kappa, nu, beta, Y, X, lam, w)
    return gt, gk, gb, (lam[0] if np.ndim(X) == 2 else lam)


def gradient_from_adjoint(L, D, tau, kappa, nu, beta, Y, X, lam, w=None):
    """The three gradient formulas for a given adjoint lambda (= G^{-1} dl/dX)."""
    A = model.powerlaw_mixing(nu, beta)
    Xb, Yb = _as_batch(X), _as_batch(Y)
    lam = _as_batch(lam)
    k = A.shape[1]
    n = L.shape[0]
    wv = np.ones(n) if w is None else np.asarray(w, np.float64)
    logf = np.log(np.asarray(nu, np.float64) / 100.0)
    g_tau = np.zeros(k)
    g_kappa = np.zeros(k)
    g_beta = np.zeros(k)
    for r in range(Xb.shape[0]):
        x, lm, y = Xb[r], lam[r], Yb[r]
        for j in range(k):
            Lx = L @ x[j]
            g_tau[j] -= lm[j] @ (kappa[j] ** 2 * wv * x[j] + Lx)
            g_kappa[j] -= 2.0 * tau[j] * kappa[j] * (lm[j] @ (wv * x[j]))
        Xa = A @ x          # (m, n): X a_c
        La = A @ lm         # (m, n): lambda a_c
        for c in range(A.shape[0]):
            for j in range(k):
                g_beta[j] += logf[c] * A[c, j] * (
                    lm[j] @ (D[c] * y[c]) - La[c] @ (D[c] * x[j]) - lm[j] @ (D[c] * Xa[c]))
    return g_tau, g_kappa, g_beta


def sensitivity_gradient(L, D, tau, kappa, nu, beta, Y, g, w=None):
    """dl/dtheta = <g, G^{-1}(db/dtheta - dG/dtheta X)> with assembled derivative matrices."""
    X, G, A = posterior_mean(L, D, tau, kappa, nu, beta, Y, w)
    dA = model.powerlaw_mixing_dbeta(nu, beta)
    k = A.shape[1]
    m = A.shape[0]
    n = L.shape[0]
    Wm = sp.identity(n) if w is None else sp.diags(np.asarray(w, np.float64))
    Yb = _as_batch(Y)
    gb = _as_batch(g)
    xs = X.reshape(X.shape[0], -1)

    def directional(dG, db):
        rhs_ = db - np.stack([dG @ xs[r] for r in range(xs.shape[0])])
        dX = solve.solve_direct(G, rhs_.reshape(X.shape))
        return float(np.sum(gb * dX))

    def Ejj(j):
        return sp.csr_matrix(([1.0], ([j], [j])), shape=(k, k))

    zero_b = np.zeros_like(xs)
    g_tau = np.array([directional(sp.kron(Ejj(j), kappa[j] ** 2 * Wm + L), zero_b)
                      for j in range(k)])
    g_kappa = np.array([directional(sp.kron(Ejj(j), 2 * tau[j] * kappa[j] * Wm), zero_b)
                        for j in range(k)])
    g_beta = np.zeros(k)
    for j in range(k):
        dGj = None
        for c in range(m):
            da = np.zeros(k)
            da[j] = dA[c, j]
            outer = np.outer(da, A[c]) + np.outer(A[c], da)      # d(a_c a_c^T)/d beta_j
            blk = sp.kron(sp.csr_matrix(outer), sp.diags(D[c]))
            dGj = blk if dGj is None else dGj + blk
        dbs = []
        for r in range(Yb.shape[0]):
            db = np.zeros((k, n))
            for c in range(m):
                db[j] += dA[c, j] * D[c] * Yb[r, c]
            dbs.append(db.reshape(-1))
        g_beta[j] = directional(dGj, np.stack(dbs))
    return g_tau, g_kappa, g_beta


def fd_gradient(loss_of_X, L, D, tau, kappa, nu, beta, Y, h=1e-6, w=None):
    """Central differences of loss(X(theta)) with X from the direct solve, step h (relative
    to max(1, |theta|))."""
    def f(t, kp, b):
        X, _, _ = posterior_mean(L, D, t, kp, nu, b, Y, w)
        return loss_of_X(X[0] if np.ndim(Y) == 2 else X)

    out = []
    for which in range(3):
        base = [np.array(tau, float), np.array(kappa, float), np.array(beta, float)]
        gr = np.zeros(len(base[which]))
        for j in range(len(gr)):
            step = h * max(1.0, abs(base[which][j]))
            plus = [v.copy() for v in base]
            minus = [v.copy() for v in base]
            plus[which][j] += step
            minus[which][j] -= step
            gr[j] = (f(*plus) - f(*minus)) / (2 * step)
        out.append(gr)
    return tuple(out)
