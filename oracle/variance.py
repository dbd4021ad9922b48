"""Posterior variances: the diagonal of the posterior covariance Qhat^{-1} = G^{-1} (eq. Q*: the
main diagonal holds the variance of each source at each pixel), TEST INFRASTRUCTURE ONLY.

* ``exact_diag``: diag(G^{-1}) column by column from the direct factorisation (small inputs).
* ``probe_diag``: the stochastic diagonal estimator of Bekas, Kokiopoulou and Saad (2007),
  diag(G^{-1}) ~ (sum_s z_s o G^{-1} z_s) / (sum_s z_s o z_s) (element-wise), for given probe
  vectors z_s; exact when the probes are the unit vectors, unbiased for Rademacher probes.
* ``lattice_homogeneous_diag``: the exact diagonal on the periodic lattice with noise constant
  per channel, where it is the same at every pixel: the average over the Fourier modes of the
  inverse k x k mode matrices.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def exact_diag(G, k, n):
    """diag(G^{-1}) as (k, n)."""
    lu = spla.splu(sp.csc_matrix(G), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    N = G.shape[0]
    out = np.empty(N)
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        out[i] = lu.solve(e)[i]
    return out.reshape(k, n)


def probe_diag(G, Z):
    """Z: (S, k, n) probes; returns the estimate (k, n)."""
    Z = np.asarray(Z, np.float64)
    S = Z.shape[0]
    lu = spla.splu(sp.csc_matrix(G), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    num = np.zeros(Z.shape[1:])
    den = np.zeros(Z.shape[1:])
    for s in range(S):
        x = lu.solve(Z[s].reshape(-1)).reshape(Z.shape[1:])
        num += Z[s] * x
        den += Z[s] * Z[s]
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def lattice_homogeneous_diag(H, W, tau, kappa, A, d, power=1):
    """Exact posterior variances (k,) on the periodic H x W lattice with d_ci = d[c]."""
    k = A.shape[1]
    lam = (4.0 - 2.0 * np.cos(2 * np.pi * np.arange(H) / H)[:, None]
           - 2.0 * np.cos(2 * np.pi * np.arange(W) / W)[None, :]) ** power
    data = np.einsum("c,cj,cl->jl", np.asarray(d, np.float64), A, A)
    M = np.broadcast_to(data, (H, W, k, k)).copy()
    for j in range(k):
        M[:, :, j, j] += tau[j] * (kappa[j] ** 2 + lam)
    Minv = np.linalg.inv(M)
    return np.real(np.einsum("hwjj->j", Minv)) / (H * W)
