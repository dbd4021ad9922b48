"""Exact solutions of special cases of G x = b that avoid the assembled matrix
(TEST INFRASTRUCTURE ONLY).

They pin ``model``/``solve`` and, at full sizes, the GPU solver, because each reaches
eq. mu* by a different route:

* ``lattice_homogeneous``: periodic lattice, noise constant per channel.  A 2-D DFT
  diagonalises L (eigenvalues 4 - 2cos(2 pi p/H) - 2cos(2 pi q/W)), hence L^2 and every Q_j at
  once; each Fourier mode leaves a k x k system.
* ``sphere_latitude_noise``: latitude-longitude sphere, noise depending on the row only.  A DFT
  in longitude decouples the modes; each is a symmetric block-tridiagonal system in latitude
  (H blocks of k x k) solved as a banded Cholesky.
* ``sylvester_separable``: separable noise d_ci = t_c nu_i (C = T kron N, Sec. 3) and a common
  prior Q_j = phi_j Q_0; the system is the Sylvester equation eq. Axb-Sylv,
  N^{-1} Q_0 M + M A^T T A P^{-1} = Y T A P^{-1}, solved by Bartels-Stewart.
* ``scalar_posterior``: k = m = 1, the textbook posterior mean of a Gaussian field observed
  with Gaussian noise, (tau (kappa^2 I + L) + a^2 D) x = a D y.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def lattice_homogeneous(H, W, tau, kappa, A, d, Y, power=1):
    """X (k, H*W) for the periodic lattice with d_ci = d[c]; Y is (m, H*W).  ``power`` = 2
    takes the prior shape L^2 (the intrinsic GMRF of App. C), whose modes are the squares of
    the Laplacian's."""
    m, k = A.shape
    Yh = np.fft.fft2(np.asarray(Y, np.float64).reshape(m, H, W), axes=(1, 2))
    # right-hand side in Fourier space: b_j = sum_c a_cj d_c y_c
    bh = np.einsum("cj,c,chw->jhw", A, np.asarray(d, np.float64), Yh)
    lam = (4.0 - 2.0 * np.cos(2 * np.pi * np.arange(H) / H)[:, None]
           - 2.0 * np.cos(2 * np.pi * np.arange(W) / W)[None, :]) ** power
    data = np.einsum("c,cj,cl->jl", np.asarray(d, np.float64), A, A)
    M = np.broadcast_to(data, (H, W, k, k)).copy()
    for j in range(k):
        M[:, :, j, j] += tau[j] * (kappa[j] ** 2 + lam)
    xh = np.linalg.solve(M, np.moveaxis(bh, 0, -1)[..., None])[..., 0]
    X = np.fft.ifft2(np.moveaxis(xh, -1, 0), axes=(1, 2)).real
    return X.reshape(k, H * W)


def _sphere_weights(H):
    phi = -np.pi / 2 + (np.arange(H) + 0.5) * np.pi / H
    ew = np.cos(phi)
    ns = np.cos(0.5 * (phi[:-1] + phi[1:]))
    return ew, ns


def sphere_latitude_noise(H, W, tau, kappa, A, d_rows, Y=None, b=None):
    """X (k, H*W) on the sphere grid with d_ci = d_rows[c, row(i)].

    Either the observations Y (m, n) or the right-hand side b (k, n) may be given."""
    m, k = A.shape
    tau = np.asarray(tau, np.float64)
    kappa = np.asarray(kappa, np.float64)
    d_rows = np.asarray(d_rows, np.float64)
    if b is None:
        Yr = np.asarray(Y, np.float64).reshape(m, H, W)
        b = np.einsum("cj,cr,crw->jrw", A, d_rows, Yr)
    else:
        b = np.asarray(b, np.float64).reshape(k, H, W)
    bh = np.fft.rfft(b, axis=2)                          # (k, H, Q)
    nq = bh.shape[2]
    ew, ns = _sphere_weights(H)
    ns_up = np.concatenate([ns, [0.0]])                  # weight to row r+1
    ns_dn = np.concatenate([[0.0], ns])                  # weight to row r-1
    data = np.einsum("cr,cj,cl->rjl", d_rows, A, A)      # (H, k, k)
    base = data.copy()
    for j in range(k):
        base[:, j, j] += tau[j] * (kappa[j] ** 2 + ns_up + ns_dn)
    N = H * k
    xh = np.empty_like(bh)
    theta = 2 * np.pi * np.arange(nq) / W
    for q in range(nq):
        blocks = base.copy()
        ewq = ew * (2.0 - 2.0 * np.cos(theta[q]))
        for j in range(k):
            blocks[:, j, j] += tau[j] * ewq
        # upper banded storage, unknown index r*k + j, bandwidth k
        ab = np.zeros((k + 1, N))
        for d in range(k):
            for j1 in range(k - d):
                j2 = j1 + d
                ab[k - d, np.arange(H) * k + j2] = blocks[:, j1, j2]
        for j in range(k):
            ab[0, np.arange(1, H) * k + j] = -tau[j] * ns
        rhs = bh[:, :, q].T.reshape(N)                   # (H, k) -> r*k + j
        sol = sla.solveh_banded(ab, np.stack([rhs.real, rhs.imag], axis=1), lower=False)
        xh[:, :, q] = (sol[:, 0] + 1j * sol[:, 1]).reshape(H, k).T
    X = np.fft.irfft(xh, n=W, axis=2)
    return X.reshape(k, H * W)


def sylvester_separable(L, nu_pix, t, phi, kappa0, A, Y):
    """Dense solve of eq. Axb-Sylv for the separable case (tiny n only).

    Noise d_ci = t_c * nu_pix_i, prior Q_j = phi_j Q_0 with Q_0 = kappa0^2 I + L.
    Returns X (k, n) (M transposed)."""
    Ld = L.toarray() if sp.issparse(L) else np.asarray(L)
    n = Ld.shape[0]
    Q0 = kappa0 ** 2 * np.eye(n) + Ld
    Ninv = np.diag(1.0 / np.asarray(nu_pix, np.float64))
    T = np.diag(np.asarray(t, np.float64))
    Pinv = np.diag(1.0 / np.asarray(phi, np.float64))
    Ymat = np.asarray(Y, np.float64).T                   # n x m, column c = map c
    left = Ninv @ Q0
    right = A.T @ T @ A @ Pinv
    F = Ymat @ T @ A @ Pinv
    M = sla.solve_sylvester(left, right, F)               # n x k
    return M.T


def scalar_posterior(L, tau, kappa, a, d, y):
    """k = m = 1: x = (tau (kappa^2 I + L) + a^2 D)^{-1} a D y."""
    n = L.shape[0]
    Qpost = tau * (kappa ** 2 * sp.identity(n) + L) + a * a * sp.diags(d)
    return spla.spsolve(sp.csc_matrix(Qpost), a * np.asarray(d) * np.asarray(y))
