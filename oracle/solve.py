"""Solves of the posterior-mean system G x = b in FP64 (TEST INFRASTRUCTURE ONLY).

* ``solve_direct``: sparse LU without pivoting of the SPD matrix G (equivalent to a Cholesky
  factorisation), the exact result every iterative method here approaches (eq. mu*).
* ``solve_dense``: dense Cholesky, for tiny inputs.
* ``cg``: the method of conjugate gradients exactly as Algorithm 2 states it (with the
  operator written B^T C B, see Sec. 2.2), stopping at ||r|| <= eps ||r_0||.
* ``pcg_block_jacobi``: the same iteration with a preconditioner (Sec. 3.2 mentions one may be
  used): the exact k x k diagonal block of G at each pixel.
"""

import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model


def solve_direct(G, b):
    """x = G^{-1} b by sparse factorisation; b may be (k, n) or (R, k, n)."""
    b = np.asarray(b, np.float64)
    shape = b.shape
    rhs = b.reshape(-1, G.shape[0]).T
    lu = spla.splu(sp.csc_matrix(G), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    x = lu.solve(np.ascontiguousarray(rhs))
    return x.T.reshape(shape)


def solve_dense(G, b):
    Gd = G.toarray() if sp.issparse(G) else np.asarray(G)
    c = sla.cho_factor(Gd)
    b = np.asarray(b, np.float64)
    return sla.cho_solve(c, b.reshape(-1)).reshape(b.shape)


def cg(apply_G, b, x0=None, eps=1e-8, maxit=100000):
    """Algorithm 2: plain CG.  ``apply_G`` maps an array shaped like b to G times it.
    Returns (x, iterations, ||r|| / ||r_0||)."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_G(x)
    p = r.copy()
    rr = float(np.vdot(r, r))
    rr0 = rr
    it = 0
    while it < maxit and np.sqrt(rr) > eps * np.sqrt(rr0):
        q = apply_G(p)
        alpha = rr / float(np.vdot(p, q))
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.vdot(r, r))
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
        it += 1
    return x, it, np.sqrt(rr / rr0) if rr0 > 0 else 0.0


def block_jacobi_blocks(L, D, tau, kappa, A, w=None):
    """P_i = diag_j(tau_j (kappa_j^2 w_i + L_ii)) + sum_c d_ci a_c a_c^T  -> (n, k, k)."""
    n = L.shape[0]
    k = A.shape[1]
    Ld = L.diagonal()
    wv = np.ones(n) if w is None else np.asarray(w, np.float64)
    P = np.einsum("ci,cj,cl->ijl", D, A, A)
    for j in range(k):
        P[:, j, j] += tau[j] * (kappa[j] ** 2 * wv + Ld)
    return P


def pcg_block_jacobi(L, D, tau, kappa, A, b, x0=None, eps=1e-8, maxit=100000, w=None,
                     max_seconds=None):
    """Preconditioned CG with the pixel-block Jacobi preconditioner.

    Returns (x, iterations, recursive relative residual, seconds)."""
    b = np.asarray(b, np.float64)
    P = block_jacobi_blocks(L, D, tau, kappa, A, w)
    Pinv = np.linalg.inv(P)                                  # (n, k, k)

    def prec(r):
        return np.einsum("ijl,li->ji", Pinv, r)

    def G(x):
        return model.apply(L, D, tau, kappa, A, x, w)

    t0 = time.perf_counter()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - G(x)
    z = prec(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    rr0 = float(np.vdot(r, r))
    rr = rr0
    it = 0
    while it < maxit and np.sqrt(rr) > eps * np.sqrt(rr0):
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
        q = G(p)
        alpha = rz / float(np.vdot(p, q))
        x += alpha * p
        r -= alpha * q
        z = prec(r)
        rz_new = float(np.vdot(r, z))
        rr = float(np.vdot(r, r))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, (np.sqrt(rr / rr0) if rr0 > 0 else 0.0), time.perf_counter() - t0


def relres(L, D, tau, kappa, A, X, b, w=None):
    """True relative residual ||b - G X||_F / ||b||_F in FP64."""
    r = b - model.apply(L, D, tau, kappa, A, X, w)
    return float(np.linalg.norm(r) / np.linalg.norm(b))
