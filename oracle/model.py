"""Operator, right-hand side and prior of the posterior-mean system (TEST INFRASTRUCTURE ONLY).

Sec. 2.1-2.2 (eq. model, eq. Q*, eq. mu*), Sec. 3.1 (eq. block-vector-mapping-matvec), App. C.
Unknowns are stored as X of shape (k, n): row j is source map j, and ``X.reshape(-1)`` is the
column-stacked vec of the n x k matrix used in Sec. 3.1 (reshape(u, N, m) convention).
"""

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------------------------
# mixing matrix
# --------------------------------------------------------------------------------------------
def powerlaw_mixing(nu, beta, nu0=100.0):
    """A[c, j] = (nu_c / nu0) ** beta_j: a straight power law in frequency per source (App. B
    form of the synchrotron and free-free columns, without the unit conversion factor)."""
    nu = np.asarray(nu, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    return np.power(nu[:, None] / nu0, beta[None, :])


def powerlaw_mixing_dbeta(nu, beta, nu0=100.0):
    """dA[c, j] / d beta_j = ln(nu_c / nu0) * A[c, j]."""
    A = powerlaw_mixing(nu, beta, nu0)
    return np.log(np.asarray(nu, dtype=np.float64) / nu0)[:, None] * A


# --------------------------------------------------------------------------------------------
# graph Laplacians, rebuilt from the grid definition through the edge incidence matrix
# --------------------------------------------------------------------------------------------
def _incidence_laplacian(n, heads, tails, weights):
    """L = E^T diag(w) E where row e of E is e_head - e_tail (a weighted graph Laplacian)."""
    ne = len(heads)
    rows = np.concatenate([np.arange(ne), np.arange(ne)])
    cols = np.concatenate([heads, tails])
    vals = np.concatenate([np.ones(ne), -np.ones(ne)])
    E = sp.csr_matrix((vals, (rows, cols)), shape=(ne, n))
    return (E.T @ sp.diags(weights) @ E).tocsr()


def laplacian_lattice(H, W):
    """Periodic H x W lattice, unit weights: L = -Delta_5pt (App. C neighbour structure)."""
    heads, tails = [], []
    for r in range(H):
        for c in range(W):
            i = r * W + c
            heads += [i, i]
            tails += [r * W + (c + 1) % W, ((r + 1) % H) * W + c]
    return _incidence_laplacian(H * W, np.array(heads), np.array(tails), np.ones(len(heads)))


def sphere_latitudes(H):
    return np.array([-np.pi / 2 + (r + 0.5) * np.pi / H for r in range(H)])


def laplacian_sphere(H, W):
    """Latitude-longitude H x W sphere grid with cos(latitude)-weighted 5-point coupling:
    east-west weight cos(phi_r), north-south weight cos of the mid latitude, no pole edges."""
    phi = sphere_latitudes(H)
    heads, tails, wts = [], [], []
    for r in range(H):
        for c in range(W):
            i = r * W + c
            heads.append(i)
            tails.append(r * W + (c + 1) % W)
            wts.append(np.cos(phi[r]))
            if r + 1 < H:
                heads.append(i)
                tails.append((r + 1) * W + c)
                wts.append(np.cos(0.5 * (phi[r] + phi[r + 1])))
    return _incidence_laplacian(H * W, np.array(heads), np.array(tails), np.array(wts))


def laplacian_bruteforce(H, W, kind):
    """Dense Laplacian by its entry-wise definition (tiny grids only): off-diagonal entry
    -weight for each neighbour pair, diagonal = minus the sum of the row's off-diagonals."""
    n = H * W
    L = np.zeros((n, n))
    phi = sphere_latitudes(H)
    for r in range(H):
        for c in range(W):
            i = r * W + c
            pairs = []
            if kind == "lattice":
                pairs = [(r * W + (c + 1) % W, 1.0), (r * W + (c - 1) % W, 1.0),
                         (((r + 1) % H) * W + c, 1.0), (((r - 1) % H) * W + c, 1.0)]
            else:
                pairs = [(r * W + (c + 1) % W, np.cos(phi[r])),
                         (r * W + (c - 1) % W, np.cos(phi[r]))]
                if r + 1 < H:
                    pairs.append(((r + 1) * W + c, np.cos(0.5 * (phi[r] + phi[r + 1]))))
                if r > 0:
                    pairs.append(((r - 1) * W + c, np.cos(0.5 * (phi[r] + phi[r - 1]))))
            for jn, wt in pairs:
                L[i, jn] -= wt
            # diagonal is minus the row sum of the off-diagonal part (Sec. 3 definition of D)
        for c in range(W):
            i = r * W + c
            L[i, i] = -(L[i].sum() - L[i, i])
    return L


def igmrf_base(L):
    """Precision shape of the intrinsic GMRF of App. C, Q = phi D^T D with D the Laplacian
    (reading of Sec. 3 / App. C: the rank N - 1 stated there holds for the Laplacian): L^T L = L^2
    as a sparse product."""
    L = sp.csr_matrix(L)
    return (L.T @ L).tocsr()


def igmrf_bruteforce(Ld):
    """(L^T L)_ij = sum_k L_ki L_kj by explicit loops over a dense L (tiny inputs only)."""
    Ld = np.asarray(Ld, np.float64)
    n = Ld.shape[0]
    Q = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            acc = 0.0
            for k in range(n):
                acc += Ld[k, i] * Ld[k, j]
            Q[i, j] = acc
    return Q


def laplacian_from_csr(rowptr, col, val, n):
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(rowptr)),
                         shape=(n, n))


# --------------------------------------------------------------------------------------------
# prior, operator, right-hand side
# --------------------------------------------------------------------------------------------
def prior_block(L, tau_j, kappa_j, w=None):
    """Q_j = tau_j (kappa_j^2 W + L), W = diag(w) or I (SPD Gaussian-field precision)."""
    n = L.shape[0]
    Wm = sp.identity(n, format="csr") if w is None else sp.diags(np.asarray(w, np.float64))
    return (tau_j * (kappa_j ** 2 * Wm + L)).tocsr()


def assemble_G(L, D, tau, kappa, A, w=None):
    """G = sum_j (e_j e_j^T) kron Q_j + sum_c (a_c a_c^T) kron D_c   (nk x nk, sparse).

    This is Q + B^T C B of eq. Q* with B = A kron I_n (Sec. 2.1) and C = blockdiag(D_c);
    (a_c a_c^T) kron D_c is the c-th channel's contribution to B^T C B."""
    k = A.shape[1]
    m = A.shape[0]
    blocks = []
    for j in range(k):
        Ej = sp.csr_matrix(([1.0], ([j], [j])), shape=(k, k))
        blocks.append(sp.kron(Ej, prior_block(L, tau[j], kappa[j], w)))
    for c in range(m):
        ac = A[c][:, None]
        blocks.append(sp.kron(sp.csr_matrix(ac @ ac.T), sp.diags(D[c])))
    G = blocks[0]
    for blk in blocks[1:]:
        G = G + blk
    return G.tocsr()


def assemble_BtCB_kron(D, A):
    """B^T C B assembled literally from B = A kron I_n and C = diag(vec of D) (Sec. 2.1)."""
    m, n = D.shape
    B = sp.kron(sp.csr_matrix(A), sp.identity(n))
    C = sp.diags(D.reshape(-1))
    return (B.T @ C @ B).tocsr()


def rhs(D, Y, A):
    """b = B^T C y of eq. mu*, returned as (k, n): column j of sum_c D_c y_c a_c^T."""
    D = np.asarray(D, np.float64)
    Y = np.asarray(Y, np.float64)
    k = A.shape[1]
    b = np.zeros((k, D.shape[1]))
    for c in range(A.shape[0]):
        for j in range(k):
            b[j] += A[c, j] * D[c] * Y[c]
    return b


def apply(L, D, tau, kappa, A, X, w=None):
    """G X matrix-free: [Q_j x_j]_j + ((X A^T) o D) A, the block mapping of
    eq. block-vector-mapping-matvec with the separable N, T replaced by per-pixel maps."""
    X = np.asarray(X, np.float64)
    k, n = X.shape
    out = np.empty_like(X)
    for j in range(k):
        out[j] = prior_block(L, tau[j], kappa[j], w) @ X[j]
    MAt = A @ X                  # (m, n): row c is (X A^T)[:, c] = X a_c
    out += A.T @ (D * MAt)       # row j: sum_c a_cj d_c (X a_c)
    return out


def apply_rows(L, D, tau, kappa, A, X, rows, w=None):
    """(G X)[:, rows] computed one pixel at a time (for sampled checks on large inputs)."""
    L = L.tocsr()
    k = X.shape[0]
    out = np.zeros((k, len(rows)))
    for t, i in enumerate(rows):
        lo, hi = L.indptr[i], L.indptr[i + 1]
        cols, vals = L.indices[lo:hi], L.data[lo:hi]
        wi = 1.0 if w is None else w[i]
        for j in range(k):
            out[j, t] = tau[j] * (kappa[j] ** 2 * wi * X[j, i] + vals @ X[j, cols])
        xi = X[:, i]
        for c in range(A.shape[0]):
            out[:, t] += A[c] * D[c, i] * (A[c] @ xi)
    return out
