"""Pins of the oracle's posterior variances diag(G^{-1}) (eq. Q*), no GPU.

The exact diagonal is checked against a dense inverse and against the lattice closed form
(translation invariance: one value per source, the mode average of the inverse mode matrices);
the probe estimator is exact for unit-vector probes and unbiased for Rademacher probes.
"""

import numpy as np

import synth
from oracle import closed_form, model, solve, variance


def _G(p):
    L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
    return model.assemble_G(L, p.D, p.tau, p.kappa, model.powerlaw_mixing(p.nu, p.beta))


def _small(kind="sphere", H=4, W=6, k=3, m=5, noise="lognormal", seed=4):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    return synth.make_problem("v", g, k, nu, None, None, [1.0, 0.6, 1.7][:k], seed,
                              beta_draw=(-3, 2), kappa_draw=(0.1, 1.0), noise=noise)


def test_exact_diag_matches_dense_inverse():
    p = _small()
    G = _G(p)
    dense = np.diag(np.linalg.inv(G.toarray())).reshape(p.k, p.n)
    ex = variance.exact_diag(G, p.k, p.n)
    assert np.abs(ex - dense).max() <= 1e-11 * np.abs(dense).max()
    assert np.all(ex > 0)


def test_unit_probes_are_exact():
    p = _small(H=3, W=5)
    G = _G(p)
    N = p.k * p.n
    Z = np.eye(N).reshape(N, p.k, p.n)
    est = variance.probe_diag(G, Z)
    assert np.abs(est - variance.exact_diag(G, p.k, p.n)).max() <= 1e-12 * est.max()


def test_lattice_closed_form_and_unbiased_probes():
    H, W, k = 6, 8, 3
    p = _small("lattice", H, W, k, noise="homogeneous")
    G = _G(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    cf = variance.lattice_homogeneous_diag(H, W, p.tau, p.kappa, A, p.D[:, 0])
    ex = variance.exact_diag(G, p.k, p.n)
    assert np.abs(ex - cf[:, None]).max() <= 1e-10 * cf.max()
    # Rademacher probes: the pixel average of the estimate converges to the exact value
    Z = synth.rademacher_probes(400, k, p.n, seed=3)
    est = variance.probe_diag(G, Z)
    assert np.abs(est.mean(axis=1) - cf).max() <= 0.05 * cf.max()
    # a plain power of the Laplacian in place of the prior's would not match
    cf2 = variance.lattice_homogeneous_diag(H, W, p.tau, p.kappa, A, p.D[:, 0], power=2)
    assert np.abs(cf2 - cf).max() > 1e-3 * cf.max()


# ---- probing with a distance colouring of the grid (Tang and Saad's probing for the diagonal
# of a matrix inverse): one 0/1 probe per (colour, source) ------------------------------------
def test_grid_colouring_separates_same_colour_pixels():
    """Brute force on small grids: any two distinct pixels of one colour are at least p steps
    apart (unweighted shortest paths of the pixel graph), and every colour is used."""
    import scipy.sparse.csgraph as csg
    for g, p in ((synth.latlong_sphere(7, 12), 3), (synth.periodic_lattice(8, 8), 4),
                 (synth.latlong_sphere(6, 8), 2), (synth.periodic_lattice(6, 9), 3)):
        adj = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n).tocsr()
        adj.data[:] = 1.0
        dist = csg.shortest_path(adj, unweighted=True)
        col = synth.grid_colouring(g, p)
        assert sorted(set(col.tolist())) == list(range(p * p))
        same = (col[:, None] == col[None, :]) & ~np.eye(g.n, dtype=bool)
        assert dist[same].min() >= p, (g.kind, p)


def test_colouring_probe_estimate_is_the_same_colour_sum():
    """With colouring probes the estimator returns, at (j, i), the sum of the entries of G^{-1}
    between (j, i) and every (j, i') of the same colour: the exact diagonal plus the
    same-colour couplings.  Checked against a dense inverse; with one pixel per colour (every
    probe a unit vector) it is the exact diagonal."""
    p = _small("sphere", 6, 8, 3)
    G = _G(p)
    Ginv = np.linalg.inv(G.toarray())
    for pc in (1, 2):
        col = synth.grid_colouring(p.graph, pc)
        est = variance.probe_diag(G, synth.colouring_probes(p.graph, p.k, pc))
        ref = np.empty((p.k, p.n))
        for j in range(p.k):
            blk = Ginv[j * p.n:(j + 1) * p.n, j * p.n:(j + 1) * p.n]
            ref[j] = np.array([blk[i, col == col[i]].sum() for i in range(p.n)])
        assert np.abs(est - ref).max() <= 1e-12 * np.abs(ref).max(), pc
    q = _small("sphere", 3, 4, 2)
    Gq = _G(q)
    est = variance.probe_diag(Gq, synth.colouring_probes(q.graph, q.k, 4))   # 12 colours
    assert np.abs(est - variance.exact_diag(Gq, q.k, q.n)).max() <= 1e-12 * est.max()


def test_probing_error_shrinks_with_distance():
    """The error is the same-colour coupling, which decays with graph distance: the largest
    error falls as the colouring distance grows, and from p = 2 every estimate is positive."""
    p = _small("sphere", 8, 24, 3, seed=9)
    G = _G(p)
    ex = variance.exact_diag(G, p.k, p.n)
    errs = []
    for pc in (1, 2, 3, 4):
        est = variance.probe_diag(G, synth.colouring_probes(p.graph, p.k, pc))
        errs.append(np.abs(est - ex).max() / ex.max())
        if pc >= 2:
            assert np.all(est > 0), pc
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-2 * errs[0], errs
