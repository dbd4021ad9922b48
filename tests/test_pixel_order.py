"""Pixel renumbering of the synthetic grids (no GPU): the blocked numbering is a permutation,
the relabelled Laplacian is P L P^T, the oracle's posterior mean of the relabelled problem is
the relabelled posterior mean (eq. mu* is invariant under a renumbering of the pixels), and the
blocked numbering keeps most stencil neighbours inside a 256-pixel tile."""

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import gradient, model


def test_blocked_order_is_a_permutation_of_whole_blocks():
    perm = synth.blocked_order(32, 64, 16, 16)
    assert np.array_equal(np.sort(perm), np.arange(32 * 64))
    # the first 256 new pixels are the top-left 16 x 16 block, row-major
    r, c = np.divmod(perm[:256], 64)
    assert np.array_equal(r, np.repeat(np.arange(16), 16))
    assert np.array_equal(c, np.tile(np.arange(16), 16))
    # the second block sits to its right
    r, c = np.divmod(perm[256:512], 64)
    assert r.min() == 0 and r.max() == 15 and c.min() == 16 and c.max() == 31
    with pytest.raises(ValueError):
        synth.blocked_order(30, 64, 16, 16)


@pytest.mark.parametrize("kind", ["sphere", "lattice"])
def test_relabelled_laplacian_is_PLPt(kind):
    g = synth.latlong_sphere(16, 32) if kind == "sphere" else synth.periodic_lattice(16, 32)
    perm = synth.blocked_order(16, 32, 8, 8)
    gp = synth.permute_graph(g, perm)
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n).toarray()
    Lp = model.laplacian_from_csr(gp.rowptr, gp.col, gp.val, gp.n).toarray()
    P = sp.csr_matrix((np.ones(g.n), (np.arange(g.n), perm)), shape=(g.n, g.n)).toarray()
    assert np.array_equal(Lp, P @ L @ P.T)
    for i in range(gp.n):   # columns sorted per row, diagonal included
        cols = gp.col[gp.rowptr[i]:gp.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols


def test_posterior_mean_commutes_with_the_renumbering():
    g = synth.latlong_sphere(16, 32)
    p = synth.make_problem("order", g, 3, synth.PLANCK_NU[[0, 3, 5, 7, 8]], [-2.0, 0.5, 1.5],
                           [0.2, 0.5, 1.0], [1.0, 2.0, 0.5], 7, noise="lognormal")
    perm = synth.blocked_order(16, 32, 8, 8)
    q = synth.permute_problem(p, perm)
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)
    Lq = model.laplacian_from_csr(q.graph.rowptr, q.graph.col, q.graph.val, q.n)
    X, _, _ = gradient.posterior_mean(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs[0])
    Xq, _, _ = gradient.posterior_mean(Lq, q.D, q.tau, q.kappa, q.nu, q.beta, q.Yobs[0])
    assert np.allclose(Xq[0], X[0][:, perm], rtol=1e-10, atol=1e-12 * np.abs(X).max())
    assert np.array_equal(q.X_true, p.X_true[:, perm])


def test_blocked_order_keeps_neighbours_in_the_tile():
    g = synth.latlong_sphere(256, 512)
    row_major = synth.outside_tile_fraction(g.rowptr, g.col, 256)
    gb = synth.permute_graph(g, synth.blocked_order(256, 512, 16, 16))
    blocked = synth.outside_tile_fraction(gb.rowptr, gb.col, 256)
    # row-major: every north/south neighbour and the east/west wrap at each tile end
    assert 0.5 < row_major < 0.52
    # 16 x 16 blocks: the 64 border pixels' outward edges out of 1024 (fewer at the poles)
    assert 0.05 < blocked < 0.0626
