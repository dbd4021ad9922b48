"""Pins of the oracle's intrinsic GMRF prior (App. C: Q_j = phi_j D^T D, D the Laplacian) and of
the physical mixing inputs (App. B), no GPU.

L^T L is checked against its entry-wise definition, the periodic lattice's spectrum (squares of
4 - 2cos - 2cos), its rank N - 1 with the constants as null space, and the posterior mean
under this prior against the Fourier closed form; G is SPD exactly when A has full column rank.
"""

import numpy as np
import pytest

import synth
from oracle import closed_form, model, physical_mixing, solve


def _L(g):
    return model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)


@pytest.mark.parametrize("kind,H,W", [("lattice", 4, 5), ("sphere", 4, 6), ("sphere", 3, 5)])
def test_igmrf_base_matches_definition(kind, H, W):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    Q = model.igmrf_base(_L(g)).toarray()
    Qb = model.igmrf_bruteforce(model.laplacian_bruteforce(H, W, kind))
    assert np.abs(Q - Qb).max() <= 1e-12 * np.abs(Qb).max()
    assert np.array_equal(Q, Q.T)


def test_igmrf_lattice_spectrum_and_rank():
    H, W = 6, 8
    Q = model.igmrf_base(_L(synth.periodic_lattice(H, W))).toarray()
    lam = (4 - 2 * np.cos(2 * np.pi * np.arange(H) / H)[:, None]
           - 2 * np.cos(2 * np.pi * np.arange(W) / W)[None, :]) ** 2
    ev = np.linalg.eigvalsh(Q)
    assert np.allclose(np.sort(ev), np.sort(lam.ravel()), atol=1e-10)
    # rank N - 1, the constants span the null space (App. C)
    assert np.abs(Q @ np.ones(H * W)).max() <= 1e-12
    assert np.sum(np.abs(ev) < 1e-9) == 1
    gs = synth.latlong_sphere(5, 8)
    evs = np.linalg.eigvalsh(model.igmrf_base(_L(gs)).toarray())
    assert np.sum(np.abs(evs) < 1e-9) == 1 and evs.min() > -1e-10


def test_igmrf_posterior_matches_fourier_closed_form():
    H, W, k = 8, 10, 3
    g = synth.periodic_lattice(H, W)
    rng = np.random.default_rng(8)
    A = synth.PLANCK_A_PRINTED[[0, 3, 5, 8]][:, :k]
    d = rng.uniform(0.5, 2.0, A.shape[0])
    D = np.repeat(d[:, None], g.n, axis=1)
    tau = np.array([2.0, 0.7, 1.3])
    kappa = np.zeros(k)
    Y = rng.standard_normal((A.shape[0], g.n))
    Q0 = model.igmrf_base(_L(g))
    G = model.assemble_G(Q0, D, tau, kappa, A)
    X_d = solve.solve_direct(G, model.rhs(D, Y, A))
    X_cf = closed_form.lattice_homogeneous(H, W, tau, kappa, A, d, Y, power=2)
    assert np.abs(X_cf - X_d).max() <= 1e-9 * np.abs(X_d).max()
    # the first-order prior's closed form does not match (the pin sees the power)
    X_1 = closed_form.lattice_homogeneous(H, W, tau, kappa + 1e-3, A, d, Y, power=1)
    assert np.abs(X_1 - X_d).max() > 1e-3 * np.abs(X_d).max()


def test_igmrf_G_spd_iff_mixing_full_rank():
    g = synth.latlong_sphere(4, 6)
    Q0 = model.igmrf_base(_L(g))
    A = synth.PLANCK_A_PRINTED[:, :3]
    D = np.repeat(synth.PLANCK_T_PRINTED[:, None] * 1e-6, g.n, axis=1)
    tau = np.ones(3)
    ev = np.linalg.eigvalsh(model.assemble_G(Q0, D, tau, np.zeros(3), A).toarray())
    assert ev.min() > 1e-8 * ev.max()
    A2 = A.copy()
    A2[:, 2] = A2[:, 1]             # rank-deficient mixing: constant maps in its null space
    ev2 = np.linalg.eigvalsh(model.assemble_G(Q0, D, tau, np.zeros(3), A2).toarray())
    assert ev2.min() < 1e-10 * ev2.max()


def test_printed_inputs_match_app_b_model():
    # the printed table the IGMRF workload feeds the solver agrees with App. B's formulas
    nu = synth.PLANCK_NU
    A = physical_mixing.physical_mixing(nu)
    assert np.abs(A - synth.PLANCK_A_PRINTED).max() <= 3e-3 * np.abs(A).max()
    T = np.loadtxt(__file__.replace("test_oracle_igmrf.py", "golden/planck_T.txt"))
    assert np.array_equal(T, synth.PLANCK_T_PRINTED)


def test_planted_mistake_in_the_square_is_caught(monkeypatch):
    orig = model.igmrf_base
    monkeypatch.setattr(model, "igmrf_base", lambda L: orig(L) + 1e-3 * sp_identity(L.shape[0]))
    with pytest.raises(AssertionError):
        test_igmrf_lattice_spectrum_and_rank()
    monkeypatch.setattr(model, "igmrf_base", lambda L: sp_csr(L))      # first power only
    with pytest.raises(AssertionError):
        test_igmrf_posterior_matches_fourier_closed_form()


def sp_identity(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


def sp_csr(L):
    import scipy.sparse as sp
    return sp.csr_matrix(L)
