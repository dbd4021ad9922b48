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
