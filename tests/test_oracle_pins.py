"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each check reaches its expected value by a route that does not go through the code under test:
closed forms, brute-force definitions, textbook special cases, identities, and the values the
paper prints (App. B).  ``test_planted_mistakes_are_caught`` plants plausible mistakes in the
oracle and confirms that at least one pin fails for each.
"""

import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import synth
from oracle import closed_form, gradient, model, physical_mixing, solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def _tiny(kind="lattice", H=5, W=6, k=3, m=5, noise="lognormal", seed=7, nrhs=1):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    return synth.make_problem("tiny", g, k, nu, None, None, [1.0, 0.7, 1.3, 0.9, 1.1, 0.8][:k],
                              seed, beta_draw=(-3, 2), kappa_draw=(0.05, 1.0), noise=noise,
                              nrhs=nrhs)


def _L(p):
    return model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)


# ---------------------------------------------------------------------------------------------
# mixing matrix
# ---------------------------------------------------------------------------------------------
def test_powerlaw_mixing_closed_form():
    A = model.powerlaw_mixing([30.0, 100.0, 200.0, 857.0], [0.0, -3.0, 1.0])
    assert A.shape == (4, 3)
    assert np.all(A[:, 0] == 1.0)                       # beta = 0: flat spectrum
    assert np.all(A[1] == 1.0)                          # reference frequency
    assert A[0, 1] == pytest.approx(1.0 / 0.027, rel=1e-14)   # (30/100)^-3
    assert A[2, 2] == pytest.approx(2.0, rel=1e-15)     # (200/100)^1
    assert A[3, 2] == pytest.approx(8.57, rel=1e-15)
    dA = model.powerlaw_mixing_dbeta([30.0, 200.0], [1.5])
    assert dA[1, 0] == pytest.approx(np.log(2.0) * 2.0 ** 1.5, rel=1e-14)


def test_physical_mixing_matches_printed_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "planck_mixing_A.txt"))
    nu, printed = rows[:, 0], rows[:, 1:]
    A = physical_mixing.physical_mixing(nu)
    # printed to 3 decimals; the constants reproduce the table to 3e-4 relative
    assert np.all(np.abs(A - printed) <= 5e-4 + 3e-4 * np.abs(printed))
    T = np.loadtxt(os.path.join(GOLDEN, "planck_T.txt"))
    assert T.shape == (9,) and np.all(T > 0)


# ---------------------------------------------------------------------------------------------
# Laplacian
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,H,W", [("lattice", 4, 5), ("lattice", 3, 3), ("sphere", 4, 6),
                                      ("sphere", 2, 3), ("sphere", 7, 4)])
def test_laplacian_three_routes_agree(kind, H, W):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    L_gen = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n).toarray()
    L_inc = (model.laplacian_lattice(H, W) if kind == "lattice"
             else model.laplacian_sphere(H, W)).toarray()
    L_bf = model.laplacian_bruteforce(H, W, kind)
    assert np.allclose(L_gen, L_bf, rtol=0, atol=1e-14)
    assert np.allclose(L_inc, L_bf, rtol=0, atol=1e-14)
    # CSR well-formed: sorted columns, diagonal present
    for i in range(g.n):
        cols = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols


@pytest.mark.parametrize("kind", ["lattice", "sphere"])
def test_laplacian_properties(kind):
    g = synth.periodic_lattice(6, 7) if kind == "lattice" else synth.latlong_sphere(6, 7)
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n).toarray()
    assert np.array_equal(L, L.T)
    assert np.allclose(L.sum(axis=1), 0.0, atol=1e-14)          # constant null vector
    ev = np.linalg.eigvalsh(L)
    assert ev[0] == pytest.approx(0.0, abs=1e-12)
    assert ev[1] > 1e-6                                          # connected: rank n - 1
    if kind == "lattice":
        H, W = 6, 7
        lam = (4 - 2 * np.cos(2 * np.pi * np.arange(H) / H)[:, None]
               - 2 * np.cos(2 * np.pi * np.arange(W) / W)[None, :])
        assert np.allclose(np.sort(lam.ravel()), ev, atol=1e-12)


def test_sphere_total_weight():
    H, W = 8, 10
    g = synth.latlong_sphere(H, W)
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)
    phi = -np.pi / 2 + (np.arange(H) + 0.5) * np.pi / H
    total = W * np.cos(phi).sum() + W * np.cos(0.5 * (phi[:-1] + phi[1:])).sum()
    assert L.diagonal().sum() == pytest.approx(2 * total, rel=1e-14)


# ---------------------------------------------------------------------------------------------
# operator identities and SPD-ness
# ---------------------------------------------------------------------------------------------
def test_vec_kron_identity():
    A = RNG.standard_normal((4, 3))
    X = RNG.standard_normal((3, 5))
    B = RNG.standard_normal((5, 2))
    lhs = (A @ X @ B).reshape(-1, order="F")
    rhs_ = np.kron(B.T, A) @ X.reshape(-1, order="F")
    assert np.allclose(lhs, rhs_, atol=1e-13)


@pytest.mark.parametrize("kind,noise", [("lattice", "lognormal"), ("sphere", "lognormal"),
                                        ("sphere", "latitude")])
def test_assembled_equals_matrix_free(kind, noise):
    p = _tiny(kind, 5, 6, noise=noise)
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    X = RNG.standard_normal((p.k, p.n))
    y1 = (G @ X.reshape(-1)).reshape(p.k, p.n)
    y2 = model.apply(L, p.D, p.tau, p.kappa, A, X)
    assert np.allclose(y1, y2, rtol=1e-13, atol=1e-12)
    rows = [0, 3, p.n - 1]
    assert np.allclose(model.apply_rows(L, p.D, p.tau, p.kappa, A, X, rows), y2[:, rows],
                       rtol=1e-13, atol=1e-12)
    # data term equals B^T C B with B = A kron I_n literally (Sec. 2.1)
    BtCB = model.assemble_BtCB_kron(p.D, A)
    prior = sum(sp.kron(sp.csr_matrix(([1.0], ([j], [j])), shape=(p.k, p.k)),
                        model.prior_block(L, p.tau[j], p.kappa[j])) for j in range(p.k))
    assert abs(G - (BtCB + prior)).max() < 1e-12


def test_rhs_is_BtCy():
    p = _tiny("sphere", 4, 5)
    A = model.powerlaw_mixing(p.nu, p.beta)
    B = sp.kron(sp.csr_matrix(A), sp.identity(p.n))
    C = sp.diags(p.D.reshape(-1))
    lit = (B.T @ (C @ p.Yobs[0].reshape(-1))).reshape(p.k, p.n)
    assert np.allclose(model.rhs(p.D, p.Yobs[0], A), lit, rtol=1e-14, atol=1e-12)


def test_G_is_spd():
    p = _tiny("lattice", 4, 4, k=3)
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A).toarray()
    assert np.array_equal(G, G.T)
    assert np.linalg.eigvalsh(G)[0] > 0
    sla.cholesky(G)


# ---------------------------------------------------------------------------------------------
# solves
# ---------------------------------------------------------------------------------------------
def test_dense_matches_sparse_direct():
    p = _tiny("sphere", 6, 8, k=3)
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    b = model.rhs(p.D, p.Yobs[0], A)
    x1 = solve.solve_direct(G, b)
    x2 = solve.solve_dense(G, b)
    assert np.allclose(x1, x2, rtol=1e-11, atol=1e-11 * np.abs(x2).max())


def test_manufactured_solution():
    p = _tiny("lattice", 8, 9, k=4, m=6)
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    Xs = RNG.standard_normal((2, p.k, p.n))
    b = np.stack([model.apply(L, p.D, p.tau, p.kappa, A, x) for x in Xs])
    Xr = solve.solve_direct(G, b)
    assert np.abs(Xr - Xs).max() < 1e-9


def test_closed_form_lattice_homogeneous():
    H, W = 8, 12
    p = _tiny("lattice", H, W, k=4, m=6, noise="homogeneous")
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    X_cf = closed_form.lattice_homogeneous(H, W, p.tau, p.kappa, A, p.D[:, 0], p.Yobs[0])
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    X_d = solve.solve_direct(G, model.rhs(p.D, p.Yobs[0], A))
    assert np.abs(X_cf - X_d).max() <= 1e-9 * np.abs(X_d).max()


def test_closed_form_sphere_latitude_noise():
    H, W = 7, 10
    p = _tiny("sphere", H, W, k=3, m=5, noise="latitude")
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    d_rows = p.D.reshape(p.m, H, W)[:, :, 0]
    X_cf = closed_form.sphere_latitude_noise(H, W, p.tau, p.kappa, A, d_rows, Y=p.Yobs[0])
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    X_d = solve.solve_direct(G, model.rhs(p.D, p.Yobs[0], A))
    assert np.abs(X_cf - X_d).max() <= 1e-9 * np.abs(X_d).max()


def test_sylvester_form_separable_noise():
    H, W = 4, 5
    g = synth.latlong_sphere(H, W)
    n, k = g.n, 3
    rng = np.random.default_rng(3)
    nu_pix = rng.uniform(0.5, 2.0, n)
    T = np.loadtxt(os.path.join(GOLDEN, "planck_T.txt"))[:5] * 1e-6
    A = physical_mixing.physical_mixing([30, 70, 100, 217, 545])[:, :k]
    phi = np.array([1.0, 2.5, 0.4])
    kappa0 = 0.3
    Y = rng.standard_normal((5, n))
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, n)
    D = T[:, None] * nu_pix[None, :]
    X_s = closed_form.sylvester_separable(L, nu_pix, T, phi, kappa0, A, Y)
    G = model.assemble_G(L, D, phi, np.full(k, kappa0), A)
    X_d = solve.solve_direct(G, model.rhs(D, Y, A))
    assert np.abs(X_s - X_d).max() <= 1e-9 * np.abs(X_d).max()


def test_scalar_case_textbook():
    g = synth.periodic_lattice(6, 6)
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 2, g.n)
    y = rng.standard_normal(g.n)
    tau, kappa, nu, beta = 1.3, 0.4, 217.0, 1.2
    a = (nu / 100.0) ** beta
    x_tb = closed_form.scalar_posterior(L, tau, kappa, a, d, y)
    A = model.powerlaw_mixing([nu], [beta])
    G = model.assemble_G(L, d[None], [tau], [kappa], A)
    x = solve.solve_direct(G, model.rhs(d[None], y[None], A))
    assert np.allclose(x[0], x_tb, rtol=1e-12, atol=1e-13)
    # one-pixel sanity: no neighbours -> x = a d y / (tau kappa^2 + a^2 d)
    assert x_tb.shape == (g.n,)


def test_cg_and_pcg_reach_direct_solution():
    p = _tiny("sphere", 10, 12, k=4, m=7)
    L = _L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    b = model.rhs(p.D, p.Yobs[0], A)
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    X_d = solve.solve_direct(G, b)
    x_cg, it_cg, rel = solve.cg(lambda x: model.apply(L, p.D, p.tau, p.kappa, A, x), b,
                                eps=1e-12)
    assert rel <= 1e-12
    assert np.abs(x_cg - X_d).max() <= 1e-6 * np.abs(X_d).max()
    x_p, it_p, relp, _ = solve.pcg_block_jacobi(L, p.D, p.tau, p.kappa, A, b, eps=1e-12)
    assert np.abs(x_p - X_d).max() <= 1e-6 * np.abs(X_d).max()
    assert it_p <= it_cg
    # block Jacobi blocks are the exact diagonal k x k blocks of G at each pixel
    P = solve.block_jacobi_blocks(L, p.D, p.tau, p.kappa, A)
    Gd = G.toarray()
    i = 17
    idx = [j * p.n + i for j in range(p.k)]
    assert np.allclose(P[i], Gd[np.ix_(idx, idx)], rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------------------------
def test_gradient_three_routes():
    p = _tiny("sphere", 4, 5, k=3, m=5, nrhs=2)
    L = _L(p)

    def loss(X):
        return float(np.sum((X - p.X_true[None]) ** 2))

    X, _, _ = gradient.posterior_mean(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs)
    g = 2 * (X - p.X_true[None])
    ga = gradient.adjoint_gradient(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs, X, g)[:3]
    gs = gradient.sensitivity_gradient(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs, g)
    gf = gradient.fd_gradient(loss, L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs, h=1e-6)
    for a, s, f in zip(ga, gs, gf):
        scale = max(np.abs(s).max(), 1e-300)
        assert np.abs(a - s).max() <= 1e-10 * scale
        assert np.abs(a - f).max() <= 1e-5 * scale


# ---------------------------------------------------------------------------------------------
# planted mistakes: each must make at least one pin fail
# ---------------------------------------------------------------------------------------------
def _pins_pass():
    try:
        test_closed_form_lattice_homogeneous()
        test_closed_form_sphere_latitude_noise()
        test_scalar_case_textbook()
        test_sylvester_form_separable_noise()
        test_assembled_equals_matrix_free("sphere", "lognormal")
        test_rhs_is_BtCy()
        test_powerlaw_mixing_closed_form()
    except AssertionError:
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    orig_prior = model.prior_block
    orig_mix = model.powerlaw_mixing
    orig_rhs = model.rhs
    orig_apply = model.apply
    plants = [
        ("prior", lambda L, t, kp, w=None: orig_prior(L, t, 0.0, w)),            # drop kappa^2
        ("prior", lambda L, t, kp, w=None: orig_prior(-L, t, kp, w)),            # wrong sign
        ("prior", lambda L, t, kp, w=None: orig_prior(L, 1.0, kp, w)),           # drop tau
        ("mix", lambda nu, b, nu0=100.0: orig_mix(nu, b, nu0) ** 1.0001),        # wrong power
        ("mix", lambda nu, b, nu0=100.0: np.power(nu0 / np.asarray(nu)[:, None],
                                                  np.asarray(b)[None, :])),      # inverted ratio
        ("rhs", lambda D, Y, A: orig_rhs(np.ones_like(D), Y, A)),                 # drop D
        ("apply", lambda L, D, t, kp, A, X, w=None: orig_apply(L, D, t, kp, A, X, w)
         - A.T @ (D * (A @ X)) + A.T @ (D * (A @ X[::-1]))),                      # wrong index
    ]
    for what, fn in plants:
        with monkeypatch.context() as mp:
            if what == "prior":
                mp.setattr(model, "prior_block", fn)
            elif what == "mix":
                mp.setattr(model, "powerlaw_mixing", fn)
            elif what == "rhs":
                mp.setattr(model, "rhs", fn)
            else:
                mp.setattr(model, "apply", fn)
            assert not _pins_pass(), f"planted mistake in {what} went unnoticed"
    assert _pins_pass()
