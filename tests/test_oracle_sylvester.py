"""Pins of the oracle's block-Lanczos Sylvester solver (Algorithms 4 and 5, Sec. 3.3), no GPU.

Expected values come from routes that do not go through the Lanczos code: the sparse direct
solve of the assembled Kronecker system, Bartels-Stewart on the dense Sylvester form, the
defining identities of the Lanczos process (N-orthonormal basis, T_j = V^T Q_0 V, the block
three-term relation), and the Sylvester residual of the explicitly formed iterate.  The last
test plants plausible mistakes and checks that a pin catches each.
"""

import numpy as np
import pytest

import synth
from oracle import closed_form, model, solve, sylvester


def _separable(H=6, W=8, k=3, m=5, kappa0=0.3, tau=(1.0, 2.0, 0.5), beta=None, seed=99):
    g = synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    p = synth.make_problem("sep", g, k, nu, beta, [kappa0] * k, list(tau)[:k], seed,
                           beta_draw=None if beta is not None else (-3, 2), noise="separable")
    L = model.laplacian_from_csr(g.rowptr, g.col, g.val, g.n)
    A = model.powerlaw_mixing(p.nu, p.beta)
    b = model.rhs(p.D, p.Yobs[0], A)
    return p, L, A, b


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_separable_factors_recover_T_and_N():
    p, L, A, b = _separable()
    nu_pix, t, phi, k0 = sylvester.separable_factors(p.D, p.tau, p.kappa)
    assert np.allclose(t[:, None] * nu_pix[None, :], p.D, rtol=1e-14, atol=0)
    assert t[0] == 1.0 and k0 == p.kappa[0] and np.all(phi == p.tau)
    with pytest.raises(ValueError):
        sylvester.separable_factors(p.D * np.linspace(1, 2, p.n)[None, :] ** np.arange(p.m)[:, None],
                                    p.tau, p.kappa)
    with pytest.raises(ValueError):
        sylvester.separable_factors(p.D, p.tau, p.kappa * np.arange(1, p.k + 1))


def test_lhat_eigendecomposition():
    p, L, A, b = _separable()
    _, t, phi, _ = sylvester.separable_factors(p.D, p.tau, p.kappa)
    rho, U, Uinv = sylvester.lhat_eig(A, t, phi)
    Lhat = A.T @ np.diag(t) @ A @ np.diag(1.0 / phi)
    assert np.allclose(Lhat @ U, U * rho[None, :], rtol=1e-10, atol=1e-10 * np.abs(Lhat).max())
    assert np.allclose(U.T @ np.diag(1.0 / phi) @ U, np.eye(p.k), atol=1e-12)
    assert np.allclose(Uinv @ U, np.eye(p.k), atol=1e-12)


def test_lanczos_relations():
    p, L, A, b = _separable(H=8, W=10)
    nu_pix, t, phi, k0 = sylvester.separable_factors(p.D, p.tau, p.kappa)
    Yhat = (b.T / nu_pix[:, None]) / phi[None, :]
    op = lambda X: sylvester.apply_NinvQ0(L, nu_pix, k0, X)
    j = 4
    V, H, B = sylvester.block_lanczos(op, nu_pix, Yhat, j)
    k = p.k
    Vall = np.hstack(V)                                   # n x (j+1)k
    # N-orthonormal basis
    assert np.abs(Vall.T @ (nu_pix[:, None] * Vall) - np.eye((j + 1) * k)).max() <= 1e-12
    # starting block reproduced
    assert _rel(V[0] @ B[0], Yhat) <= 1e-13
    # T_j = V_j^T Q_0 V_j (eq. tridiag-factorization), Q_0 = kappa0^2 I + L assembled
    Q0 = k0 ** 2 * np.eye(p.n) + L.toarray()
    Vj = Vall[:, :j * k]
    T = sylvester.tridiag(H, B)
    assert np.abs(Vj.T @ Q0 @ Vj - T).max() <= 1e-12 * np.abs(T).max()
    # Lanczos relation N^{-1} Q_0 V_j = V_{j+1} Tbar_j (eq. lanczos-relation)
    Tbar = np.zeros(((j + 1) * k, j * k))
    Tbar[:j * k] = T
    Tbar[j * k:, (j - 1) * k:] = B[j + 1]
    assert _rel(Vall @ Tbar, op(Vj)) <= 1e-12
    for i in range(2, j + 2):
        assert np.allclose(np.tril(B[i], -1), 0) and np.all(np.diag(B[i]) > 0)


@pytest.mark.parametrize("assembly", ["basis", "rerun"])
def test_solution_matches_direct_and_bartels_stewart(assembly):
    # tau varied, so P != I and the U^{-1} = U^T P^{-1} reading is exercised
    p, L, A, b = _separable(beta=[0.0, -3.0, 1.5])
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    X_d = solve.solve_direct(G, b)
    nu_pix, t, phi, k0 = sylvester.separable_factors(p.D, p.tau, p.kappa)
    X_bs = closed_form.sylvester_separable(L, nu_pix, t, phi, k0, A, p.Yobs[0])
    assert _rel(X_bs, X_d) <= 1e-10
    out = sylvester.solve_separable(L, p.D, p.tau, p.kappa, A, b, eps=1e-12, maxit=120,
                                    assembly=assembly)
    assert out["relgamma"][-1] <= 1e-12
    assert _rel(out["X"], X_d) <= 1e-9


def test_residual_estimate_is_the_true_sylvester_residual():
    p, L, A, b = _separable(H=8, W=10)
    nu_pix, t, phi, k0 = sylvester.separable_factors(p.D, p.tau, p.kappa)
    Yhat = (b.T / nu_pix[:, None]) / phi[None, :]
    Lhat = A.T @ np.diag(t) @ A @ np.diag(1.0 / phi)
    op = lambda X: sylvester.apply_NinvQ0(L, nu_pix, k0, X)
    nB0 = np.linalg.norm(sylvester.n_qr(Yhat, nu_pix)[1])
    for i in (1, 2, 5, 9):
        out = sylvester.sylvester_lanczos(L, nu_pix, t, phi, k0, A, Yhat, eps=0.0, maxit=i)
        assert out["iterations"] == i
        M = out["M"]
        R = op(M) + M @ Lhat - Yhat
        RU = R @ out["U"]
        true = np.sqrt(np.sum(nu_pix[:, None] * RU * RU))
        assert abs(true - out["relgamma"][-1] * nB0) <= 1e-7 * true


def test_workload_shaped_case_reaches_relres():
    # six power laws over the nine Planck channels: cond(B_0) ~ 1e8; the kept-basis assembly
    # reaches the tolerance on the true residual of G x = b
    p = synth.separable_problem(2, scale=64)
    L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
    A = model.powerlaw_mixing(p.nu, p.beta)
    b = model.rhs(p.D, p.Yobs[0], A)
    out = sylvester.solve_separable(L, p.D, p.tau, p.kappa, A, b, eps=1e-10)
    assert solve.relres(L, p.D, p.tau, p.kappa, A, out["X"], b) <= 1e-8
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    assert _rel(out["X"], solve.solve_direct(G, b)) <= 1e-6


# ---------------------------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------------------------
def _pins_pass():
    try:
        test_lanczos_relations()
        test_solution_matches_direct_and_bartels_stewart("basis")
        test_residual_estimate_is_the_true_sylvester_residual()
    except (AssertionError, np.linalg.LinAlgError):
        return False
    return True


def test_planted_mistakes_are_caught(monkeypatch):
    assert _pins_pass()
    step = sylvester.lanczos_step
    coef = sylvester.coefficients
    gam = sylvester.residual_gamma

    def step_B_not_transposed(op, nu_pix, V, Vold, Bi):
        return step(op, nu_pix, V, Vold, None if Bi is None else Bi.T)

    def qr_euclidean(W, nu_pix):
        q, r = np.linalg.qr(W)
        sg = np.sign(np.diag(r))
        return q * sg[None, :], sg[:, None] * r

    def coef_drop_Pinv(phi_T, Q, B0, U, Uinv, rho):
        return coef(phi_T, Q, B0, U, U.T, rho)

    def gamma_last_columns(T, Bnext, B0, U, rho):
        k = B0.shape[0]
        phi_T, Q = np.linalg.eigh(T)
        S = (U.T @ B0.T) @ Q[:k, :]
        J = Q[:, -k:] @ Bnext.T                   # Q_i E_i literally: last k columns
        g = sum(float(np.sum(((S[l] / (rho[l] + phi_T)) @ J) ** 2)) for l in range(k))
        return g, phi_T, Q

    def gamma_no_shift(T, Bnext, B0, U, rho):
        return gam(T, Bnext, B0, U, np.zeros_like(rho))

    plants = [("lanczos_step", step_B_not_transposed), ("n_qr", qr_euclidean),
              ("coefficients", coef_drop_Pinv), ("residual_gamma", gamma_last_columns),
              ("residual_gamma", gamma_no_shift)]
    for name, fn in plants:
        with monkeypatch.context() as mp:
            mp.setattr(sylvester, name, fn)
            assert not _pins_pass(), f"planted mistake in {name} went unnoticed"
    assert _pins_pass()
