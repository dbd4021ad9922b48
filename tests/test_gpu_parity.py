"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Tolerances:
* FP64 operator apply: |Y - Y_oracle| <= 64 u64 (|G| |X|) element-wise, the forward error
  bound of a sum of at most ~40 products per output (u64 = 2^-53).
* FP32 operator apply: |Y - Y_oracle| <= 64 u32 (|G| |X|) element-wise (u32 = 2^-24).
* Solves: relative solution error ||X - X_oracle||_F / ||X_oracle||_F <= 1e-8 in FP64 mode and
  <= 1e-6 in mixed mode (FP32 inner, FP64 refinement).
"""

import numpy as np
import pytest

import synth
from gpu_common import (device_batch, operator_for, oracle_L, oracle_solution, relerr,
                        small_problem)
from oracle import model

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08057_gb300 import build
    build.build()


def abs_apply(p, X, A):
    """|G| |X| with the same terms as the apply (for rounding-error bounds)."""
    L = oracle_L(p)
    absL = abs(L)
    out = np.empty_like(X)
    for j in range(p.k):
        out[j] = p.tau[j] * (p.kappa[j] ** 2 * np.abs(X[j]) + absL @ np.abs(X[j]))
    out += np.abs(A).T @ (p.D * (np.abs(A) @ np.abs(X)))
    return out


CASES = [
    ("lattice", 37, 41, 3, 5, 0),     # 1517 px: 6 tiles of 256, ragged tail
    ("sphere", 20, 33, 6, 9, 5),      # ld > n
    ("lattice", 9, 11, 1, 1, 3),      # scalar case
    ("sphere", 16, 17, 8, 16, 0),     # largest k and m the library takes
    ("lattice", 12, 30, 4, 7, 64),
    ("sphere", 3, 4, 2, 3, 1),        # smaller than one tile
    ("sphere", 16, 64, 6, 9, 0),      # whole tiles, aligned rows: staged FP32 apply
    ("lattice", 32, 32, 4, 7, 0),     # idem, lattice (neighbour windows two tiles away)
]


@pytest.mark.parametrize("kind,H,W,k,m,pad", CASES)
def test_apply_parity(kind, H, W, k, m, pad):
    import torch
    p = small_problem(kind, H, W, k, m, seed=100 + k + m)
    ld = p.n + pad
    op = operator_for(p, ld=ld)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, k, p.n))
    A = model.powerlaw_mixing(p.nu, p.beta)
    L = oracle_L(p)
    ref = np.stack([model.apply(L, p.D, p.tau, p.kappa, A, x) for x in X])
    bound = np.stack([abs_apply(p, x, A) for x in X])
    Xd = device_batch(X, ld)
    Y64 = op.apply(Xd).cpu().numpy()[:, :, :p.n]
    assert np.all(np.abs(Y64 - ref) <= 64 * U64 * bound + 1e-300)
    Y32 = op.apply(Xd.to(torch.float32)).cpu().numpy()[:, :, :p.n].astype(np.float64)
    X32 = Xd.to(torch.float32).cpu().numpy()[:, :, :p.n].astype(np.float64)
    ref32 = np.stack([model.apply(L, p.D, p.tau, p.kappa, A, x) for x in X32])
    # inputs rounded to FP32 first; then the FP32 arithmetic bound
    assert np.all(np.abs(Y32 - ref32) <= 64 * U32 * bound * 1.01 + 1e-30)
    op.close()


@pytest.mark.parametrize("nrhs", [3, 8, 16])
def test_staged_apply_many_columns(nrhs):
    """The staged stand-alone apply stages a tile's operator rows once for all its columns
    (more columns than ring stages): every column against the oracle, within the FP32 bound."""
    import torch
    p = small_problem("sphere", 16, 64, 6, 9, seed=77)   # n = 1024: whole tiles
    op = operator_for(p)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((nrhs, p.k, p.n))
    A = model.powerlaw_mixing(p.nu, p.beta)
    L = oracle_L(p)
    Xd = device_batch(X, p.n).to(torch.float32)
    Y32 = op.apply(Xd).cpu().numpy().astype(np.float64)
    X32 = Xd.cpu().numpy().astype(np.float64)
    for r in range(nrhs):
        ref = model.apply(L, p.D, p.tau, p.kappa, A, X32[r])
        bound = abs_apply(p, X32[r], A)
        assert np.all(np.abs(Y32[r] - ref) <= 64 * U32 * bound * 1.01 + 1e-30), r
    op.close()


def test_rhs_parity():
    p = small_problem("sphere", 19, 23, 5, 7, seed=9, nrhs=3)
    ld = p.n + 7
    op = operator_for(p, ld=ld)
    A = model.powerlaw_mixing(p.nu, p.beta)
    ref = np.stack([model.rhs(p.D, y, A) for y in p.Yobs])
    got = op.rhs(device_batch(p.Yobs, ld)).cpu().numpy()[:, :, :p.n]
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    op.close()


def test_explicit_mixing_matrix_override():
    from oracle import physical_mixing
    p = small_problem("lattice", 14, 15, 4, 9, seed=4)
    A = physical_mixing.physical_mixing(synth.PLANCK_NU)
    op = operator_for(p, A=A)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((1, 4, p.n))
    ref = model.apply(oracle_L(p), p.D, p.tau, p.kappa, A, X[0])
    got = op.apply(device_batch(X, p.n)).cpu().numpy()[0]
    assert np.abs(got - ref).max() <= 64 * U64 * abs_apply(p, X[0], A).max()
    Xo, b = oracle_solution(p, A=A)
    Xs, info = op.solve(device_batch(b, p.n), tol=1e-12, precision=0)
    assert info["code"] == 0
    assert relerr(Xs.cpu().numpy(), Xo) <= 1e-8
    op.close()


SOLVE_CASES = [
    ("lattice", 24, 24, 3, 5, 1),
    ("sphere", 18, 36, 6, 9, 1),
    ("lattice", 21, 19, 4, 7, 3),     # several right-hand sides, ragged
    ("sphere", 10, 12, 8, 12, 2),
    ("lattice", 7, 9, 1, 2, 1),
]


@pytest.mark.parametrize("kind,H,W,k,m,nrhs", SOLVE_CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_parity(kind, H, W, k, m, nrhs, precision):
    p = small_problem(kind, H, W, k, m, seed=7 + k, nrhs=nrhs)
    ld = p.n + 3
    op = operator_for(p, ld=ld)
    Xo, b = oracle_solution(p)
    tol = 1e-12 if precision == 0 else 1e-11
    X, info = op.solve(device_batch(b, ld), tol=tol, precision=precision)
    assert info["code"] == 0, info
    assert info["relres"] <= tol
    X = X.cpu().numpy()[:, :, :p.n]
    assert relerr(X, Xo) <= (1e-8 if precision == 0 else 1e-6)
    op.close()


@pytest.mark.parametrize("nrhs", [1, 2, 3])
def test_staged_residual_parity(nrhs, monkeypatch):
    """With the FP64 residual selected (SYLV_RESIDUAL=f64): whole tiles, an even caller leading
    dimension and at most two columns stage its streams (reported in the info); otherwise the
    direct kernel runs.  Cold and warm starts, one to three right-hand sides, against the
    oracle's direct solve.  The tile configuration is pinned to 256-pixel tiles with both
    staged inner kernels (the staged residual needs 256-pixel tiles; the tuner may prefer 128
    on a problem this small)."""
    monkeypatch.setenv("SYLV_TUNE_FORCE", "256,1,1,1")
    monkeypatch.setenv("SYLV_RESIDUAL", "f64")
    p = small_problem("sphere", 16, 64, 6, 9, seed=33, nrhs=nrhs)   # n = 1024, (k, m, E) = (6, 9, 4)
    Xo, b = oracle_solution(p)
    for ldu in (p.n, p.n + 1):
        op = operator_for(p, ld=ldu)
        assert op.ld == ldu
        Bd = device_batch(b, ldu)
        X, info = op.solve(Bd, tol=1e-11, precision=1)
        assert info["code"] == 0, info
        assert info["residual_staged"] == (1 if ldu % 2 == 0 and nrhs <= 2 else 0)
        assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
        X0 = device_batch(Xo + 1e-3, ldu)
        X, info = op.solve(Bd, X0=X0, tol=1e-11, precision=1)
        assert info["code"] == 0
        assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
        op.close()


def _df_bound(p, E, X, b, A):
    """(k + E + 4) 2^-45 (|b| + |G||X|) element-wise: the stated error bound of the
    double-float residual (each output sums at most k + 1 products and a stencil of E, every
    product leaving below 2^-45 of itself in the compensation and the operand splits)."""
    return (p.k + E + 4) * 2.0 ** -45 * (np.abs(b) + abs_apply(p, X, A))


RESID_CASES = [
    ("lattice", 37, 41, 3, 5, 2),     # ragged last tile, two columns
    ("sphere", 20, 33, 6, 9, 1),
    ("sphere", 16, 17, 8, 16, 3),     # largest k and m
    ("lattice", 9, 11, 1, 1, 1),      # scalar case
]


@pytest.mark.parametrize("kind,H,W,k,m,nrhs", RESID_CASES)
def test_residual_double_float_elementwise(kind, H, W, k, m, nrhs):
    """sylv_residual (the refinement's true residual, double-float on the FP32 pipe) against
    the oracle's FP64 b - G X element by element, on a nearly converged X (|r| ~ 1e-9 |b|, so
    b and G X cancel to nine digits), within the stated bound; its typical error is far below."""
    p = small_problem(kind, H, W, k, m, seed=60 + k, nrhs=nrhs)
    ld = p.n + 3
    op = operator_for(p, ld=ld)
    A = model.powerlaw_mixing(p.nu, p.beta)
    L = oracle_L(p)
    rng = np.random.default_rng(k + m)
    X = rng.standard_normal((nrhs, k, p.n)) * np.exp(rng.uniform(-3, 3, size=(nrhs, k, 1)))
    X[:, :, ::7] = 0.0                                   # exact zeros are split too
    GX = np.stack([model.apply(L, p.D, p.tau, p.kappa, A, x) for x in X])
    b = GX + 1e-9 * np.abs(GX).max() * rng.standard_normal(GX.shape)
    ref = b - GX
    R = op.residual(device_batch(b, ld), device_batch(X, ld)).cpu().numpy()[:, :, :p.n]
    E = op_degree_of(p)
    err = np.abs(R - ref)
    scale = np.stack([np.abs(b[r]) + abs_apply(p, X[r], A) for r in range(nrhs)])
    assert np.all(err <= np.stack([_df_bound(p, E, X[r], b[r], A) for r in range(nrhs)]))
    assert np.sqrt(np.mean((err / scale) ** 2)) <= 2.0 ** -46
    op.close()


def test_residual_outside_double_float_range_uses_fp64():
    """Pixels whose X lies outside the split's range, and a handle whose tau exceeds 2^40, are
    computed in FP64: still within the FP64 bound of the oracle's residual."""
    p = small_problem("sphere", 12, 20, 4, 6, seed=3)
    A = model.powerlaw_mixing(p.nu, p.beta)
    L = oracle_L(p)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((1, p.k, p.n))
    X[0, 1, 5] = 1e-30                                   # below 2^-60
    X[0, 2, 40] = 3e20                                   # above 2^61
    for tau_scale in (1.0, 1e13):
        q = synth.Problem(p.name, p.graph, p.k, p.m, p.tau * tau_scale, p.kappa, p.nu, p.beta,
                          p.D, p.Yobs, p.X_true, p.tol, {})
        op = operator_for(q)
        GX = model.apply(L, q.D, q.tau, q.kappa, A, X[0])
        b = GX + 1e-6 * rng.standard_normal(GX.shape)
        R = op.residual(device_batch(b, p.n), device_batch(X, p.n)).cpu().numpy()[0]
        bound = 64 * U64 * (np.abs(b) + abs_apply(q, X[0], A)) + \
            _df_bound(q, op_degree_of(q), X[0], b, A)
        assert np.all(np.abs(R - (b - GX)) <= bound), tau_scale
        op.close()


@pytest.mark.parametrize("nrhs,pad", [(1, 0), (2, 0), (3, 0), (8, 0), (1, 1), (3, 1)])
def test_double_float_residual_in_the_solve(nrhs, pad, monkeypatch):
    """Mixed solves whose true residual is formed in double-float: staged (whole tiles, an even
    caller leading dimension) for one to eight right-hand sides, plain otherwise (odd ld); cold
    and warm starts against the oracle's direct solve, and a warm start holding values below
    the double-float range at some pixels (recomputed in FP64 inside the kernel).  (Values
    whose squares overflow FP32 cannot start a mixed solve with either residual kernel: the
    inner solve's dot products are FP32.)"""
    monkeypatch.setenv("SYLV_TUNE_FORCE", "256,1,1,1")
    p = small_problem("sphere", 16, 64, 6, 9, seed=35, nrhs=nrhs)   # n = 1024: whole tiles
    ldu = p.n + pad
    op = operator_for(p, ld=ldu)
    Xo, b = oracle_solution(p)
    Bd = device_batch(b, ldu)
    X, info = op.solve(Bd, tol=1e-11, precision=1)
    assert info["code"] == 0, info
    assert info["residual_staged"] == (3 if pad == 0 else 2), info
    assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    X0 = Xo + 1e-3
    X, info = op.solve(Bd, X0=device_batch(X0, ldu), tol=1e-11, precision=1)
    assert info["code"] == 0 and relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    X0[:, :, ::37] = 1e-30                  # below the split's range: FP64 at those pixels
    X, info = op.solve(Bd, X0=device_batch(X0, ldu), tol=1e-11, precision=1)
    assert info["code"] == 0 and relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


def op_degree_of(p):
    """Off-diagonal entries per row of the problem's prior shape."""
    deg = int(np.max(np.diff(p.graph.rowptr))) - 1
    return 3 * deg if p.prior == "igmrf" else deg


MC_CASES = [
    ("sphere", 16, 64, 6, 9, 5, 1),    # whole tiles: the staged FP64 residual is skipped (R > 2)
    ("sphere", 20, 30, 6, 9, 8, 1),    # ragged last tile
    ("lattice", 24, 24, 4, 7, 6, 1),
    ("lattice", 21, 19, 3, 5, 7, 1),
    ("sphere", 18, 40, 5, 7, 8, 0),    # no preconditioner: empty operator slots in the update
    ("sphere", 16, 32, 6, 8, 2, 1),    # two columns through the multi-column pair as well
]


@pytest.mark.parametrize("kind,H,W,k,m,nrhs,precond", MC_CASES)
def test_multi_column_solve_parity(kind, H, W, k, m, nrhs, precond, monkeypatch):
    """The multi-column inner kernels (a tile's operator data staged once and kept in
    registers for all its columns; pixel block formed from the noise maps) pinned by the
    tuner override: every right-hand side against the oracle's direct solve (mixed, 1e-6),
    with a caller leading dimension above n."""
    from paper_2204_08057_gb300 import binding as Bn
    monkeypatch.setenv("SYLV_TUNE_FORCE", "256,1,2,2")
    p = small_problem(kind, H, W, k, m, seed=90 + nrhs, nrhs=nrhs)
    ld = p.n + 7
    op = operator_for(p, ld=ld)
    Xo, b = oracle_solution(p)
    pc = Bn.SYLV_PRECOND_BLOCK_JACOBI if precond else Bn.SYLV_PRECOND_NONE
    X, info = op.solve(device_batch(b, ld), tol=1e-11, precision=1, precond=pc,
                       maxit=100000)
    assert info["code"] == 0, info
    assert (info["apply_staged"], info["update_staged"]) == (2, 2), info
    X = X.cpu().numpy()[:, :, :p.n]
    for r in range(nrhs):
        assert relerr(X[r], Xo[r]) <= 1e-6, r
    # a warm start (the first inner iteration skips p and q) from a perturbed solution
    X0 = device_batch(Xo + 1e-3, ld)
    X, info = op.solve(device_batch(b, ld), X0=X0, tol=1e-11, precision=1, precond=pc,
                       maxit=100000)
    assert info["code"] == 0, info
    assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


def test_multi_column_igmrf_shape(monkeypatch):
    """The multi-column pair on the intrinsic GMRF shape (L^2: 12 off-diagonals per row) with
    the printed App. B mixing, four right-hand sides, against the oracle's direct solve."""
    monkeypatch.setenv("SYLV_TUNE_FORCE", "256,1,2,2")
    g = synth.latlong_sphere(16, 32)
    rng = np.random.default_rng(8)
    A = synth.PLANCK_A_PRINTED
    nu_pix = np.exp(0.3 * rng.standard_normal(g.n))
    D = (synth.PLANCK_T_PRINTED * 1e-6)[:, None] * nu_pix[None, :]
    Xt = rng.standard_normal((4, 4, g.n))
    Y = np.stack([A @ x + rng.standard_normal((9, g.n)) / np.sqrt(D) for x in Xt])
    p = synth.Problem("paper_sphere16x32", g, 4, 9, np.array([2.0, 0.5, 1.0, 3.0]),
                      np.full(4, 0.3), synth.PLANCK_NU, np.zeros(4), D, Y, Xt[0], 1e-8, {},
                      A=A.copy(), prior="igmrf")
    op = operator_for(p)
    Xo, b = oracle_solution(p)
    X, info = op.solve(device_batch(b, p.n), tol=1e-10, precision=1)
    assert info["code"] == 0, info
    assert (info["apply_staged"], info["update_staged"]) == (2, 2), info
    assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_blocked_pixel_order_parity(precision, monkeypatch):
    """The workload's grid in 16 x 16-pixel blocks (a renumbering that keeps most stencil
    neighbours inside a pixel's own 256-pixel tile): the staged kernels' solution is the
    oracle's solution of the row-major problem, renumbered."""
    monkeypatch.setenv("SYLV_TUNE_FORCE", "256,1,1,1")
    p = small_problem("sphere", 32, 64, 6, 9, seed=41)   # n = 2048: 8 tiles of 16 x 16 blocks
    perm = synth.blocked_order(32, 64, 16, 16)
    q = synth.permute_problem(p, perm)
    Xo, b = oracle_solution(p)
    op = operator_for(q)
    # cond(G) is ~8.7e5 here, so a relative solution error of 1e-8 needs relres ~1e-12
    X, info = op.solve(device_batch(b[:, :, perm], q.n), tol=1e-12 if precision == 0 else 1e-11,
                       precision=precision)
    assert info["code"] == 0, info
    assert relerr(X.cpu().numpy()[:, :, :q.n], Xo[:, :, perm]) <= (1e-8 if precision == 0
                                                                  else 1e-6)
    op.close()


@pytest.mark.parametrize("kind,H,W,nrhs", [("sphere", 16, 24, 1), ("sphere", 128, 256, 2)])
def test_solve_from_host_buffers(kind, H, W, nrhs):
    """sylv_solve_host (observations and solution in host memory, copies overlapped with the
    right-hand side and the refinement steps) gives the device path's solution bit for bit:
    one and eight pixel slices, page-locked and pageable buffers, a warm start, and a zero
    right-hand side (answered by the first residual, before any update)."""
    import torch
    p = small_problem(kind, H, W, 4, 7, seed=44, nrhs=nrhs)
    op = operator_for(p)
    Yd = device_batch(p.Yobs, op.ld)
    Xd, info_d = op.solve(op.rhs(Yd), tol=1e-10)
    assert info_d["code"] == 0
    ref = Xd.cpu()
    Yh = Yd.cpu().pin_memory()
    X, info = op.solve_host(Yh, tol=1e-10)
    assert info["code"] == 0 and info["iterations"] == info_d["iterations"]
    assert torch.equal(X, ref)
    X2, _ = op.solve_host(Yd.cpu(), out=torch.empty_like(ref), tol=1e-10)   # pageable
    assert torch.equal(X2, ref)
    X3, info3 = op.solve_host(Yh, X0=ref, tol=1e-10)
    assert info3["code"] == 0 and info3["iterations"] == 0
    assert torch.equal(X3, ref)
    Xz, infz = op.solve_host(torch.zeros_like(Yh), out=torch.full_like(ref, 7.0), tol=1e-10)
    assert infz["code"] == 0 and float(Xz.abs().max()) == 0.0
    Xo, _ = oracle_solution(p)
    assert relerr(X.numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


def test_solve_options_paths():
    """No preconditioner, no graph, profiling, warm start: same solution."""
    p = small_problem("sphere", 16, 20, 4, 6, seed=21)
    op = operator_for(p)
    Xo, b = oracle_solution(p)
    Bd = device_batch(b, p.n)
    for kw in (dict(precond=0, precision=0), dict(use_graph=0), dict(profile=1),
               dict(profile=1, use_graph=0), dict(check_every=1), dict(check_every=100),
               dict(inner_tol=1e-2)):
        X, info = op.solve(Bd, tol=1e-11, **kw)
        assert info["code"] == 0, (kw, info)
        assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6, kw
        if kw.get("profile"):
            assert info["n_apply"] > 0 and info["ms_apply"] > 0 and info["n_residual"] > 0
    X0 = device_batch(Xo + 1e-3, p.n)
    X, info = op.solve(Bd, X0=X0, tol=1e-11)
    assert info["code"] == 0
    assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


def test_config1_plain_fp64_cg():
    """64 x 64 periodic lattice, k=3, m=5, plain FP64 CG (no preconditioner) to 1e-10."""
    p = synth.config_problem(1)
    op = operator_for(p)
    Xo, b = oracle_solution(p)
    X, info = op.solve(device_batch(b, p.n), tol=1e-10, precision=0, precond=0)
    assert info["code"] == 0 and info["relres"] <= 1e-10
    # relres 1e-10 bounds the error by cond(G) * 1e-10; check against the oracle at 1e-6 and
    # at the FP64 parity bar after tightening the tolerance
    assert relerr(X.cpu().numpy()[0], Xo[0]) <= 1e-6
    X2, info2 = op.solve(device_batch(b, p.n), tol=1e-13, precision=0, precond=0)
    assert relerr(X2.cpu().numpy()[0], Xo[0]) <= 1e-8
    op.close()


def test_batched_parity():
    from paper_2204_08057_gb300.operator import solve_batched
    specs = [("lattice", 17, 19, 3, 5, 1), ("sphere", 12, 20, 6, 8, 2),
             ("lattice", 30, 31, 4, 6, 1), ("lattice", 9, 10, 5, 7, 1),
             ("sphere", 22, 25, 3, 5, 1), ("lattice", 5, 6, 6, 8, 3)]
    probs = [small_problem(*s[:5], seed=40 + i, nrhs=s[5]) for i, s in enumerate(specs)]
    ops = [operator_for(p, ld=p.n + i) for i, p in enumerate(probs)]
    refs = [oracle_solution(p) for p in probs]
    Bs = [device_batch(b, op.ld) for (_, b), op in zip(refs, ops)]
    for precision, bar in ((1, 1e-6), (0, 1e-8)):
        Xs, infos = solve_batched(ops, Bs, tol=1e-12 if precision == 0 else 1e-11,
                                  precision=precision)
        for X, (Xo, _), p, info in zip(Xs, refs, probs, infos):
            assert info["status"] == 0
            assert relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= bar
    # the same systems one by one give the same answers (independent scalars per system)
    X1, _ = ops[2].solve(Bs[2], tol=1e-11)
    assert relerr(X1.cpu().numpy()[:, :, :probs[2].n], refs[2][0]) <= 1e-6
    for op in ops:
        op.close()


def test_backward_matches_oracle_gradient():
    from oracle import gradient
    p = small_problem("sphere", 8, 10, 3, 5, seed=77, nrhs=2)
    op = operator_for(p)
    L = oracle_L(p)
    Xo, _ = oracle_solution(p)
    g = 2 * (Xo - p.X_true[None])
    ga = gradient.adjoint_gradient(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs, Xo, g)
    gt, gk, gb, lam, info = op.backward(device_batch(Xo, p.n), device_batch(g, p.n),
                                        device_batch(p.Yobs, p.n), tol=1e-12, precision=0)
    assert info["status"] == 0
    for got, ref in zip((gt, gk, gb), ga[:3]):
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    assert relerr(lam.cpu().numpy(), ga[3]) <= 1e-8
    op.close()


def test_autograd_function_fd():
    import torch
    from paper_2204_08057_gb300.autograd import SylvProblem, sylv_solve_differentiable
    from oracle import gradient
    p = small_problem("lattice", 8, 9, 3, 5, seed=5)
    prob = SylvProblem(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=p.D, nu=p.nu)
    tau = torch.tensor(p.tau, dtype=torch.float64, requires_grad=True)
    kappa = torch.tensor(p.kappa, dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(p.beta, dtype=torch.float64, requires_grad=True)
    Y = device_batch(p.Yobs, p.n)[0]
    Xt = torch.as_tensor(p.X_true, device="cuda")
    X = sylv_solve_differentiable(Y, tau, kappa, beta, prob, tol=1e-12, precision=0)
    loss = ((X - Xt) ** 2).sum()
    loss.backward()
    L = oracle_L(p)
    fd = gradient.fd_gradient(lambda Z: float(np.sum((Z - p.X_true) ** 2)), L, p.D, p.tau,
                              p.kappa, p.nu, p.beta, p.Yobs[0], h=1e-6)
    for got, ref in zip((tau.grad, kappa.grad, beta.grad), fd):
        assert np.allclose(got.numpy(), ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


def test_autograd_reuses_one_handle_across_parameters():
    """Two forwards at different parameters and their backwards in reverse order: each result
    and gradient against the oracle at its own parameters, with one sylv_create in total (the
    handle moves between parameter values by sylv_set_params)."""
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    from paper_2204_08057_gb300.autograd import SylvProblem, sylv_solve_differentiable
    from oracle import gradient
    p = small_problem("sphere", 8, 10, 3, 5, seed=17)
    prob = SylvProblem(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=p.D, nu=p.nu)
    Y = device_batch(p.Yobs, p.n)[0]
    Xt = torch.as_tensor(p.X_true, device="cuda")
    L = oracle_L(p)
    thetas = [(p.tau, p.kappa, p.beta), (p.tau * 1.3, p.kappa * 0.8, p.beta + 0.1)]
    made = Bn.calls["sylv_create"]
    leaves, losses = [], []
    for tau0, kappa0, beta0 in thetas:
        t = [torch.tensor(v, dtype=torch.float64, requires_grad=True)
             for v in (tau0, kappa0, beta0)]
        X = sylv_solve_differentiable(Y, *t, prob, tol=1e-12, precision=0)
        Xo = gradient.posterior_mean(L, p.D, tau0, kappa0, p.nu, beta0, p.Yobs[0])[0][0]
        assert relerr(X.detach().cpu().numpy()[:, :p.n], Xo) <= 1e-8
        leaves.append(t)
        losses.append(((X - Xt) ** 2).sum())
    for q in (1, 0):           # the second forward's backward first, then the first's
        losses[q].backward()
        tau0, kappa0, beta0 = thetas[q]
        Xo = gradient.posterior_mean(L, p.D, tau0, kappa0, p.nu, beta0, p.Yobs[0])[0][0]
        ga = gradient.adjoint_gradient(L, p.D, tau0, kappa0, p.nu, beta0, p.Yobs[0], Xo,
                                       2 * (Xo - p.X_true))
        for got, ref in zip((x.grad for x in leaves[q]), ga[:3]):
            assert np.abs(got.numpy() - ref).max() <= 1e-7 * np.abs(ref).max(), (q, got, ref)
    assert Bn.calls["sylv_create"] - made == 1
    prob.close()


@pytest.mark.parametrize("force,nrhs,precision,precond", [
    ("128,1,0,0", 1, 0, 1),     # FP64 PCG (direct kernels), block-Jacobi
    ("128,1,0,0", 2, 0, 0),     # FP64 CG
    ("128,1,0,0", 2, 1, 0),     # direct FP32 kernels
    ("256,1,1,1", 1, 1, 0),     # staged pair, consumer-side sums
    ("256,1,1,1", 2, 1, 0),
    ("256,1,2,2", 3, 1, 0),     # multi-column pair
])
def test_capped_iterates_match_oracle_pcg_steps(force, nrhs, precision, precond, monkeypatch):
    """Capping the iterations at j (1, 2, 7) stops the solve on the j-th CG iterate from X = 0:
    it must equal the oracle's CG (Algorithm 2) or block-Jacobi PCG after exactly j steps.
    This pins every step of the iteration, in particular the solution step that the operator
    kernel of the next iteration performs and its completion by the X update when the solve
    ends on an update (after one step, the only contribution).  The FP32 kernels are compared
    without the preconditioner: their preconditioner applies an FP16 copy of the block factor,
    a different (approximate) block-Jacobi operator than the oracle's exact one, so only the
    converged solutions agree there (the solve-parity tests)."""
    from oracle import solve as osolve
    from paper_2204_08057_gb300 import binding as Bn
    monkeypatch.setenv("SYLV_TUNE_FORCE", force)
    p = small_problem("sphere", 16, 64, 6, 9, seed=61, nrhs=nrhs)   # whole tiles: staged
    op = operator_for(p)
    _, b = oracle_solution(p)
    L, A = oracle_L(p), model.powerlaw_mixing(p.nu, p.beta)
    Bd = device_batch(b, p.n)
    for j in (1, 2, 7):
        X, info = op.solve(Bd, tol=1e-14, maxit=j, precision=precision, precond=precond,
                           allow_not_converged=True)
        assert info["code"] == Bn.SYLV_E_NOT_CONVERGED and info["iterations"] == j, (j, info)
        Xg = X.cpu().numpy()[:, :, :p.n]
        for r in range(nrhs):
            if precond:
                xo, it, _, _ = osolve.pcg_block_jacobi(L, p.D, p.tau, p.kappa, A, b[r], maxit=j)
            else:
                xo, it, _ = osolve.cg(lambda x: model.apply(L, p.D, p.tau, p.kappa, A, x),
                                      b[r], maxit=j)
            assert it == j
            err = relerr(Xg[r], xo)
            assert err <= (1e-11 if precision == 0 else 1e-4), (j, r, err)
    op.close()


@pytest.mark.parametrize("force,nrhs,stall", [
    ("256,1,1,1", 1, 1),     # staged double-float residual
    ("256,1,1,1", 1, 2),     # operator kernel, consumer-side sums
    ("256,1,1,1", 2, 4),     # update kernel
    ("256,1,2,2", 3, 2),     # multi-column operator kernel
    ("256,1,2,2", 3, 4),     # multi-column update kernel
])
def test_expired_wait_returns_timeout_and_the_handle_recovers(force, nrhs, stall, monkeypatch):
    """Failure detection without a device fault: a staged kernel whose producer issues nothing
    (SYLV_INJECT_STALL, a flag set on the host) leaves its consumers waiting on a stage that
    nothing fills; their bounded waits (budget cut to ~10 ms by SYLV_WAIT_BUDGET_CYCLES) run
    out, the CTAs record the timeout and leave, and the solve returns SYLV_E_TIMEOUT.  The same
    handle then solves correctly (the next solve's set-up resets the counters and column states
    the aborted kernels left)."""
    from paper_2204_08057_gb300 import binding as Bn
    monkeypatch.setenv("SYLV_TUNE_FORCE", force)
    p = small_problem("sphere", 16, 64, 6, 9, seed=51, nrhs=nrhs)   # whole tiles: staged
    op = operator_for(p)
    Xo, b = oracle_solution(p)
    Bd = device_batch(b, p.n)
    X, info = op.solve(Bd, tol=1e-11, precision=1)        # plan, tuner and kernels in place
    assert info["code"] == 0
    monkeypatch.setenv("SYLV_WAIT_BUDGET_CYCLES", "20000000")
    monkeypatch.setenv("SYLV_INJECT_STALL", str(stall))
    with pytest.raises(Bn.SylvError) as e:
        op.solve(Bd, tol=1e-11, precision=1, check_every=2)
    assert e.value.code == Bn.SYLV_E_TIMEOUT
    assert "wait" in str(e.value)
    monkeypatch.delenv("SYLV_INJECT_STALL")
    monkeypatch.delenv("SYLV_WAIT_BUDGET_CYCLES")
    X, info = op.solve(Bd, tol=1e-11, precision=1)
    assert info["code"] == 0 and relerr(X.cpu().numpy()[:, :, :p.n], Xo) <= 1e-6
    op.close()


def test_single_pixel_and_isolated_pixels():
    """n = 1 (no neighbours, ELL width 0): G is the k x k block itself."""
    import torch
    from paper_2204_08057_gb300.operator import Operator
    k, m = 3, 4
    nu = np.array([30.0, 100.0, 217.0, 545.0])
    beta = np.array([0.5, -2.0, 1.2])
    tau = np.array([1.0, 2.0, 0.5])
    kappa = np.array([0.3, 0.1, 1.0])
    d = np.array([[1.5], [0.7], [2.0], [1.1]])
    op = Operator(rowptr=np.array([0, 1]), col=np.array([0]), val=np.array([0.0]), D=d,
                  tau=tau, kappa=kappa, nu=nu, beta=beta)
    A = model.powerlaw_mixing(nu, beta)
    Gk = np.diag(tau * kappa ** 2) + (A.T * d[:, 0]) @ A
    b = np.array([[1.0], [-2.0], [0.5]])
    X, info = op.solve(torch.as_tensor(b[None], device="cuda"), tol=1e-13, precision=0)
    assert info["code"] == 0
    assert np.allclose(X.cpu().numpy()[0, :, 0], np.linalg.solve(Gk, b[:, 0]), rtol=1e-10)
    op.close()


def test_zero_rhs_gives_zero():
    p = small_problem("lattice", 6, 7, 3, 5, seed=3)
    op = operator_for(p)
    X, info = op.solve(op.zeros(1), tol=1e-10)
    assert info["code"] == 0 and float(X.abs().max()) == 0.0
    op.close()


def test_error_statuses():
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    from paper_2204_08057_gb300.operator import Operator
    p = small_problem("lattice", 6, 7, 3, 5, seed=3)
    bad_col = p.graph.col.copy()
    bad_col[5] = p.n + 3                               # out of range
    with pytest.raises(Bn.SylvError) as e:
        Operator(rowptr=p.graph.rowptr, col=bad_col, val=p.graph.val, D=p.D, tau=p.tau,
                 kappa=p.kappa, nu=p.nu, beta=p.beta)
    assert e.value.code == Bn.SYLV_E_INVALID
    bad_ptr = p.graph.rowptr.copy()
    bad_ptr[3], bad_ptr[4] = bad_ptr[4], bad_ptr[3]    # non-monotone
    with pytest.raises(Bn.SylvError) as e:
        Operator(rowptr=bad_ptr, col=p.graph.col, val=p.graph.val, D=p.D, tau=p.tau,
                 kappa=p.kappa, nu=p.nu, beta=p.beta)
    assert e.value.code == Bn.SYLV_E_INVALID
    D = p.D.copy()
    D[1, 4] = -1.0
    with pytest.raises(Bn.SylvError) as e:
        Operator(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=D, tau=p.tau,
                 kappa=p.kappa, nu=p.nu, beta=p.beta)
    assert e.value.code == Bn.SYLV_E_INVALID
    D[1, 4] = np.nan
    with pytest.raises(Bn.SylvError):
        Operator(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=D, tau=p.tau,
                 kappa=p.kappa, nu=p.nu, beta=p.beta)
    # a row with 9 off-diagonal entries exceeds the library's ELL width
    n = 10
    rowptr = np.array([0, 10] + list(range(12, 12 + 2 * 9, 2)), dtype=np.int32)
    col = np.concatenate([np.arange(10), np.ravel([[i, 0] for i in range(1, 10)])])
    val = np.concatenate([[9.0], -np.ones(9), np.ravel([[1.0, -1.0]] * 9)])
    with pytest.raises(Bn.SylvError) as e:
        Operator(rowptr=rowptr, col=col, val=val, D=np.ones((2, n)), tau=[1.0], kappa=[1.0],
                 nu=[30.0, 70.0], beta=[1.0])
    assert e.value.code == Bn.SYLV_E_UNSUPPORTED
    # iteration cap: NOT_CONVERGED with a finite last iterate and the reached residual
    op = operator_for(p)
    _, b = oracle_solution(p)
    X, info = op.solve(device_batch(b, p.n), tol=1e-12, maxit=2, precision=0,
                       allow_not_converged=True)
    assert info["code"] == Bn.SYLV_E_NOT_CONVERGED
    assert np.isfinite(X.cpu().numpy()).all() and 0 < info["relres"] < 1
    with pytest.raises(Bn.SylvError) as e:
        op.solve(device_batch(b, p.n), tol=0.0)
    assert e.value.code == Bn.SYLV_E_INVALID
    # non-finite right-hand side: reported, not hung
    bn = b.copy()
    bn[0, 1, 3] = np.inf
    X, info = op.solve(device_batch(bn, p.n), tol=1e-8, allow_not_converged=True,
                       allow=(Bn.SYLV_E_BREAKDOWN,))
    assert info["code"] in (Bn.SYLV_E_BREAKDOWN, Bn.SYLV_E_NOT_CONVERGED)
    assert torch.cuda.is_available()
    op.close()
