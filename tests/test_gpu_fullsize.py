"""Parity at the workloads' full sizes (GPU), where the oracle's direct solve is too slow.

* 1024 x 2048 sphere (n = 2,097,152, k = 6, m = 9) with noise constant along each latitude
  row: the solve against the closed form (longitude DFT + banded Cholesky per mode), mixed
  (relerr <= 1e-6) and FP64 (relerr <= 1e-8).
* The bench workload itself (lognormal per-pixel noise): operator rows sampled one by one by
  the oracle (poles, wrap-around columns, random pixels), and the solve's true FP64 residual
  recomputed by the oracle's matrix-free apply (a property that holds at any size).
* 512 x 1024 sphere (k = 4, m = 7), latitude noise: the adjoint gradient against the oracle's
  formulas evaluated with closed-form solutions for X and lambda.
* The 64-system batch: every member's residual by the oracle; the two smallest members
  against the direct solve.
* 1024 x 3072 sphere with 8 right-hand sides (the multi-RHS workload at a quarter of its
  sides): every right-hand side's residual by the oracle.
"""

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_L, oracle_solution, relerr
from oracle import closed_form, gradient, model

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


def _rows(p):
    H, W = p.graph.H, p.graph.W
    rng = np.random.default_rng(11)
    picks = [0, W - 1, W, (H - 1) * W, p.n - 1, (H // 2) * W + W // 2]
    return np.unique(np.concatenate([picks, rng.integers(0, p.n, 400)]))


def test_sphere_2M_latitude_noise_against_closed_form():
    p = synth.config_problem(2, noise="latitude")
    A = model.powerlaw_mixing(p.nu, p.beta)
    d_rows = p.D.reshape(p.m, p.graph.H, p.graph.W)[:, :, 0]
    Xc = closed_form.sphere_latitude_noise(p.graph.H, p.graph.W, p.tau, p.kappa, A, d_rows,
                                           Y=p.Yobs[0])
    op = operator_for(p)
    import torch
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(B, tol=1e-10)
    assert info["code"] == 0
    assert relerr(X.cpu().numpy()[0], Xc) <= 1e-6
    X64, info64 = op.solve(B, tol=1e-12, precision=0)
    assert info64["code"] == 0
    assert relerr(X64.cpu().numpy()[0], Xc) <= 1e-8
    op.close()


def test_sphere_2M_bench_workload_rows_and_residual():
    import torch
    p = synth.config_problem(2)
    op = operator_for(p)
    L = oracle_L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    rng = np.random.default_rng(5)
    Xr = rng.standard_normal((1, p.k, p.n))
    rows = _rows(p)
    ref = model.apply_rows(L, p.D, p.tau, p.kappa, A, Xr[0], rows)
    absx = np.abs(Xr[0])
    bound = model.apply_rows(abs(L), p.D, np.abs(p.tau), np.abs(p.kappa), np.abs(A), absx, rows)
    Y64 = op.apply(device_batch(Xr, p.n)).cpu().numpy()[0][:, rows]
    assert np.all(np.abs(Y64 - ref) <= 64 * U64 * bound)
    X32 = device_batch(Xr, p.n).to(torch.float32)
    Y32 = op.apply(X32).cpu().numpy()[0][:, rows].astype(np.float64)
    ref32 = model.apply_rows(L, p.D, p.tau, p.kappa, A,
                             X32.cpu().numpy()[0].astype(np.float64), rows)
    assert np.all(np.abs(Y32 - ref32) <= 64 * U32 * bound * 1.01)
    # solve, then the true residual by the oracle's matrix-free FP64 apply
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(B, tol=1e-8)
    assert info["code"] == 0
    b = model.rhs(p.D, p.Yobs[0], A)
    assert np.allclose(B.cpu().numpy()[0], b, rtol=1e-12, atol=1e-12 * np.abs(b).max())
    Xh = X.cpu().numpy()[0]
    r = b - model.apply(L, p.D, p.tau, p.kappa, A, Xh)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.0e-8 * 1.001
    assert abs(rel - info["relres"]) <= 1e-3 * rel
    # the refinement's double-float residual of that solution, element by element on the
    # sampled rows (b and G X cancel to eight digits there)
    assert info["residual_staged"] in (2, 3)     # double-float (staged where the rows allow)
    Rd = op.residual(B, X).cpu().numpy()[0][:, rows]
    ref_rows = b[:, rows] - model.apply_rows(L, p.D, p.tau, p.kappa, A, Xh, rows)
    scale = np.abs(b[:, rows]) + model.apply_rows(abs(L), p.D, np.abs(p.tau), np.abs(p.kappa),
                                                  np.abs(A), np.abs(Xh), rows)
    E = int(np.max(np.diff(p.graph.rowptr))) - 1
    assert np.all(np.abs(Rd - ref_rows) <= (p.k + E + 4) * 2.0 ** -45 * scale)
    op.close()


def test_sphere_512x1024_gradient_against_closed_forms():
    p = synth.config_problem(4, noise="latitude")
    H, W = p.graph.H, p.graph.W
    A = model.powerlaw_mixing(p.nu, p.beta)
    d_rows = p.D.reshape(p.m, H, W)[:, :, 0]
    Xc = closed_form.sphere_latitude_noise(H, W, p.tau, p.kappa, A, d_rows, Y=p.Yobs[0])
    g = 2.0 * (Xc - p.X_true)
    lam = closed_form.sphere_latitude_noise(H, W, p.tau, p.kappa, A, d_rows, b=g)
    L = oracle_L(p)
    ref = gradient.gradient_from_adjoint(L, p.D, p.tau, p.kappa, p.nu, p.beta, p.Yobs[0], Xc,
                                         lam)
    op = operator_for(p)
    gt, gk, gb, lam_d, info = op.backward(device_batch(Xc, p.n), device_batch(g, p.n),
                                          device_batch(p.Yobs, p.n), tol=1e-12, precision=0)
    assert info["status"] == 0
    assert relerr(lam_d.cpu().numpy()[0], lam) <= 1e-8
    for got, want in zip((gt, gk, gb), ref):
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    op.close()


def test_batch_of_64_every_member():
    import torch
    from paper_2204_08057_gb300.operator import solve_batched
    probs = synth.batch_problems(64)
    ops = [operator_for(p) for p in probs]
    Bs = [op.rhs(torch.from_numpy(p.Yobs).cuda()) for op, p in zip(ops, probs)]
    Xs, infos = solve_batched(ops, Bs, tol=1e-8)
    for p, X, info in zip(probs, Xs, infos):
        assert info["status"] == 0
        L = oracle_L(p)
        A = model.powerlaw_mixing(p.nu, p.beta)
        b = model.rhs(p.D, p.Yobs[0], A)
        r = b - model.apply(L, p.D, p.tau, p.kappa, A, X.cpu().numpy()[0])
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.0e-8 * 1.001, p.name
    small = sorted(range(len(probs)), key=lambda t: probs[t].n)[:2]
    for t in small:
        Xo, _ = oracle_solution(probs[t])
        Xt, _ = solve_batched([ops[t]], [Bs[t]], tol=1e-11)
        assert relerr(Xt[0].cpu().numpy(), Xo) <= 1e-6
    for op in ops:
        op.close()


def test_multi_rhs_8_on_3M_pixels():
    import torch
    p = synth.config_problem(5, scale=4)         # 1024 x 3072 sphere, k = 6, m = 9, R = 8
    assert p.nrhs == 8
    op = operator_for(p)
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(B, tol=1e-8)
    assert info["code"] == 0
    L = oracle_L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    Xh = X.cpu().numpy()
    for r in range(p.nrhs):
        b = model.rhs(p.D, p.Yobs[r], A)
        res = b - model.apply(L, p.D, p.tau, p.kappa, A, Xh[r])
        assert np.linalg.norm(res) / np.linalg.norm(b) <= 1.0e-8 * 1.001
    op.close()
