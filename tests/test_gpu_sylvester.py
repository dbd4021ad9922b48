"""GPU parity of the block-Lanczos Sylvester solver (sylv_solve_sylvester, Sec. 3.3,
Algorithms 4 and 5) against the oracle, through the C ABI.

The solution is compared with the oracle's direct solve of the assembled system (FP64 mode:
relative error <= 1e-8, mixed: <= 1e-6) on separable problems (d_ci = t_c nu_i, one prior
shape) over lattices, spheres and a degree-6 graph (generic ELL width), ragged tiles, ld > n,
k = 1..8, several right-hand sides, warm starts, graph and direct launches; the reported
residual is recomputed by the oracle; non-separable problems are refused.
"""

import dataclasses

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_L, oracle_solution, relerr
from oracle import model

pytestmark = pytest.mark.gpu

SYLV_E_UNSUPPORTED = 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08057_gb300 import build
    build.build()


def _sep(kind, H, W, k, m, seed, nrhs=1, kappa0=0.2, tau=None):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    tau = np.linspace(0.5, 2.0, k) if tau is None else tau
    return synth.make_problem(f"sep_{kind}{H}x{W}_k{k}", g, k, nu, None, [kappa0] * k, tau,
                              seed, beta_draw=(-3, 2), noise="separable", nrhs=nrhs)


def _triangular(H, W, k, m, seed):
    """Periodic lattice plus one diagonal per cell: degree 6, so the generic ELL path runs."""
    p = _sep("lattice", H, W, k, m, seed)
    r = np.repeat(np.arange(H), W)
    c = np.tile(np.arange(W), H)
    i = r * W + c
    u = np.concatenate([i, i, i])
    v = np.concatenate([r * W + (c + 1) % W, ((r + 1) % H) * W + c,
                        ((r + 1) % H) * W + (c + 1) % W])
    w = np.concatenate([np.ones(H * W), np.ones(H * W), 0.5 * np.ones(H * W)])
    rowptr, col, val = synth.laplacian_csr_from_edges(H * W, u, v, w)
    p.graph = dataclasses.replace(p.graph, rowptr=rowptr, col=col, val=val)
    return p


def _solve(p, precision, ld=None, **kw):
    import torch
    op = operator_for(p, ld=ld)
    Bv = op.rhs(device_batch(p.Yobs, op.ld))
    X, info = op.solve_sylvester(Bv, precision=precision, **kw)
    torch.cuda.synchronize()
    return op, X.cpu().numpy()[:, :, :p.n], info


CASES = [
    ("sphere", 24, 40, 3, 5, 0),      # n = 960: ragged last tile
    ("lattice", 32, 32, 4, 7, 0),
    ("sphere", 16, 64, 6, 9, 64),     # ld > n
    ("lattice", 20, 24, 8, 12, 0),
    ("sphere", 12, 20, 1, 3, 0),
]


@pytest.mark.parametrize("kind,H,W,k,m,pad", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_sylvester_solve_parity(kind, H, W, k, m, pad, precision):
    p = _sep(kind, H, W, k, m, seed=100 + H + k)
    Xd, b = oracle_solution(p)
    ld = None if pad == 0 else ((p.n + 255) // 256) * 256 + pad
    op, X, info = _solve(p, precision, ld=ld, tol=1e-12 if precision == 0 else 1e-10)
    assert info["code"] == 0, info
    assert relerr(X, Xd) <= (1e-8 if precision == 0 else 1e-6)
    # the reported residual is the true one
    L = oracle_L(p)
    A = model.powerlaw_mixing(p.nu, p.beta)
    r = b[0] - model.apply(L, p.D, p.tau, p.kappa, A, X[0])
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1.01 * info["relres"] + 1e-15
    op.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_sylvester_generic_ell_width(precision):
    p = _triangular(18, 22, 5, 7, seed=7)
    Xd, _ = oracle_solution(p)
    op, X, info = _solve(p, precision, tol=1e-12 if precision == 0 else 1e-10)
    assert info["code"] == 0
    assert relerr(X, Xd) <= (1e-8 if precision == 0 else 1e-6)
    op.close()


def test_sylvester_multiple_rhs_and_options():
    import torch
    p = _sep("sphere", 20, 36, 4, 7, seed=5, nrhs=3)
    Xd, _ = oracle_solution(p)
    op = operator_for(p)
    Bv = op.rhs(device_batch(p.Yobs, op.ld))
    for kw in ({"use_graph": 1}, {"use_graph": 0, "profile": 1}, {"check_every": 3},
               {"profile": 1}, {"inner_tol": 1e-2}):
        X, info = op.solve_sylvester(Bv, tol=1e-10, **kw)
        assert info["code"] == 0, (kw, info)
        assert relerr(X.cpu().numpy()[:, :, :p.n], Xd) <= 1e-6, kw
        if kw.get("profile"):
            assert info["ms_apply"] > 0 and info["ms_update"] > 0 and info["ms_residual"] > 0
    # warm start from the answer: one residual, no Lanczos step
    X0 = torch.from_numpy(np.ascontiguousarray(Xd)).cuda()
    X0p = torch.zeros((3, p.k, op.ld), dtype=torch.float64, device="cuda")
    X0p[:, :, :p.n] = X0
    X, info = op.solve_sylvester(Bv, X0=X0p, tol=1e-8)
    assert info["code"] == 0 and info["iterations"] == 0
    # iteration cap
    from paper_2204_08057_gb300 import binding as B
    X, info = op.solve_sylvester(Bv, tol=1e-12, maxit=3, allow_not_converged=True)
    assert info["code"] == B.SYLV_E_NOT_CONVERGED and info["iterations"] <= 3
    op.close()


def test_sylvester_matches_pcg_on_workload_shape():
    # the separable 1024 x 2048 workload at 1/16 of its sides (64 x 128, k = 6, m = 9)
    # (relres <= 1e-8 bounds the error only up to cond(G), so the error is checked at 1e-11)
    p = synth.separable_problem(2, scale=16)
    Xd, _ = oracle_solution(p)
    op, X, info = _solve(p, 1, tol=1e-8)
    assert info["code"] == 0 and info["relres"] <= 1e-8
    op.close()
    op, X, info = _solve(p, 1, tol=1e-11)
    assert info["code"] == 0
    assert relerr(X, Xd) <= 1e-6
    op.close()


def test_zero_rhs_and_refusals():
    import torch
    from paper_2204_08057_gb300 import binding as B
    p = _sep("lattice", 16, 16, 3, 5, seed=3)
    op = operator_for(p)
    Z = torch.zeros((1, p.k, op.ld), dtype=torch.float64, device="cuda")
    X, info = op.solve_sylvester(Z)
    assert info["code"] == 0 and float(X.abs().max()) == 0.0
    op.close()
    # per-pixel noise that is not separable
    q = synth.make_problem("nonsep", synth.periodic_lattice(16, 16), 3,
                           synth.PLANCK_NU[[0, 3, 5, 7, 8]], None, [0.2] * 3, 1.0, 9,
                           beta_draw=(-3, 2), noise="lognormal")
    op = operator_for(q)
    Bv = op.rhs(device_batch(q.Yobs, op.ld))
    with pytest.raises(B.SylvError) as e:
        op.solve_sylvester(Bv)
    assert e.value.code == SYLV_E_UNSUPPORTED and "separable" in B.sylv_last_error()
    op.close()
    # prior shapes that differ
    r = _sep("lattice", 16, 16, 3, 5, seed=4)
    r.kappa = np.array([0.2, 0.3, 0.2])
    op = operator_for(r)
    Bv = op.rhs(device_batch(r.Yobs, op.ld))
    with pytest.raises(B.SylvError) as e:
        op.solve_sylvester(Bv)
    assert e.value.code == SYLV_E_UNSUPPORTED and "kappa" in B.sylv_last_error()
    op.close()


@pytest.mark.parametrize("staged", ["0", "1"])
def test_sylvester_plain_and_staged_kernels_agree(monkeypatch, staged):
    # the staged FP32 passes (bulk copies) and the plain ones give the same solution
    monkeypatch.setenv("SYLV_LZ_STAGED", staged)
    p = _sep("sphere", 32, 48, 6, 9, seed=21)
    Xd, _ = oracle_solution(p)
    op, X, info = _solve(p, 1, tol=1e-10)
    assert info["code"] == 0
    assert info["apply_staged"] == int(staged)
    assert relerr(X, Xd) <= 1e-6
    op.close()
