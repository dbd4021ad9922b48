"""GPU parity of the intrinsic GMRF prior (App. C: Q_j = phi_j D^T D, D the Laplacian; the
library forms L^2 on the device) with the physical mixing matrix and channel weights of
App. B, through the C ABI.

The device-built operator is compared element-wise with the oracle's (L^T L from a sparse
product), and the solves with the oracle's direct solve (FP64 <= 1e-8, mixed <= 1e-6) for the
improper prior (kappa = 0) and with a mass term, by PCG and by the Lanczos-Sylvester solver
(the paper's model is separable: C = T kron N, one prior shape); at full size on the lattice
against the Fourier closed form with squared modes.
"""

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_A, oracle_L, oracle_solution, relerr
from oracle import closed_form, model

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


def _paper_model(kind, H, W, seed, kappa0=0.0, phi=(2.0, 0.5, 1.0, 3.0)):
    """The paper's model on a small grid: printed A (k = 4) and T, per-pixel N, IGMRF prior."""
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    rng = np.random.default_rng(seed)
    A = synth.PLANCK_A_PRINTED
    nu_pix = np.exp(0.3 * rng.standard_normal(g.n))
    D = (synth.PLANCK_T_PRINTED * 1e-6)[:, None] * nu_pix[None, :]
    X = rng.standard_normal((4, g.n))
    Y = A @ X + rng.standard_normal((9, g.n)) / np.sqrt(D)
    return synth.Problem(f"paper_{kind}{H}x{W}", g, 4, 9, np.array(phi), np.full(4, kappa0),
                         synth.PLANCK_NU, np.zeros(4), D, Y[None], X, 1e-8, {},
                         A=A.copy(), prior="igmrf")


@pytest.mark.parametrize("kind,H,W", [("sphere", 12, 20), ("lattice", 16, 18)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_igmrf_apply_parity(kind, H, W, dtype):
    import torch
    p = _paper_model(kind, H, W, seed=3, kappa0=0.25)
    op = operator_for(p)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((2, p.k, p.n))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Y = op.apply(device_batch(X, op.ld).to(tdt)).double().cpu().numpy()[:, :, :p.n]
    L2 = oracle_L(p)
    A = oracle_A(p)
    Xin = X if dtype == "f64" else X.astype(np.float32).astype(np.float64)
    ref = np.stack([model.apply(L2, p.D, p.tau, p.kappa, A, x) for x in Xin])
    absL = abs(L2)
    bound = np.stack([model.apply(absL, p.D, p.tau, p.kappa, abs(A), abs(x)) for x in Xin])
    u = U64 if dtype == "f64" else U32
    assert np.all(np.abs(Y - ref) <= 64 * u * bound + 1e-300)
    op.close()


@pytest.mark.parametrize("kind,H,W,kappa0", [("sphere", 12, 20, 0.0), ("lattice", 16, 18, 0.0),
                                             ("sphere", 16, 24, 0.3)])
@pytest.mark.parametrize("precision", [0, 1])
def test_igmrf_solve_parity(kind, H, W, kappa0, precision):
    p = _paper_model(kind, H, W, seed=5, kappa0=kappa0)
    Xd, _ = oracle_solution(p)
    op = operator_for(p)
    Bv = op.rhs(device_batch(p.Yobs, op.ld))
    tol = 1e-12 if precision == 0 else 1e-10
    X, info = op.solve(Bv, tol=tol, precision=precision)
    assert info["code"] == 0, info
    assert relerr(X.cpu().numpy()[:, :, :p.n], Xd) <= (1e-8 if precision == 0 else 1e-6)
    # the paper's model is separable: the Lanczos-Sylvester solver applies as well
    Xl, infol = op.solve_sylvester(Bv, tol=tol, precision=precision, inner_tol=1e-5)
    assert infol["code"] == 0, infol
    assert relerr(Xl.cpu().numpy()[:, :, :p.n], Xd) <= (1e-8 if precision == 0 else 1e-6)
    op.close()


def test_igmrf_lattice_full_size_closed_form():
    # 512 x 512 periodic lattice, noise constant per channel (the printed T), improper prior
    import torch
    H = W = 512
    g = synth.periodic_lattice(H, W)
    rng = np.random.default_rng(17)
    A = synth.PLANCK_A_PRINTED
    d = synth.PLANCK_T_PRINTED * 1e-6
    D = np.repeat(d[:, None], g.n, axis=1)
    tau = np.array([3.0, 0.5, 1.0, 2.0])
    Y = rng.standard_normal((9, g.n))
    p = synth.Problem("lattice512_igmrf", g, 4, 9, tau, np.zeros(4), synth.PLANCK_NU,
                      np.zeros(4), D, Y[None], np.zeros((4, g.n)), 1e-8, {}, A=A.copy(),
                      prior="igmrf")
    Xc = closed_form.lattice_homogeneous(H, W, tau, np.zeros(4), A, d, Y, power=2)
    op = operator_for(p)
    Bv = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(Bv, tol=1e-11)
    assert info["code"] == 0
    assert relerr(X.cpu().numpy()[0], Xc) <= 1e-6
    X64, info64 = op.solve(Bv, tol=1e-12, precision=0)
    assert info64["code"] == 0
    assert relerr(X64.cpu().numpy()[0], Xc) <= 1e-8
    op.close()


def test_igmrf_paper_workload_residual_by_oracle():
    # the 1024 x 2048 paper-model workload: the reported residual recomputed by the oracle
    import torch
    p = synth.igmrf_problem(2)
    op = operator_for(p)
    Bv = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(Bv, tol=1e-8)
    assert info["code"] == 0 and info["relres"] <= 1e-8
    L2 = oracle_L(p)
    A = oracle_A(p)
    b = model.rhs(p.D, p.Yobs[0], A)
    r = b - model.apply(L2, p.D, p.tau, p.kappa, A, X.cpu().numpy()[0][:, :p.n])
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.01 * info["relres"] + 1e-14
    op.close()
