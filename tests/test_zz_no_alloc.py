"""sylv_solve_noalloc, the allocation-free solve, against sylv_solve (GPU).

The entry point serves callers that cannot allocate device memory when they solve (a
pipeline with memory reserved at start-up, a fixed memory budget, or a loop that must avoid
an allocator's synchronisation); its workspace is a fixed device array inside the library.
This file is collected last so that a run stopping at its first failure has run every other
test; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_solution, relerr, small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08057_gb300 import build
    build.build()


@pytest.mark.parametrize("kind,H,W,k,m,nrhs,precision", [
    ("lattice", 40, 40, 3, 5, 1, 1),
    ("sphere", 24, 48, 6, 9, 2, 1),
    ("sphere", 20, 30, 4, 7, 1, 0),
    ("lattice", 9, 13, 8, 12, 3, 1),
])
def test_noalloc_matches_sylv_solve_twice(kind, H, W, k, m, nrhs, precision):
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    p = small_problem(kind, H, W, k, m, seed=300 + k, nrhs=nrhs)
    ld = p.n + 5
    op = operator_for(p, ld=ld)
    Xo, b = oracle_solution(p)
    Bd = device_batch(b, ld)
    tol = 1e-11 if precision == 1 else 1e-12
    bar = 1e-6 if precision == 1 else 1e-8
    X_ref, info_ref = op.solve(Bd, tol=tol, precision=precision)
    assert info_ref["code"] == 0
    for call in range(2):     # the scratch array keeps the previous call's contents
        X = torch.full_like(Bd, float("nan"))
        opts = Bn.make_opts(tol=tol, precision=precision)
        code, info = Bn.sylv_solve_noalloc(op.handle, Bd, X, nrhs, opts, k=k, ld=ld, n=p.n)
        assert code == Bn.SYLV_OK and info.relres <= tol, (call, info.as_dict())
        Xn = X.cpu().numpy()[:, :, :p.n]
        assert relerr(Xn, X_ref.cpu().numpy()[:, :, :p.n]) <= bar
        assert relerr(Xn, Xo) <= bar
    op.close()


def test_noalloc_rejects_workspace_beyond_the_array():
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    p = small_problem("lattice", 400, 400, 6, 8, seed=5)   # 160k px x 6 x 8 RHS > 16 MiB
    op = operator_for(p)
    Bd = torch.zeros((8, 6, p.n), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(Bd)
    with pytest.raises(Bn.SylvError) as e:
        Bn.sylv_solve_noalloc(op.handle, Bd, X, 8, Bn.make_opts(), k=6, ld=p.n, n=p.n)
    assert e.value.code == Bn.SYLV_E_UNSUPPORTED
    assert "scratch" in str(e.value)
    op.close()


def _noalloc(op, p, Bd, nrhs, k, ld, tol, precision):
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    X = torch.full_like(Bd, float("nan"))
    code, info = Bn.sylv_solve_noalloc(op.handle, Bd, X, nrhs,
                                       Bn.make_opts(tol=tol, precision=precision),
                                       k=k, ld=ld, n=p.n)
    assert code == Bn.SYLV_OK and info.relres <= tol, info.as_dict()
    return X.cpu().numpy()[:, :, :p.n]


def test_noalloc_back_to_back_layouts_move():
    """Consecutive calls whose workspace sections sit at different offsets of the shared array
    (the counter, CG states and partial sums move when nrhs, k or the CTA count change): a
    3-RHS k = 8 lattice, then a 1-RHS k = 3 lattice, then a 2-RHS sphere, then the first again;
    each against the oracle's direct solve."""
    cases = [("lattice", 9, 13, 8, 12, 3), ("lattice", 40, 40, 3, 5, 1),
             ("sphere", 24, 48, 6, 9, 2), ("lattice", 9, 13, 8, 12, 3)]
    for t, (kind, H, W, k, m, nrhs) in enumerate(cases):
        p = small_problem(kind, H, W, k, m, seed=700 + k, nrhs=nrhs)
        ld = p.n + 3 * t
        op = operator_for(p, ld=ld)
        Xo, b = oracle_solution(p)
        Xn = _noalloc(op, p, device_batch(b, ld), nrhs, k, ld, 1e-11, 1)
        assert relerr(Xn, Xo) <= 1e-6, (t, kind, relerr(Xn, Xo))
        op.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_intrinsic_gmrf_prior(precision):
    """A handle built with the intrinsic GMRF prior (App. C: L^2 formed on the device, 12
    off-diagonals per row) and the printed App. B mixing, against the oracle's direct solve."""
    g = synth.latlong_sphere(12, 20)
    rng = np.random.default_rng(41)
    A = synth.PLANCK_A_PRINTED
    nu_pix = np.exp(0.3 * rng.standard_normal(g.n))
    D = (synth.PLANCK_T_PRINTED * 1e-6)[:, None] * nu_pix[None, :]
    X = rng.standard_normal((4, g.n))
    Y = A @ X + rng.standard_normal((9, g.n)) / np.sqrt(D)
    p = synth.Problem("paper_sphere12x20", g, 4, 9, np.array([2.0, 0.5, 1.0, 3.0]),
                      np.zeros(4), synth.PLANCK_NU, np.zeros(4), D, Y[None], X, 1e-8, {},
                      A=A.copy(), prior="igmrf")
    ld = p.n + 1
    op = operator_for(p, ld=ld)
    Xo, b = oracle_solution(p)
    tol = 1e-10 if precision == 1 else 1e-12
    for call in range(2):
        Xn = _noalloc(op, p, device_batch(b, ld), 1, 4, ld, tol, precision)
        assert relerr(Xn, Xo) <= (1e-6 if precision == 1 else 1e-8), (call, relerr(Xn, Xo))
    op.close()
