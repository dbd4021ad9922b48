"""sylv_solve_noalloc, the allocation-free solve, against sylv_solve (GPU).

The entry point serves callers that cannot allocate device memory when they solve (a
pipeline with memory reserved at start-up, a fixed memory budget, or a loop that must avoid
an allocator's synchronisation); its workspace is a fixed device array inside the library.
This file is collected last so that a run stopping at its first failure has run every other
test; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

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
