"""GPU parity of the posterior variances (sylv_variance: diag(G^{-1}) of eq. Q* by the probe
estimator of Bekas, Kokiopoulou and Saad), through the C ABI.

Unit-vector probes give the exact diagonal (compared with the oracle's exact diag(G^{-1}));
Rademacher probes are compared with the oracle's estimator on the same probes, including a
ragged last chunk of probes; on a 128 x 128 lattice with homogeneous noise the pixel average of
the estimate is compared with the closed form.
"""

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_A, oracle_L
from oracle import model, variance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08057_gb300 import build
    build.build()


def _problem(kind, H, W, k, m, seed, noise="lognormal"):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    return synth.make_problem("var", g, k, nu, None, None, np.linspace(0.7, 1.5, k), seed,
                              beta_draw=(-3, 2), kappa_draw=(0.05, 1.0), noise=noise)


def _G(p):
    return model.assemble_G(oracle_L(p), p.D, p.tau, p.kappa, oracle_A(p))


@pytest.mark.parametrize("precision", [0, 1])
def test_unit_probes_give_the_exact_diagonal(precision):
    p = _problem("sphere", 4, 6, 3, 5, seed=2)
    N = p.k * p.n
    Z = np.eye(N).reshape(N, p.k, p.n)
    op = operator_for(p)
    var, info = op.variance(device_batch(Z, op.ld), tol=1e-12 if precision == 0 else 1e-10,
                            precision=precision)
    assert info["code"] == 0
    ex = variance.exact_diag(_G(p), p.k, p.n)
    err = np.abs(var.cpu().numpy()[:, :p.n] - ex).max() / ex.max()
    assert err <= (1e-9 if precision == 0 else 1e-6)
    op.close()


def test_rademacher_probes_match_the_oracle_estimator():
    p = _problem("lattice", 12, 14, 4, 6, seed=6)
    Z = synth.rademacher_probes(40, p.k, p.n, seed=11)      # 16 + 16 + 8
    op = operator_for(p)
    var, info = op.variance(device_batch(Z, op.ld), tol=1e-12, precision=0)
    assert info["code"] == 0
    ref = variance.probe_diag(_G(p), Z)
    assert np.abs(var.cpu().numpy()[:, :p.n] - ref).max() <= 1e-9 * np.abs(ref).max()
    # zero probes leave zero
    var0, _ = op.variance(device_batch(np.zeros((2, p.k, p.n)), op.ld))
    assert float(var0.abs().max()) == 0.0
    op.close()


def test_lattice_average_matches_closed_form():
    H = W = 128
    p = _problem("lattice", H, W, 3, 5, seed=9, noise="homogeneous")
    Z = synth.rademacher_probes(64, p.k, p.n, seed=12)
    op = operator_for(p)
    var, info = op.variance(device_batch(Z, op.ld), tol=1e-8)
    assert info["code"] == 0
    cf = variance.lattice_homogeneous_diag(H, W, p.tau, p.kappa, oracle_A(p), p.D[:, 0])
    avg = var.cpu().numpy()[:, :p.n].mean(axis=1)
    assert np.abs(avg - cf).max() <= 0.02 * cf.max()
    op.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_colouring_probes_match_exact_diagonal_within_the_coupling_bound(precision):
    """sylv_variance_probing (probes generated on the device from a distance colouring) against
    the exact diagonal of a dense inverse: at every (source, pixel) the error lies within the
    sum of the magnitudes of the G^{-1} entries between same-colour pixels (the estimator's
    value is the diagonal plus those entries), it equals the oracle's estimator on the same
    probes, and the largest error falls as the colouring distance grows."""
    p = _problem("sphere", 12, 24, 4, 6, seed=21)
    op = operator_for(p)
    G = _G(p)
    Ginv = np.linalg.inv(G.toarray())
    exact = np.diag(Ginv).reshape(p.k, p.n)
    slack = 1e-9 if precision == 0 else 1e-5            # solve tolerance
    errs = []
    for pc in (1, 2, 3, 4):
        col = synth.grid_colouring(p.graph, pc)
        var, info = op.variance_probing(col, pc * pc, tol=1e-11, precision=precision)
        assert info["code"] == 0, info
        est = var.cpu().numpy()[:, :p.n]
        bound = np.empty_like(exact)
        for j in range(p.k):
            blk = np.abs(Ginv[j * p.n:(j + 1) * p.n, j * p.n:(j + 1) * p.n])
            for i in range(p.n):
                same = col == col[i]
                bound[j, i] = blk[i, same].sum() - blk[i, i]
        assert np.all(np.abs(est - exact) <= bound + slack * exact), pc
        ref = variance.probe_diag(G, synth.colouring_probes(p.graph, p.k, pc))
        assert np.abs(est - ref).max() <= slack * np.abs(ref).max(), pc
        errs.append(np.abs(est - exact).max() / exact.max())
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    op.close()


def test_colouring_out_of_range_is_refused():
    import torch
    from paper_2204_08057_gb300 import binding as Bn
    p = _problem("sphere", 8, 12, 3, 5, seed=2)
    op = operator_for(p)
    col = synth.grid_colouring(p.graph, 2)
    col[5] = 4                                            # outside [0, 4)
    with pytest.raises(Bn.SylvError) as e:
        op.variance_probing(col, 4, tol=1e-10)
    assert e.value.code == Bn.SYLV_E_INVALID
    op.close()
