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
