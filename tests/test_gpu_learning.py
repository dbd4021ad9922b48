"""GPU parity of the parameter-learning path (Sec. 5: repeated solves across the prior and
mixing parameters), through the C ABI: sylv_set_params against a fresh handle, warm starts, the
learning driver's trajectory against the oracle's loop, and invalid updates."""

import numpy as np
import pytest

import synth
from gpu_common import device_batch, operator_for, oracle_L, oracle_solution, relerr
from oracle import learning

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08057_gb300 import build
    build.build()


def _problem():
    g = synth.latlong_sphere(12, 20)
    nu = synth.PLANCK_NU[[0, 2, 3, 5, 7, 8]]
    return synth.make_problem("learn", g, 3, nu, [-2.0, 0.5, 1.5], [0.2, 0.5, 1.0],
                              [1.0, 2.0, 0.5], 31, noise="lognormal")


def test_set_params_equals_a_fresh_handle():
    import torch
    p = _problem()
    op = operator_for(p)
    Y = device_batch(p.Yobs, op.ld)
    tau2, kappa2, beta2 = np.array([0.7, 1.3, 2.2]), np.array([0.4, 0.1, 0.6]), p.beta - 0.3
    op.solve(op.rhs(Y), tol=1e-12, precision=0)            # solve with the old parameters
    op.set_params(tau2, kappa2, beta=beta2)
    X, info = op.solve(op.rhs(Y), tol=1e-12, precision=0)
    q = synth.make_problem("learn2", p.graph, 3, p.nu, beta2, kappa2, tau2, 31, noise="lognormal")
    q.D, q.Yobs = p.D, p.Yobs
    Xd, _ = oracle_solution(q)
    assert info["code"] == 0 and relerr(X.cpu().numpy()[:, :, :p.n], Xd) <= 1e-9
    fresh = operator_for(q)
    Xf, _ = fresh.solve(fresh.rhs(Y), tol=1e-12, precision=0)
    assert float(torch.max(torch.abs(X - Xf))) <= 1e-12 * float(torch.max(torch.abs(Xf)))
    # invalid values are refused and leave the handle as it was
    from paper_2204_08057_gb300 import binding as B
    with pytest.raises(B.SylvError):
        op.set_params(np.array([1.0, -1.0, 1.0]), kappa2, beta=beta2)
    X2, _ = op.solve(op.rhs(Y), tol=1e-12, precision=0)
    assert float(torch.max(torch.abs(X2 - X))) <= 1e-12 * float(torch.max(torch.abs(X)))
    fresh.close()
    op.close()


def test_learning_trajectory_matches_oracle_and_warm_starts_save_iterations():
    import torch
    from paper_2204_08057_gb300.learn import HyperLearner
    p = _problem()
    op = operator_for(p)
    Y = device_batch(p.Yobs, op.ld)
    Xt = device_batch(p.X_true[None], op.ld)
    n = p.n

    def loss_grad_gpu(X):
        d = X - Xt
        d[:, :, n:] = 0.0
        return float(torch.sum(d * d)), 2.0 * d

    def loss_grad_cpu(X):
        d = X - p.X_true
        return float(np.sum(d * d)), 2.0 * d

    tau0, kappa0, beta0 = [0.5, 3.0, 2.0], [0.5, 0.2, 0.3], p.beta + 0.2
    lr = 2e-4                     # the loss decreases at this rate (oracle: 171 -> 68)
    ref = learning.learn(oracle_L(p), p.D, p.nu, p.Yobs[0], loss_grad_cpu, tau0, kappa0, beta0,
                         steps=5, lr=lr)
    hl = HyperLearner(op, Y, loss_grad_gpu, tau0, kappa0, beta0, lr=lr, tol=1e-12, precision=0)
    recs = [hl.step() for _ in range(5)]
    for a, b in zip(recs, ref):
        assert abs(a["loss"] - b["loss"]) <= 1e-8 * abs(b["loss"])
        assert np.allclose(a["tau"], b["tau"], rtol=1e-8)
        assert np.allclose(a["kappa"], b["kappa"], rtol=1e-8)
        assert np.allclose(a["beta"], b["beta"], rtol=1e-8, atol=1e-10)
    # the same steps from cold starts take more iterations
    cold = HyperLearner(op, Y, loss_grad_gpu, tau0, kappa0, beta0, lr=lr, warm=False, tol=1e-12,
                        precision=0)
    crec = [cold.step() for _ in range(5)]
    warm_its = sum(r["forward_iterations"] + r["adjoint_iterations"] for r in recs[1:])
    cold_its = sum(r["forward_iterations"] + r["adjoint_iterations"] for r in crec[1:])
    assert warm_its < cold_its
    op.close()


def test_lanczos_sees_new_parameters():
    p = synth.separable_problem(2, scale=32)
    op = operator_for(p)
    Y = device_batch(p.Yobs, op.ld)
    op.solve_sylvester(op.rhs(Y), tol=1e-10)
    tau2 = np.array([0.5, 1.0, 2.0, 0.7, 1.4, 3.0])
    op.set_params(tau2, p.kappa, beta=p.beta)
    X, info = op.solve_sylvester(op.rhs(Y), tol=1e-12, precision=0)
    q = synth.separable_problem(2, scale=32)
    q.tau = tau2
    Xd, _ = oracle_solution(q)
    assert info["code"] == 0 and relerr(X.cpu().numpy()[:, :, :p.n], Xd) <= 1e-8
    op.close()
