"""Helpers shared by the GPU tests: upload seeded problems, run the oracle on the same inputs."""

import numpy as np

import synth
from oracle import model, solve


def device_batch(arr, ld, device="cuda"):
    """(R, rows, n) or (rows, n) numpy -> (R, rows, ld) float64 CUDA tensor (zero padded)."""
    import torch
    a = np.asarray(arr, np.float64)
    if a.ndim == 2:
        a = a[None]
    out = torch.zeros((a.shape[0], a.shape[1], ld), dtype=torch.float64, device=device)
    out[:, :, :a.shape[2]] = torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return out


def operator_for(p, ld=None, A=None, use_powerlaw=True):
    from paper_2204_08057_gb300.operator import Operator
    A = p.A if A is None else A
    return Operator(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=p.D, tau=p.tau,
                    kappa=p.kappa, nu=p.nu if A is None else None,
                    beta=p.beta if A is None else None, A=A, ld=ld, prior=p.prior)


def oracle_L(p):
    """The prior shape the problem's operator uses: L, or L^T L for the intrinsic GMRF."""
    L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
    return model.igmrf_base(L) if p.prior == "igmrf" else L


def oracle_A(p):
    return model.powerlaw_mixing(p.nu, p.beta) if p.A is None else p.A


def oracle_solution(p, A=None):
    L = oracle_L(p)
    A = oracle_A(p) if A is None else A
    G = model.assemble_G(L, p.D, p.tau, p.kappa, A)
    b = np.stack([model.rhs(p.D, y, A) for y in p.Yobs])
    return solve.solve_direct(G, b), b


def relerr(X, Xref):
    return float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))


def small_problem(kind, H, W, k, m, seed, noise="lognormal", nrhs=1, tau=None):
    g = synth.periodic_lattice(H, W) if kind == "lattice" else synth.latlong_sphere(H, W)
    nu = synth.PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]
    tau = tau if tau is not None else np.linspace(0.6, 1.4, k)
    return synth.make_problem(f"{kind}{H}x{W}_k{k}_m{m}", g, k, nu, None, None, tau, seed,
                              beta_draw=(-3, 2), kappa_draw=(0.02, 1.0), noise=noise,
                              nrhs=nrhs)
