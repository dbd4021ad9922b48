"""Seeded problem instances shaped like the paper's workloads (Sec. 2, Sec. 4, App. B).

An instance carries only inputs: the pixel graph (Laplacian in CSR), per-channel per-pixel
noise precision maps d_{c,i} > 0, prior hyperparameters tau_j, kappa_j, channel frequencies
nu_c and spectral indices beta_j, and simulated observed maps ``Yobs`` (R x m x n).  The solver
side (CUDA library or oracle) derives the mixing matrix, the right-hand side and the operator
from these itself.

Observations are simulated from the linear mixing model (eq. model) with a sky that is
deliberately a little richer than the solver's model: smooth source maps s_j, each mixed with a
power-law spectrum whose index varies smoothly over the sky (beta_j + delta_beta_j(pixel)),
plus white noise of precision d_{c,i}.  Source maps come from spectrally filtered white noise.

Random draws use numpy ``Generator(PCG64(seed))`` in this fixed order:
beta, kappa (only where drawn), noise maps D, source maps, spectral-index fluctuations,
observation noise, further right-hand-side perturbations.
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .grids import GridGraph, latlong_sphere, periodic_lattice

CONFIG_SEED_BASE = 2204080570
PLANCK_NU = np.array([30.0, 44.0, 70.0, 100.0, 143.0, 217.0, 353.0, 545.0, 857.0])


@dataclass
class Problem:
    name: str
    graph: GridGraph
    k: int
    m: int
    tau: np.ndarray          # (k,)
    kappa: np.ndarray        # (k,)
    nu: np.ndarray           # (m,) GHz
    beta: np.ndarray         # (k,)
    D: np.ndarray            # (m, n) float64 noise precision maps
    Yobs: np.ndarray         # (R, m, n) float64 observed maps
    X_true: np.ndarray       # (k, n) float64 simulated source maps
    tol: float = 1e-8
    meta: dict = field(default_factory=dict)
    A: Optional[np.ndarray] = None   # (m, k) explicit mixing matrix (else the power law)
    prior: str = "gmrf"              # "gmrf": Q_j = tau_j (kappa_j^2 W + L); "igmrf": L^2 for L

    @property
    def n(self) -> int:
        return self.graph.n

    @property
    def nrhs(self) -> int:
        return self.Yobs.shape[0]


def _smooth_fields(rng, count, H, W, corr_len):
    """``count`` unit-variance smooth random maps on an H x W grid (filtered white noise)."""
    out = np.empty((count, H * W), dtype=np.float64)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f2 = fy * fy + fx * fx
    filt = 1.0 / (1.0 + f2 * (corr_len * 2 * np.pi) ** 2)
    for t in range(count):
        white = rng.standard_normal((H, W))
        f = np.fft.irfft2(np.fft.rfft2(white) * filt, s=(H, W))
        f -= f.mean()
        f /= max(f.std(), 1e-300)
        out[t] = f.ravel()
    return out


def _noise_maps(rng, m, graph, noise, sigma):
    n = graph.n
    if noise == "lognormal":        # per channel, per pixel
        z = rng.standard_normal((m, n))
    elif noise == "homogeneous":    # one value per channel
        z = np.repeat(rng.standard_normal((m, 1)), n, axis=1)
    elif noise == "latitude":       # per channel, per grid row
        z = np.repeat(rng.standard_normal((m, graph.H)), graph.W, axis=1)
    elif noise == "separable":      # d_ci = t_c * nu_i (the paper's C = T kron N)
        t = rng.standard_normal((m, 1))
        s = rng.standard_normal((1, n))
        z = t + s
    else:
        raise ValueError(noise)
    return np.exp(0.3 * z) / (np.asarray(sigma, dtype=np.float64)[:, None] ** 2)


def make_problem(name, graph: GridGraph, k, nu, beta, kappa, tau, seed, *, nrhs=1,
                 noise="lognormal", sigma=None, kappa_draw=None, beta_draw=None,
                 sky_amp=None, tol=1e-8, meta=None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    m = len(nu)
    nu = np.asarray(nu, dtype=np.float64)
    if beta_draw is not None:
        beta = rng.uniform(beta_draw[0], beta_draw[1], size=k)
    beta = np.asarray(beta, dtype=np.float64)
    if kappa_draw is not None:
        kappa = np.exp(np.linspace(np.log(kappa_draw[0]), np.log(kappa_draw[1]), k))
        kappa = kappa[rng.permutation(k)]
    kappa = np.asarray(kappa, dtype=np.float64)
    tau = np.broadcast_to(np.asarray(tau, dtype=np.float64), (k,)).copy()
    sigma = np.ones(m) if sigma is None else np.asarray(sigma, dtype=np.float64)
    D = _noise_maps(rng, m, graph, noise, sigma)
    H, W = graph.H, graph.W
    corr = max(2.0, min(H, W) / 16.0)
    S = _smooth_fields(rng, k, H, W, corr)
    amp = np.ones(k) if sky_amp is None else np.asarray(sky_amp, dtype=np.float64)
    S *= amp[:, None]
    dbeta = 0.05 * _smooth_fields(rng, k, H, W, 2 * corr)
    logf = np.log(nu / 100.0)
    sky = np.zeros((m, graph.n))
    for j in range(k):
        for c in range(m):
            sky[c] += np.exp((beta[j] + dbeta[j]) * logf[c]) * S[j]
    Yobs = np.empty((nrhs, m, graph.n))
    for r in range(nrhs):
        Yobs[r] = sky + rng.standard_normal((m, graph.n)) / np.sqrt(D)
    return Problem(name, graph, k, m, tau, kappa, nu, beta, D, Yobs, S, tol, dict(meta or {}))


def _grid(kind, H, W):
    return periodic_lattice(H, W) if kind == "lattice" else latlong_sphere(H, W)


def _nu_for(m):
    if m == 9:
        return PLANCK_NU.copy()
    return PLANCK_NU[np.round(np.linspace(0, 8, m)).astype(int)]


def config_problem(config_id: int, *, scale: Optional[int] = None, noise="lognormal",
                   nrhs: Optional[int] = None) -> Problem:
    """Workload ``config_id`` (1, 2, 4 or 5; 3 is ``batch_problems``).

    ``scale`` divides both grid sides (a scaled-down instance from the same recipe).
    """
    seed = CONFIG_SEED_BASE + config_id
    s = 1 if scale is None else int(scale)
    if config_id == 1:
        g = _grid("lattice", 64 // s, 64 // s)
        return make_problem("lattice64x64_k3_m5", g, 3, [30.0, 70.0, 100.0, 143.0, 217.0],
                            [0.0, -3.0, 1.5], [0.1, 0.3, 1.0], 1.0, seed, noise=noise,
                            nrhs=nrhs or 1, tol=1e-10, meta={"config": 1})
    if config_id == 2:
        g = _grid("sphere", 1024 // s, 2048 // s)
        return make_problem("sphere1024x2048_k6_m9", g, 6, PLANCK_NU, None, None, 1.0, seed,
                            beta_draw=(-3.0, 2.0), kappa_draw=(0.01, 1.0), noise=noise,
                            nrhs=nrhs or 1, tol=1e-8, meta={"config": 2})
    if config_id == 4:
        g = _grid("sphere", 512 // s, 1024 // s)
        return make_problem("sphere512x1024_k4_m7", g, 4, _nu_for(7), None, None, 1.0, seed,
                            beta_draw=(-3.0, 2.0), kappa_draw=(0.01, 1.0), noise=noise,
                            nrhs=nrhs or 1, tol=1e-8, meta={"config": 4})
    if config_id == 5:
        g = _grid("sphere", 4096 // s, 12288 // s)
        return make_problem("sphere4096x12288_k6_m9_r8", g, 6, PLANCK_NU, None, None, 1.0,
                            seed, beta_draw=(-3.0, 2.0), kappa_draw=(0.01, 1.0), noise=noise,
                            nrhs=nrhs or 8, tol=1e-8, meta={"config": 5})
    raise ValueError(f"unknown config {config_id}")


def separable_problem(config_id: int = 2, *, scale: Optional[int] = None, kappa0: float = 0.1,
                      nrhs: Optional[int] = None) -> Problem:
    """The separable special case of workload ``config_id`` (2, 4 or 5): the same grid,
    channels and spectral-index draw, noise precision d_ci = t_c nu_i (C = T kron N) and one
    prior shape for every source (all kappa_j = kappa0, the geometric middle of 0.01..1), so
    that the system is the Sylvester equation eq. Axb-Sylv."""
    sides = {2: (1024, 2048, 6, 9), 4: (512, 1024, 4, 7), 5: (4096, 12288, 6, 9)}
    if config_id not in sides:
        raise ValueError(f"no separable variant of config {config_id}")
    H, W, k, m = sides[config_id]
    s = 1 if scale is None else int(scale)
    g = _grid("sphere", H // s, W // s)
    return make_problem(f"sphere{H // s}x{W // s}_k{k}_m{m}_separable", g, k, _nu_for(m), None,
                        [kappa0] * k, 1.0, CONFIG_SEED_BASE + 20 + config_id,
                        beta_draw=(-3.0, 2.0), noise="separable",
                        nrhs=nrhs or (8 if config_id == 5 else 1), tol=1e-8,
                        meta={"config": config_id, "separable": True})


def igmrf_problem(config_id: int = 2, *, scale: Optional[int] = None, phi: float = 1e6,
                  kappa0: float = 0.0, nrhs: Optional[int] = None) -> Problem:
    """The paper's own model on the grid of workload ``config_id`` (2 or 4): the four physical
    sources (CMB, synchrotron, dust, free-free) with the mixing matrix and channel weights T
    printed in App. B over the nine Planck channels, noise precision d_ci = t_c nu_i with a
    log-normal per-pixel map nu (C = T kron N), and the intrinsic GMRF prior of App. C,
    Q_j = phi_j L^2 (kappa0 = 0; kappa0 > 0 adds kappa0^2 W).  The sky is the physical mixing of
    smooth source maps with amplitudes of order 1e-3 (the scale where T's weights and the prior
    phi ~ 1e6 are comparable), plus white noise of precision d_ci."""
    from .physical import PLANCK_A_PRINTED, PLANCK_T_PRINTED
    sides = {2: (1024, 2048), 4: (512, 1024)}
    if config_id not in sides:
        raise ValueError(f"no IGMRF variant of config {config_id}")
    H, W = sides[config_id]
    s = 1 if scale is None else int(scale)
    g = _grid("sphere", H // s, W // s)
    A = PLANCK_A_PRINTED.copy()
    m, k = A.shape
    R = nrhs or 1
    rng = np.random.Generator(np.random.PCG64(CONFIG_SEED_BASE + 40 + config_id))
    nu_pix = np.exp(0.3 * rng.standard_normal(g.n))
    D = PLANCK_T_PRINTED[:, None] * nu_pix[None, :]
    corr = max(2.0, min(g.H, g.W) / 16.0)
    S = 1e-3 * _smooth_fields(rng, k, g.H, g.W, corr)
    sky = A @ S
    Yobs = np.empty((R, m, g.n))
    for r in range(R):
        Yobs[r] = sky + rng.standard_normal((m, g.n)) / np.sqrt(D)
    return Problem(f"sphere{g.H}x{g.W}_k{k}_m{m}_igmrf_physical", g, k, m,
                   np.full(k, float(phi)), np.full(k, float(kappa0)), _nu_for(m), np.zeros(k),
                   D, Yobs, S, 1e-8, {"config": config_id, "igmrf": True}, A=A, prior="igmrf")


def rademacher_probes(count: int, k: int, n: int, seed: int) -> np.ndarray:
    """(count, k, n) probe vectors with independent +-1 entries (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 2, size=(count, k, n)).astype(np.float64) * 2.0 - 1.0


def _batch_draws(count, side_range, seed):
    seed = CONFIG_SEED_BASE + 3 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(side_range[0]), np.log(side_range[1])
    sides = np.round(np.exp(rng.uniform(lo, hi, size=count))).astype(int)
    ks = rng.integers(3, 7, size=count)
    sub = rng.integers(0, 2**62, size=count)
    return sides, ks, sub


def batch_shapes(count=64, side_range=(128, 1024), *, seed=None):
    """(side, k) of each system of ``batch_problems`` (same draws), without building them."""
    sides, ks, _ = _batch_draws(count, side_range, seed)
    return [(int(a), int(b)) for a, b in zip(sides, ks)]


def grid_colouring(graph: GridGraph, p: int) -> np.ndarray:
    """Colour of every pixel of a grid graph, (r mod p) * p + (c mod p): p^2 colours, and two
    distinct pixels of one colour are at least p steps apart on the grid (a distance-(p - 1)
    colouring).  A periodic side must be a multiple of p (longitude always; latitude too on
    the periodic lattice) so that the wrap-around keeps that property."""
    if p < 1:
        raise ValueError("p must be >= 1")
    if graph.W % p or (graph.kind == "lattice" and graph.H % p):
        raise ValueError(f"a periodic side of the {graph.kind} is not a multiple of p = {p}")
    r = np.repeat(np.arange(graph.H, dtype=np.int64), graph.W)
    c = np.tile(np.arange(graph.W, dtype=np.int64), graph.H)
    return ((r % p) * p + c % p).astype(np.int64)


def colouring_probes(graph: GridGraph, k: int, p: int) -> np.ndarray:
    """(p^2 k, k, n) probing vectors of a distance-(p - 1) colouring: probe (q, j) is 1 on the
    pixels of colour q in source j and 0 elsewhere, so every (source, pixel) entry is covered
    by exactly one probe."""
    col = grid_colouring(graph, p)
    Z = np.zeros((p * p * k, k, graph.n))
    for q in range(p * p):
        mask = col == q
        for j in range(k):
            Z[q * k + j, j, mask] = 1.0
    return Z


def batch_problems(count=64, side_range=(128, 1024), *, seed=None,
                   indices=None) -> List[Problem]:
    """Batched workload: ``count`` independent periodic lattices of log-uniform side, k in
    {3,4,5,6} uniform, m = k + 2, own kappa (log-spaced 0.01..1, permuted), beta and noise.
    ``indices``: build only these members (the same problems as in the whole batch)."""
    sides, ks, sub = _batch_draws(count, side_range, seed)
    out = []
    for b in (range(count) if indices is None else indices):
        k = int(ks[b])
        m = k + 2
        g = _grid("lattice", int(sides[b]), int(sides[b]))
        out.append(make_problem(f"batch{b}_lattice{sides[b]}_k{k}", g, k, _nu_for(m), None, None,
                                1.0, int(sub[b]), beta_draw=(-3.0, 2.0),
                                kappa_draw=(0.01, 1.0), tol=1e-8, meta={"config": 3, "index": b}))
    return out
