"""Seeded synthetic inputs for the posterior-mean system of the CMB source-separation model.

This module is shared by the CPU oracle (``oracle/``), the tests and ``bench.py``.  It holds
input synthesis only: pixel graphs and their Laplacian in CSR form (the neighbour structure a
user of the solver supplies, Sec. 2.2 / App. C), noise-precision maps, spectral parameters and
simulated observations, and the mixing matrix and channel weights App. B prints (input data as
printed).  It computes no part of the solve: no mixing matrix derived from a model, no
right-hand side, no operator application.
"""

from .grids import (  # noqa: F401
    GridGraph,
    periodic_lattice,
    latlong_sphere,
    laplacian_csr_from_edges,
)
from .physical import PLANCK_A_PRINTED, PLANCK_T_PRINTED  # noqa: F401
from .order import (  # noqa: F401
    blocked_order,
    permute_graph,
    permute_problem,
    outside_tile_fraction,
)
from .problems import (  # noqa: F401
    PLANCK_NU,
    Problem,
    make_problem,
    config_problem,
    batch_problems,
    batch_shapes,
    colouring_probes,
    grid_colouring,
    separable_problem,
    igmrf_problem,
    rademacher_probes,
    CONFIG_SEED_BASE,
)
