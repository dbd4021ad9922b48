"""GB300 solver for the posterior-mean system of the CMB source-separation model
(arxiv 2204.08057): matrix-free operator, fused preconditioned CG, FP32/FP64 iterative
refinement, batched and multi-right-hand-side solves and an adjoint gradient, all in the CUDA
library ``_build/libsylv.so`` behind the C ABI ``include/sylv.h``.

``binding`` mirrors the C entry points by name; ``Operator`` is a tensor-level wrapper and
``SylvSolve`` a torch.autograd.Function.  Import does not load the library; the first call
does, and fails if it has not been built.
"""

from . import binding  # noqa: F401
from .binding import SylvError, load, make_opts, sylv_opts_default  # noqa: F401


def __getattr__(name):
    if name in ("Operator", "solve_batched"):
        from . import operator as _op
        return getattr(_op, name)
    if name in ("SylvSolve", "SylvProblem", "sylv_solve_differentiable"):
        from . import autograd as _ag
        return getattr(_ag, name)
    raise AttributeError(name)
