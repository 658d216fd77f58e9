"""GB300 library for entropic optimal transport by the truncated Newton method of
Kemertas, Farahmand and Jepson (ICLR 2025, arXiv 2504.02067).

The compute path is libeot.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/eot.h); this package only builds it and marshals arguments.
"""
from .binding import (COST_DENSE_F32, COST_DENSE_F64, COST_SQEUCLID_POINTS, PRECISIONS,  # noqa: F401
                      EotError, EotParams, EotProblem, EotStats, Handle, Problem,
                      PROJECT_NEWTON, PROJECT_SINKHORN, NEWTON_REDUCED, NEWTON_FULL, default_params, load_library,
                      solve_batched)
from .buildlib import build  # noqa: F401


def __getattr__(name):
    # the autograd layer imports torch's autograd machinery; load it on first use
    if name in ("EOTFunction", "eot_value"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
