"""GB300 (sm_103a) implementation of MUSTER's registration loop (arXiv 2412.14671).

The CUDA library ``libmuster.so`` (C ABI in ``include/muster.h`` and
``include/muster_ops.h``) does all the work; this package is its binding.
"""
from ._native import (  # noqa: F401
    ADAM,
    GRADIENT,
    IMAGE,
    JACOBIAN,
    LNCC,
    PAIR_DISP,
    PAIR_FLOW,
    PARAMETERS,
    SGD,
    SILNCC,
    VELOCITY,
    WARPED,
    MusterError,
)
from .api import (  # noqa: F401
    Muster,
    MusterLoss,
    default_params,
    footprint,
    op_deformation_metrics,
    op_downsample,
    op_exp,
    op_jacobian_det,
    op_similarity,
)
