"""GB300 (sm_103a) implementation of the data-parallel hot path of differentiable
radio ray tracing (Hoydis et al., arXiv 2311.18558): specular path tracing,
per-path field computation, CFR synthesis, their adjoints, behind the C ABI of
include/rt103.h.  The Python layer only marshals arguments."""
from ._lib import LIB_PATH, RtError, load  # noqa: F401
from .api import (Context, Paths, Scene, cfr, cfr_backward, cfr_power_mse_fused, eval_fields,  # noqa: F401
                  eval_fields_backward, import_paths, trace_paths)
from .autograd import Cfr, CfrPowerMSE, EvalFields, LogMaterials, calibration_loss  # noqa: F401
