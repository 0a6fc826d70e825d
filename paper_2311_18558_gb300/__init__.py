"""GB300 (sm_103a) implementation of the data-parallel hot path of differentiable
radio ray tracing (Hoydis et al., arXiv 2311.18558): specular path tracing,
per-path field computation, CFR synthesis, their adjoints, and the trainable
extensions (the paper's loss, antenna and scattering patterns, diffuse
reflection, first-order diffraction, material embeddings), behind the C ABI of include/rt103.h.  The Python layer only marshals arguments."""
from ._lib import LIB_PATH, RtError, load  # noqa: F401
from .api import (MLP_NB, MLP_NW, Context, Paths, Scene, antenna_apply, antenna_apply_backward,  # noqa: F401
                  autotune_trace, cfr, cfr_backward, cfr_power_mse_fused, cir, cir_metrics, cir_stats,
                  delay_spread_power_loss, eval_fields, eval_fields_backward, eval_fields_diffraction,
                  eval_fields_diffraction_backward, eval_fields_diffuse, eval_fields_diffuse_backward,
                  import_paths, mlp_backward, mlp_forward, pack_mlp, power_scale_ema, rx_merge, rx_split,
                  scene_wedges, set_cfr_tensor_cores, set_diffuse_phases, set_trace_async, set_tuning, set_wait_limit,
                  specular_reduction, specular_reduction_backward, trace_batch, trace_diffraction,
                  trace_diffuse, trace_paths)
from .autograd import (AntennaApply, AntennaPattern, Cfr, CfrPowerMSE, DelaySpreadPowerLoss,  # noqa: F401
                       EvalFields, EvalFieldsDiffraction, EvalFieldsDiffuse, LogMaterials, MaterialEmbeddings,
                       NeuralMaterials, NeuralMaterialsFn, RxMerge, ScatteringPattern, SpecularReduction,
                       calibration_loss, pack_scattering, paper_calibration_loss)
