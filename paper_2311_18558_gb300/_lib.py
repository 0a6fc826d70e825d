"""ctypes declarations of librt103 (include/rt103.h).  Loading fails loudly if the
library has not been built: there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librt103.so")

_lib = None
_lock = threading.Lock()

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F32 = ctypes.c_float
F64 = ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); mirrors include/rt103.h
SIGNATURES = {
    "rt_create": (I32, [ctypes.c_int, P, PP]),
    "rt_destroy": (I32, [P]),
    "rt_set_stream": (I32, [P, P]),
    "rt_last_error": (ctypes.c_char_p, [P]),
    "rt_status_word": (I32, [P, ctypes.POINTER(I32)]),
    "rt_version": (ctypes.c_char_p, []),
    "rt_set_profiling": (I32, [P, I32]),
    "rt_profile_read": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(F64), ctypes.POINTER(I64)]),
    "rt_scene_upload": (I32, [P, P, I32, P, I32, P, I32, P, PP]),
    "rt_scene_free": (I32, [P]),
    "rt_scene_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(F64)]),
    "rt_trace_paths": (I32, [P, P, P, P, I32, I64, I32, PP]),
    "rt_paths_import": (I32, [P, P, I64, I32, I32, P, P, P, P, PP]),
    "rt_paths_count": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "rt_paths_rx_offsets": (I32, [P, P]),
    "rt_paths_export": (I32, [P, P, P, P, P, P]),
    "rt_paths_candidates": (I32, [P, P]),
    "rt_paths_device_views": (I32, [P, PP, PP]),
    "rt_paths_free": (I32, [P]),
    "rt_trace_batch": (I32, [P, P, I32, P, P, P, I64, I32, PP]),
    "rt_paths_batch_info": (I32, [P, ctypes.POINTER(I32), P, P]),
    "rt_set_tuning": (I32, [P, I32, I32, I32]),
    "rt_set_cfr_tensor_cores": (I32, [P, I32]),
    "rt_set_wait_limit": (I32, [P, I32]),
    "rt_set_trace_async": (I32, [P, I32]),
    "rt_paths_resolve": (I32, [P]),
    "rt_trace_diffuse": (I32, [P, P, P, P, I32, I64, I32, PP]),
    "rt_eval_fields_diffuse": (I32, [P, P, P, P, P, F64, F32, F32, P, P]),
    "rt_eval_fields_diffuse_backward": (I32, [P, P, P, P, P, F64, F32, F32, P, P, P, P]),
    "rt_set_diffuse_phases": (I32, [P, P, P]),
    "rt_specular_reduction": (I32, [P, P, P, P, P]),
    "rt_specular_reduction_backward": (I32, [P, P, P, P, P, P, P]),
    "rt_scene_wedges": (I32, [P, P, ctypes.POINTER(I32), P, P]),
    "rt_trace_diffraction": (I32, [P, P, P, P, P, I32, PP]),
    "rt_eval_fields_diffraction": (I32, [P, P, P, P, I32, F64, F32, F32, P, P]),
    "rt_eval_fields_diffraction_backward": (I32, [P, P, P, P, I32, F64, F32, F32, P, P, P, P]),
    "rt_rx_merge": (I32, [P, I32, P, P, P, P, P, P]),
    "rt_rx_split": (I32, [P, I32, P, P, P, P, P]),
    "rt_antenna_apply": (I32, [P, P, P, I32, P, I32, P, P, P, P]),
    "rt_antenna_apply_backward": (I32, [P, P, P, I32, P, I32, P, P, P, P, P, P, P]),
    "rt_cir": (I32, [P, P, I32, I32, P]),
    "rt_cir_stats": (I32, [P, P, I32, I32, F64, P, P]),
    "rt_power_scale_ema": (I32, [P, P, P, I32, F32, P]),
    "rt_delay_spread_power_loss": (I32, [P, P, I32, I32, F64, P, P, P, P, P, P, P]),
    "rt_cir_metrics": (I32, [P, P, P, P, P, I32, P, P, P]),
    "rt_autotune_trace": (I32, [P, P, P, P, I32, I64, I32, P, ctypes.POINTER(F64)]),
    "rt_eval_fields": (I32, [P, P, P, P, I32, F64, F32, F32, P, P]),
    "rt_eval_fields_backward": (I32, [P, P, P, P, I32, F64, F32, F32, P, P, P, P]),
    "rt_cfr": (I32, [P, P, I32, P, P, F64, F64, I32, P]),
    "rt_cfr_backward": (I32, [P, P, I32, P, F64, F64, I32, P, P]),
    "rt_cfr_power_mse_fused": (I32, [P, P, I32, P, P, F64, F64, I32, P, P, P, P, P]),
    "rt_cfr_power_mse_fused_noalloc": (I32, [P, P, I32, P, P, F64, F64, I32, P, P, P, P, P]),
    "rt_mlp_forward": (I32, [P, P, P, P, P, P, P]),
    "rt_mlp_backward": (I32, [P, P, P, P, P, P, P, P, P, P, P]),
}

STATUS = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_CUDA", 3: "RT_ERR_OOM", 4: "RT_ERR_CAPACITY",
          5: "RT_ERR_STACK_OVERFLOW", 6: "RT_ERR_ITER_LIMIT", 7: "RT_ERR_TIMEOUT", 8: "RT_ERR_NUMERIC",
          9: "RT_ERR_UNSUPPORTED"}


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load() -> ctypes.CDLL:
    """Load librt103.so (built by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librt103.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
