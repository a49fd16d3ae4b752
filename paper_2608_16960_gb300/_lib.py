"""ctypes loader for libtsp.so (the C ABI of include/tsp.h).

The product path has no fallback: if the CUDA library is missing or fails to
load, every call raises. Symbols keep their C names.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import nvbuild as _build

_lock = threading.Lock()
_lib = None

TSP_OK = 0
TSP_SIRT_NONNEG = 1
TSP_SIRT_REUSE_WEIGHTS = 2
STATUS_NAMES = {0: "TSP_OK", 1: "TSP_EINVAL", 2: "TSP_ENOTMONO", 3: "TSP_ENOMEM", 4: "TSP_ECUDA",
                5: "TSP_ETIMEOUT", 6: "TSP_EDEVICE", 7: "TSP_ENOTSUP"}


class TspError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class tsp_batch_item(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("geom", ctypes.c_void_p), ("y", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class tsp_launch(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("warp_tile_w", ctypes.c_int), ("scatter", ctypes.c_int)]


# (name, restype, argtypes) for every symbol declared in include/tsp.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_I64P = ctypes.POINTER(ctypes.c_int64)
_LP = ctypes.POINTER(tsp_launch)
SIGNATURES = {
    "tsp_grid_create": (_I, [_DP, _I, _DP, _I, _DP, _I, ctypes.POINTER(_P)]),
    "tsp_grid_shape": (_I, [_P, _IP, _IP, _IP]),
    "tsp_grid_destroy": (None, [_P]),
    "tsp_geom_cone": (_I, [_I, _DP, _DP, _DP, _I, _I, _D, _D, ctypes.POINTER(_P)]),
    "tsp_geom_parallel": (_I, [_I, _DP, _DP, _I, _I, _D, _D, ctypes.POINTER(_P)]),
    "tsp_geom_rays": (_I, [_I64, _P, _P, _I, ctypes.POINTER(_P)]),
    "tsp_geom_num_rays": (_I, [_P, _I64P]),
    "tsp_geom_destroy": (None, [_P]),
    "tsp_forward": (_I, [_P, _P, _P, _P, _I, _P]),
    "tsp_forward_ex": (_I, [_P, _P, _P, _P, _I, _LP, _P]),
    "tsp_adjoint": (_I, [_P, _P, _P, _P, _I, _I, _P]),
    "tsp_adjoint_ex": (_I, [_P, _P, _P, _P, _I, _I, _LP, _P]),
    "tsp_count_segments": (_I, [_P, _P, _P, _P]),
    "tsp_segments_build": (_I, [_P, _P, _I, ctypes.POINTER(_P), _P]),
    "tsp_segments_info": (_I, [_P, _I64P, _I64P, ctypes.POINTER(ctypes.c_size_t)]),
    "tsp_segments_export": (_I, [_P, _P, _P, _P]),
    "tsp_segments_export_transposed": (_I, [_P, _P, _P, _P]),
    "tsp_segments_sirt_weights": (_I, [_P, _P, _P, _P]),
    "tsp_debug_fail_allocation": (_I, [_I64]),
    "tsp_debug_allocation_count": (_I, [_I64P]),
    "tsp_debug_tc_stall": (_I, [_I64]),
    "tsp_segments_forward": (_I, [_P, _P, _P, _I, _P]),
    "tsp_segments_adjoint": (_I, [_P, _P, _P, _I, _I, _P]),
    "tsp_segments_sirt_workspace_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "tsp_segments_sirt": (_I, [_P, _P, _P, _I, _I, _P, ctypes.c_size_t, _P]),
    "tsp_segments_destroy": (None, [_P]),
    "tsp_sirt_workspace_bytes": (_I, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "tsp_sirt": (_I, [_P, _P, _P, _P, _I, _I, _P, ctypes.c_size_t, _LP, _P]),
    "tsp_sirt_noalloc": (_I, [_P, _P, _P, _P, _I, _I, _P]),
    "tsp_autotune": (_I, [_P, _P, _LP, _LP, _P]),
    "tsp_autotune_lookup": (_I, [_P, _P, _LP, _LP]),
    "tsp_autotune_clear": (None, []),
    "tsp_autotune_store": (_I, [_P, _P, _LP, _LP]),
    "tsp_batch_create": (_I, [ctypes.POINTER(tsp_batch_item), _I, ctypes.POINTER(_P)]),
    "tsp_batch_workspace_bytes": (_I, [_P, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "tsp_batch_sirt": (_I, [_P, _I, _I, _P, ctypes.c_size_t, _P]),
    "tsp_batch_sirt_capture": (_I, [_P, _I, _I, _P, ctypes.c_size_t]),
    "tsp_batch_sirt_launch": (_I, [_P, _P]),
    "tsp_batch_info": (_I, [_P, _I64P, _I64P, _IP]),
    "tsp_batch_destroy": (None, [_P]),
    "tsp_shbs_create": (_I, [_I, _I, _DP, _I, _DP, _I, _DP, _I, _D, _D, ctypes.POINTER(_P)]),
    "tsp_shbs_tables": (_I, [_P, _P, _P]),
    "tsp_shbs_render": (_I, [_P, _P, _P, _P]),
    "tsp_shbs_render_adjoint": (_I, [_P, _P, _P, _P]),
    "tsp_shbs_destroy": (None, [_P]),
    "tsp_adam": (_I, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, _I, _P]),
    "tsp_sq_residual": (_I, [_P, _P, _I64, _P, _P, _P]),
    "tsp_geom_polar": (_I, [_I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), _I, _I, ctypes.c_double, ctypes.POINTER(_P)]),
    "tsp_shbs_create_shells": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(ctypes.c_double), _I,
                                    ctypes.POINTER(_P)]),
    "tsp_tikhonov_radial": (_I, [_P, _I, _I, ctypes.c_float, _P, _P, _P]),
    "tsp_sq_residual_weighted": (_I, [_P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "tsp_vec_dot": (_I, [_P, _P, ctypes.c_int64, _P, _P]),
    "tsp_vec_axpby": (_I, [ctypes.c_float, _P, ctypes.c_float, _P, ctypes.c_int64, _P]),
    "tsp_vec_mul": (_I, [_P, _P, _P, ctypes.c_int64, _P]),
    "tsp_sirt_chunked": (_I, [_P, _I, _I, _I, ctypes.c_size_t, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t), _P]),
    "tsp_forward_dynamic": (_I, [_P, _P, _P, _P, _P]),
    "tsp_adjoint_dynamic": (_I, [_P, _P, _P, _P, _I, _P]),
    "tsp_sunward_rays": (_I, [_P, ctypes.POINTER(ctypes.c_double), _P, _P, _P]),
    "tsp_atten_optical_depth": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "tsp_atten_optical_depth_adjoint": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _I, _P]),
    "tsp_atten_forward": (_I, [_P, _P, _P, _P, _P, _P, _I, _P]),
    "tsp_atten_backward": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P]),
    "tsp_net_create": (_I, [_I, _I, _I, _I, ctypes.POINTER(_P)]),
    "tsp_net_destroy": (None, [_P]),
    "tsp_net_num_params": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "tsp_net_set_params": (_I, [_P, _P, ctypes.c_size_t]),
    "tsp_net_get_params": (_I, [_P, _P, ctypes.c_size_t]),
    "tsp_net_get_grads": (_I, [_P, _P, ctypes.c_size_t]),
    "tsp_net_get_state": (_I, [_P, _P, _P, _P, ctypes.c_size_t, _IP]),
    "tsp_net_set_state": (_I, [_P, _P, _P, _P, ctypes.c_size_t, _I]),
    "tsp_net_forward": (_I, [_P, _P, _I, _P, _P]),
    "tsp_net_loss_grad": (_I, [_P, _P, _P, _I, ctypes.POINTER(ctypes.c_double), _P]),
    "tsp_net_adam": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "tsp_net_activation": (_I, [_P, _I, _I, _P]),
    "tsp_sirt_weights": (_I, [_P, _P, _P, _P, _P]),
    "tsp_phantoms": (_I, [_P, _P, _I, _I, _P, _P]),
    "tsp_batch_max": (_I, [_P, _I64, _I, _P, _P]),
    "tsp_add_noise": (_I, [_P, _I64, _I, _P, ctypes.c_float, _P, _P]),
    "tsp_mul_bcast": (_I, [_P, _P, _I64, _I, _P]),
    "tsp_scale_batch": (_I, [_P, _P, _I64, _I, _I, _P]),
    "tsp_device_status": (_I, [_P, _IP]),
    "tsp_last_error": (ctypes.c_char_p, []),
    "tsp_version": (_I, []),
}


def extra_signatures():
    """Signatures of the entry points declared beyond the projector core
    (reconstruction, batching, training); merged in by their modules."""
    return _EXTRA


_EXTRA: dict = {}


def register(sigs: dict):
    _EXTRA.update(sigs)
    if _lib is not None:
        _apply(_lib, sigs)


def _apply(L, sigs):
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def so_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libtsp.so (building it first if asked and absent). Raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.SO
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            _apply(L, SIGNATURES)
            _apply(L, _EXTRA)
            _lib = L
    return _lib


def check(status: int, what: str = ""):
    if status != TSP_OK:
        msg = load().tsp_last_error().decode(errors="replace")
        raise TspError(status, f"{what}: {msg}" if what else msg)
