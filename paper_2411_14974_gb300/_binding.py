"""ctypes declarations of the C ABI in include/convex_splat.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from .build import LIB


class CsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("z_near", ctypes.c_float)]


class CsSettings(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("dist_mode", ctypes.c_int32), ("dist_power", ctypes.c_float),
                ("tile_test", ctypes.c_int32), ("tile_split", ctypes.c_int32)]


class CsScene(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("delta", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("k", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("activation", ctypes.c_int32),
                ("storage", ctypes.c_int32)]


class CsAdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("grad_abs_sum", ctypes.c_void_p), ("n", ctypes.c_int64), ("lr", ctypes.c_float)]


class CsAdamSettings(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("zero_grad", ctypes.c_int32)]


class CsParamArrays(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("delta", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class CsRefineSettings(ctypes.Structure):
    _fields_ = [("split_threshold", ctypes.c_float), ("split_scale", ctypes.c_float),
                ("split_sigma_scale", ctypes.c_float), ("split_opacity_scale", ctypes.c_float),
                ("prune_opacity", ctypes.c_float), ("prune_size", ctypes.c_float)]


class CsCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


# every entry point declared in include/convex_splat.h, with (restype, argtypes)
_P = ctypes.c_void_p
_PROTOTYPES = {
    "cs_default_settings": (None, [ctypes.POINTER(CsSettings)]),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_context_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P)]),
    "cs_context_destroy": (None, [_P]),
    "cs_forward": (ctypes.c_int, [_P, ctypes.POINTER(CsScene), ctypes.POINTER(CsCamera), ctypes.c_int32,
                                  ctypes.POINTER(CsSettings), _P, _P, ctypes.POINTER(_P), _P]),
    "cs_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cs_backward_write": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cs_state_release": (None, [_P]),
    "cs_state_copy": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_state_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "cs_step_host": (ctypes.c_int, [_P, ctypes.POINTER(CsScene), ctypes.POINTER(CsCamera), ctypes.c_int32,
                                    ctypes.POINTER(CsSettings), _P, _P, _P, _P, _P, _P, _P, _P]),
    "cs_step_host_submit": (ctypes.c_int, [_P, ctypes.POINTER(CsScene), ctypes.POINTER(CsCamera),
                                           ctypes.POINTER(CsSettings), _P, _P, _P, _P, _P, _P, _P,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "cs_step_host_wait": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "cs_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cs_profile_read": (ctypes.c_int, [_P, _P, _P]),
    "cs_kernel_launch_count": (ctypes.c_uint64, []),
    "cs_work_counts": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "cs_measure_alu_rates": (ctypes.c_int, [ctypes.c_int32, _P]),
    "cs_debug_set_pair_value": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_uint32]),
    "cs_forward_static": (ctypes.c_int, [ctypes.POINTER(CsScene), ctypes.POINTER(CsCamera),
                                         ctypes.POINTER(CsSettings), _P, _P, _P]),
    "cs_loss_l1_dssim": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                        _P, _P, _P]),
    "cs_adam_step": (ctypes.c_int, [_P, ctypes.POINTER(CsAdamGroup), ctypes.c_int32, ctypes.POINTER(CsAdamSettings),
                                    ctypes.c_int64, _P]),
    "cs_refine": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(CsParamArrays),
                                 ctypes.POINTER(CsParamArrays), ctypes.POINTER(CsParamArrays), _P, ctypes.c_int32,
                                 ctypes.POINTER(CsRefineSettings), ctypes.c_int64, ctypes.POINTER(CsParamArrays),
                                 ctypes.POINTER(CsParamArrays), ctypes.POINTER(CsParamArrays), _P,
                                 ctypes.POINTER(ctypes.c_int64), _P]),
    "cs_server_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, ctypes.c_int32,
                                        ctypes.POINTER(CsSettings), ctypes.POINTER(_P)]),
    "cs_server_destroy": (None, [_P]),
    "cs_server_set_pipelining": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cs_server_add_scene": (ctypes.c_int, [_P, ctypes.POINTER(CsScene), ctypes.POINTER(ctypes.c_int32)]),
    "cs_server_remove_scene": (ctypes.c_int, [_P, ctypes.c_int32]),
    "cs_server_submit": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(CsCamera), _P,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "cs_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(CsCompletion), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "cs_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
}

STAGES = ("preprocess", "depth_sort", "scan_emit", "tile_sort", "blend", "blend_backward", "preprocess_backward",
          "loss", "optimizer")
ADAM_MAX_GROUPS = 16

_lib = None


def lib():
    """Load the compiled library; fails loudly if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        handle = ctypes.CDLL(LIB)
        for name, (res, args) in _PROTOTYPES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def exported_symbols():
    return list(_PROTOTYPES)


class CsError(RuntimeError):
    pass


def check(code: int, what: str):
    if code != 0:
        msg = lib().cs_last_error().decode(errors="replace")
        raise CsError(f"{what} failed (status {code}): {msg}")
