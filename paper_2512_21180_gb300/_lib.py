"""ctypes loader for libcbct.so: argument marshalling only.

The library is built in-tree by `build.py`. There is no fallback: if the shared
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcbct.so")
_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_longlong
F32 = ctypes.c_float
F64 = ctypes.c_double
U64 = ctypes.c_uint64


class LpdDesc(ctypes.Structure):
    _fields_ = [("n_iter", I32), ("n_mem", I32), ("width", I32), ("slope", F32), ("mu_ref", F32),
                ("bp_scale", F32), ("seed", U64), ("residual_input", I32), ("max_batch", I32),
                ("reversible", I32), ("lire", I32), ("p4", I32), ("unet", I32),
                ("weight_norm", I32)]


class GeomDesc(ctypes.Structure):
    _fields_ = [
        ("nx", I32), ("ny", I32), ("nz", I32),
        ("vox", F64 * 3), ("center", F64 * 3),
        ("nu", I32), ("nv", I32),
        ("du", F64), ("dv", F64), ("u_offset", F64), ("v_offset", F64),
        ("sid", F64), ("sdd", F64),
        ("n_angles", I32), ("angles", P), ("normalize", I32),
    ]


# name -> (restype, argtypes); kept beside the declarations in include/cbct.h
SIGNATURES = {
    "cbct_last_error": (ctypes.c_char_p, []),
    "geometry_create": (I32, [ctypes.POINTER(GeomDesc), ctypes.POINTER(P)]),
    "geometry_destroy": (None, [P]),
    "geometry_scale": (F64, [P]),
    "forward_project": (I32, [P, P, P, I32, I32, P]),
    "back_project": (I32, [P, P, P, I32, I32, P]),
    "forward_project_f64": (I32, [P, P, P, I32, I32, P]),
    "back_project_f64": (I32, [P, P, P, I32, I32, P]),
    "back_project_noalloc": (I32, [P, P, P, I32, I32, P]),
    "cbct_count_samples": (I32, [P, ctypes.POINTER(I64), P]),
    "cbct_device_status": (I32, [P, ctypes.POINTER(I32), I32]),
    "lpd_device_status": (I32, [P, ctypes.POINTER(I32), I32]),
    "cbct_forward_config": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(F64), ctypes.POINTER(F64)]),
    "cbct_phantom": (I32, [P, P, I32, I32, P, P]),
    "cbct_poisson": (I32, [P, I64, F64, U64, P, P]),
    "cbct_neglog": (I32, [P, I64, F64, P, P]),
    "cbct_simulate": (I32, [P, P, I32, F64, U64, P, P, P]),
    "cbct_redundancy_weight": (I32, [P, P, P]),
    "cbct_detector_response": (I32, [P, I32, P]),
    "cbct_water_bone": (I32, [P, I64, I32, F64, P, P]),
    "cbct_poly_reading": (I32, [P, I32, I64, I32, I32, P, P, P, P, U64, I32, P, P, P, P]),
    "cbct_poly_simulate": (I32, [P, P, I32, F64, I32, P, P, P, P, U64, I32, P, P, P]),
    "cbct_fov": (I32, [P, P, P]),
    "cbct_fdk_pad": (I32, [P]),
    "cbct_fdk": (I32, [P, P, P, I32, I32, P]),
    "cbct_opnorm": (I32, [P, F64, I32, ctypes.POINTER(F64), P]),
    "cbct_pdhg": (I32, [P, P, P, P, I32, I32, F64, F64, F64, F64, I32, P]),
    "cbct_landweber": (I32, [P, P, P, I32, I32, F64, I32, P]),
    "cbct_conv": (I32, [P, I32, I32, I32, I32, I32, I32, P, P, I32, I32, I32, I32, F32, P, I32, P, P, I64, P, P]),
    "cbct_conv_wgrad": (I32, [P, I32, I32, P, I32, I32, I32, I32, I32, I32, I32, P, P, I32, P, P]),
    "cbct_conv_plan": (I32, [I32, I32, I32, I32, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I64),
                             ctypes.POINTER(I32), ctypes.POINTER(I32)]),
    "lpd_create": (I32, [P, ctypes.POINTER(LpdDesc), ctypes.POINTER(P)]),
    "lpd_destroy": (None, [P]),
    "lpd_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(F32)]),
    "lpd_forward": (I32, [P, P, P, P, I32, I32, P]),
    "lpd_backward": (I32, [P, P, P, P, P]),
    "lpd_forward_latent": (I32, [P, P, P, P, P, P, I32, P]),
    "lpd_get_state": (I32, [P, P, P, P]),
    "lpd_backward_latent": (I32, [P, P, P, P, P, P, P, P, P]),
    "cbct_resample_down": (I32, [P, I64, I32, I32, I32, I32, I32, I32, I32, F32, P, P]),
    "cbct_resample_up": (I32, [P, I64, I32, I32, I32, I32, I32, I32, P, P]),
    "lpd_zero_grad": (I32, [P, P]),
    "lpd_clip_grads": (I32, [P, F32, F32, P, P]),
    "lpd_adam_step": (I32, [P, F32, F32, F32, F32, I32, F32, P]),
    "lpd_set_params": (I32, [P, P, I64]),
    "lpd_get_params": (I32, [P, P, I64]),
    "lpd_get_grads": (I32, [P, P, I64]),
    "cbct_masked_mse": (I32, [P, P, P, F32, I64, P, P, P]),
    "cbct_wait_probe": (I32, [P, I64, P, P]),
    "lpd_get_perms": (I32, [P, P]),
    "cbct_smem_probe": (I32, [I32, I32, P, ctypes.POINTER(I64), P]),
    "lpd_set_perms": (I32, [P, P]),
}

EXTRA_SIGNATURES: dict = {}


class CbctError(RuntimeError):
    pass


def load():
    """Load libcbct.so (raises if it is absent: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise CbctError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in {**SIGNATURES, **EXTRA_SIGNATURES}.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, what: str = ""):
    if rc != 0:
        msg = load().cbct_last_error().decode(errors="replace")
        raise CbctError(f"{what} failed ({rc}): {msg}")
