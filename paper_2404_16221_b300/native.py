"""ctypes binding of libnerfxl.so (the C ABI in include/nerfxl.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. PyTorch supplies device memory and the current stream. There is no
fallback: if the shared library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnerfxl.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "nerfxl.h")

MAX_LEVELS = 32

OK, E_INVALID, E_WORKSPACE, E_CUDA, E_TIMEOUT, E_UNSUPPORTED, E_OVERFLOW = range(7)
F32, F16, BF16, E4M3 = range(4)
ARCH_FUSED, ARCH_SPLIT = 0, 1
STATUS_NAMES = {0: "OK", 1: "E_INVALID", 2: "E_WORKSPACE", 3: "E_CUDA", 4: "E_TIMEOUT", 5: "E_UNSUPPORTED",
                6: "E_OVERFLOW"}


class NerfxlError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__("%s: %s (%s)" % (what, STATUS_NAMES.get(status, status), msg))
        self.status = status


class FieldDesc(C.Structure):
    _fields_ = [("K", C.c_int32), ("L", C.c_int32), ("F", C.c_int32), ("log2_T", C.c_int32),
                ("mlp_in", C.c_int32), ("mlp_width", C.c_int32), ("level_res", C.c_int32 * MAX_LEVELS),
                ("boxes", C.c_void_p), ("tables", C.c_void_p), ("mlp", C.c_void_p), ("table_dtype", C.c_int32),
                ("mlp_dtype", C.c_int32), ("mlp_scales", C.c_void_p), ("occupancy", C.c_void_p),
                ("occ_res", C.c_int32), ("arch", C.c_int32)]


class AdamDesc(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int64)]


class TrainStateDesc(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("tables", "mlp", "grad_tables", "grad_mlp", "m_tables", "v_tables",
                                          "m_mlp", "v_mlp")]


class CameraDesc(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3), ("forward", C.c_float * 3),
                ("tan_half_fov", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("reserved", C.c_int32)]


class RayItemDesc(C.Structure):
    _fields_ = [("batch_offset", C.c_int64), ("first_pixel", C.c_int64), ("out_offset", C.c_int64),
                ("camera", C.c_int32), ("count", C.c_int32)]


class SamplingDesc(C.Structure):
    _fields_ = [("n_samples", C.c_int32), ("max_segments", C.c_int32), ("t_min", C.c_float), ("flags", C.c_int32)]


_lib = None

_vp, _i64, _i32, _sz = C.c_void_p, C.c_int64, C.c_int32, C.c_size_t
_FP, _SP = C.POINTER(FieldDesc), C.POINTER(SamplingDesc)

# name -> (restype, argtypes)
SIGNATURES = {
    "nerfxl_table_entries": (_i64, [_vp, _i32, _i32]),
    "nerfxl_mlp_params": (_i64, [_i32, _i32]),
    "nerfxl_field_mlp_params": (_i64, [_FP]),
    "nerfxl_max_chunks": (_i32, [_SP, _i32]),
    "nerfxl_workspace_bytes": (_sz, [_FP, _SP, _i64, _i32]),
    "nerfxl_render_fwd": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_check": (C.c_int, [_vp, _sz, _vp]),
    "nerfxl_render_fwd_static": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nerfxl_static_check": (C.c_int, [_vp]),
    "nerfxl_last_error": (C.c_char_p, []),
    "nerfxl_workspace_stats": (C.c_int, [_vp, _sz, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp]),
    "nerfxl_set_profile_events": (C.c_int, [_vp, _vp]),
    "nerfxl_launch_count": (_i64, []),
    "nerfxl_set_gather_groups": (C.c_int, [_sz, _sz, _i64, _i64]),
    "nerfxl_render_bwd": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_loss": (C.c_int, [_i64, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_adam_update": (C.c_int, [_i64, _vp, _vp, _vp, _vp, C.c_void_p, _vp, _i32, _vp]),
    "nerfxl_quantize_e4m3": (C.c_int, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "nerfxl_step_workspace_bytes": (_sz, [_FP, _SP, _i64]),
    "nerfxl_step_sub_batch": (_i64, [_FP, _SP, _i64, _sz]),
    "nerfxl_step": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_render_cameras_workspace_bytes": (_sz, [_FP, _SP, _i64]),
    "nerfxl_render_cameras": (C.c_int, [_FP, _SP, _i64, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_debug_wait_probe": (C.c_int, [_vp, C.c_uint32, _i32, _vp]),
    "nerfxl_probe_reduction_rate": (C.c_int, [_vp, _sz, _i32, _vp, _vp]),
    "nerfxl_probe_load_rate": (C.c_int, [_vp, _sz, _i32, _vp, _vp]),
    "nerfxl_debug_camera_rays": (C.c_int, [_i64, _i32, _vp, _vp, _i32, _vp, _vp, _vp]),
    "nerfxl_partition": (C.c_int, [_vp, _i64, _vp, _i32, _vp, _vp]),
    "nerfxl_occupancy_update": (C.c_int, [_FP, _i32, _i64, C.c_uint64, C.c_float, C.c_float, _vp, _vp, _vp]),
    "nerfxl_region_chunks": (C.c_int, [_vp, _sz, _i32, _vp, _vp]),
    "nerfxl_debug_segments": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "nerfxl_debug_samples": (C.c_int, [_FP, _SP, _i64, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}


def header_functions(path: str = HEADER):
    """Function names the C header declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nerfxl_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libnerfxl.so (built in-tree) and bind every declared function."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnerfxl.so is not built; run `python -m paper_2404_16221_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str):
    if status != OK:
        raise NerfxlError(status, what, lib().nerfxl_last_error().decode())


def table_entries(level_res, log2_T: int) -> int:
    arr = (C.c_int32 * len(level_res))(*[int(v) for v in level_res])
    return int(lib().nerfxl_table_entries(arr, len(level_res), int(log2_T)))


def mlp_params(mlp_in: int, width: int) -> int:
    return int(lib().nerfxl_mlp_params(int(mlp_in), int(width)))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)
