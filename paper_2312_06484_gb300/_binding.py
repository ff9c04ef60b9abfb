"""ctypes declarations of the C ABI in include/airpf.h (argument marshalling only).

``load()`` returns the in-tree library ``_build/libairpf.so``, building it with nvcc
if it is missing or stale.  There is no fallback: if the library cannot be built or
loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_uint32, c_int64, c_double, c_uint64 = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64,
                                                  ctypes.c_double, ctypes.c_uint64)
c_void_p, c_size_t = ctypes.c_void_p, ctypes.c_size_t
P_double = ctypes.POINTER(ctypes.c_double)


class AirpfConfig(ctypes.Structure):
    _fields_ = [("model", c_int32), ("dx", c_int32), ("dy", c_int32), ("m", c_int32),
                ("M", c_int32), ("T", c_int32), ("B", c_int32), ("mode", c_int32),
                ("tau", c_double), ("precision", c_int32), ("record", c_int32),
                ("seed", c_uint64), ("launch", c_int32), ("reserved", c_int32), ("ppt", c_int32),
                ("islands_per_cta", c_int32), ("ckpt", c_int32), ("tau_int", c_double),
                ("radix", c_int32)]


# every symbol include/airpf.h declares, with (restype, argtypes)
SIGNATURES = {
    "airpf_workspace_bytes": (c_int32, [ctypes.POINTER(AirpfConfig), ctypes.POINTER(c_size_t)]),
    "airpf_create": (c_int32, [ctypes.POINTER(AirpfConfig), c_void_p, c_size_t, c_void_p, c_void_p,
                               ctypes.POINTER(c_void_p)]),
    "airpf_destroy": (c_int32, [c_void_p]),
    "airpf_run": (c_int32, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint32, c_void_p, c_void_p,
                            c_void_p, c_void_p, c_void_p]),
    "airpf_run_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint32, c_void_p]),
    "airpf_pmmh": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                             c_uint32, c_uint32, c_int32, c_void_p, c_void_p, c_void_p]),
    "airpf_run_static": (c_int32, [ctypes.POINTER(AirpfConfig), c_void_p, c_void_p, c_void_p, c_uint32,
                                   c_uint32, c_void_p, c_void_p]),
    "airpf_group_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "airpf_group_destroy": (c_int32, [c_void_p]),
    "airpf_group_run": (c_int32, [c_void_p, ctypes.POINTER(c_void_p), c_void_p, ctypes.POINTER(c_uint32),
                                  c_uint32, ctypes.POINTER(c_void_p)]),
    "airpf_group_pmmh": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_void_p), ctypes.POINTER(c_uint32), c_uint32, c_int32,
                                   ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p)]),
    "airpf_group_sync": (c_int32, [c_void_p]),
    "airpf_autotune": (c_int32, [ctypes.POINTER(AirpfConfig), c_void_p, c_size_t, c_void_p, c_void_p, c_void_p,
                                 c_int32, c_void_p, ctypes.POINTER(AirpfConfig), ctypes.POINTER(ctypes.c_float)]),
    "airpf_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint32, c_void_p, c_void_p, c_void_p]),
    "airpf_pmmh_langevin": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_uint32, c_uint32, c_int32, c_void_p, c_void_p, c_void_p]),
    "airpf_step_begin": (c_int32, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint32]),
    "airpf_step_islands": (c_int32, [c_void_p, c_int32, c_int32, c_int32]),
    "airpf_step_cascade": (c_int32, [c_void_p, c_int32]),
    "airpf_step_end": (c_int32, [c_void_p, c_void_p]),
    "airpf_step_regions": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_size_t), ctypes.POINTER(c_size_t),
                                     ctypes.POINTER(c_int32)]),
    "airpf_step_levels": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "airpf_sync": (c_int32, [c_void_p]),
    "airpf_launch_mode": (c_int32, [c_void_p]),
    "airpf_tiling": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "airpf_moments": (c_int32, [c_void_p, c_void_p]),
    "airpf_kernel_times": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "airpf_debug_inject": (c_int32, [c_void_p, c_int32]),
    "airpf_debug_math": (c_int32, [c_int32, c_void_p, c_void_p, ctypes.c_int64, c_void_p]),
    "airpf_theta_dim": (c_int32, [c_int32, c_int32]),
    "airpf_last_launch_count": (c_int64, [c_void_p]),
    "airpf_last_error": (ctypes.c_char_p, [c_void_p]),
    "airpf_status_string": (ctypes.c_char_p, [c_int32]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """The loaded CUDA library (raises if it is not there and cannot be built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"AIRPF CUDA library missing at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AirpfError(RuntimeError):
    pass


def check(status: int, ctx=None):
    if status != 0:
        lib = load()
        msg = lib.airpf_last_error(ctx).decode(errors="replace")
        name = lib.airpf_status_string(status).decode()
        raise AirpfError(f"{name}: {msg}")
