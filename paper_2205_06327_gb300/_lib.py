"""ctypes binding of libptycho.so (include/ptycho.h): argument marshalling only.

The library is built in-tree by ``paper_2205_06327_gb300.build``; importing
this module loads it and fails loudly if it is missing.  There is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptycho.so")

PTYCHO_OK = 0
PTYCHO_ERR_ARG = -1
PTYCHO_ERR_POSITION = -2
PTYCHO_ERR_CUDA = -3
PTYCHO_ERR_NOMEM = -4
PTYCHO_ERR_TIMEOUT = -5
PTYCHO_ERR_UNSUPPORTED = -6
PTYCHO_FP32 = 0
PTYCHO_BF16X3 = 1
PTYCHO_FP16X3 = 2
PTYCHO_FLAG_ASYNC_CHECK = 1
PTYCHO_FLAG_TIMING = 2
PTYCHO_FLAG_SELFTEST_TIMEOUT = 4
PTYCHO_CKPT_AUTO = -1

ERROR_NAMES = {
    PTYCHO_ERR_ARG: "PTYCHO_ERR_ARG",
    PTYCHO_ERR_POSITION: "PTYCHO_ERR_POSITION",
    PTYCHO_ERR_CUDA: "PTYCHO_ERR_CUDA",
    PTYCHO_ERR_NOMEM: "PTYCHO_ERR_NOMEM",
    PTYCHO_ERR_TIMEOUT: "PTYCHO_ERR_TIMEOUT",
    PTYCHO_ERR_UNSUPPORTED: "PTYCHO_ERR_UNSUPPORTED",
}

# Every symbol include/ptycho.h declares.
EXPORTED = [
    "ptycho_plan_create", "ptycho_plan_destroy", "ptycho_plan_info", "ptycho_plan_status",
    "ptycho_forward", "ptycho_loss_grad", "ptycho_loss_grad_host", "ptycho_step", "ptycho_plan_timing",
    "ptycho_loss_grad_noalloc",
    "ptycho_potential_to_transmission", "ptycho_potential_grad", "ptycho_last_error", "ptycho_version",
    "ptycho_multi_loss_grad", "ptycho_multi_step", "ptycho_step_accumulate",
]


class PtychoParams(C.Structure):
    _fields_ = [
        ("M", C.c_int32), ("S", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("N", C.c_int32),
        ("lambda_A", C.c_double), ("dz_A", C.c_double), ("pixel_A", C.c_double),
        ("precision", C.c_int32), ("flags", C.c_int32),
        ("workspace_bytes", C.c_int64),
        ("tile_h", C.c_int32), ("tile_w", C.c_int32),
        ("ckpt_every", C.c_int32),
    ]


class PtychoTiming(C.Structure):
    _fields_ = [
        ("chain_ms", C.c_double), ("accum_ms", C.c_double), ("probe_ms", C.c_double), ("other_ms", C.c_double),
        ("chain_launches", C.c_int64), ("accum_launches", C.c_int64), ("launches", C.c_int64),
        ("chain_positions", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class PtychoProblem(C.Structure):
    """One entry of a multi-problem call (ptycho_problem)."""
    _fields_ = [
        ("plan", C.c_void_p),
        ("pos_yx", C.c_void_p),
        ("probe", C.c_void_p),
        ("obj", C.c_void_p),
        ("meas_I", C.c_void_p),
        ("loss_out", C.c_void_p),
        ("grad_obj", C.c_void_p),
        ("grad_probe", C.c_void_p),
    ]


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the library once and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "ptycho_plan_create": ([C.POINTER(vp), C.POINTER(PtychoParams)], C.c_int),
        "ptycho_plan_destroy": ([vp], C.c_int),
        "ptycho_plan_info": ([vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)], C.c_int),
        "ptycho_plan_status": ([vp], C.c_int),
        "ptycho_forward": ([vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "ptycho_loss_grad": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "ptycho_loss_grad_host": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "ptycho_step": ([vp, vp, vp, vp, vp, dbl, dbl, i32, vp, vp, vp], C.c_int),
        "ptycho_step_accumulate": ([vp, vp, vp, vp, vp, dbl, dbl, vp, i32, vp, vp], C.c_int),
        "ptycho_plan_timing": ([vp, C.POINTER(PtychoTiming), i32], C.c_int),
        "ptycho_loss_grad_noalloc": ([C.POINTER(PtychoParams), vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "ptycho_potential_to_transmission": ([vp, vp, C.c_int64, dbl, vp], C.c_int),
        "ptycho_potential_grad": ([vp, vp, vp, C.c_int64, dbl, vp], C.c_int),
        "ptycho_multi_loss_grad": ([C.POINTER(PtychoProblem), i32, vp], C.c_int),
        "ptycho_multi_step": ([C.POINTER(PtychoProblem), i32, dbl, dbl, vp], C.c_int),
        "ptycho_last_error": ([], C.c_char_p),
        "ptycho_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != PTYCHO_OK:
        raise PtychoError(rc, load().ptycho_last_error().decode())
