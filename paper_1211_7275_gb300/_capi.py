"""ctypes binding of the C ABI in include/qew.h (``libqew.so``).  Argument marshalling only:
every step of the relaxation runs in the library's CUDA kernels.  There is no fallback: if the
library is missing or cannot be loaded, loading raises."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqew.so")

QEW_OK = 0
QEW_EINVAL = -1
QEW_ENOMEM = -2
QEW_ECUDA = -3
QEW_ETIMEOUT = -4
QEW_ENONFINITE = -5
QEW_ESTATE = -6

RF_GAUSS_LINEAR = 0
RB_UNIFORM_CATMULLROM = 1
NONE = 2
RB_GAUSS_LINEAR = 3
RB_GAUSS_CATMULLROM = 4

FP32_SPLIT = 0
FP64 = 1

# every entry point declared in include/qew.h, with (restype, argtypes)
_P = ctypes.c_void_p
_H = ctypes.c_void_p
SIGNATURES = {
    "qew_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int32, ctypes.c_uint64]),
    "qew_create_batch": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int32, _P, _P, _P, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_int32]),
    "qew_set_precision": (ctypes.c_int, [_H, ctypes.c_int32]),
    "qew_set_stream": (ctypes.c_int, [_H, _P]),
    "qew_set_disorder_period": (ctypes.c_int, [_H, ctypes.c_int64]),
    "qew_set_samples": (ctypes.c_int, [_H, _P]),
    "qew_set_tuning": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "qew_get_tuning": (ctypes.c_int, [_H, _P, _P, _P]),
    "qew_advance": (ctypes.c_int, [_H, ctypes.c_int64]),
    "qew_observe": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P]),
    "qew_observe_ex": (ctypes.c_int, [_H, _P, ctypes.c_int32, _P, _P, _P]),
    "qew_get_state": (ctypes.c_int, [_H, _P, _P]),
    "qew_get_cells": (ctypes.c_int, [_H, _P]),
    "qew_set_state": (ctypes.c_int, [_H, _P]),
    "qew_reset": (ctypes.c_int, [_H]),
    "qew_num_sites": (ctypes.c_int, [_H, _P]),
    "qew_structure_factor": (ctypes.c_int, [_H, ctypes.c_int32, _P]),
    "qew_disorder_values": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                           _P, _P, ctypes.c_int64, _P]),
    "qew_philox_words": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "qew_measure_alu_peaks": (ctypes.c_int, [_P, ctypes.c_int32]),
    "qew_enable_stats": (ctypes.c_int, [_H, ctypes.c_int32]),
    "qew_get_stats": (ctypes.c_int, [_H, _P, _P, _P, _P, _P]),
    "qew_observe_state_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_int32, ctypes.c_uint64, _P, _P, _P, _P]),
    "qew_critical_force_rf": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_double, ctypes.c_double,
                                             _P, _P, _P, _P]),
    "qew_selftest_bounded_wait": (ctypes.c_int, [_H, ctypes.c_int32]),
    "qew_last_error": (ctypes.c_char_p, [_H]),
    "qew_destroy": (None, [_H]),
}

_lock = threading.Lock()
_lib = None


class QewError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qew status {code}: {msg}")
        self.code = code


def load(build_if_missing: bool = True):
    """Load libqew.so (building it first when missing or stale and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import _build
                try:
                    _build.build()
                except RuntimeError:
                    if not os.path.exists(LIB_PATH):
                        raise
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1211_7275_gb300._build.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, handle=None) -> None:
    if rc != QEW_OK:
        msg = load().qew_last_error(handle)
        raise QewError(rc, msg.decode() if msg else "")
