"""ctypes binding of libeq.so (include/eq.h).  Argument marshalling only: every step of the
projection runs in the library's CUDA kernels.  There is no fallback: if the library is missing
or fails to load, every call raises."""
from __future__ import annotations

import ctypes
import os

from . import _build

c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p

EQ_OK, EQ_ERR_INVALID, EQ_ERR_OOM, EQ_ERR_CUDA, EQ_ERR_TIMEOUT = 0, 1, 2, 3, 4
EQ_ERR_BUSY, EQ_PENDING, EQ_ERR_NOT_FOUND = 5, 6, 7
EQ_F32, EQ_F64 = 0, 1
EQ_OP_DDO, EQ_OP_CDO = 0, 1
EQ_NYQ_KEEP, EQ_NYQ_ZERO = 0, 1
EQ_TARGET_EQUILIBRIUM, EQ_TARGET_COMPATIBILITY = 0, 1
EQ_FLAG_NONFINITE, EQ_FLAG_NO_LINF = 1, 2
EQ_NUM_PASSES = 7
PASS_NAMES = ["z_forward", "mean_finalise", "y_forward", "x_fwd_project_inv", "y_inverse",
              "z_inverse", "norms_finalise"]

STATUS_NAMES = {0: "EQ_OK", 1: "EQ_ERR_INVALID", 2: "EQ_ERR_OOM", 3: "EQ_ERR_CUDA",
                4: "EQ_ERR_TIMEOUT", 5: "EQ_ERR_BUSY", 6: "EQ_PENDING", 7: "EQ_ERR_NOT_FOUND"}


class EqPlanOpts(ctypes.Structure):
    _fields_ = [("op", c_int), ("hx", c_double), ("hy", c_double), ("hz", c_double),
                ("nyq", c_int), ("want_linf", c_int), ("graph", c_int), ("target", c_int)]


class EqNorms(ctypes.Structure):
    _fields_ = [("mean", c_double * 6), ("norm_in", c_double), ("norm_out", c_double),
                ("resid_l2", c_double), ("resid_rel", c_double), ("resid_linf", c_double),
                ("div_in_l2", c_double), ("div_out_l2", c_double), ("flags", c_int)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "mean"}
        d["mean"] = list(self.mean)
        return d


class EqServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("admitted", ctypes.c_ulonglong),
                ("completed", ctypes.c_ulonglong), ("failed", ctypes.c_ulonglong),
                ("rejected", ctypes.c_ulonglong), ("cancelled", ctypes.c_ulonglong),
                ("plans_created", ctypes.c_ulonglong), ("plans_reused", ctypes.c_ulonglong),
                ("plans_evicted", ctypes.c_ulonglong), ("plan_create_seconds", c_double),
                ("queued", ctypes.c_longlong), ("inflight", ctypes.c_longlong),
                ("inflight_peak", ctypes.c_longlong), ("hbm_in_use", ctypes.c_ulonglong),
                ("hbm_in_use_peak", ctypes.c_ulonglong), ("hbm_budget", ctypes.c_ulonglong),
                ("plans_cached", ctypes.c_longlong)]

    def to_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) of every entry point declared in include/eq.h
SIGNATURES = [
    ("eq_plan_opts_default", None, [ctypes.POINTER(EqPlanOpts)]),
    ("eq_plan_create", c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(EqPlanOpts),
                               ctypes.POINTER(c_void_p)]),
    ("eq_plan_create_varlen", c_int, [ctypes.POINTER(c_int), c_int, c_int,
                                      ctypes.POINTER(EqPlanOpts), ctypes.POINTER(c_void_p)]),
    ("eq_project", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_project_host", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_project_host_async", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_project_hodge", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_project_padded", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("eq_norms", c_int, [c_void_p, ctypes.POINTER(EqNorms)]),
    ("eq_selftest_wait_timeout", c_int, [c_void_p, ctypes.c_longlong, c_void_p]),
    ("eq_plan_workspace_bytes", c_size_t, [c_void_p]),
    ("eq_plan_autotune", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_plan_set_timing", c_int, [c_void_p, c_int]),
    ("eq_plan_pass_ms", c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int)]),
    ("eq_plan_destroy", None, [c_void_p]),
    ("eq_project_static", c_int, [c_int, c_int, c_int, ctypes.POINTER(EqPlanOpts), c_void_p,
                                  c_void_p, c_void_p, c_void_p]),
    ("eq_server_create", c_int, [c_size_t, c_int, ctypes.POINTER(c_void_p)]),
    ("eq_serve_submit", c_int, [c_void_p, c_int, c_int, c_int, c_int, ctypes.POINTER(EqPlanOpts),
                                c_void_p, c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]),
    ("eq_serve_poll", c_int, [c_void_p, ctypes.c_ulonglong, c_int, ctypes.POINTER(EqNorms),
                              ctypes.POINTER(c_double)]),
    ("eq_serve_cancel", c_int, [c_void_p, ctypes.c_ulonglong]),
    ("eq_server_stats", c_int, [c_void_p, ctypes.POINTER(EqServerStats)]),
    ("eq_server_destroy", None, [c_void_p]),
    ("eq_grains_create", c_int, [ctypes.POINTER(c_int), c_int, c_int, c_int, c_int,
                                 ctypes.POINTER(c_void_p)]),
    ("eq_grain_average", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("eq_grains_destroy", None, [c_void_p]),
    ("eq_last_error", ctypes.c_char_p, []),
]

_LIB = None


class EqError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    """libeq.so, or the bounds-checked libeq_check.so when the environment sets
    EQ_BOUNDS_CHECK=1 (read when the library is first loaded)."""
    return _build.LIB_CHECK if os.environ.get("EQ_BOUNDS_CHECK") == "1" else _build.LIB


def load() -> ctypes.CDLL:
    """Load libeq.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def check(status: int, where: str) -> None:
    if status != EQ_OK:
        msg = load().eq_last_error()
        raise EqError(status, where, msg.decode() if msg else "")
