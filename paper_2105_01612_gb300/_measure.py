"""ctypes binding of libeqm.so, the benchmark's measurement kernels (csrc/measure/eqm.cu): FMA
throughput probes and the per-mode projector of the cuFFT comparison baseline.  Not part of the
projection path; used by bench.py only."""
from __future__ import annotations

import ctypes
import os

from . import _build

_LIB = None


def load() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.MEASURE_LIB):
            raise RuntimeError(f"{_build.MEASURE_LIB} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.MEASURE_LIB)
        v, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        lib.eqm_fma_probe.restype = i
        lib.eqm_fma_probe.argtypes = [i, v, i, i, ll, v]
        lib.eqm_project_half.restype = i
        lib.eqm_project_half.argtypes = [i, v, i, i, i, v, v, v, v]
        _LIB = lib
    return _LIB


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise RuntimeError(f"{where}: CUDA error {rc}")


def fma_probe(dtype_code: int, out_ptr: int, blocks: int, threads: int, iters: int,
              stream: int) -> None:
    """dtype_code 1: FP64, 0: FP32; 16 * iters flops per thread."""
    _check(load().eqm_fma_probe(dtype_code, out_ptr, blocks, threads, iters, stream or None),
           "eqm_fma_probe")


def project_half(dtype_code: int, spec_ptr: int, nz: int, ny: int, nxh: int, xi_x: int,
                 xi_y: int, xi_z: int, stream: int) -> None:
    _check(load().eqm_project_half(dtype_code, spec_ptr, nz, ny, nxh, xi_x, xi_y, xi_z,
                                   stream or None), "eqm_project_half")
