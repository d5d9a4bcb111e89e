"""Build libeq.so from csrc/ with nvcc for sm_103a (in-tree, parallel per translation unit), and
the benchmark's measurement kernels into libeqm.so."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libeq.so")
# the same library with device-side bounds checks (EQ_BOUNDS_CHECK): an out-of-range index raises
# the plan's error word (reported by eq_norms) and the access is skipped; loaded instead of
# libeq.so when the environment sets EQ_BOUNDS_CHECK=1
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libeq_check.so")
# measurement kernels of the benchmark (throughput probes, the cuFFT baseline's projector): a
# library of their own, not on the projection path
MEASURE_SRC = os.path.join(CSRC, "measure", "eqm.cu")
MEASURE_LIB = os.path.join(HERE, "libeqm.so")

SOURCES = ["eq_f32.cu", "eq_f64.cu", "eq_gen_f32.cu", "eq_gen_f64.cu", "eq_gen_dd.cu", "eq_gen_host.cu", "eq_api.cu", "eq_serve.cu", "eq_static.cu",
           "eq_grains.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libeq.so")
    return path


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, checked: bool = True) -> str:
    """Compile every CUDA translation unit and link libeq.so (and, with `checked`, the
    bounds-checked libeq_check.so, compiled alongside) and the measurement library libeqm.so;
    returns the path of libeq.so."""
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "eq.h"))
    procs = []
    mp = None
    if force or _stale(MEASURE_LIB, [MEASURE_SRC]):
        cmd = [nvcc(), *ARCH, *FLAGS, "-shared", MEASURE_SRC, "-o", MEASURE_LIB]
        mp = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    variants = [(BUILD, LIB, [])]
    if checked:
        variants.append((BUILD_CHECK, LIB_CHECK, ["-DEQ_BOUNDS_CHECK=1"]))
    objs_of = {}
    for bdir, lib, extra in variants:
        os.makedirs(bdir, exist_ok=True)
        objs = objs_of.setdefault(lib, [])
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src.replace(".cu", ".o"))
            objs.append(o)
            if force or _stale(o, [s] + headers):
                cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
                if verbose:
                    print(" ".join(cmd), file=sys.stderr)
                procs.append((lib, src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                         stderr=subprocess.STDOUT, text=True)))
    errors, rebuilt = [], set()
    for lib, src, p in procs:
        out, _ = p.communicate()
        rebuilt.add(lib)
        if p.returncode != 0:
            errors.append(f"{src}:\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    for _, lib, _ in variants:
        objs = objs_of[lib]
        if force or lib in rebuilt or _stale(lib, objs):
            cmd = [nvcc(), *ARCH, "-shared", "-o", lib, *objs]
            r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed:\n" + r.stdout)
    if mp is not None:
        out, _ = mp.communicate()
        if mp.returncode != 0:
            raise RuntimeError("nvcc failed (measurement kernels):\n" + out)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
