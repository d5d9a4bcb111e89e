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
# measurement kernels of the benchmark (throughput probes, the cuFFT baseline's projector): a
# library of their own, not on the projection path
MEASURE_SRC = os.path.join(CSRC, "measure", "eqm.cu")
MEASURE_LIB = os.path.join(HERE, "libeqm.so")

SOURCES = ["eq_f32.cu", "eq_f64.cu", "eq_gen_f32.cu", "eq_gen_f64.cu", "eq_gen_host.cu", "eq_api.cu", "eq_serve.cu", "eq_static.cu",
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


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every CUDA translation unit and link libeq.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "eq.h"))
    procs, objs = [], []
    mp = None
    if force or _stale(MEASURE_LIB, [MEASURE_SRC]):
        cmd = [nvcc(), *ARCH, *FLAGS, "-shared", MEASURE_SRC, "-o", MEASURE_LIB]
        mp = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc(), *ARCH, *FLAGS, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    if force or procs or _stale(LIB, objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs]
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
