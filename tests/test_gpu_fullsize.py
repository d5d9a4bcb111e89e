"""Parity with the FP64 oracle on generic 3-D modes at full size: the 512^3 Voronoi workload the
bench times (5000 grains ~ N(0, 200 MPa), voxel noise ~ N(0, 20 MPa), DDO; Sec. 4.2 operator on
grain-boundary fields, Sec. 5.1), and two cross-sections that run the 512-point kernels along
x and y, and along x and z.

The fields are drawn on the host (the noise by a CPU generator), so the GPU and the oracle see
the same FP32 values.  The 512^3 oracle run takes a minute or two on the host cores; its result
is cached as .npy (key: a hash of the input bytes and the options) in $EQ_ORACLE_CACHE, default
.oracle_cache/ at the repository root, and its wall time is printed.
"""
import hashlib
import json
import math
import os
import time

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CACHE = os.environ.get("EQ_ORACLE_CACHE", os.path.join(ROOT, ".oracle_cache"))
W = np.array([1.0, 1, 1, 2, 2, 2])
TOL = 2e-6          # FP32 path against the FP64 oracle, relative L2 (A:B-weighted)
NTOL = 1e-5         # FP32 norms
EPS32 = 1.2e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def host_field(shape, grains, sigma, noise, seed):
    return voronoi_stress_field(shape, grains, sigma, noise, seed, dtype=torch.float32,
                                device="cpu").numpy()


def oracle_cached(s32, op="ddo"):
    """oracle.project_large of s32 (FP32 values read in FP64), from the cache when present."""
    h = hashlib.blake2b(s32.tobytes(), digest_size=16)
    h.update(f"{s32.shape}|{op}|keep|h=1".encode())
    key = "project_large_" + h.hexdigest()
    path = os.path.join(CACHE, key + ".npy")
    if os.path.exists(path):
        with open(os.path.join(CACHE, key + ".json")) as f:
            meta = json.load(f)
        return np.load(path, mmap_mode="r"), meta
    t0 = time.perf_counter()
    ref = oracle.project_large(s32, op)
    dt = time.perf_counter() - t0
    meta = {"seconds": dt, "cores": os.cpu_count(), "shape": list(s32.shape), "op": op}
    try:
        os.makedirs(CACHE, exist_ok=True)
        np.save(path, ref)
        with open(os.path.join(CACHE, key + ".json"), "w") as f:
            json.dump(meta, f)
    except OSError:
        pass                                    # a read-only or full disk only loses the cache
    return ref, meta


def rel_by_component(out_gpu, ref):
    """A:B-weighted relative L2 of a (6, ...) CUDA tensor against a (6, ...) FP64 array, one
    component at a time (host memory stays bounded)."""
    num = den = 0.0
    for c in range(6):
        o = out_gpu[c].double().cpu().numpy()
        r = np.asarray(ref[c], dtype=np.float64)
        num += W[c] * float(((o - r) ** 2).sum())
        den += W[c] * float((r * r).sum())
    return math.sqrt(num / den)


def check_against_oracle(s32, want_div=True):
    ref, meta = oracle_cached(s32)
    nz, ny, nx = s32.shape[1:]
    plan = eq.Plan(nx, ny, nz, torch.float32, 1, "ddo")
    x = torch.from_numpy(s32).cuda().unsqueeze(0)
    out = plan.project(x)
    nrm = plan.norms()[0]
    plan.close()
    err = rel_by_component(out[0], ref)
    del out, x
    torch.cuda.empty_cache()
    assert err <= TOL, err
    want = oracle.norms_large(s32, ref, "ddo", div_out=False)
    for k in ("norm_in", "norm_out", "resid_l2", "resid_rel"):
        assert nrm[k] == pytest.approx(want[k], rel=NTOL), k
    if want_div:
        assert nrm["div_in_l2"] == pytest.approx(want["div_in_l2"], rel=NTOL)
    assert nrm["resid_linf"] == pytest.approx(want["resid_linf"], rel=NTOL,
                                              abs=100 * EPS32 * float(np.abs(s32).max()))
    assert nrm["div_out_l2"] <= 1e3 * EPS32 * want["norm_in"]
    assert np.allclose(nrm["mean"], want["mean"], rtol=NTOL, atol=NTOL * want["norm_in"])
    return err, meta


# (nz, ny, nx): generic modes through the 512-point x pass and 512-point y passes, and through the
# 512-point x pass and 512-point z passes
@pytest.mark.parametrize("shape", [(64, 512, 512), (512, 64, 512)])
def test_generic_modes_through_the_512_point_kernels(shape):
    s32 = host_field(shape, 625, 200.0, 20.0, 210501614 + shape[0])
    err, meta = check_against_oracle(s32)
    print(f"\n{shape}: rel L2 {err:.3e}; oracle {meta['seconds']:.1f} s on {meta['cores']} cores")


def test_512cubed_voronoi_workload_against_the_oracle():
    """The bench's 512^3 field (seed 210501614), element by element against one oracle run."""
    s32 = host_field((512, 512, 512), 5000, 200.0, 20.0, 210501614)
    err, meta = check_against_oracle(s32)
    print(f"\n512^3: rel L2 {err:.3e}; oracle {meta['seconds']:.1f} s on {meta['cores']} cores")
