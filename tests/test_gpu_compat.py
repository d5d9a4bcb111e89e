"""Parity of the strain-compatibility target (c0 + S - S_equil, the dual constraint) with the
FP64 oracle, through the C ABI on every path that runs the projector: compile-time lengths (the
TMA, warp and plain x kernels), runtime lengths, the static-scratch entry point and serving.

Bars as for the equilibrium target: relative L2 <= 1e-12 (FP64) / 2e-6 (FP32); norms within
1e-10 / 1e-5; the returned field has a vanishing inc (checked in real space on the GPU result).
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq
from paper_2105_01612_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-6}
NTOL = {torch.float64: 1e-10, torch.float32: 1e-5}
W = np.array([1.0, 1, 1, 2, 2, 2])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    w = W.reshape((6,) + (1,) * (a.ndim - 1))
    return math.sqrt(float((w * (a - b) ** 2).sum() / max((w * b ** 2).sum(), 1e-300)))


def field(shape, seed, grains=40):
    return voronoi_stress_field(shape, grains, 150.0, 15.0, seed).numpy()


def run(s, dtype, op="ddo", nyq="keep", h=(1.0, 1.0, 1.0)):
    x = torch.as_tensor(s).to(dtype).cuda().unsqueeze(0).contiguous()
    plan = eq.Plan(x.shape[4], x.shape[3], x.shape[2], dtype, 1, op, h, nyq,
                   target="compatibility")
    out = plan.project(x)
    nrm = plan.norms()[0]
    plan.close()
    return out[0].double().cpu().numpy(), nrm


def check(out, nrm, s, ref, dtype, op="ddo", h=(1.0, 1.0, 1.0)):
    assert rel(out, ref) <= TOL[dtype]
    want = oracle.norms(s, ref, op, h)
    tol = NTOL[dtype]
    for k in ("norm_in", "norm_out", "resid_l2", "resid_rel", "div_in_l2", "div_out_l2"):
        assert nrm[k] == pytest.approx(want[k], rel=tol, abs=tol * want["norm_in"] * 1e-3), k
    assert nrm["resid_linf"] == pytest.approx(want["resid_linf"], rel=tol,
                                              abs=1e-5 * np.abs(s).max())


@pytest.mark.parametrize("op", ["ddo", "cdo"])
def test_16cubed_fp64(op):
    s = field((16, 16, 16), 210501612, grains=8)
    ref = oracle.project_compat(s, op)
    out, nrm = run(s, torch.float64, op)
    check(out, nrm, s, ref, torch.float64, op)


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 64, 128), (16, 64, 512)])
def test_power_of_two_fp32_and_real_space_compatibility(shape):
    s = field(shape, 3 + shape[2])
    ref = oracle.project_compat(s, "ddo")
    out, nrm = run(s, torch.float32)
    check(out, nrm, s, ref, torch.float32)
    # independent of the oracle's transforms: inc of the result vanishes (central differences)
    inc = oracle.inc_central_diff(out)
    assert np.abs(inc).max() <= 1e-4 * np.abs(s).max()


def test_512_point_rows_fp64_and_nyquist_zero():
    s = field((8, 16, 512), 77)
    for nyq in ("keep", "zero"):
        ref = oracle.project_compat(s, "ddo", nyq=nyq)
        out, nrm = run(s, torch.float64, nyq=nyq)
        assert rel(out, ref) <= 1e-12, nyq


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_runtime_lengths(dtype):
    s = field((18, 25, 30), 91)
    h = (1.0, 0.7, 1.3)
    ref = oracle.project_compat(s, "ddo", h)
    out, nrm = run(s, dtype, h=h)
    check(out, nrm, s, ref, dtype, h=h)


def test_static_entry_point_and_equilibrium_plus_compat_split_the_field():
    s = field((32, 32, 64), 123)
    x = torch.as_tensor(s).float().cuda().contiguous()
    out = torch.empty_like(x)
    opts = eq._opts("ddo", target="compatibility")
    lib = _lib.load()
    st = lib.eq_project_static(64, 32, 32, ctypes.byref(opts), x.data_ptr(), out.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream)
    _lib.check(st, "eq_project_static")
    torch.cuda.synchronize()
    ref = oracle.project_compat(s, "ddo")
    assert rel(out.double().cpu().numpy(), ref) <= 2e-6
    # S_equil + compat = S + c0, with both from the GPU
    eqo, _ = eq.project(x)
    c0 = s.mean(axis=(1, 2, 3))[:, None, None, None]
    both = eqo.double().cpu().numpy() + out.double().cpu().numpy()
    assert rel(both, s + c0) <= 4e-6


def test_served_request_with_the_compatibility_target():
    s = field((20, 24, 28), 5)
    x = torch.as_tensor(s).float().contiguous().pin_memory()
    y = torch.empty_like(x).pin_memory()
    srv = eq.Server(1 << 30, 2)
    try:
        t = srv.submit(x, y, target="compatibility")
        srv.wait(t)
    finally:
        srv.close()
    assert rel(y.double().numpy(), oracle.project_compat(s, "ddo")) <= 2e-6
