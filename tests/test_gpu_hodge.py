"""Parity of eq_project_hodge (the projection plus the Hodge potential y of Theorem 2) with the
FP64 oracle, through the C ABI.

y is compared with oracle.hodge_potential (relative L2 over the three components <= 1e-12 FP64,
2e-6 FP32); d_out must be bit-identical to eq_project's; independently of the oracle's
transforms, sym grad y built in real space (central differences) must equal S - S_out.
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


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def vrel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return math.sqrt(float(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def same_projection(out, plain, dtype):
    """The Hodge form returns the plain projection: bit for bit in FP32; in FP64, where plain
    projections run in double-float arithmetic and the Hodge form in FP64 instructions, to the
    formats' rounding."""
    if dtype == torch.float64:
        assert vrel(out, plain) <= 1e-13
    else:
        assert np.array_equal(out, plain)


def field(shape, seed, grains=30):
    return voronoi_stress_field(shape, grains, 150.0, 15.0, seed).numpy()


def run_hodge(s, dtype, op="ddo", target="equilibrium", h=(1.0, 1.0, 1.0)):
    x = torch.as_tensor(np.asarray(s)).to(dtype).cuda().contiguous()
    xb = x if x.dim() == 5 else x.unsqueeze(0)
    b, _, nz, ny, nx = xb.shape
    plan = eq.Plan(nx, ny, nz, dtype, b, op, h, target=target)
    out, y = plan.project_hodge(xb)
    plain = plan.project(xb)
    torch.cuda.synchronize()
    plan.close()
    return (out.double().cpu().numpy(), y.double().cpu().numpy(), plain.double().cpu().numpy())


@pytest.mark.parametrize("op", ["ddo", "cdo"])
def test_16cubed_fp64(op):
    s = field((16, 16, 16), 210501612, grains=8)
    out, y, plain = run_hodge(s, torch.float64, op)
    same_projection(out, plain, torch.float64)
    assert vrel(out, oracle.project(s, op)) <= 1e-12
    ref = oracle.hodge_potential(s, op)
    assert vrel(y[0, :3], ref) <= 1e-12
    assert np.abs(y[0, 3]).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(64, 64, 64), (512, 32, 64), (16, 32, 512)])
def test_fp32_against_the_oracle_and_real_space(shape):
    s = field(shape, 11 + shape[0])
    out, y, plain = run_hodge(s, torch.float32)
    assert np.array_equal(out, plain)
    ref = oracle.hodge_potential(s, "ddo")
    assert vrel(y[0, :3], ref) <= TOL[torch.float32]
    # sym grad y with central differences rebuilds what the projection removed
    sg = oracle.symgrad_field(y[0, :3], (1.0, 1.0, 1.0), "ddo")
    removed = s - out[0]
    w = np.array([1.0, 1, 1, 2, 2, 2]).reshape(6, 1, 1, 1)
    err = math.sqrt(float((w * (sg - removed) ** 2).sum() / (w * removed ** 2).sum()))
    assert err <= 5e-6


@pytest.mark.parametrize("shape,dtype", [((8, 16, 512), torch.float64), ((8, 16, 256), torch.float32),
                                         ((8, 16, 256), torch.float64)])
def test_warp_kernel_rows(shape, dtype):
    # x rows of 256 and 512 points run the potential in the warp-per-row x kernel
    s = field(shape, 40 + shape[2])
    out, y, plain = run_hodge(s, dtype)
    same_projection(out, plain, dtype)
    assert vrel(y[0, :3], oracle.hodge_potential(s, "ddo")) <= TOL[dtype]


def test_batch_spacing_and_compatibility_target_fp64():
    h = (1.0, 0.8, 1.25)
    s = np.stack([field((16, 32, 8), 21), field((16, 32, 8), 22)])
    out, y, plain = run_hodge(s, torch.float64, target="compatibility", h=h)
    same_projection(out, plain, torch.float64)
    for f in range(2):
        assert vrel(y[f, :3], oracle.hodge_potential(s[f], "ddo", h)) <= 1e-12
        assert vrel(out[f], oracle.project_compat(s[f], "ddo", h)) <= 1e-12


def test_runtime_length_plans_and_bad_buffers_are_rejected():
    lib = _lib.load()
    x = torch.zeros(1, 6, 12, 10, 9, device="cuda")
    plan = eq.Plan(9, 10, 12, torch.float32, 1)
    y = torch.zeros(1, 4, 12, 10, 9, device="cuda")
    st = lib.eq_project_hodge(ctypes.c_void_p(plan.handle), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), None)
    assert st == _lib.EQ_ERR_INVALID and b"power-of-two" in lib.eq_last_error()
    plan.close()
    x = torch.zeros(1, 6, 8, 8, 8, device="cuda")
    plan = eq.Plan(8, 8, 8, torch.float32, 1)
    st = lib.eq_project_hodge(ctypes.c_void_p(plan.handle), ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), None)
    assert st == _lib.EQ_ERR_INVALID and b"overlaps" in lib.eq_last_error()
    plan.close()
