"""Parity of eq_project_padded (a non-periodic specimen projected inside a zero-stress buffer,
Sec. 5.2) with the FP64 oracle, through the C ABI."""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field, gaussian_array
import paper_2105_01612_gb300 as eq
from paper_2105_01612_gb300 import _lib

pytestmark = pytest.mark.gpu
W = np.array([1.0, 1, 1, 2, 2, 2])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def rel(a, b):
    w = W.reshape((6,) + (1,) * (np.ndim(a) - 1))
    return math.sqrt(float((w * (a - b) ** 2).sum() / max((w * b ** 2).sum(), 1e-300)))


def run(s, grid, dtype, inplace=False):
    x = torch.as_tensor(np.asarray(s)).to(dtype).cuda().contiguous()
    xb = x if x.dim() == 5 else x.unsqueeze(0)
    nz, ny, nx = grid
    plan = eq.Plan(nx, ny, nz, dtype, xb.shape[0])
    out = plan.project_padded(xb, xb if inplace else None)
    nrm = plan.norms()
    torch.cuda.synchronize()
    plan.close()
    return out.view(x.shape).double().cpu().numpy(), nrm


@pytest.mark.parametrize("spec", [(12, 14, 10), (16, 12, 10)])
def test_fp64_against_the_oracle_with_norms(spec):
    s = voronoi_stress_field(spec, 6, 100.0, 10.0, 70).numpy()
    grid = (16, 16, 16)
    out, nrm = run(s, grid, torch.float64)
    ref = oracle.project_padded(s, grid)
    assert rel(out, ref) <= 1e-12
    big = np.zeros((6,) + grid)
    big[:, :spec[0], :spec[1], :spec[2]] = s
    want = oracle.norms(big, oracle.project(big))
    for k in ("norm_in", "norm_out", "resid_l2", "div_in_l2"):
        assert nrm[0][k] == pytest.approx(want[k], rel=1e-10), k
    assert nrm[0]["resid_linf"] == pytest.approx(float(np.abs(s - ref).max()), rel=1e-10)
    assert not (nrm[0]["flags"] & 2)


def test_fp32_batch_and_in_place():
    spec, grid = (100, 120, 90), (128, 128, 128)
    s = np.stack([voronoi_stress_field(spec, 60, 150.0, 15.0, 71 + f).numpy() for f in range(2)])
    out, nrm = run(s, grid, torch.float32)
    for f in range(2):
        assert rel(out[f], oracle.project_padded(s[f], grid)) <= 2e-6
    out2, _ = run(s, grid, torch.float32, inplace=True)
    assert np.array_equal(out, out2)


def test_equilibrated_specimen_with_compact_stress_function_is_kept():
    shape = (12, 14, 16)
    mask = np.zeros(shape)
    mask[3:-3, 3:-3, 3:-3] = 1.0
    s = oracle.beltrami_field(gaussian_array((6,) + shape, seed=72) * mask)
    out, _ = run(s, (16, 16, 16), torch.float64)
    assert rel(out, s) <= 1e-12


def test_rejections():
    lib = _lib.load()
    x = torch.zeros(1, 6, 8, 8, 8, device="cuda")
    plan = eq.Plan(12, 10, 9, torch.float32, 1)            # runtime lengths
    st = lib.eq_project_padded(ctypes.c_void_p(plan.handle), 8, 8, 8, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), None)
    assert st == _lib.EQ_ERR_INVALID and b"power-of-two" in lib.eq_last_error()
    plan.close()
    plan = eq.Plan(8, 8, 4, torch.float32, 1)
    st = lib.eq_project_padded(ctypes.c_void_p(plan.handle), 8, 8, 8, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), None)
    assert st == _lib.EQ_ERR_INVALID and b"fit" in lib.eq_last_error()
    plan.close()


@pytest.mark.parametrize("spec,grid,dtype", [
    ((100, 120, 92), (128, 128, 128), torch.float32),     # fused: TMA z passes, 16-byte rows
    ((40, 50, 36), (64, 64, 64), torch.float64),
    ((64, 40, 28), (64, 64, 64), torch.float32),          # no padding along z
    ((30, 64, 64), (64, 64, 64), torch.float64),          # padding along z only
])
def test_fused_padding_matches_the_separate_kernels_and_the_oracle(spec, grid, dtype, monkeypatch):
    s = voronoi_stress_field(spec, 20, 150.0, 15.0, 80 + spec[0]).numpy()
    fused, nf = run(s, grid, dtype)
    monkeypatch.setenv("EQ_PAD_UNFUSED", "1")
    sep, ns = run(s, grid, dtype)
    assert np.array_equal(fused, sep)
    for k in ("norm_in", "norm_out", "resid_l2", "resid_linf", "div_in_l2"):
        assert nf[0][k] == ns[0][k], k
    assert rel(fused, oracle.project_padded(s, grid)) <= (1e-12 if dtype == torch.float64 else 2e-6)
