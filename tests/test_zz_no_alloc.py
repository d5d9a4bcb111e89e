"""eq_project_static: the projection for callers that cannot allocate device memory when they
project (a fixed memory budget, a caller-owned allocator, or a loop where CUDA allocation calls
are not allowed).  Its scratch is a fixed array declared by the library, so the call allocates
nothing; its results must match eq_project's.

This file is named to be collected last, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq
from paper_2105_01612_gb300 import _lib

pytestmark = pytest.mark.gpu

W = torch.tensor([1.0, 1, 1, 2, 2, 2], dtype=torch.float64).view(6, 1, 1, 1)
TOL_F32 = 2e-6          # the FP32 parity bar used by the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def rel(a, b):
    """A:B-weighted relative L2 difference, in FP64 on the tensors' device."""
    w = W.to(a.device)
    a = a.double()
    b = b.double()
    return math.sqrt(float((w * (a - b) ** 2).sum() / (w * b ** 2).sum()))


def static_project(x, out, norms_dev, op="ddo"):
    lib = _lib.load()
    opts = eq._opts(op)
    stream = torch.cuda.current_stream().cuda_stream
    nz, ny, nx = x.shape[-3:]
    st = lib.eq_project_static(nx, ny, nz, ctypes.byref(opts), x.data_ptr(), out.data_ptr(),
                               norms_dev.data_ptr(), stream)
    _lib.check(st, "eq_project_static")


def _field(shape, seed, dev):
    """Voronoi grains for the small grids; a seeded Gaussian field on the device for the large
    ones (any field serves: both entry points see the same tensor)."""
    if shape[0] * shape[1] * shape[2] <= 1 << 18:
        return voronoi_stress_field(shape, 40, 150.0, 10.0, seed, dtype=torch.float32,
                                    device=dev).contiguous()
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    return (100.0 * torch.randn((6,) + shape, generator=g, device=dev, dtype=torch.float32)
            + 5.0).contiguous()


# (nz, ny, nx): a generic grid; degenerate axes (nz = 1 and ny = 2, ny = 1) whose row-pair
# counts take the special cases of the scratch layout; and 512^3, the largest grid accepted,
# whose row-pair list and partials need the most scratch
@pytest.mark.parametrize("shape", [(32, 64, 128), (1, 2, 64), (2, 1, 32), (512, 512, 512)])
def test_static_scratch_entry_point_matches_eq_project_on_two_calls_in_a_row(shape):
    dev = torch.device("cuda")
    norms_dev = torch.zeros(ctypes.sizeof(_lib.EqNorms), dtype=torch.uint8, device=dev)
    plan = eq.Plan(shape[2], shape[1], shape[0], torch.float32, 1, "ddo", device=dev)
    for call, seed in enumerate((2105, 1612)):
        x = _field(shape, seed, dev)
        out_static = torch.empty_like(x)
        static_project(x, out_static, norms_dev)
        out_plan = plan.project(x.unsqueeze(0))[0]
        nrm_plan = plan.norms()[0]
        torch.cuda.synchronize()
        assert rel(out_static, out_plan) <= TOL_F32, f"call {call}"
        got = _lib.EqNorms.from_buffer_copy(bytes(norms_dev.cpu().numpy()))
        for k in ("norm_in", "norm_out", "resid_l2", "resid_linf", "div_in_l2"):
            assert getattr(got, k) == pytest.approx(nrm_plan[k], rel=1e-5), (call, k)
        assert np.allclose(list(got.mean), nrm_plan["mean"], rtol=1e-6, atol=1e-9)
        del x, out_static, out_plan
    plan.close()


def test_static_scratch_entry_point_rejects_grids_beyond_its_limit():
    lib = _lib.load()
    dev = torch.device("cuda")
    x = torch.zeros(6, 2, 2, 1024, dtype=torch.float32, device=dev)
    st = lib.eq_project_static(1024, 2, 2, None, x.data_ptr(), x.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream)
    assert st == _lib.EQ_ERR_INVALID
    assert b"powers of two" in lib.eq_last_error()
