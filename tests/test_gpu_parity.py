"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: relative L2 (A:B-weighted, over all voxels) <= 1e-12 for FP64 and <= 2e-6 for FP32; norms
within 1e-10 (FP64) / 1e-5 (FP32) relative; div_out_l2 (round-off level by construction) within
a small multiple of the precision times div_in_l2.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from fieldgen import gaussian_array, voronoi_stress_field, periodic_voronoi_map
import paper_2105_01612_gb300 as eq

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-6}
NTOL = {torch.float64: 1e-10, torch.float32: 1e-5}
EPS = {torch.float64: 2.2e-16, torch.float32: 1.2e-7}
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


def gpu_project(s, dtype, op="ddo", h=(1.0, 1.0, 1.0), nyq="keep", inplace=False):
    x = torch.as_tensor(np.asarray(s)).to(dtype).cuda().contiguous()
    b = x if x.dim() == 5 else x.unsqueeze(0)
    plan = eq.Plan(b.shape[4], b.shape[3], b.shape[2], dtype, b.shape[0], op, h, nyq)
    out = plan.project(b, b if inplace else None)
    nrm = plan.norms()
    plan.close()
    return out.view(x.shape).double().cpu().numpy(), nrm


def check_norms(got, s64, ref_out, op, h, dtype, linf=True):
    want = oracle.norms(s64, ref_out, op, h)
    tol = NTOL[dtype]
    for k in ("norm_in", "norm_out", "resid_l2", "resid_rel", "div_in_l2"):
        assert got[k] == pytest.approx(want[k], rel=tol, abs=tol * want["norm_in"] * 1e-3), k
    if linf:
        assert got["resid_linf"] == pytest.approx(want["resid_linf"], rel=tol,
                                                  abs=100 * EPS[dtype] * np.abs(s64).max()), "linf"
    # the projected spectrum is divergence-free up to round-off of the working precision
    assert got["div_out_l2"] <= 1e3 * EPS[dtype] * want["norm_in"] / min(h), "div_out"
    assert np.allclose(got["mean"], want["mean"], rtol=tol, atol=tol * want["norm_in"])


def field(shape, grains, sigma, noise, seed):
    return voronoi_stress_field(shape, grains, sigma, noise, seed).numpy()


# ------------------------------------------------------------------ configs 1 and 2

@pytest.mark.parametrize("op", ["ddo", "cdo"])
def test_16cubed_fp64_voronoi_8_grains(op):
    s = field((16, 16, 16), 8, 100.0, 10.0, 210501612)
    ref = oracle.project(s, op)
    out, nrm = gpu_project(s, torch.float64, op)
    assert rel(out, ref) <= 1e-12
    check_norms(nrm[0], s, ref, op, (1.0, 1.0, 1.0), torch.float64)
    naive = oracle.project(s, op, transform="direct")
    assert rel(out, naive) <= 1e-12


_CFG2 = {}


def _config2(op):
    """128^3 truth = inc(H) of a smooth random potential (spectrum ~ |k|^-4), RMS 100 MPa, plus a
    200-grain piecewise-constant perturbation ~ N(0, 50 MPa)."""
    if op not in _CFG2:
        shape = (128, 128, 128)
        pot = oracle.smooth_potential(gaussian_array((6,) + shape, 210501613))
        truth = oracle.beltrami_field(pot, op=op)
        truth *= 100.0 / math.sqrt(oracle.frob2(truth).mean())
        delta = field(shape, 200, 50.0, 0.0, 210501614)
        _CFG2[op] = (truth, delta)
    return _CFG2[op]


@pytest.mark.parametrize("op", ["ddo", "cdo"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_128cubed_beltrami_truth_plus_grain_perturbation(op, dtype):
    truth, delta = _config2(op)
    s = truth + delta
    if dtype == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
    ref = oracle.project(s, op)
    out, nrm = gpu_project(s, dtype, op)
    assert rel(out, ref) <= TOL[dtype]
    check_norms(nrm[0], s, ref, op, (1.0, 1.0, 1.0), dtype)
    # recovery error equals the projection of the perturbation (linearity, Sec. 5.1)
    pd, _ = gpu_project(delta, dtype, op)
    err = out - truth
    scale = math.sqrt(oracle.frob2(truth).mean())
    assert math.sqrt(oracle.frob2(err - pd).mean()) <= 10 * TOL[dtype] * scale


# ------------------------------------------------------------------ shapes, options, edge cases

@pytest.mark.parametrize("shape", [(16, 16, 16), (8, 32, 16), (4, 8, 64), (32, 16, 8),
                                   (2, 4, 128), (16, 256, 4), (8, 2, 512), (4, 4, 1024),
                                   (64, 128, 32), (256, 64, 16), (1024, 64, 16)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_shapes(shape, dtype):
    s = field(shape, 6, 100.0, 10.0, sum(shape))
    if dtype == torch.float32:
        s = s.astype(np.float32).astype(np.float64)
    for op in ("ddo", "cdo"):
        h = (1.0, 0.8, 1.3)
        ref = oracle.project(s, op, h)
        out, nrm = gpu_project(s, dtype, op, h)
        assert rel(out, ref) <= TOL[dtype], op
        check_norms(nrm[0], s, ref, op, h, dtype)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 8), (1, 4, 1), (2, 1, 1), (2, 2, 2),
                                   (1, 8, 16), (4, 1, 32)])
def test_degenerate_and_tiny_shapes(shape):
    s = gaussian_array((6,) + shape, 5, 50.0) + 3.0
    for dtype in (torch.float64, torch.float32):
        ss = s.astype(np.float32).astype(np.float64) if dtype == torch.float32 else s
        for nyq in ("keep", "zero"):
            ref = oracle.project(ss, "ddo", nyq=nyq)
            out, _ = gpu_project(ss, dtype, "ddo", nyq=nyq)
            assert rel(out, ref) <= TOL[dtype], (dtype, nyq)


@pytest.mark.parametrize("op", ["ddo", "cdo"])
def test_nyquist_zero_policy_matches_literal_route(op):
    s = field((8, 16, 32), 5, 100.0, 10.0, 77)
    ref = oracle.project_literal(s, op)
    out, _ = gpu_project(s, torch.float64, op, nyq="zero")
    assert rel(out, ref) <= 1e-12


def test_batch_inplace_and_host_entry():
    shape = (16, 32, 64)
    fields = np.stack([field(shape, 7, 100.0, 10.0, 900 + i) for i in range(3)])
    x = torch.as_tensor(fields).cuda()
    plan = eq.Plan(64, 32, 16, torch.float64, 3, "ddo")
    out = plan.project(x)
    nrm = plan.norms()
    for i in range(3):
        ref = oracle.project(fields[i], "ddo")
        assert rel(out[i].cpu().numpy(), ref) <= 1e-12
        check_norms(nrm[i], fields[i], ref, "ddo", (1.0, 1.0, 1.0), torch.float64)
    y = x.clone()
    plan.project(y, y)
    torch.testing.assert_close(y, out, rtol=0, atol=0)
    assert all(n["flags"] & 2 for n in plan.norms())            # no L-inf in place
    hin = x.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    plan.project_host(hin, hout)
    torch.testing.assert_close(hout, out.cpu(), rtol=0, atol=0)
    # asynchronous host entry: two plans on two streams, two fields in flight
    plan2 = eq.Plan(64, 32, 16, torch.float64, 3, "ddo")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.empty_like(hin).pin_memory() for _ in range(4)]
    for k in range(4):
        (plan if k % 2 == 0 else plan2).project_host(hin, outs[k], stream=s1 if k % 2 == 0 else s2,
                                                    wait=False)
    nrm2 = plan2.norms()                                        # waits for plan2's last call
    torch.cuda.synchronize()
    for k in range(4):
        torch.testing.assert_close(outs[k], out.cpu(), rtol=0, atol=0)
    assert nrm2[0]["norm_out"] == nrm[0]["norm_out"]
    plan2.close()
    plan.close()


def test_tma_and_plain_passes_agree(monkeypatch):
    """The TMA / bulk-copy fed passes compute what the plain-load passes compute."""
    s = field((64, 128, 64), 9, 100.0, 10.0, 55)
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("EQ_NO_TMA", flag)
        for dtype in (torch.float32, torch.float64):
            o, n = gpu_project(s, dtype)
            outs.append((dtype, o, n))
    for dtype in (torch.float32, torch.float64):
        a = [o for d, o, _ in outs if d == dtype]
        b = [n for d, _, n in outs if d == dtype]
        # identical transforms; only the FP64 mean substituted at k = 0 can differ in its last
        # bit, because the two first passes reduce it over different block grids
        assert rel(a[0], a[1]) <= 4 * EPS[dtype]
        # the two paths split the FP64 reductions over different block grids
        # (FP32 partials are Kahan-compensated FP32 sums, FP64 ones plain FP64 sums)
        tol = 1e-7 if dtype == torch.float32 else 1e-12
        for k in ("norm_in", "norm_out", "resid_l2", "resid_linf", "div_in_l2"):
            assert b[0][0][k] == pytest.approx(b[1][0][k], rel=tol), k


def test_deterministic_and_nonfinite_flag():
    s = field((32, 32, 32), 9, 100.0, 10.0, 31)
    a, na = gpu_project(s, torch.float32)
    b, nb = gpu_project(s, torch.float32)
    assert np.array_equal(a, b) and na == nb
    s[3, 5, 7, 9] = np.nan
    _, nn = gpu_project(s, torch.float32)
    assert nn[0]["flags"] & 1


def test_errors_surface_as_status():
    with pytest.raises(eq.EqError):
        eq.Plan(2048, 64, 64)
    plan = eq.Plan(16, 16, 16, torch.float32)
    x = torch.zeros(1, 6, 16, 16, 16, device="cuda")
    with pytest.raises(eq.EqError):
        eq.eq_project(plan.handle, x.data_ptr(), x.data_ptr() + 4, 0)   # partial overlap
    plan.close()


# ------------------------------------------------------------------ full size (512^3, FP32)

def test_512cubed_fp32_planes_against_oracle_and_properties():
    """At the benchmark size and launch configuration: (1) a field that is a sum of three
    functions of two coordinates each has its spectrum on the three coordinate planes, so the
    oracle projects it exactly on 512 x 512 slabs; (2) on a Voronoi field, idempotence,
    Pythagoras and zero divergence hold."""
    n = 512
    f_xy = gaussian_array((6, 1, n, n), 1)
    f_yz = gaussian_array((6, n, n, 1), 2)
    f_zx = gaussian_array((6, n, 1, n), 3)
    dev = torch.device("cuda")
    x = (torch.as_tensor(f_xy, dtype=torch.float32, device=dev)
         + torch.as_tensor(f_yz, dtype=torch.float32, device=dev)
         + torch.as_tensor(f_zx, dtype=torch.float32, device=dev)).contiguous()
    # the oracle sees exactly the FP32 values the GPU sees: project each slab separately
    ref = (torch.as_tensor(oracle.project(f_xy.astype(np.float32).astype(np.float64)), device=dev)
           + torch.as_tensor(oracle.project(f_yz.astype(np.float32).astype(np.float64)), device=dev)
           + torch.as_tensor(oracle.project(f_zx.astype(np.float32).astype(np.float64)), device=dev))
    plan = eq.Plan(n, n, n, torch.float32, 1, "ddo")
    out = plan.project(x.unsqueeze(0))[0]
    w = torch.tensor(W, device=dev, dtype=torch.float64).view(6, 1, 1, 1)
    d = out.double() - ref
    err = math.sqrt(float((w * d * d).sum() / (w * ref * ref).sum()))
    # the three slab sums overlap on lines; linearity makes the sum exact
    assert err <= 2e-6, err
    del x, ref, d
    s = voronoi_stress_field((n, n, n), 5000, 200.0, 20.0, 210501614, dtype=torch.float32,
                             device="cuda").unsqueeze(0)
    ps = plan.project(s)
    nr = plan.norms()[0]
    pps = plan.project(ps)
    num = float((w * (pps[0].double() - ps[0].double()) ** 2).sum())
    den = float((w * ps[0].double() ** 2).sum())
    assert math.sqrt(num / den) <= 2e-6
    assert abs(nr["norm_in"] ** 2 - nr["norm_out"] ** 2 - nr["resid_l2"] ** 2) <= 1e-5 * nr["norm_in"] ** 2
    assert nr["div_out_l2"] <= 1e-5 * nr["div_in_l2"]
    assert nr["flags"] == 0
    plan.close()
