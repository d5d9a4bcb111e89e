"""Parity of the runtime-length path (mixed radix 2..13 and Bluestein) and of uneven batches
(one launch per pass over all fields) with the FP64 CPU oracle."""
import json
import math

import numpy as np
import pytest
import torch

import oracle
from fieldgen import voronoi_stress_field
import paper_2105_01612_gb300 as eq

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-6}
W = np.array([1.0, 1, 1, 2, 2, 2])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def rel(a, b):
    w = W.reshape((6,) + (1,) * (np.ndim(a) - 1))
    return math.sqrt(float((w * (a - b) ** 2).sum() / max((w * b ** 2).sum(), 1e-300)))


def as_dtype(s, dtype):
    return s.astype(np.float32).astype(np.float64) if dtype == torch.float32 else s


@pytest.mark.parametrize("shape", [(3, 5, 7), (6, 10, 9), (26, 13, 11), (23, 19, 17), (4, 34, 67),
                                   (2, 3, 97), (5, 2, 250), (37, 31, 33), (1, 1, 7), (7, 1, 1),
                                   # power-of-two transform lengths (the fixed-size register
                                   # FFT): Bluestein convolutions of 128, 256 and 512 points on
                                   # each axis, and direct transforms of 128 and 256 points
                                   (139, 3, 5), (4, 151, 6), (3, 2, 179), (47, 90, 5), (256, 6, 5),
                                   (3, 128, 4), (5, 3, 256)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_any_size_matches_oracle(shape, dtype):
    s = as_dtype(voronoi_stress_field(shape, 5, 100.0, 10.0, sum(shape)).numpy(), dtype)
    for op, nyq, h in (("ddo", "keep", (1.0, 1.0, 1.0)), ("cdo", "zero", (0.7, 1.1, 1.3))):
        ref = oracle.project(s, op, h, nyq)
        x = torch.as_tensor(s).to(dtype).cuda().unsqueeze(0)
        plan = eq.Plan(shape[2], shape[1], shape[0], dtype, 1, op, h, nyq)
        out = plan.project(x)
        nrm = plan.norms()[0]
        plan.close()
        got = out[0].double().cpu().numpy()
        assert rel(got, ref) <= TOL[dtype], (op, nyq)
        want = oracle.norms(s, ref, op, h)
        for k in ("norm_in", "norm_out", "resid_l2", "div_in_l2"):
            assert nrm[k] == pytest.approx(want[k], rel=10 * TOL[dtype] + 1e-12, abs=1e-9), k


def _varlen_run(dims, dtype, seed0, op="ddo"):
    fields = [voronoi_stress_field((nz, ny, nx), 7, 150.0, 5.0, seed0 + i, dtype=dtype).numpy()
              for i, (nx, ny, nz) in enumerate(dims)]
    plan = eq.VarlenPlan(dims, dtype, op)
    flat = plan.pack([torch.as_tensor(f) for f in fields])
    out = torch.empty_like(flat)
    plan.project(flat, out)
    nrm = plan.norms()
    outs = [o.double().cpu().numpy() for o in plan.unpack(out)]
    plan.close()
    return fields, outs, nrm


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_uneven_batch_matches_oracle_and_single_runs(dtype):
    dims = [(16, 16, 16), (12, 20, 9), (33, 7, 14), (64, 8, 8), (5, 97, 3), (30, 30, 30)]
    fields, outs, nrm = _varlen_run(dims, dtype, 4000)
    for i, (f, o) in enumerate(zip(fields, outs)):
        f64 = f.astype(np.float64)
        ref = oracle.project(f64, "ddo")
        assert rel(o, ref) <= TOL[dtype], dims[i]
        want = oracle.norms(f64, ref, "ddo")
        assert nrm[i]["resid_rel"] == pytest.approx(want["resid_rel"], rel=1e-5)
        # the field alone gives the same output bits as inside the batch
        _, alone, _ = _varlen_run([dims[i]], dtype, 4000 + i)
        assert np.array_equal(alone[0], o), dims[i]


def test_batch_of_64_uneven_fields_config_sizes_sampled():
    """Uneven batch at the sizes of the 64-field workload (each axis uniform in 64..256, FP32):
    every field's norms are consistent and two sampled fields match the oracle."""
    rng = np.random.Generator(np.random.PCG64(210501612 + 3))
    dims = [tuple(int(v) for v in rng.integers(64, 257, size=3)) for _ in range(64)]
    grains = [int(g) for g in rng.integers(50, 2001, size=64)]
    plan = eq.VarlenPlan(dims, torch.float32, "ddo")
    fields = [voronoi_stress_field((nz, ny, nx), grains[i], 150.0, 0.0, 5000 + i,
                                   dtype=torch.float32, device="cuda")
              for i, (nx, ny, nz) in enumerate(dims)]
    flat = plan.pack(fields)
    out = torch.empty_like(flat)
    plan.project(flat, out)
    nrm = plan.norms()
    outs = plan.unpack(out)
    for i in (0, 37):
        f = fields[i].double().cpu().numpy()
        ref = oracle.project(f, "ddo")
        assert rel(outs[i].double().cpu().numpy(), ref) <= 2e-6, dims[i]
    for n in nrm:
        assert abs(n["norm_in"] ** 2 - n["norm_out"] ** 2 - n["resid_l2"] ** 2) <= 1e-5 * n["norm_in"] ** 2
        assert n["div_out_l2"] <= 1e-5 * n["div_in_l2"]
    plan.close()


def test_autotune_keeps_results_and_writes_the_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("EQ_TUNE_CACHE", str(cache))
    dims = [(24, 20, 18), (33, 16, 40), (64, 12, 10)]
    fields, ref_outs, _ = _varlen_run(dims, torch.float32, 6000)
    plan = eq.VarlenPlan(dims, torch.float32, "ddo")
    flat = plan.pack([torch.as_tensor(f) for f in fields])
    out = torch.empty_like(flat)
    plan.autotune(flat, out)
    plan.project(flat, out)
    for o, r in zip(plan.unpack(out), ref_outs):
        assert rel(o.double().cpu().numpy(), r) <= 2e-6
    plan.close()
    txt = cache.read_text()
    assert txt.strip().startswith("{") and "gen|f32" in txt
    # a new plan with the same key starts from the cached shapes and still matches
    _, again, _ = _varlen_run(dims, torch.float32, 6000)
    for a, r in zip(again, ref_outs):
        assert rel(a, r) <= 2e-6
    # power-of-two plan: TMA / plain choice per pass
    s = voronoi_stress_field((64, 64, 64), 9, 100.0, 5.0, 61).numpy()
    x = torch.as_tensor(s).float().cuda().unsqueeze(0)
    p2 = eq.Plan(64, 64, 64, torch.float32)
    y = torch.empty_like(x)
    p2.autotune(x, y)
    p2.project(x, y)
    assert rel(y[0].double().cpu().numpy(), oracle.project(x[0].double().cpu().numpy(), "ddo")) <= 2e-6
    p2.close()


@pytest.mark.parametrize("dims", [(32, 32, 32), (30, 20, 18)])
def test_pass_timing_covers_the_asked_calls_then_turns_off(dims):
    nx, ny, nz = dims
    x = torch.randn(1, 6, nz, ny, nx, device="cuda")
    plan = eq.Plan(nx, ny, nz, torch.float32, 1)
    ref = plan.project(x)
    plan.set_timing(2)
    for _ in range(2):
        out = plan.project(x)
    ms, n = plan.pass_ms()
    assert n == 2 and all(v >= 0.0 for v in ms.values()) and sum(ms.values()) > 0.0
    plan.project(x, out)                              # after pass_ms: untimed again
    _, n2 = plan.pass_ms()
    assert n2 == 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    plan.close()


def test_every_pass_kernel_choice_matches_the_oracle(tmp_path, monkeypatch):
    """The tuning cache picks each pass's kernel: the shared-memory strided kernel or the
    warp-per-column one (z, y), the shared-memory x kernel, the warp-per-row one or the
    warp-per-plane-pair one.  Every
    combination gives the oracle's result on lengths served directly (256) and by Bluestein
    (18..130 through 256- and 512-point transforms); an entry that does not fit is passed over."""
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("EQ_TUNE_CACHE", str(cache))
    dims = [(24, 20, 18), (33, 16, 40), (64, 12, 10), (130, 5, 256), (7, 256, 129)]
    fields = [voronoi_stress_field((nz, ny, nx), 6, 100.0, 5.0, 7100 + i, dtype=torch.float32)
              for i, (nx, ny, nz) in enumerate(dims)]
    refs = [oracle.project(f.double().numpy(), "ddo") for f in fields]
    plan = eq.VarlenPlan(dims, torch.float32, "ddo")
    flat = plan.pack([f.cuda() for f in fields])
    out = torch.empty_like(flat)
    plan.autotune(flat, out)
    plan.close()
    key = json.loads(cache.read_text())
    assert len(key) == 1
    key = next(iter(key))
    for zc, yc, xp in [(0, 0, 4), (0, 0, 0), (16, 16, 2), (0, 8, 2), (8, 0, 0), (0, 0, 1), (16, 8, 4)]:
        cache.write_text(json.dumps({key: [zc, 256, yc, 256, xp]}))
        plan = eq.VarlenPlan(dims, torch.float32, "ddo")
        out = torch.empty_like(flat)
        plan.project(flat, out)
        nrm = plan.norms()
        for i, (o, r) in enumerate(zip(plan.unpack(out), refs)):
            assert rel(o.double().cpu().numpy(), r) <= 2e-6, (zc, yc, xp, dims[i])
            assert nrm[i]["div_out_l2"] <= 1e-5 * nrm[i]["div_in_l2"]
        plan.close()
    # a stale entry (a shape that does not fit) falls back to the default shapes
    cache.write_text(json.dumps({key: [999, 256, 0, 256, 0]}))
    plan = eq.VarlenPlan(dims, torch.float32, "ddo")
    out = torch.empty_like(flat)
    plan.project(flat, out)
    for o, r in zip(plan.unpack(out), refs):
        assert rel(o.double().cpu().numpy(), r) <= 2e-6
    plan.close()


def test_fp64_runtime_length_plans_in_double_float_match_the_oracle(monkeypatch):
    """FP64 runtime-length plans whose lengths are 512 or at most 256 run every pass in
    double-float arithmetic (FP64 at the ends, FP32 pairs between the passes).  Their results and
    norms agree with the FP64 oracle to 1e-12 and with the FP64-instruction passes to 1e-13."""
    dims = [(24, 20, 18), (130, 5, 256), (7, 256, 129), (512, 4, 6), (1, 1, 7)]
    fields = [voronoi_stress_field((nz, ny, nx), 6, 100.0, 5.0, 7300 + i, dtype=torch.float64)
              for i, (nx, ny, nz) in enumerate(dims)]
    results = {}
    for arith in ("native", "paired"):
        if arith == "native":
            monkeypatch.setenv("EQ_F64_ARITH", "native")
        else:
            monkeypatch.delenv("EQ_F64_ARITH", raising=False)
        plan = eq.VarlenPlan(dims, torch.float64, "ddo")
        flat = plan.pack([f.cuda() for f in fields])
        out = torch.empty_like(flat)
        plan.project(flat, out)
        results[arith] = ([o.cpu().numpy() for o in plan.unpack(out)], plan.norms())
        plan.close()
    for i, f in enumerate(fields):
        ref = oracle.project(f.numpy(), "ddo")
        ref_n = oracle.norms(f.numpy(), ref, "ddo")
        o, nrm = results["paired"][0][i], results["paired"][1][i]
        assert rel(o, ref) <= 1e-12, dims[i]
        assert rel(o, results["native"][0][i]) <= 1e-13, dims[i]
        for k in ("norm_in", "norm_out", "resid_l2"):
            assert abs(nrm[k] - ref_n[k]) <= 1e-12 * ref_n["norm_in"], (dims[i], k)
        assert nrm["div_out_l2"] <= 1e-12 * nrm["div_in_l2"]


def test_fp64_power_of_two_plan_autotune_then_plain_and_hodge():
    """An FP64 power-of-two plan tunes the variants of its own (FP64-instruction) passes, which
    its Hodge form runs, while plain projections go through its double-float sub-plan: both stay
    within 1e-12 of the oracle after tuning."""
    s = voronoi_stress_field((64, 64, 64), 9, 100.0, 5.0, 67).numpy()
    x = torch.as_tensor(s).cuda().unsqueeze(0)
    p = eq.Plan(64, 64, 64, torch.float64)
    y = torch.empty_like(x)
    p.autotune(x, y)
    p.project(x, y)
    ref = oracle.project(s, "ddo")
    assert rel(y[0].cpu().numpy(), ref) <= 1e-12
    out, pot = p.project_hodge(x)
    assert rel(out[0].cpu().numpy(), ref) <= 1e-12
    yref = oracle.hodge_potential(s, "ddo")
    assert np.linalg.norm(pot[0, :3].cpu().numpy() - yref) <= 1e-11 * np.linalg.norm(yref)
    p.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_lengths_beyond_the_register_transforms_take_the_shared_memory_kernels(dtype):
    """Lengths between 256 and 1024 other than 512 have no 256- or 512-point register transform:
    such plans run the shared-memory mixed-radix / Bluestein kernels (and FP64 keeps FP64
    instructions) and still give the oracle's result."""
    dims = [(300, 4, 5), (6, 7, 263), (9, 270, 3)]
    fields, outs, nrm = _varlen_run(dims, dtype, 7700)
    for i, f in enumerate(fields):
        ref = oracle.project(f.astype(np.float64), "ddo")
        assert rel(outs[i], ref) <= TOL[dtype], dims[i]
        assert nrm[i]["div_out_l2"] <= (1e-12 if dtype == torch.float64 else 1e-5) * nrm[i]["div_in_l2"]
