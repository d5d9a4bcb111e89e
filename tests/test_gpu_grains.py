"""Grain averaging on the GPU (Sec. 5.1) against the FP64 oracle, through the C ABI, and the
grain-averaged recovery workload of Table 1 (grain-average an equilibrated field, then project
it) end to end."""
import numpy as np
import pytest
import torch

import oracle
from fieldgen import periodic_voronoi_map, voronoi_stress_field, gaussian_array
import paper_2105_01612_gb300 as eq

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2105_01612_gb300 import _build
    _build.build()


def _map(shape, n, seed, empty=None):
    g = periodic_voronoi_map(shape, n, seed=seed).numpy()
    if empty is not None:
        g = np.where(g == empty, (empty + 1) % n, g)
    return g


def _scattered_map(shape, n, seed, empty):
    # an independent id per voxel: no spatial coherence at all (Voronoi grains are compact)
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.integers(0, n, size=shape).astype(np.int32)
    return np.where(g == empty, (empty + 1) % n, g)


@pytest.mark.parametrize("kind", ["voronoi", "scattered"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_means_and_field_match_the_oracle_batch_of_two(dtype, kind):
    shape = (24, 20, 28)
    gmap = _map(shape, 40, 12, empty=7) if kind == "voronoi" else _scattered_map(shape, 40, 12, 7)
    s = np.stack([voronoi_stress_field(shape, 30, 100.0, 10.0, 31 + f).numpy() for f in range(2)])
    gr = eq.Grains(gmap, 41)                       # ids 7 and 40 have no voxel
    x = torch.as_tensor(s).to(dtype).cuda().contiguous()
    means, avg = gr.average(x)
    torch.cuda.synchronize()
    xs = x.double().cpu().numpy()                 # the values the GPU actually averaged
    for f in range(2):
        want = oracle.grain_means(xs[f], gmap, 41)
        got = means[f].cpu().numpy()
        # FP64 data: FP64 sums; FP32 data: compensated FP32 per thread, FP64 across threads
        mtol = 1e-12 if dtype == torch.float64 else 2e-6
        assert np.abs(got - want).max() <= mtol * np.abs(want).max()
        assert np.all(got[7] == 0.0) and np.all(got[40] == 0.0)
        ref = oracle.grain_average(xs[f], gmap, 41)
        tol = 1e-13 if dtype == torch.float64 else 2e-6
        assert np.abs(avg[f].double().cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    # fixed-order sums: a second call gives the same bits; in place gives the same field
    means2, _ = gr.average(x)
    x2 = x.clone()
    gr.average(x2, out=x2)
    torch.cuda.synchronize()
    assert torch.equal(means, means2)
    assert torch.equal(x2, avg)
    gr.close()


def test_grain_averaged_recovery_workload_fp32():
    # Sec. 5.1 / Table 1 on synthetic grains: an equilibrated truth, its grain average, and the
    # projection of the grain average, each step on the GPU, against the oracle's pipeline
    shape = (32, 32, 32)
    truth = oracle.beltrami_field(oracle.smooth_potential(gaussian_array((6,) + shape, seed=50)))
    truth *= 100.0 / np.sqrt(oracle.frob2(truth).mean())
    gmap = _map(shape, 100, 51)
    gr = eq.Grains(gmap, 100)
    x = torch.as_tensor(truth).float().cuda().unsqueeze(0).contiguous()
    _, avg = gr.average(x)
    rec, _ = eq.project(avg)
    torch.cuda.synchronize()
    ref_avg = oracle.grain_average(x[0].double().cpu().numpy(), gmap, 100)
    ref_rec = oracle.project(ref_avg, "ddo")
    w = np.array([1.0, 1, 1, 2, 2, 2]).reshape(6, 1, 1, 1)
    got = rec[0].double().cpu().numpy()
    err = np.sqrt((w * (got - ref_rec) ** 2).sum() / (w * ref_rec ** 2).sum())
    assert err <= 2e-6
    # the recovery is closer to the truth than the grain average it started from
    e_avg = np.sqrt((w * (ref_avg - truth) ** 2).sum())
    e_rec = np.sqrt((w * (got - truth) ** 2).sum())
    assert e_rec < e_avg
    gr.close()
