"""Pins of the oracle's grain averaging (Sec. 5.1) against things other than itself: a plain
voxel-by-voxel loop, fields that are constant per grain, the total sum, idempotence, and a
planted off-by-one in the grain ids."""
import numpy as np

import oracle
from fieldgen import gaussian_array, periodic_voronoi_map


def _loop_means(s6, gmap, ngrains):
    sums = np.zeros((ngrains, 6))
    counts = np.zeros(ngrains)
    nz, ny, nx = gmap.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                g = gmap[z, y, x]
                counts[g] += 1
                sums[g] += s6[:, z, y, x]
    return np.where(counts[:, None] > 0, sums / np.maximum(counts, 1)[:, None], 0.0)


def test_means_equal_a_voxel_loop_including_an_empty_grain():
    gmap = periodic_voronoi_map((6, 7, 8), 9, seed=3).numpy()
    gmap = np.where(gmap == 4, 5, gmap)                   # grain 4 left empty
    s = gaussian_array((6, 6, 7, 8), seed=4)
    got = oracle.grain_means(s, gmap, 10)
    assert np.allclose(got, _loop_means(s, gmap, 10), rtol=1e-13, atol=1e-14)
    assert np.all(got[4] == 0.0) and np.all(got[9] == 0.0)


def test_piecewise_constant_fields_are_fixed_points_and_sums_are_kept():
    gmap = periodic_voronoi_map((8, 8, 8), 12, seed=5).numpy()
    vals = gaussian_array((12, 6), seed=6)
    s = np.stack([vals[:, c][gmap] for c in range(6)])
    assert np.allclose(oracle.grain_average(s, gmap, 12), s, rtol=0, atol=1e-14)
    noisy = s + gaussian_array(s.shape, seed=7)
    avg = oracle.grain_average(noisy, gmap, 12)
    assert np.allclose(avg.sum(axis=(1, 2, 3)), noisy.sum(axis=(1, 2, 3)), rtol=1e-12)
    assert np.allclose(oracle.grain_average(avg, gmap, 12), avg, rtol=0, atol=1e-13)


def test_planted_off_by_one_grain_id_is_caught():
    gmap = periodic_voronoi_map((6, 6, 6), 8, seed=8).numpy()
    s = gaussian_array((6, 6, 6, 6), seed=9)
    good = oracle.grain_means(s, gmap, 8)
    bad = oracle.grain_means(s, (gmap + 1) % 8, 8)
    assert not np.allclose(good, bad)
    assert np.allclose(good, _loop_means(s, gmap, 8), rtol=1e-13, atol=1e-14)
