"""Pins of the oracle's buffered (non-periodic) projection against things other than itself:
no padding is the periodic projection, an equilibrated specimen whose stress function vanishes
near its boundary comes back unchanged (built in real space, no FFT), and placing the specimen
elsewhere in the buffer (a periodic shift) changes nothing."""
import numpy as np

import oracle
from fieldgen import gaussian_array


def _rel(a, b):
    return float(np.sqrt(oracle.frob2(a - b).sum() / max(oracle.frob2(b).sum(), 1e-300)))


def test_no_padding_is_the_periodic_projection():
    s = gaussian_array((6, 8, 6, 10), seed=60)
    assert _rel(oracle.project_padded(s, (8, 6, 10)), oracle.project(s)) < 1e-14


def test_equilibrated_specimen_with_a_compact_stress_function_is_unchanged():
    # H vanishes within 3 voxels of the specimen faces, so inc(H) (central differences) is the
    # same on the specimen and on the padded grid, and it is equilibrated there
    shape = (12, 14, 16)
    hpot = gaussian_array((6,) + shape, seed=61)
    mask = np.zeros(shape)
    mask[3:-3, 3:-3, 3:-3] = 1.0
    s = oracle.beltrami_field(hpot * mask)
    assert np.abs(s[:, 0]).max() == 0.0 and np.abs(s[:, -1]).max() == 0.0
    out = oracle.project_padded(s, (16, 24, 20))
    assert _rel(out, s) < 1e-12


def test_position_of_the_specimen_in_the_buffer_does_not_matter():
    s = gaussian_array((6, 6, 8, 10), seed=62)
    grid = (10, 12, 16)
    corner = oracle.project_padded(s, grid)
    big = np.zeros((6,) + grid)
    big[:, 2:8, 3:11, 4:14] = s
    centred = oracle.project(big)[:, 2:8, 3:11, 4:14]
    assert _rel(centred, corner) < 1e-13
    # and the buffer changes the answer compared with treating the specimen as periodic
    assert _rel(corner, oracle.project(s)) > 1e-3
