"""Pins of the oracle's compatibility projection and Hodge potential (no GPU).

Each is checked against something other than itself: brute-force least squares over explicit
symmetric gradients, real-space central differences (inc of a compatible field is 0; sym grad of
the potential rebuilds the removed part), fields with a known decomposition, and a planted sign
mistake that the pins must reject.
"""
import numpy as np
import pytest

import oracle
from oracle.projection import VOIGT_IJ, VOIGT_W
from fieldgen import gaussian_array


def _rel(a, b):
    return float(np.sqrt(oracle.frob2(a - b).sum() / max(oracle.frob2(b).sum(), 1e-300)))


def _symgrad_matrix(shape, h):
    """Dense matrix y (3V) -> sym grad y (6V) with periodic central differences (DDO)."""
    v = int(np.prod(shape))
    cols = []
    for i in range(3):
        for idx in range(v):
            e = np.zeros((3,) + tuple(shape))
            e.reshape(3, v)[i, idx] = 1.0
            cols.append(oracle.symgrad_field(e, h, "ddo").reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 2)])
def test_compat_is_the_least_squares_closest_compatible_field(shape):
    # compatible = sym grad y + c (y periodic, c constant): minimise the A:A distance directly
    h = (1.0, 1.0, 1.0)
    s = gaussian_array((6,) + shape, seed=41)
    v = int(np.prod(shape))
    g = _symgrad_matrix(shape, h)
    consts = np.zeros((6 * v, 6))
    for c in range(6):
        consts[c * v:(c + 1) * v, c] = 1.0
    basis = np.concatenate([g, consts], axis=1)
    sw = np.repeat(np.sqrt(VOIGT_W), v)                       # rows weighted by sqrt(w)
    coef, *_ = np.linalg.lstsq(basis * sw[:, None], s.reshape(-1) * sw, rcond=None)
    best = (basis @ coef).reshape(s.shape)
    assert _rel(oracle.project_compat(s, "ddo", h), best) < 1e-12


@pytest.mark.parametrize("shape", [(6, 8, 10), (7, 9, 5)])
def test_compat_keeps_symmetric_gradients_and_maps_equilibrated_fields_to_their_mean(shape):
    h = (1.0, 0.8, 1.3)
    c = np.arange(1.0, 7.0)[:, None, None, None]
    a = gaussian_array((3,) + shape, seed=5)
    sg = oracle.symgrad_field(a, h, "ddo") + c
    assert _rel(oracle.project_compat(sg, "ddo", h), sg) < 1e-12
    hpot = oracle.smooth_potential(gaussian_array((6,) + shape, seed=6))
    eq = oracle.beltrami_field(hpot, h, "ddo") + c
    out = oracle.project_compat(eq, "ddo", h)
    assert np.abs(out - np.broadcast_to(c, out.shape)).max() < 1e-10 * np.abs(eq).max()


def test_compat_output_is_compatible_by_central_differences():
    # inc of a compatible field vanishes; checked in real space without any FFT
    s = gaussian_array((6, 8, 6, 10), seed=7)
    out = oracle.project_compat(s, "ddo")
    inc = oracle.inc_central_diff(out)
    assert np.abs(inc).max() < 1e-11 * np.abs(s).max()
    # and the two projections split the field: P S + C S = S + c0
    c0 = s.mean(axis=(1, 2, 3))[:, None, None, None]
    assert _rel(oracle.project(s, "ddo") + out, s + c0) < 1e-13
    # idempotent
    assert _rel(oracle.project_compat(out, "ddo"), out) < 1e-12


@pytest.mark.parametrize("op", ["ddo", "cdo"])
def test_potential_rebuilds_the_removed_part(op):
    h = (1.0, 1.2, 0.9)
    s = gaussian_array((6, 6, 8, 10), seed=8)
    y = oracle.hodge_potential(s, op, h)
    removed = s - oracle.project(s, op, h)
    assert _rel(oracle.symgrad_field(y, h, op), removed) < 1e-12
    assert np.abs(y.mean(axis=(1, 2, 3))).max() < 1e-12 * np.abs(y).max()


def test_potential_recovers_the_generating_vector_field_on_odd_grids():
    # odd sizes: Xi = 0 only at k = 0, so sym grad is injective on mean-free fields
    a = gaussian_array((3, 5, 7, 9), seed=9)
    a -= a.mean(axis=(1, 2, 3), keepdims=True)
    y = oracle.hodge_potential(oracle.symgrad_field(a, (1.0, 1.0, 1.0), "ddo"), "ddo")
    assert np.abs(y - a).max() < 1e-11 * np.abs(a).max()


def test_planted_sign_mistake_in_the_potential_is_caught():
    s = gaussian_array((6, 6, 8, 10), seed=10)
    y = oracle.hodge_potential(s, "ddo")
    removed = s - oracle.project(s, "ddo")
    assert _rel(oracle.symgrad_field(-y, (1.0, 1.0, 1.0), "ddo"), removed) > 1.0
