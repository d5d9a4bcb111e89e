"""Grain averaging of a stress field (test infrastructure: only tests, smoke() and the bench's
CPU baseline use this package).

Sec. 5.1 builds its synthetic measurement by averaging the equilibrated stress over each grain
of a Voronoi polycrystal ("grain-averaged stress field"), the kind of data a grain-resolved
diffraction reconstruction provides, and then projects it (Table 1, Fig. 4).  By definition the
mean of grain g is the sum of the field over the voxels whose grain id is g divided by their
count; the grain-averaged field puts that mean on every voxel of the grain.

Reading where the paper is silent (listed in the design notes): a grain id with no voxel has
mean 0.
"""
from __future__ import annotations

import numpy as np


def grain_means(s6: np.ndarray, gmap: np.ndarray, ngrains: int) -> np.ndarray:
    """(ngrains, 6) float64 means of the Voigt components of ``s6`` (6, nz, ny, nx) per grain id
    of ``gmap`` (nz, ny, nx), ids in [0, ngrains)."""
    s6 = np.asarray(s6, dtype=np.float64)
    g = np.asarray(gmap).reshape(-1)
    counts = np.bincount(g, minlength=ngrains).astype(np.float64)
    out = np.zeros((ngrains, 6))
    for c in range(6):
        sums = np.bincount(g, weights=s6[c].reshape(-1), minlength=ngrains)
        out[:, c] = np.where(counts > 0, sums / np.where(counts > 0, counts, 1.0), 0.0)
    return out


def grain_average(s6: np.ndarray, gmap: np.ndarray, ngrains: int) -> np.ndarray:
    """The grain-averaged field: every voxel carries the mean of its grain (6, nz, ny, nx)."""
    m = grain_means(s6, gmap, ngrains)
    return np.stack([m[:, c][np.asarray(gmap)] for c in range(6)])
