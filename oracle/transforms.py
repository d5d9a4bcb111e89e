"""Discrete Fourier transforms of the oracle (Sec. 4, eqs. eqnFFT / eqniFFT).

The paper's two DFT formulas are garbled (exponent 2 pi i / L instead of 2 pi i / N, a repeated
index, swapped labels, no normalisation).  Reading used here: forward transform unnormalised with
exp(-2 pi i m x / N) per axis, inverse with exp(+2 pi i m x / N) and a factor 1/N per axis.  The
projection's result does not depend on this convention.

Three routes, pinned against each other and against numpy.fft in the tests:
  * ``dft3_naive``  - the full triple sum as one dense matrix (tiny grids only);
  * ``dft3_direct`` - the same sum done one axis at a time, O(N^2) per axis, any N;
  * ``fft3``        - scipy.fft (a library FFT used as one step), for large grids.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft

_WORKERS = max(1, os.cpu_count() or 1)


def _dft_matrix(n: int, sign: int) -> np.ndarray:
    m = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(m, m) / n)


def dft_axis_direct(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """Direct O(N^2) DFT of ``x`` along ``axis`` (1/N applied when ``inverse``)."""
    n = x.shape[axis]
    mat = _dft_matrix(n, +1 if inverse else -1)
    y = np.moveaxis(np.tensordot(mat, np.moveaxis(x, axis, 0), axes=(1, 0)), 0, axis)
    return y / n if inverse else y


def dft3_direct(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """3-D DFT over the last three axes, one direct per-axis DFT after another."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in (-1, -2, -3):
        y = dft_axis_direct(y, ax, inverse)
    return y


def dft3_naive(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """3-D DFT over the last three axes as the literal triple sum over all voxel/mode pairs.

    Builds the (N^3 x N^3) kernel exp(-+2 pi i (mx x/nx + my y/ny + mz z/nz)); for grids with at
    most a few thousand voxels.
    """
    nz, ny, nx = x.shape[-3:]
    if nx * ny * nz > 4096:
        raise ValueError("dft3_naive is for tiny grids (<= 4096 voxels)")
    z, y, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = (np.outer(xx.ravel(), xx.ravel()) / nx + np.outer(y.ravel(), y.ravel()) / ny
          + np.outer(z.ravel(), z.ravel()) / nz)
    sign = 1.0 if inverse else -1.0
    kern = np.exp(sign * 2j * np.pi * ph)
    lead = x.shape[:-3]
    flat = np.asarray(x, dtype=np.complex128).reshape(-1, nx * ny * nz)
    out = flat @ kern.T
    if inverse:
        out /= nx * ny * nz
    return out.reshape(lead + (nz, ny, nx))


def fft3(x: np.ndarray) -> np.ndarray:
    """Forward 3-D DFT over the last three axes (library FFT, complex128)."""
    return scipy.fft.fftn(np.asarray(x, dtype=np.complex128), axes=(-3, -2, -1),
                          workers=_WORKERS)


def ifft3(x: np.ndarray) -> np.ndarray:
    """Inverse 3-D DFT over the last three axes, with the 1/(nx ny nz) factor."""
    return scipy.fft.ifftn(x, axes=(-3, -2, -1), workers=_WORKERS)
