"""Brute-force closest equilibrated field on tiny grids (Sec. 3.2, the argmin problem itself).

No Fourier projector is involved: the divergence is assembled as an explicit real matrix D acting
on all 6 x V stored components, and the minimiser of sum_voxels (S - S_exp):(S - S_exp) subject to
D S = 0 is found by weighted least squares with Lagrange multipliers:

    S = S_exp - W^-1 D^T lam,   (D W^-1 D^T) lam = D S_exp,

with W the Voigt weights (1, 1, 1, 2, 2, 2) of the tensor inner product.  D comes from the
real-space central differences (DDO, eq. eq:diff) or from the spectral derivative (CDO, Sec. 4.1)
applied to unit fields.
"""
from __future__ import annotations

import numpy as np

from .projection import VOIGT_W, divergence, divergence_central_diff


def divergence_matrix(shape, op: str, h) -> np.ndarray:
    """Dense matrix of S -> div S for fields of ``shape`` (nz, ny, nx); size (3V, 6V)."""
    v = int(np.prod(shape))
    cols = []
    for c in range(6):
        for idx in range(v):
            e = np.zeros((6,) + tuple(shape))
            e.reshape(6, v)[c, idx] = 1.0
            d = divergence_central_diff(e, h) if op == "ddo" else divergence(e, op, h)
            cols.append(d.reshape(-1))
    return np.stack(cols, axis=1)


def project_bruteforce(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Closest divergence-free field under A:B, by constrained least squares (tiny grids)."""
    s6 = np.asarray(s6, dtype=np.float64)
    shape = s6.shape[1:]
    v = int(np.prod(shape))
    if v > 512:
        raise ValueError("project_bruteforce is for tiny grids (<= 512 voxels)")
    dmat = divergence_matrix(shape, op, h)
    winv = np.repeat(1.0 / VOIGT_W, v)
    e = s6.reshape(-1)
    a = (dmat * winv[None, :]) @ dmat.T
    lam = np.linalg.lstsq(a, dmat @ e, rcond=1e-12)[0]
    return (e - winv * (dmat.T @ lam)).reshape(s6.shape)
