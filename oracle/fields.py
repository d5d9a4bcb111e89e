"""Fields with a known projection, built from the Hodge decomposition (Sec. 3.1, Theorem 2).

* ``beltrami_field``: inc(H) of a symmetric potential H; it is divergence-free, so the projection
  leaves it unchanged (Sec. 3.2; the divergence-free perturbation case of Sec. 5.1, Fig. 3c,d).
* ``symgrad_field``: (D a + (D a)^T)/2 of a vector field a; the projection removes it entirely
  (the symmetrised-gradient perturbation of Sec. 5.1, Fig. 3a,b).

For DDO both are built in real space with periodic central differences (eq. eq:diff), with no
Fourier transform, so they test the spectral projector against an independent construction.
For CDO they are built with the spectral derivative i Xi.
"""
from __future__ import annotations

import numpy as np

from .operators import central_diff, wavevector_grids
from .transforms import fft3, ifft3
from .projection import VOIGT_IJ, to_tensor, to_voigt, _EPS


def _deriv(f: np.ndarray, axis_xyz: int, h, op: str) -> np.ndarray:
    if op == "ddo":
        return central_diff(f, axis_xyz, h[axis_xyz])
    xi = wavevector_grids(f.shape[-3:], h, op)[axis_xyz]
    return np.real(ifft3(1j * xi * fft3(f)))


def inc_central_diff(h6: np.ndarray, h=(1.0, 1.0, 1.0), op: str = "ddo") -> np.ndarray:
    """(inc H)_kn = eps_ijk eps_lmn d_i d_l H_jm (Theorem 2) with the operator's derivative."""
    t = to_tensor(np.asarray(h6, dtype=np.float64))
    out = np.zeros_like(t)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                if _EPS[i, j, k] == 0.0:
                    continue
                for l in range(3):
                    for m in range(3):
                        for n in range(3):
                            e = _EPS[i, j, k] * _EPS[l, m, n]
                            if e == 0.0:
                                continue
                            out[k, n] += e * _deriv(_deriv(t[j, m], l, h, op), i, h, op)
    return to_voigt(out)


def beltrami_field(h6: np.ndarray, h=(1.0, 1.0, 1.0), op: str = "ddo") -> np.ndarray:
    """An equilibrated field: inc(H) for the symmetric potential ``h6`` (6 Voigt components)."""
    return inc_central_diff(h6, h, op)


def symgrad_field(a3: np.ndarray, h=(1.0, 1.0, 1.0), op: str = "ddo") -> np.ndarray:
    """(D a + (D a)^T) / 2 of a vector field ``a3`` of shape (3, nz, ny, nx), as Voigt."""
    a3 = np.asarray(a3, dtype=np.float64)
    return np.stack([0.5 * (_deriv(a3[i], j, h, op) + _deriv(a3[j], i, h, op))
                     for (i, j) in VOIGT_IJ])


def smooth_potential(white6: np.ndarray, power: float = 4.0) -> np.ndarray:
    """Smooth random symmetric potential: white noise filtered by |m|^-power (m the signed
    integer frequency vector, m != 0; the mean is removed)."""
    shape = white6.shape[-3:]
    nz, ny, nx = shape
    fz = np.fft.fftfreq(nz) * nz
    fy = np.fft.fftfreq(ny) * ny
    fx = np.fft.fftfreq(nx) * nx
    m2 = fz[:, None, None] ** 2 + fy[None, :, None] ** 2 + fx[None, None, :] ** 2
    filt = np.where(m2 > 0, np.where(m2 > 0, m2, 1.0) ** (-power / 2.0), 0.0)
    return np.real(ifft3(fft3(white6) * filt))
