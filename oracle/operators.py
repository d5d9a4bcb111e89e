"""Differential operators of Sec. 4: the CDO wavevector (Sec. 4.1), the DDO modified wavevector
from central differences (Sec. 4.2, eq. eq:diff), and the consistent 25-point biharmonic stencil
with its Fourier symbol (end of Sec. 4.2).
"""
from __future__ import annotations

import numpy as np


def wavevector(n: int, h: float, op: str) -> np.ndarray:
    """Per-axis symbol Xi[m], m = 0..n-1, such that d/dx <-> i Xi (float64).

    CDO (Sec. 4.1, eq. eq:cdo and the case list after it): Xi = 2 pi s / (n h) with the signed
    frequency s = m for m < n/2 and s = m - n for m > n/2; the Nyquist index m = n/2 (even n)
    gets Xi = 0.  The paper writes the cases with a 1-based index; read with 0-based m.
    DDO (Sec. 4.2, eq. eq:diff and the substitution after it): the central difference
    (f(i+1) - f(i-1)) / (2h) has symbol i sin(2 pi m / n) / h, so Xi = sin(2 pi m / n) / h (the
    paper's (m - 1) is its 1-based index).
    """
    m = np.arange(n, dtype=np.float64)
    s = np.where(m < n / 2.0, m, m - n)
    if op == "cdo":
        xi = 2.0 * np.pi * s / (n * h)
    elif op == "ddo":
        # sin(2 pi m / n) = sin(2 pi s / n); the signed form makes Xi[n - m] = -Xi[m] exactly
        xi = np.sin(2.0 * np.pi * s / n) / h
    else:
        raise ValueError(f"unknown operator {op!r}")
    if n % 2 == 0:
        xi[n // 2] = 0.0        # exact zero (sin(pi) is not 0 in floating point)
    return xi


def wavevector_grids(shape, h, op: str):
    """Broadcastable grids (Xi_x, Xi_y, Xi_z) for a grid ``(nz, ny, nx)``, spacing (hx, hy, hz)."""
    nz, ny, nx = shape
    hx, hy, hz = h
    xi_x = wavevector(nx, hx, op)[None, None, :]
    xi_y = wavevector(ny, hy, op)[None, :, None]
    xi_z = wavevector(nz, hz, op)[:, None, None]
    return xi_x, xi_y, xi_z


def biharmonic_symbol_paper(shape, h: float) -> np.ndarray:
    """Fourier symbol of the 25-point biharmonic stencil as the paper prints it (Sec. 4.2).

    (42 - 24 sum_j cos(4 pi m_j / N_j) + 2 sum_j cos(8 pi m_j / N_j)
        + 8 sum_{j<l} cos(4 pi m_j / N_j) cos(4 pi m_l / N_l)) / (16 h^4)
    The printed left-hand side xi_x^4 + xi_y^4 + xi_z^4 and the misplaced parenthesis are read
    as (sum_j xi_j^2)^2 with every cosine term inside the bracket; one spacing h as in the paper.
    """
    nz, ny, nx = shape
    cz = np.cos(4 * np.pi * np.arange(nz) / nz)[:, None, None]
    cy = np.cos(4 * np.pi * np.arange(ny) / ny)[None, :, None]
    cx = np.cos(4 * np.pi * np.arange(nx) / nx)[None, None, :]
    c2z = np.cos(8 * np.pi * np.arange(nz) / nz)[:, None, None]
    c2y = np.cos(8 * np.pi * np.arange(ny) / ny)[None, :, None]
    c2x = np.cos(8 * np.pi * np.arange(nx) / nx)[None, None, :]
    val = (42.0 - 24.0 * (cx + cy + cz) + 2.0 * (c2x + c2y + c2z)
           + 8.0 * (cx * cy + cy * cz + cx * cz))
    return val / (16.0 * h ** 4)


def central_diff(f: np.ndarray, axis_xyz: int, h: float) -> np.ndarray:
    """Periodic central difference (f(i+1) - f(i-1)) / (2h) along x/y/z = 0/1/2 (eq. eq:diff)."""
    ax = -1 - axis_xyz
    return (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / (2.0 * h)


def stencil25_apply(f: np.ndarray, h: float, weights=None) -> np.ndarray:
    """Apply the 25-point biharmonic stencil of Sec. 4.2 in real space, divided by 16 h^4.

    ``weights`` maps offsets (dx, dy, dz) to coefficients; by default the paper's printed ones
    (centre 42; -12 at distance 2 along an axis; 1 at distance 4; 2 at the twelve (+-2, +-2)
    in-plane diagonals).  The 1/(16 h^4) factor is the one of the printed Fourier symbol.
    """
    if weights is None:
        weights = paper_stencil_weights()
    out = np.zeros_like(f, dtype=np.float64)
    for (dx, dy, dz), w in weights.items():
        out += w * np.roll(f, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))
    return out / (16.0 * h ** 4)


def paper_stencil_weights() -> dict:
    """Offsets and coefficients of the printed 25-point stencil (Sec. 4.2)."""
    w = {(0, 0, 0): 42.0}
    for a in (0, 1, 2):
        for s in (-1, 1):
            off2 = [0, 0, 0]
            off2[a] = 2 * s
            w[tuple(off2)] = -12.0
            off4 = [0, 0, 0]
            off4[a] = 4 * s
            w[tuple(off4)] = 1.0
    for a, b in ((0, 1), (1, 2), (0, 2)):
        for sa in (-2, 2):
            for sb in (-2, 2):
                off = [0, 0, 0]
                off[a] = sa
                off[b] = sb
                w[tuple(off)] = 2.0
    return w
