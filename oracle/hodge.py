"""The other parts of the Hodge decomposition (test infrastructure: only tests, smoke() and the
bench's CPU baseline use this package).

Theorem 2 (Sec. 3.1) splits a symmetric field A into inc(H) + sym grad y + c0.  The equilibrium
projection (``projection.project``) keeps inc(H) + c0.  The two functions here return the rest:

* ``project_compat``: the strain-compatibility projection, the dual constraint named in the
  Conclusions.  A field is compatible when it is sym grad y + c0 for a periodic y, i.e. when its
  inc vanishes.  The closest compatible field under A:B is c0 + (A - S_equil): the
  sym-gradient part of the decomposition plus the mean.
* ``hodge_potential``: the vector field y of Theorem 2 itself (mean-free), the solution of
  sym grad y = A - S_equil in Fourier space.

Reading where the paper is silent (listed in the design notes): at modes where Xi = 0 but k != 0
no y reaches the field, so y is 0 there; ``project_compat`` with ``nyq='keep'`` returns 0 there
(every field is divergence-free at those modes, so S_equil keeps them) and with ``nyq='zero'``
keeps them (S_equil drops them).
"""
from __future__ import annotations

import numpy as np

from .projection import project, _forward, _inverse, _xi_full, to_tensor


def project_compat(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0), nyq: str = "keep",
                   transform: str = "fft") -> np.ndarray:
    """Closest strain-compatible field: c0 + (S - S_equil) (Theorem 2; Conclusions)."""
    s6 = np.asarray(s6, dtype=np.float64)
    c0 = s6.mean(axis=(1, 2, 3))
    return s6 - project(s6, op, h, nyq, transform) + c0[:, None, None, None]


def hodge_potential(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0),
                    transform: str = "fft") -> np.ndarray:
    """The mean-free vector field y of Theorem 2, shape (3, nz, ny, nx).

    With a derivative acting as i Xi (Sec. 4), sym grad y has the spectrum
    (i/2)(Xi y^T + y Xi^T).  The part removed by the projector at a mode with Xi != 0 is
    n v^T + v n^T - s n n^T with n = Xi / |Xi|, v = S_hat n and s = n . v (S_hat - Q S_hat Q
    written out), which that form reaches with y_hat = -(i / |Xi|) (2 v - s n).  y_hat = 0 where
    Xi = 0.
    """
    s6 = np.asarray(s6, dtype=np.float64)
    shape = s6.shape[1:]
    c0 = s6.mean(axis=(1, 2, 3))
    t = to_tensor(_forward(s6 - c0[:, None, None, None], transform))
    xi = _xi_full(shape, h, op)
    k2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    degenerate = k2 == 0.0
    kn = np.sqrt(np.where(degenerate, 1.0, k2))
    n = np.stack([a / kn for a in xi])                            # (3, nz, ny, nx)
    v = np.einsum("ij...,j...->i...", t, n)
    s = np.einsum("i...,i...->...", n, v)
    yhat = -1j / kn * (2.0 * v - s * n)
    yhat = np.where(degenerate[None], 0.0, yhat)
    return np.real(_inverse(yhat, transform))
