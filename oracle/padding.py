"""Non-periodic specimens in a zero-stress buffer (test infrastructure: only tests, smoke() and
the bench's CPU baseline use this package).

Sec. 5.2 makes a measured specimen periodic by surrounding it with a buffer region of zero stress
(free lateral surfaces) and projects the enlarged field.  The function below writes that out:
zero field on the enlarged grid, specimen copied in, the equilibrium projection of the whole
grid, and the specimen region cut back out.

Reading (listed in the design notes): the specimen sits at the origin corner of the enlarged
grid and the buffer fills the high end of every padded axis.  On a periodic grid that is the
same as a buffer on both sides (a shift of the whole field, which the projection commutes with);
an axis with no padding stays periodically connected, as the paper does along z.
"""
from __future__ import annotations

import numpy as np

from .projection import project


def project_padded(s6: np.ndarray, grid_shape, op: str = "ddo", h=(1.0, 1.0, 1.0),
                   nyq: str = "keep", transform: str = "fft") -> np.ndarray:
    """Equilibrium projection of specimen ``s6`` (6, sz, sy, sx) embedded with zero stress in a
    periodic grid ``grid_shape`` = (nz, ny, nx) >= the specimen; returns the specimen region."""
    s6 = np.asarray(s6, dtype=np.float64)
    sz, sy, sx = s6.shape[1:]
    nz, ny, nx = grid_shape
    if sz > nz or sy > ny or sx > nx:
        raise ValueError("the grid must contain the specimen")
    big = np.zeros((6, nz, ny, nx))
    big[:, :sz, :sy, :sx] = s6
    return project(big, op, h, nyq, transform)[:, :sz, :sy, :sx]
