"""The equilibrium projection, its literal Euler-Lagrange route, divergence and norms (float64).

Definition followed (Sec. 3.2): S_equil is the field closest to S_exp in L^2 among periodic
symmetric fields with zero divergence.  With the Hodge decomposition (Sec. 3.1, Theorem 2) the
removed part is a symmetric gradient and the kept part is inc(H) + c0 with c0 = mean(S_exp)
(Sec. 3.2, eq. eq:sequil and the averaging argument after it).  In Fourier space a derivative is
multiplication by i Xi (Sec. 4); the divergence-free condition at mode k reads S_hat(k) n = 0
with n = Xi / |Xi|, and the closest such matrix under A:B is Q S_hat Q with Q = I - n n^T.

Readings where the paper is silent (each listed in the design notes):
  * modes with Xi(k) = 0 but k != 0 (the Nyquist corners): ``nyq='keep'`` leaves them
    unchanged (every field is divergence-free there, so the closest field keeps them);
    ``nyq='zero'`` removes them, which is what the literal route inc(inc(S)/biharmonic) gives.
  * the k = 0 mode is the mean c0 and is always kept.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .operators import wavevector_grids, biharmonic_symbol_paper, central_diff
from .transforms import dft3_direct, dft3_naive, fft3, ifft3

VOIGT_IJ = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
VOIGT_W = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])


def to_tensor(s6: np.ndarray) -> np.ndarray:
    """(6, ...) Voigt array -> (3, 3, ...) symmetric tensor array."""
    t = np.empty((3, 3) + s6.shape[1:], dtype=s6.dtype)
    for c, (i, j) in enumerate(VOIGT_IJ):
        t[i, j] = s6[c]
        t[j, i] = s6[c]
    return t


def to_voigt(t: np.ndarray) -> np.ndarray:
    """(3, 3, ...) tensor array -> (6, ...) Voigt array (upper triangle)."""
    return np.stack([t[i, j] for (i, j) in VOIGT_IJ])


def frob2(s6: np.ndarray) -> np.ndarray:
    """Per-voxel A:A of a Voigt field (off-diagonals weigh 2)."""
    return np.einsum("c,c...->...", VOIGT_W, np.abs(s6) ** 2)


def inner(a6: np.ndarray, b6: np.ndarray) -> float:
    """<A, B> = sum over voxels of A:B."""
    w = VOIGT_W.reshape((6,) + (1,) * (np.ndim(a6) - 1))
    return float((w * a6 * b6).sum())


def _forward(x, transform):
    if transform == "fft":
        return fft3(x)
    if transform == "direct":
        return dft3_direct(x)
    if transform == "naive":
        return dft3_naive(x)
    raise ValueError(transform)


def _inverse(x, transform):
    if transform == "fft":
        return ifft3(x)
    if transform == "direct":
        return dft3_direct(x, inverse=True)
    if transform == "naive":
        return dft3_naive(x, inverse=True)
    raise ValueError(transform)


def _xi_full(shape, h, op):
    xi = wavevector_grids(shape, h, op)
    return [np.broadcast_to(a, shape) for a in xi]


def project_spectrum(shat6: np.ndarray, h, op: str, nyq: str = "keep", grid=None,
                     z0: int = 0) -> np.ndarray:
    """Apply the per-mode projector to a Voigt spectrum ``(6, nz, ny, nx)`` (complex).

    At every mode with Xi != 0: S_hat <- Q S_hat Q, Q = I - n n^T, n = Xi / |Xi| (the orthogonal
    projection, under A:B, onto matrices with S_hat n = 0).  Xi = 0: identity at k = 0; at k != 0
    identity (``keep``) or zero (``zero``).

    ``grid``/``z0``: ``shat6`` is the slab of z indices z0, z0 + 1, ... of the spectrum of a grid
    ``(nz, ny, nx)`` (default: the whole spectrum); each mode gets the Xi of its own index.
    """
    shape = shat6.shape[1:]
    if grid is None:
        xi = _xi_full(shape, h, op)
    else:
        xi_x, xi_y, xi_z = wavevector_grids(tuple(grid), h, op)
        xi = [np.broadcast_to(a, shape) for a in (xi_x, xi_y, xi_z[z0:z0 + shape[0]])]
    k2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    degenerate = k2 == 0.0
    inv = np.where(degenerate, 0.0, 1.0 / np.sqrt(np.where(degenerate, 1.0, k2)))
    n = np.stack([a * inv for a in xi])                       # (3, nz, ny, nx)
    q = np.eye(3)[:, :, None, None, None] - n[:, None] * n[None, :]
    t = to_tensor(shat6)
    out = np.einsum("ij...,jk...,kl...->il...", q, t, q)
    if nyq == "keep":
        out = np.where(degenerate[None, None], t, out)
    elif nyq == "zero":
        out = np.where(degenerate[None, None], 0.0, out)
        if z0 == 0:
            out[:, :, 0, 0, 0] = t[:, :, 0, 0, 0]
    else:
        raise ValueError(nyq)
    return to_voigt(out)


def project(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0), nyq: str = "keep",
            transform: str = "fft") -> np.ndarray:
    """S_equil of Sec. 3.2 by the solution strategy of Sec. 3.3, in closed form.

    1. c0 = mean of S over voxels, per component (Sec. 3.2, eq. after eq:sequil).
    2. S_hat = DFT(S - c0) (the demeaned field of eq. eqnOptH).
    3. per-mode projector (``project_spectrum``).
    4. S_equil = IDFT(S_hat) + c0.
    """
    s6 = np.asarray(s6, dtype=np.float64)
    c0 = s6.mean(axis=(1, 2, 3))
    st = s6 - c0[:, None, None, None]
    shat = _forward(st, transform)
    out = project_spectrum(shat, h, op, nyq)
    return np.real(_inverse(out, transform)) + c0[:, None, None, None]


def project_large(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0), nyq: str = "keep",
                  slab: int = 2) -> np.ndarray:
    """``project`` for grids whose whole (3, 3)-tensor spectrum does not fit in host memory
    (512^3: about 20 GB for one complex tensor array, several of them alive at once).

    The same four steps of Sec. 3.2-3.3 with the same arithmetic per mode: the mean and the
    transforms run one Voigt component at a time, and ``project_spectrum`` runs on z-slabs of
    ``slab`` planes of the spectrum, each with the Xi of its own modes.  Only the grouping of modes
    into arrays differs from ``project`` (the per-mode projector has no coupling between modes).
    ``s6`` may be float32; it is read one component at a time in float64.
    """
    nz, ny, nx = s6.shape[1:]
    c0 = np.array([np.asarray(s6[c], dtype=np.float64).mean() for c in range(6)])
    shat = np.empty((6, nz, ny, nx), dtype=np.complex128)
    for c in range(6):
        shat[c] = fft3(np.asarray(s6[c], dtype=np.float64) - c0[c])

    def one_slab(z0):
        z1 = min(nz, z0 + slab)
        shat[:, z0:z1] = project_spectrum(shat[:, z0:z1], h, op, nyq, grid=(nz, ny, nx), z0=z0)

    # slabs are independent (disjoint modes), so they may run on the host cores side by side
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        list(ex.map(one_slab, range(0, nz, slab)))
    out = np.empty((6, nz, ny, nx), dtype=np.float64)
    for c in range(6):
        out[c] = np.real(ifft3(shat[c])) + c0[c]
    return out


_EPS = np.zeros((3, 3, 3))
for _i, _j, _k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    _EPS[_i, _j, _k] = 1.0
    _EPS[_i, _k, _j] = -1.0


def inc_hat(t: np.ndarray, xi) -> np.ndarray:
    """(inc A)^_kn = eps_ijk eps_lmn (i Xi_i)(i Xi_l) A^_jm for a (3, 3, ...) spectrum
    (Sec. 3.1, Theorem 2, with nabla -> i Xi as in Sec. 4)."""
    d = np.stack([1j * a for a in xi])                          # i Xi, (3, nz, ny, nx)
    return np.einsum("ijk,lmn,i...,l...,jm...->kn...", _EPS, _EPS, d, d, t, optimize=True)


def project_literal(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0),
                    transform: str = "fft") -> np.ndarray:
    """S_equil by the literal route of Sec. 3.2-3.3: solve the Euler-Lagrange equation
    nabla^4 H = inc(S~) (eq. eqnELH) in Fourier space, with the gauge mean(H) = 0, then
    S_equil = inc(H) + c0 (eq. eq:sequil).

    The biharmonic symbol is the paper's 25-point-stencil symbol for DDO with one spacing
    (Sec. 4.2) and |Xi|^4 otherwise.  Modes where it vanishes get H = 0 there.
    """
    s6 = np.asarray(s6, dtype=np.float64)
    shape = s6.shape[1:]
    c0 = s6.mean(axis=(1, 2, 3))
    t = to_tensor(_forward(s6 - c0[:, None, None, None], transform))
    xi = _xi_full(shape, h, op)
    k2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    if op == "ddo" and h[0] == h[1] == h[2]:
        bih = biharmonic_symbol_paper(shape, h[0])
    else:
        bih = k2 ** 2
    degenerate = k2 == 0.0
    hh = inc_hat(t, xi) / np.where(degenerate, 1.0, bih)
    hh = np.where(degenerate[None, None], 0.0, hh)
    out = to_voigt(inc_hat(hh, xi))
    return np.real(_inverse(out, transform)) + c0[:, None, None, None]


def divergence(s6: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0)) -> np.ndarray:
    """(div S)_i = sum_j d_j S_ij with d_j <-> i Xi_j of the chosen operator; shape (3, ...)."""
    t = to_tensor(fft3(np.asarray(s6, dtype=np.float64)))
    xi = _xi_full(s6.shape[1:], h, op)
    dhat = sum(1j * xi[j] * t[:, j] for j in range(3))
    return np.real(ifft3(dhat))


def divergence_central_diff(s6: np.ndarray, h=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Divergence with plain periodic central differences in real space (eq. eq:diff), no FFT."""
    t = to_tensor(np.asarray(s6, dtype=np.float64))
    return np.stack([sum(central_diff(t[i, j], j, h[j]) for j in range(3)) for i in range(3)])


def norms(s_in: np.ndarray, s_out: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0)) -> dict:
    """Per-field diagnostics by definition, in real space.

    RMS norms ||A|| = sqrt(mean over voxels of A:A); resid = S_in - S_out; resid_linf is the
    largest |component| of resid over voxels and Voigt components; div_*_l2 is the RMS of the
    divergence vector with the chosen operator.  (Table 1 and Fig. 3 do not say how their L^2
    error is normalised; these definitions are this library's.)
    """
    s_in = np.asarray(s_in, dtype=np.float64)
    s_out = np.asarray(s_out, dtype=np.float64)
    resid = s_in - s_out
    norm_in = float(np.sqrt(frob2(s_in).mean()))
    d_in = divergence(s_in, op, h)
    d_out = divergence(s_out, op, h)
    return {
        "mean": s_in.mean(axis=(1, 2, 3)),
        "norm_in": norm_in,
        "norm_out": float(np.sqrt(frob2(s_out).mean())),
        "resid_l2": float(np.sqrt(frob2(resid).mean())),
        "resid_rel": float(np.sqrt(frob2(resid).mean())) / norm_in if norm_in > 0 else 0.0,
        "resid_linf": float(np.abs(resid).max()),
        "div_in_l2": float(np.sqrt((d_in ** 2).sum(axis=0).mean())),
        "div_out_l2": float(np.sqrt((d_out ** 2).sum(axis=0).mean())),
    }


def _div2_sum(s6: np.ndarray, op: str, h) -> float:
    """Sum over voxels of |div S|^2 with the operator of ``divergence``, one row
    (div S)_i = sum_j d_j S_ij at a time, each S_ij transformed on its own."""
    shape = s6.shape[1:]
    xi = _xi_full(shape, h, op)
    total = 0.0
    for i in range(3):
        dhat = np.zeros(shape, dtype=np.complex128)
        for j in range(3):
            c = VOIGT_IJ.index((min(i, j), max(i, j)))
            dhat += 1j * xi[j] * fft3(np.asarray(s6[c], dtype=np.float64))
        d = np.real(ifft3(dhat))
        total += float((d * d).sum())
    return total


def norms_large(s_in: np.ndarray, s_out: np.ndarray, op: str = "ddo", h=(1.0, 1.0, 1.0),
                div_out: bool = True) -> dict:
    """``norms`` for grids too large for whole-field tensor arrays: the same definitions,
    evaluated one Voigt component (real-space terms) or one row of the divergence at a time.
    ``div_out=False`` leaves the output divergence out (reported as NaN)."""
    nv = float(np.prod(s_in.shape[1:]))
    mean = np.empty(6)
    a2 = b2 = r2 = 0.0
    linf = 0.0
    for c in range(6):
        a = np.asarray(s_in[c], dtype=np.float64)
        b = np.asarray(s_out[c], dtype=np.float64)
        r = a - b
        mean[c] = a.mean()
        a2 += VOIGT_W[c] * float((a * a).sum())
        b2 += VOIGT_W[c] * float((b * b).sum())
        r2 += VOIGT_W[c] * float((r * r).sum())
        linf = max(linf, float(np.abs(r).max()))
    norm_in = float(np.sqrt(a2 / nv))
    resid = float(np.sqrt(r2 / nv))
    return {
        "mean": mean,
        "norm_in": norm_in,
        "norm_out": float(np.sqrt(b2 / nv)),
        "resid_l2": resid,
        "resid_rel": resid / norm_in if norm_in > 0 else 0.0,
        "resid_linf": linf,
        "div_in_l2": float(np.sqrt(_div2_sum(s_in, op, h) / nv)),
        "div_out_l2": float(np.sqrt(_div2_sum(s_out, op, h) / nv)) if div_out else float("nan"),
    }
