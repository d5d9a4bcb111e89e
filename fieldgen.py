"""Seeded synthetic stress-field generators shared by the tests, the bench and the oracle checks.

This module draws the inputs only: it holds none of the projection's arithmetic (no transform,
no wavevector, no projector, no difference operator). Every field it returns has the boundary
layout used everywhere in this repository: shape ``(6, nz, ny, nx)``, x fastest, components in
Voigt order (xx, yy, zz, yz, xz, xy).

Workload recipe (stand-in for the paper's EVPFFT Cu polycrystal, Sec. 5.1, and its Gum Metal DCT
field, Sec. 5.2, neither of which is available): a periodic Voronoi tessellation of the box,
a constant stress per grain drawn i.i.d. normal per Voigt component, plus i.i.d. normal voxel
noise. The grain of a voxel is the seed nearest to the voxel centre ``(i + 1/2) h`` under the
periodic minimum-image distance; equal distances go to the lower grain index.
"""
from __future__ import annotations

import math

import numpy as np
import torch

SEED_BASE = 210501612


def workload_seed(config_index: int, field_index: int = 0) -> int:
    """Seed of field ``field_index`` of workload ``config_index`` (0-based)."""
    return SEED_BASE + int(config_index) + int(field_index)


def _grain_seeds(shape, n_grains: int, seed: int) -> np.ndarray:
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    # seed positions in voxel units, columns (x, y, z)
    return rng.uniform(0.0, 1.0, size=(n_grains, 3)) * np.array([nx, ny, nz], dtype=np.float64)


def _grain_stress(n_grains: int, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.normal(0.0, sigma, size=(n_grains, 6))


def periodic_voronoi_map(shape, n_grains: int, seed: int, device="cpu",
                         chunk: int = 1 << 14) -> torch.Tensor:
    """Grain index (int32, shape ``(nz, ny, nx)``) of every voxel of a periodic Voronoi map.

    Seeds are uniform in the box.  Periodic images of the seeds that lie within a margin of the
    box are added as candidates, so a plain Euclidean nearest-candidate search equals the
    minimum-image search; the margin is doubled until it exceeds every voxel's nearest distance.
    Candidates are ordered by grain index so the first minimum is the lowest grain index.
    """
    nz, ny, nx = shape
    box = np.array([nx, ny, nz], dtype=np.float64)
    seeds = _grain_seeds(shape, n_grains, seed)
    dev = torch.device(device)
    spacing = (nx * ny * nz / max(n_grains, 1)) ** (1.0 / 3.0)
    margin = 3.0 * spacing
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)],
                      dtype=np.float64)
    while True:
        imgs = seeds[:, None, :] + shifts[None, :, :] * box[None, None, :]   # (G, 27, 3)
        inside = np.all((imgs > -margin) & (imgs < box + margin), axis=2)     # (G, 27)
        gidx = np.repeat(np.arange(n_grains), 27).reshape(n_grains, 27)[inside]
        cand = torch.tensor(imgs[inside], dtype=torch.float32, device=dev)
        cand_g = torch.tensor(gidx, dtype=torch.int32, device=dev)
        out = torch.empty(nz * ny * nx, dtype=torch.int32, device=dev)
        worst = 0.0
        total = nz * ny * nx
        for s in range(0, total, chunk):
            e = min(total, s + chunk)
            lin = torch.arange(s, e, device=dev, dtype=torch.int64)
            x = (lin % nx).to(torch.float32) + 0.5
            y = ((lin // nx) % ny).to(torch.float32) + 0.5
            z = (lin // (nx * ny)).to(torch.float32) + 0.5
            pts = torch.stack([x, y, z], dim=1)
            d = torch.cdist(pts, cand, compute_mode="donot_use_mm_for_euclid_dist")
            dmin, arg = torch.min(d, dim=1)
            out[s:e] = cand_g[arg]
            worst = max(worst, float(dmin.max()))
        if worst < margin or margin > float(box.max()):
            return out.reshape(nz, ny, nx)
        margin *= 2.0


def voronoi_stress_field(shape, n_grains: int, grain_sigma: float, noise_sigma: float,
                         seed: int, dtype=torch.float64, device="cpu") -> torch.Tensor:
    """Piecewise-constant grain stress plus voxel noise, shape ``(6, nz, ny, nx)``.

    Per-grain Voigt components ~ N(0, grain_sigma) (numpy PCG64 from ``seed``); voxel noise
    ~ N(0, noise_sigma) from a torch generator on ``device`` seeded with ``seed`` (so the noise
    of a given seed depends on the device; the tests always feed one tensor to both sides).
    """
    gmap = periodic_voronoi_map(shape, n_grains, seed, device=device).to(torch.int64)
    stress = torch.tensor(_grain_stress(n_grains, grain_sigma, seed), dtype=dtype, device=device)
    field = stress[gmap].permute(3, 0, 1, 2).contiguous()    # (6, nz, ny, nx)
    if noise_sigma > 0.0:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        field += noise_sigma * torch.randn(field.shape, generator=gen, dtype=dtype, device=device)
    return field


def gaussian_field(shape, seed: int, sigma: float = 1.0, dtype=torch.float64,
                   device="cpu") -> torch.Tensor:
    """I.i.d. N(0, sigma) symmetric field (6 Voigt components), drawn on the CPU with PCG64."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.normal(0.0, sigma, size=(6, nz, ny, nx))
    return torch.tensor(a, dtype=dtype, device=device)


def gaussian_array(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    """I.i.d. N(0, sigma) float64 numpy array of any shape (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, sigma, size=shape)


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    """Integer in [lo, hi] drawn log-uniformly (rounded)."""
    return int(min(hi, max(lo, round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))))
