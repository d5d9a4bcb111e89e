"""Seeded synthetic stress-field generators shared by the tests, the bench and the oracle checks.

This module draws the inputs only: it holds none of the projection's arithmetic (no transform,
no wavevector, no projector, no difference operator). Every field it returns has the boundary
layout used everywhere in this repository: shape ``(6, nz, ny, nx)``, x fastest, components in
Voigt order (xx, yy, zz, yz, xz, xy).

Workload recipe (stand-in for the paper's EVPFFT Cu polycrystal, Sec. 5.1, and its Gum Metal DCT
field, Sec. 5.2, neither of which is available): a periodic Voronoi tessellation of the box,
a constant stress per grain drawn i.i.d. normal per Voigt component, plus i.i.d. normal voxel
noise. The grain of a voxel is the seed nearest to the voxel centre ``(i + 1/2) h`` under the
periodic minimum-image distance.
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


def periodic_voronoi_map(shape, n_grains: int, seed: int, device="cpu") -> torch.Tensor:
    """Grain index (int32, shape ``(nz, ny, nx)``) of every voxel of a periodic Voronoi map.

    Seeds are uniform in the box; each voxel centre takes its nearest seed under the periodic
    minimum-image distance (a periodic k-d tree, queried one z-slab at a time on all host cores;
    exact ties, a measure-zero event, are resolved by the tree).
    """
    from scipy.spatial import cKDTree
    nz, ny, nx = shape
    seeds = _grain_seeds(shape, n_grains, seed)
    box = np.array([nx, ny, nz], dtype=np.float64)
    tree = cKDTree(np.mod(seeds, box), boxsize=box)
    out = np.empty((nz, ny, nx), dtype=np.int32)
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    plane = np.stack([xx.ravel(), yy.ravel(), np.zeros(nx * ny)], axis=1)
    step = max(1, (1 << 22) // max(1, nx * ny))
    for z0 in range(0, nz, step):
        z1 = min(nz, z0 + step)
        pts = np.concatenate([plane + np.array([0.0, 0.0, z + 0.5]) for z in range(z0, z1)])
        _, idx = tree.query(pts, k=1, workers=-1)
        out[z0:z1] = idx.reshape(z1 - z0, ny, nx)
    return torch.from_numpy(out).to(device)


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
