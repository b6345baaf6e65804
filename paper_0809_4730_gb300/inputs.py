"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
oracle's tests.

This module holds no arithmetic of the lattice Boltzmann method: only the
workload descriptions (grid sizes, wall planes, physical parameters) and the
seeded body-force fields and initial perturbations that both sides receive as
plain arrays.  Every array is float64, in the C-ABI layout
``[component][z][y][x]`` (x fastest).
"""
from __future__ import annotations

import numpy as np


def duct_force_x(nx: int, ny: int, nz: int, F0: float = 1e-6) -> np.ndarray:
    """Streamwise force of the square-duct workload,
    F_x(y, z) = F0 (1 + 0.5 sin(2 pi y / L_y) cos(2 pi z / L_z)),
    with y, z the node indices and L_y = ny, L_z = nz.  Returns [3, nz, ny, nx]
    (only the x component is non-zero)."""
    y = np.arange(ny, dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)
    fx = F0 * (1.0 + 0.5 * np.sin(2.0 * np.pi * y[None, :] / ny) * np.cos(2.0 * np.pi * z[:, None] / nz))
    F = np.zeros((3, nz, ny, nx))
    F[0] = fx[:, :, None]
    return F


def gaussian_force(nx: int, ny: int, nz: int, F0: float = 1e-6, sigma_rel: float = 0.2,
                   seed: int = 1) -> np.ndarray:
    """Per-node body force with F_x ~ N(F0, (sigma_rel F0)^2) and
    F_y, F_z ~ N(0, (sigma_rel F0)^2), seeded.  Returns [3, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    F = rng.normal(0.0, sigma_rel * F0, size=(3, nz, ny, nx))
    F[0] += F0
    return F


def random_force(nx: int, ny: int, nz: int, scale: float, seed: int) -> np.ndarray:
    """Unstructured random force field (uniform in [-scale, scale]) for parity
    tests.  Returns [3, nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(3, nz, ny, nx))


def perturbation(q: int, nx: int, ny: int, nz: int, scale: float, seed: int) -> np.ndarray:
    """Random perturbation [q, nz, ny, nx] added to an initial state so that
    parity tests exercise every term of the update."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(q, nz, ny, nx))


def batch_sizes(n_domains: int = 64, lo: int = 32, hi: int = 160, seed: int = 0) -> np.ndarray:
    """Seeded edge lengths of the batched cubic ducts, uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_domains)
