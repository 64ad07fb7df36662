"""Seeded synthetic inputs for the EIFMM workloads.

This module only draws random numbers (numpy PCG64); it holds none of the
method's arithmetic, so both the GPU path and its CPU checker can use it.
The point sets follow the paper's test cases (Section 5.2: points drawn from a
uniform law in a cube) and the workload shapes used to exercise the library:

  * ``uniform_cube``      -- N iid points in [0, 1)^3;
  * ``gaussian_mixture``  -- N points from 8 equal-weight isotropic Gaussians
                              (std 0.05, centres U[0.2, 0.8]^3), clipped to
                              [0, 1]^3: strongly non-uniform leaves;
  * ``sigma_uniform`` / ``sigma_normal`` -- potentials, column-major N x R;
  * ``batch_sizes``       -- log-uniform problem sizes for batched runs.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(n: int, seed: int) -> np.ndarray:
    """(n, 3) float64 points iid uniform in [0, 1)^3."""
    return rng(seed).random((n, 3))


def gaussian_mixture(n: int, seed: int, n_centres: int = 8, std: float = 0.05,
                     centre_lo: float = 0.2, centre_hi: float = 0.8) -> np.ndarray:
    """(n, 3) points from an equal-weight isotropic Gaussian mixture, clipped
    to [0, 1]^3."""
    g = rng(seed)
    centres = g.uniform(centre_lo, centre_hi, size=(n_centres, 3))
    which = g.integers(0, n_centres, size=n)
    pts = centres[which] + std * g.standard_normal((n, 3))
    return np.clip(pts, 0.0, 1.0)


def sigma_uniform(n: int, nrhs: int, seed: int) -> np.ndarray:
    """(n, nrhs) Fortran-ordered potentials iid U[-1, 1]."""
    return np.asfortranarray(rng(seed).uniform(-1.0, 1.0, size=(nrhs, n)).T)


def sigma_normal(n: int, nrhs: int, seed: int) -> np.ndarray:
    """(n, nrhs) Fortran-ordered potentials iid N(0, 1)."""
    return np.asfortranarray(rng(seed).standard_normal(size=(nrhs, n)).T)


def batch_sizes(n_problems: int, lo: int, hi: int, seed: int) -> list[int]:
    """Problem sizes round(exp(U[ln lo, ln hi]))."""
    u = rng(seed).uniform(np.log(lo), np.log(hi), size=n_problems)
    return [int(round(float(np.exp(v)))) for v in u]


def sample_targets(n: int, n_sample: int, seed: int) -> np.ndarray:
    """Sorted distinct target indices for sampled accuracy checks."""
    return np.sort(rng(seed).choice(n, size=min(n, n_sample), replace=False)).astype(np.int64)


def sphere_surface(n: int, seed: int, radius: float = 0.5) -> np.ndarray:
    """(n, 3) points iid uniform on the sphere of the given radius centred in
    the unit cube (the paper's "sphere" test case, Section 5.2), clipped to
    [0, 1]^3 against rounding."""
    g = rng(seed).standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return np.clip(0.5 + radius * g, 0.0, 1.0)
