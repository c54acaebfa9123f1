"""Seeded synthetic inputs for the Poisson workloads.

This module only draws and shapes input data (right-hand sides, manufactured
solutions, batch size mixes).  It holds none of the multigrid arithmetic and
is the one module that both the CUDA path's callers and the CPU oracle's
callers share.  Arrays hold all (n+1)^d nodes, x fastest, boundary nodes 0.

Recipes (random streams: numpy ``Generator(PCG64(seed))``):

* ``rhs_sine_plus_uniform`` -- d pi^2 prod sin(pi x_m) + amp * U[-1,1]
  (2D 257^2 workload: amp = 1e-3, seed 1).
* ``rhs_uniform`` -- i.i.d. U[-1,1] (3D 257^3 workload, seed 2; batch, seed 4).
* ``rhs_sine_plus_gauss`` -- d pi^2 prod sin(pi x_m) + sigma * N(0,1)
  (3D 513^3 workload: sigma = 1e-2, seed 3).
* ``rhs_grf`` -- Gaussian random field: white noise in the sine (DST-I) basis
  shaped by |k|^-1 amplitude (power ~ |k|^-2), normalised to unit RMS (3D
  257^3 learned-smoother workload, seed 5).
* ``batch_mix`` -- 512 size classes drawn uniformly from 2D (2^k+1)^2,
  k = 6..10 and 3D (2^k+1)^3, k = 4..7 (seed 4).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _interior_mask_view(a: np.ndarray) -> np.ndarray:
    return a[(slice(1, -1),) * a.ndim]


def manufactured_u(d: int, n: int) -> np.ndarray:
    """prod_m sin(pi x_m) on all nodes (zero on the boundary up to rounding,
    forced to exactly zero)."""
    x = np.arange(n + 1) / n
    s = np.sin(np.pi * x)
    s[0] = 0.0
    s[-1] = 0.0
    if d == 2:
        return np.ascontiguousarray(s[:, None] * s[None, :])
    return np.ascontiguousarray(s[:, None, None] * s[None, :, None] * s[None, None, :])


def rhs_uniform(d: int, n: int, seed: int) -> np.ndarray:
    f = np.zeros((n + 1,) * d)
    g = _rng(seed)
    _interior_mask_view(f)[...] = g.uniform(-1.0, 1.0, size=(n - 1,) * d)
    return f


def rhs_sine_plus_uniform(d: int, n: int, seed: int, amp: float = 1e-3) -> np.ndarray:
    f = d * np.pi ** 2 * manufactured_u(d, n)
    g = _rng(seed)
    _interior_mask_view(f)[...] += amp * g.uniform(-1.0, 1.0, size=(n - 1,) * d)
    return f


def rhs_sine_plus_gauss(d: int, n: int, seed: int, sigma: float = 1e-2) -> np.ndarray:
    f = d * np.pi ** 2 * manufactured_u(d, n)
    g = _rng(seed)
    _interior_mask_view(f)[...] += sigma * g.standard_normal(size=(n - 1,) * d)
    return f


def rhs_grf(d: int, n: int, seed: int) -> np.ndarray:
    """White noise coefficients on the sine modes k = 1..n-1 per axis, scaled
    by 1/|k|, synthesised with an (orthonormal) DST-I and normalised to unit
    RMS over the interior."""
    from scipy.fft import idstn

    g = _rng(seed)
    c = g.standard_normal(size=(n - 1,) * d)
    ks = np.arange(1, n)
    k2 = np.zeros((n - 1,) * d)
    for ax in range(d):
        shape = [1] * d
        shape[ax] = n - 1
        k2 = k2 + (ks.reshape(shape) ** 2)
    c = c / np.sqrt(k2)
    field = idstn(c, type=1, norm="ortho")
    field = field / np.sqrt(np.mean(field ** 2))
    f = np.zeros((n + 1,) * d)
    _interior_mask_view(f)[...] = field
    return f


BATCH_CLASSES = [(2, 2 ** k) for k in range(6, 11)] + [(3, 2 ** k) for k in range(4, 8)]


def batch_mix(count: int = 512, seed: int = 4):
    """List of (d, n) for ``count`` solves, classes drawn uniformly."""
    g = _rng(seed)
    idx = g.integers(0, len(BATCH_CLASSES), size=count)
    return [BATCH_CLASSES[i] for i in idx]


def batch_rhs(mix, seed: int = 4):
    """One U[-1,1] right-hand side per solve, seeds seed*100000 + index."""
    return [rhs_uniform(d, n, seed * 100000 + s) for s, (d, n) in enumerate(mix)]
