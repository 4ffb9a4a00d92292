"""Seeded synthetic particle sets.

These stand in for the paper's datasets (Table 1 of arXiv 2404.02826: Nyx and
HACC cosmology, SPH dam-break and FPM fluid runs), none of which is available
here.  Every generator is deterministic in (n, seed) and uses numpy's PCG64
``default_rng``.  This module only draws positions; it holds none of the
compressor's arithmetic, and both the oracle tests and the CUDA tests use it.

Recipes:
  * ``uniform``    - n points i.i.d. uniform in [0, box)^3 (random storage order).
  * ``cosmology``  - periodic box [0, 256)^3; 70 % of the points in 20,000
                     isotropic Gaussian clumps (centres uniform, sigma
                     log-uniform in [0.05, 2.0], clump weights classical Pareto
                     with alpha = 1.8 and x_m = 1, counts multinomial), wrapped
                     into the box; 30 % uniform background; one global shuffle.
  * ``fluid``      - cubic lattice of spacing h = 1/384 on 384 x 192 x 228
                     sites (x fastest), the first n sites in lattice-index
                     order, each jittered by U(-0.3h, 0.3h) per axis; sites with
                     z >= 0.3 are displaced by a smooth sinusoidal flow of
                     amplitude 0.05.  Stored in lattice-index order.
  * ``near_ties``  - points placed on or next to the midpoints of a given
                     lattice, to exercise round-half-even decisions.
"""
from __future__ import annotations

import numpy as np

__all__ = ["uniform", "cosmology", "fluid", "near_ties", "by_name"]


def uniform(n: int, seed: int = 0, box: float = 256.0, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, box, (n, 3)).astype(dtype)


def cosmology(n: int, seed: int = 0, box: float = 256.0, n_clumps: int = 20000, clump_frac: float = 0.7,
              sigma_lo: float = 0.05, sigma_hi: float = 2.0, alpha: float = 1.8, dtype=np.float32,
              chunk: int = 1 << 22) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n_clumped = int(round(clump_frac * n))
    centres = rng.uniform(0.0, box, (n_clumps, 3))
    sigma = np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi), n_clumps))
    weight = rng.pareto(alpha, n_clumps) + 1.0
    counts = rng.multinomial(n_clumped, weight / weight.sum())
    owner = np.repeat(np.arange(n_clumps, dtype=np.int32), counts)
    out = np.empty((n, 3), dtype=dtype)
    for a in range(0, n_clumped, chunk):
        b = min(n_clumped, a + chunk)
        c = owner[a:b]
        p = centres[c] + sigma[c, None] * rng.standard_normal((b - a, 3))
        out[a:b] = np.mod(p, box)
    for a in range(n_clumped, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = rng.uniform(0.0, box, (b - a, 3))
    # values that round up to the box edge wrap to 0 (periodic box)
    out[out >= box] = 0
    perm = rng.permutation(n)
    return out[perm]


def fluid(n: int, seed: int = 0, h: float = 1.0 / 384, dims=(384, 192, 228), jitter: float = 0.3,
          amplitude: float = 0.05, dtype=np.float64) -> np.ndarray:
    nx, ny, nz = dims
    if n > nx * ny * nz:
        raise ValueError("n exceeds the lattice")
    rng = np.random.default_rng(seed)
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    x0 = i * h
    y0 = j * h
    z0 = k * h
    pos = np.stack([x0, y0, z0], axis=1)
    pos += rng.uniform(-jitter * h, jitter * h, (n, 3))
    moved = z0 >= 0.3
    ly, lz = ny * h, 0.6
    two_pi = 2.0 * np.pi
    ux = np.sin(two_pi * y0 / ly) * np.cos(two_pi * z0 / lz)
    uy = np.sin(two_pi * z0 / lz) * np.cos(two_pi * x0)
    uz = np.sin(two_pi * x0) * np.cos(two_pi * y0 / ly)
    disp = amplitude * np.stack([ux, uy, uz], axis=1)
    pos[moved] += disp[moved]
    return pos.astype(dtype)


def near_ties(n: int, origin, step: float, seed: int = 0, dtype=np.float32, spread: int = 64) -> np.ndarray:
    """Points at o + step*(k + 1/2) (and their neighbours one unit in the last place)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, spread, (n, 3))
    half = np.asarray(origin, np.float64) + step * (k + 0.5)
    p = half.astype(dtype)
    nudge = rng.integers(-1, 2, (n, 3))
    p = np.where(nudge > 0, np.nextafter(p, np.asarray(np.inf, dtype)), p)
    p = np.where(nudge < 0, np.nextafter(p, np.asarray(-np.inf, dtype)), p)
    return p.astype(dtype)


def by_name(name: str, n: int, seed: int = 0, dtype=None) -> np.ndarray:
    if name == "uniform":
        return uniform(n, seed, dtype=dtype or np.float32)
    if name == "cosmology":
        return cosmology(n, seed, dtype=dtype or np.float32)
    if name == "fluid":
        return fluid(n, seed, dtype=dtype or np.float64)
    raise KeyError(name)
