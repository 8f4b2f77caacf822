"""Seeded synthetic inputs for the gasket stencils.

This module is shared by the tests, the benchmark and the smoke check; it
holds none of the method's arithmetic (no block map, no stencil, no write
pass).  It knows only the problem statement: the level-r gasket is the set of
cells (x, y) of the n x n grid (n = 2^r) with (x & y) == 0, stored row-major,
and random fields are drawn from a counter-based generator:

    key   = y * n + x
    h     = SplitMix64 output for state (seed * 0x9E3779B97F4A7C15) XOR key
            (Steele, Lea, Flood, OOPSLA 2014; Mix13 finaliser)
    u     = (h >> 40) * 2^-24          -- U[0,1), exact in float32
    alive = u < p                      -- Bernoulli(p)

Initial states are zero off the gasket, as the step kernels require.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_next(state: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each state (uint64 array, wrapping arithmetic)."""
    z = np.asarray(state, dtype=np.uint64) + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def cell_hash(r: int, xs: np.ndarray, ys: np.ndarray, seed: int) -> np.ndarray:
    xs = np.asarray(xs, dtype=np.uint64)
    ys = np.asarray(ys, dtype=np.uint64)
    key = (ys << np.uint64(r)) | xs
    with np.errstate(over="ignore"):
        s = np.uint64((int(seed) * 0x9E3779B97F4A7C15) & (2**64 - 1))
    return splitmix64_next(s ^ key)


def uniform_at(r: int, xs, ys, seed: int) -> np.ndarray:
    """U[0,1) draw of every listed cell, float32 (exact 24-bit values)."""
    h = cell_hash(r, xs, ys, seed)
    return ((h >> np.uint64(40)).astype(np.float64) * 2.0**-24).astype(np.float32)


def gasket_cells(r: int) -> tuple[np.ndarray, np.ndarray]:
    """Coordinates (xs, ys) of the 3^r gasket cells, row-major order."""
    xs = np.zeros(1, dtype=np.int64)
    ys = np.zeros(1, dtype=np.int64)
    for k in range(r):
        h = 1 << k
        xs, ys = np.concatenate([xs, xs + h, xs]), np.concatenate([ys, ys, ys + h])
    order = np.argsort((ys << r) | xs, kind="stable")
    return xs[order], ys[order]


def _region_coords(x0: int, y0: int, w: int, h: int):
    ys, xs = np.mgrid[y0:y0 + h, x0:x0 + w]
    return xs.astype(np.int64), ys.astype(np.int64)


def _on_gasket(r: int, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    n = 1 << r
    inside = (xs >= 0) & (xs < n) & (ys >= 0) & (ys < n)
    return inside & ((xs & ys) == 0)


def ca_seed_region(r: int, p: float, seed: int, x0: int, y0: int, w: int,
                   h: int) -> np.ndarray:
    """Bernoulli(p) live cells on the gasket inside a region (uint8, h x w);
    0 off the gasket and outside the grid."""
    xs, ys = _region_coords(x0, y0, w, h)
    on = _on_gasket(r, xs, ys)
    out = np.zeros((h, w), dtype=np.uint8)
    if on.any():
        u = uniform_at(r, xs[on], ys[on], seed).astype(np.float64)
        out[on] = (u < p).astype(np.uint8)
    return out


def uniform_region(r: int, seed: int, x0: int, y0: int, w: int,
                   h: int) -> np.ndarray:
    """U[0,1) field on the gasket inside a region (float32); 0 elsewhere."""
    xs, ys = _region_coords(x0, y0, w, h)
    on = _on_gasket(r, xs, ys)
    out = np.zeros((h, w), dtype=np.float32)
    if on.any():
        out[on] = uniform_at(r, xs[on], ys[on], seed)
    return out


def ca_seed_grid(r: int, p: float, seed: int) -> np.ndarray:
    n = 1 << r
    return ca_seed_region(r, p, seed, 0, 0, n, n)


def uniform_grid(r: int, seed: int) -> np.ndarray:
    n = 1 << r
    return uniform_region(r, seed, 0, 0, n, n)


def ca_seed_sparse(r: int, p: float, seed: int):
    """Flat row-major indices (int64) of the gasket cells and their Bernoulli
    states (uint8): for scattering a full-size initial state on the device."""
    xs, ys = gasket_cells(r)
    u = uniform_at(r, xs, ys, seed).astype(np.float64)
    return (ys << r) | xs, (u < p).astype(np.uint8)


def uniform_sparse(r: int, seed: int):
    """Flat row-major indices (int64) of the gasket cells and their U[0,1)
    values (float32)."""
    xs, ys = gasket_cells(r)
    return (ys << r) | xs, uniform_at(r, xs, ys, seed)


def batch_levels(count: int, lo: int, hi: int, seed: int) -> list[int]:
    """Levels of a batch of gaskets drawn uniformly from lo..hi (numpy PCG64
    stream seeded with `seed`)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, count)]


def instance_seed(seed: int, i: int) -> int:
    """Seed of gasket i of a batch: seed + i * 2^32 (distinct streams)."""
    return int(seed) + (int(i) << 32)

