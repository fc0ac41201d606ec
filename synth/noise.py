"""Improved gradient noise (K. Perlin, "Improving noise", SIGGRAPH 2002), written from the
published description, for seeded 3D perturbations of the synthetic fields.

At integer lattice points the noise is zero; each corner of the unit cell around a point
contributes the dot product of its pseudo-random gradient (one of the twelve directions to the
edge midpoints of a cube, hashed through a seeded permutation of 0..255) with the offset to the
point, and the eight contributions are blended with the quintic fade 6t^5 - 15t^4 + 10t^3.
Values lie in about [-1, 1]; the lattice repeats every 256 units.
"""
from __future__ import annotations

import numpy as np

from .rng import Stream

# the twelve cube-edge directions, padded to sixteen by repeating four of them
_GRAD = np.array([[1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
                  [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
                  [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1],
                  [1, 1, 0], [0, -1, 1], [-1, 1, 0], [0, -1, -1]], dtype=np.float64)


def permutation_table(seed: int) -> np.ndarray:
    """Seeded permutation of 0..255, stored twice so that p[i + j] needs no wrap."""
    p = Stream(seed, "perlin-permutation").permutation(256)
    return np.concatenate([p, p]).astype(np.int64)


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def noise3(x, y, z, perm: np.ndarray) -> np.ndarray:
    """Gradient noise at the points (x, y, z) (arrays of equal shape)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    xi, yi, zi = np.floor(x), np.floor(y), np.floor(z)
    fx, fy, fz = x - xi, y - yi, z - zi
    X = xi.astype(np.int64) & 255
    Y = yi.astype(np.int64) & 255
    Z = zi.astype(np.int64) & 255
    u, v, w = _fade(fx), _fade(fy), _fade(fz)
    out = np.zeros_like(fx)
    # trilinear blend of the eight corner contributions
    for dx in (0, 1):
        hx = perm[X + dx]
        wx = u if dx else 1.0 - u
        for dy in (0, 1):
            hy = perm[hx + Y + dy]
            wy = v if dy else 1.0 - v
            for dz in (0, 1):
                g = _GRAD[perm[hy + Z + dz] & 15]
                dot = g[..., 0] * (fx - dx) + g[..., 1] * (fy - dy) + g[..., 2] * (fz - dz)
                out += (wx * wy * (w if dz else 1.0 - w)) * dot
    return out


def fractal3(x, y, z, perm: np.ndarray, octaves: int = 3, lacunarity: float = 2.0,
             gain: float = 0.5) -> np.ndarray:
    """Sum of octaves of noise3, normalised by the sum of their amplitudes."""
    tot = np.zeros(np.broadcast(x, y, z).shape)
    amp, freq, norm = 1.0, 1.0, 0.0
    for _ in range(octaves):
        tot += amp * noise3(np.asarray(x) * freq, np.asarray(y) * freq, np.asarray(z) * freq, perm)
        norm += amp
        amp *= gain
        freq *= lacunarity
    return tot / norm
