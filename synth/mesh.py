"""Seeded synthetic unstructured meshes in LDU face addressing (cells -> graph nodes, faces ->
edges), the stand-in for the unstructured combustor meshes of the sparse-solver workload.

Recipe: the cells of an nx x ny x nz hexahedral grid; a face joins every pair of cells that
share a grid face, and with probability ``p_extra`` also a cell and each of its three forward
edge-diagonal neighbours (+1,+1,0), (+1,0,+1), (0,+1,+1), so that cells have 3 to 12 faces
(hexahedra, and polyhedra of a hybrid mesh). Cells are then numbered in a random order (a
mesh generator's arbitrary numbering) and faces are oriented owner < neighbour and sorted by
(owner, neighbour), the upper-triangular face order of LDU addressing.

Per face a positive coefficient g_f (a diffusivity times area over distance: log-normal, the
diagonal faces weaker) and per cell a positive diagonal source s_c (volume over time step:
log-normal) are drawn; neither is computed from geometry. Nothing here is the method's
arithmetic: it draws numbers.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Mesh:
    n_cells: int
    owner: np.ndarray        # int32 [n_faces], owner < neighbour
    neighbour: np.ndarray    # int32 [n_faces]
    face_coeff: np.ndarray   # float64 [n_faces], g_f > 0
    cell_source: np.ndarray  # float64 [n_cells], s_c > 0

    @property
    def n_faces(self) -> int:
        return int(self.owner.shape[0])


def grid_mesh(nx: int, ny: int, nz: int, seed: int = 7, p_extra: float = 0.15,
              shuffle: bool = True) -> Mesh:
    """The mesh described in the module docstring. ``shuffle=False`` keeps the lexicographic
    grid numbering (x fastest)."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    pairs = [
        (idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel(), 1.0),
        (idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel(), 1.0),
        (idx[:-1, :, :].ravel(), idx[1:, :, :].ravel(), 1.0),
    ]
    if p_extra > 0.0:
        diag = [(idx[:, :-1, :-1], idx[:, 1:, 1:]), (idx[:-1, :, :-1], idx[1:, :, 1:]),
                (idx[:-1, :-1, :], idx[1:, 1:, :])]
        for a, b in diag:
            keep = rng.random(a.size) < p_extra
            pairs.append((a.ravel()[keep], b.ravel()[keep], 0.3))
    a = np.concatenate([p[0] for p in pairs])
    b = np.concatenate([p[1] for p in pairs])
    scale = np.concatenate([np.full(p[0].size, p[2]) for p in pairs])
    g = scale * np.exp(rng.normal(0.0, 0.5, a.size))
    s = np.exp(rng.normal(0.0, 0.3, n)) * 0.5
    if shuffle:
        new_of_old = rng.permutation(n).astype(np.int64)
        a, b = new_of_old[a], new_of_old[b]
        s = s[np.argsort(new_of_old)]
    own = np.minimum(a, b)
    nei = np.maximum(a, b)
    order = np.argsort(own * n + nei, kind="stable")
    return Mesh(n, own[order].astype(np.int32), nei[order].astype(np.int32),
                np.ascontiguousarray(g[order]), np.ascontiguousarray(s))


def rhs_vector(n: int, seed: int = 11) -> np.ndarray:
    """A right-hand side b with values of order one."""
    return np.random.default_rng(seed).normal(0.0, 1.0, n)


def tiny_mesh() -> Mesh:
    """A hand-made 5-cell mesh (a ring of four cells around a centre cell, plus one ring
    face) used by the oracle's brute-force pins."""
    owner = np.array([0, 0, 0, 0, 1, 2, 3], dtype=np.int32)
    neighbour = np.array([1, 2, 3, 4, 2, 4, 4], dtype=np.int32)
    g = np.array([1.0, 2.0, 0.5, 1.5, 0.25, 0.75, 1.25])
    s = np.array([0.5, 1.0, 2.0, 0.25, 1.5])
    return Mesh(5, owner, neighbour, g, s)
