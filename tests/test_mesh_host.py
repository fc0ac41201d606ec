"""Host logic of the sparse-solver module (no GPU): mesh decomposition into block rows,
Cuthill-McKee + level numbering, renumbering into LDU face order, argument checks."""
import numpy as np
import pytest

from synth import mesh as smesh


@pytest.fixture(scope="module")
def sol():
    import __graft_entry__ as g
    g.build()
    from paper_2508_18969_gb300 import solver
    return solver


def _levels_in_numbering(n, owner, neighbour, part_ptr):
    """Dependency level of every cell in the given numbering: 1 + the highest level among its
    earlier-numbered neighbours of the same block row."""
    part = np.repeat(np.arange(len(part_ptr) - 1), np.diff(part_ptr))
    nbrs = [[] for _ in range(n)]
    for a, b in zip(owner.tolist(), neighbour.tolist()):
        if part[a] == part[b]:
            lo, hi = min(a, b), max(a, b)
            nbrs[hi].append(lo)
    lv = np.zeros(n, dtype=np.int64)
    for r in range(n):
        if nbrs[r]:
            lv[r] = 1 + max(lv[c] for c in nbrs[r])
    return lv


def test_decompose_permutation_balance_and_levels(sol):
    m = smesh.grid_mesh(20, 18, 16, seed=4)
    t = 12
    new_of_old, part_ptr = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, t)
    assert np.array_equal(np.sort(new_of_old), np.arange(m.n_cells))
    assert part_ptr[0] == 0 and part_ptr[-1] == m.n_cells
    sizes = np.diff(part_ptr)
    assert sizes.min() >= 1
    assert sizes.max() - sizes.min() <= 4                     # ceil(log2 12) levels of rounding
    own, nei, face_old, flip = sol.mesh_renumber(m.n_cells, m.owner, m.neighbour, new_of_old)
    lv = _levels_in_numbering(m.n_cells, own, nei, part_ptr)
    for I in range(t):
        seg = lv[part_ptr[I]:part_ptr[I + 1]]
        assert (np.diff(seg) >= 0).all(), "cells of a block row are not in level order"


def test_decompose_quality_on_a_grid(sol):
    """Recursive bisection of a 32^3 grid into 8 parts: axis planes would cut 3 x 32^2 = 3072
    of ~95k faces. Breadth-first fronts grown from a corner are diagonal planes, whose cross
    sections hold up to ~2.3x as many faces; the bound allows that and no more."""
    m = smesh.grid_mesh(32, 32, 32, seed=6, p_extra=0.0)
    new_of_old, part_ptr = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, 8)
    part = np.repeat(np.arange(8), np.diff(part_ptr))
    cut = (part[new_of_old[m.owner]] != part[new_of_old[m.neighbour]]).sum()
    assert cut <= 2.5 * 3072, cut


def test_decompose_deterministic(sol):
    m = smesh.grid_mesh(30, 25, 20, seed=2)
    a = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, 7)
    b = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, 7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_decompose_edge_cases(sol):
    m = smesh.grid_mesh(6, 5, 4, seed=3)
    p, pp = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, 1)
    assert list(pp) == [0, m.n_cells] and np.array_equal(np.sort(p), np.arange(m.n_cells))
    p, pp = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, m.n_cells)
    assert np.array_equal(pp, np.arange(m.n_cells + 1))
    # two disconnected grids and an isolated cell
    a = smesh.grid_mesh(5, 4, 3, seed=1, shuffle=False)
    n = 2 * a.n_cells + 1
    own = np.concatenate([a.owner, a.owner + a.n_cells])
    nei = np.concatenate([a.neighbour, a.neighbour + a.n_cells])
    p, pp = sol.mesh_decompose(n, own, nei, 5)
    assert np.array_equal(np.sort(p), np.arange(n)) and pp[-1] == n


def test_renumber_faces(sol):
    m = smesh.grid_mesh(9, 8, 7, seed=5)
    rng = np.random.default_rng(0)
    perm = rng.permutation(m.n_cells).astype(np.int32)
    own, nei, face_old, flip = sol.mesh_renumber(m.n_cells, m.owner, m.neighbour, perm)
    assert (own < nei).all()
    key = own.astype(np.int64) * m.n_cells + nei
    assert (np.diff(key) > 0).all()
    assert np.array_equal(np.sort(face_old), np.arange(m.n_faces))
    a, b = perm[m.owner[face_old]], perm[m.neighbour[face_old]]
    assert np.array_equal(np.minimum(a, b), own) and np.array_equal(np.maximum(a, b), nei)
    assert np.array_equal(flip.astype(bool), a > b)


def test_host_argument_checks(sol):
    from paper_2508_18969_gb300 import DFError
    m = smesh.tiny_mesh()
    with pytest.raises(DFError, match="INVALID_ARG"):
        sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, 6)
    bad = m.neighbour.copy()
    bad[0] = 9
    with pytest.raises(DFError, match="INVALID_ARG"):
        sol.mesh_decompose(m.n_cells, m.owner, bad, 2)
    with pytest.raises(DFError, match="INVALID_ARG"):
        sol.mesh_renumber(m.n_cells, m.owner, m.neighbour, np.zeros(m.n_cells, np.int32))
