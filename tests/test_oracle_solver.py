"""Pins of the sparse-solver oracle (Sec. 3.2) against facts that do not come from the oracle:
hand-written matrices, textbook in-place Gauss-Seidel and Jacobi loops on tiny inputs,
closed-form invariants of the finite-volume Laplacian, and dense linear algebra."""
import numpy as np
import pytest

import synth
from synth import mesh as smesh
from oracle import solver as osol


def _tiny_ldu():
    m = smesh.tiny_mesh()
    upper = np.arange(1.0, 8.0)
    lower = -np.arange(1.0, 8.0)
    diag = np.array([10.0, 11.0, 12.0, 13.0, 14.0])
    return m, lower, diag, upper


def test_ldu_matrix_hand_written():
    m, lower, diag, upper = _tiny_ldu()
    A = osol.ldu_matrix(m.n_cells, m.owner, m.neighbour, lower, diag, upper).toarray()
    want = np.array([[10.0, 1.0, 2.0, 3.0, 4.0],
                     [-1.0, 11.0, 5.0, 0.0, 0.0],
                     [-2.0, -5.0, 12.0, 0.0, 6.0],
                     [-3.0, 0.0, 0.0, 13.0, 7.0],
                     [-4.0, 0.0, -6.0, -7.0, 14.0]])
    assert np.array_equal(A, want)
    x = np.array([1.0, -2.0, 0.5, 3.0, -1.0])
    assert np.array_equal(osol.spmv(osol.ldu_matrix(m.n_cells, m.owner, m.neighbour, lower, diag,
                                                    upper), x), want @ x)


def test_ldu_swap_is_transpose():
    mesh = smesh.grid_mesh(5, 4, 3, seed=3)
    rng = np.random.default_rng(0)
    lo, up = rng.normal(size=mesh.n_faces), rng.normal(size=mesh.n_faces)
    d = rng.normal(size=mesh.n_cells)
    A = osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, lo, d, up)
    At = osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, up, d, lo)
    assert (A.T - At).count_nonzero() == 0


def test_fv_laplacian_invariants():
    """Row sums equal the source (constants are in the operator's kernel apart from s), the
    operator is symmetric, and x^T A x = sum s x^2 + sum_f g (x_o - x_n)^2."""
    mesh = smesh.grid_mesh(6, 5, 4, seed=5)
    lo, d, up = osol.fv_laplacian(mesh.n_cells, mesh.owner, mesh.neighbour, mesh.face_coeff,
                                  mesh.cell_source)
    A = osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, lo, d, up)
    np.testing.assert_allclose(A @ np.ones(mesh.n_cells), mesh.cell_source, rtol=1e-13, atol=1e-13)
    assert abs(A - A.T).max() == 0.0
    x = np.random.default_rng(1).normal(size=mesh.n_cells)
    energy = (mesh.cell_source * x * x).sum() + (
        mesh.face_coeff * (x[mesh.owner] - x[mesh.neighbour]) ** 2).sum()
    assert abs(x @ (A @ x) - energy) <= 1e-12 * energy


def test_fv_laplacian_tiny_by_hand():
    m = smesh.tiny_mesh()
    lo, d, up = osol.fv_laplacian(m.n_cells, m.owner, m.neighbour, m.face_coeff, m.cell_source)
    # cell 0 touches faces 0-3 (g = 1, 2, 0.5, 1.5); cell 2 faces 1, 4, 5 (2, 0.25, 0.75)
    assert d[0] == 0.5 + 1.0 + 2.0 + 0.5 + 1.5
    assert d[2] == 2.0 + 2.0 + 0.25 + 0.75
    assert d[4] == 1.5 + 1.5 + 0.75 + 1.25
    assert np.array_equal(lo, -m.face_coeff) and np.array_equal(up, -m.face_coeff)


def _dd_matrix(n, seed, asym=True):
    """A random diagonally dominant sparse matrix on a small mesh graph."""
    mesh = smesh.grid_mesh(n, 3, 2, seed=seed)
    rng = np.random.default_rng(seed)
    up = -rng.random(mesh.n_faces)
    lo = up * (1.0 + (0.3 * rng.random(mesh.n_faces) if asym else 0.0))
    d = 7.0 + rng.random(mesh.n_cells)
    return mesh, osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, lo, d, up)


def _textbook_block_gs(Ad, b, x, part_ptr):
    """In-place Gauss-Seidel row by row inside each block; values of other blocks frozen at
    the start of the sweep (brute force on a dense matrix)."""
    n = Ad.shape[0]
    x_old = x.copy()
    x = x.copy()
    for I in range(len(part_ptr) - 1):
        lo, hi = part_ptr[I], part_ptr[I + 1]
        for r in range(lo, hi):
            acc = b[r]
            for c in range(n):
                if c == r:
                    continue
                v = x[c] if lo <= c < hi else x_old[c]
                acc -= Ad[r, c] * v
            x[r] = acc / Ad[r, r]
    return x


def test_gs_one_block_is_textbook_gauss_seidel():
    mesh, A = _dd_matrix(7, 21)
    n = mesh.n_cells
    rng = np.random.default_rng(2)
    b, x0 = rng.normal(size=n), rng.normal(size=n)
    got = osol.gauss_seidel(A, b, x0, [0, n], sweeps=1)
    want = _textbook_block_gs(A.toarray(), b, x0, [0, n])
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)


def test_gs_blocks_match_textbook():
    mesh, A = _dd_matrix(8, 22)
    n = mesh.n_cells
    parts = [0, 10, 11, 30, n]
    rng = np.random.default_rng(3)
    b, x0 = rng.normal(size=n), rng.normal(size=n)
    got = osol.gauss_seidel(A, b, x0, parts, sweeps=2)
    want = _textbook_block_gs(A.toarray(), b, _textbook_block_gs(A.toarray(), b, x0, parts), parts)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14)


def test_gs_singleton_blocks_is_jacobi():
    mesh, A = _dd_matrix(6, 23)
    n = mesh.n_cells
    rng = np.random.default_rng(4)
    b, x0 = rng.normal(size=n), rng.normal(size=n)
    Ad = A.toarray()
    D = np.diag(Ad)
    jacobi = (b - (Ad - np.diag(D)) @ x0) / D
    got = osol.gauss_seidel(A, b, x0, np.arange(n + 1), sweeps=1)
    np.testing.assert_allclose(got, jacobi, rtol=1e-13, atol=1e-14)


def test_gs_fixed_point_and_convergence():
    mesh = smesh.grid_mesh(6, 6, 5, seed=8)
    lo, d, up = osol.fv_laplacian(mesh.n_cells, mesh.owner, mesh.neighbour, mesh.face_coeff,
                                  mesh.cell_source)
    A = osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, lo, d, up)
    b = smesh.rhs_vector(mesh.n_cells)
    xs = np.linalg.solve(A.toarray(), b)
    parts = [0, 40, 95, 150, mesh.n_cells]
    np.testing.assert_allclose(osol.gauss_seidel(A, b, xs, parts, 1), xs, rtol=1e-11, atol=1e-12)
    x = osol.gauss_seidel(A, b, np.zeros(mesh.n_cells), parts, 300)
    assert np.abs(x - xs).max() <= 1e-9 * np.abs(xs).max()


def test_spmv_permutation_equivariance():
    """(P A P^T)(P x) = P (A x): renumbering cells and faces changes nothing but the order."""
    mesh = smesh.grid_mesh(5, 5, 4, seed=9, shuffle=False)
    rng = np.random.default_rng(5)
    lo, up = rng.normal(size=mesh.n_faces), rng.normal(size=mesh.n_faces)
    d = rng.normal(size=mesh.n_cells)
    x = rng.normal(size=mesh.n_cells)
    y = osol.spmv(osol.ldu_matrix(mesh.n_cells, mesh.owner, mesh.neighbour, lo, d, up), x)
    p = rng.permutation(mesh.n_cells)                   # new index of old cell
    a, b_ = p[mesh.owner], p[mesh.neighbour]
    flip = a > b_
    own, nei = np.where(flip, b_, a), np.where(flip, a, b_)
    lo2, up2 = np.where(flip, up, lo), np.where(flip, lo, up)
    d2 = np.empty_like(d); d2[p] = d
    x2 = np.empty_like(x); x2[p] = x
    y2 = osol.spmv(osol.ldu_matrix(mesh.n_cells, own, nei, lo2, d2, up2), x2)
    np.testing.assert_allclose(y2[p], y, rtol=1e-14, atol=1e-14)


def test_mesh_generator_shape():
    mesh = smesh.grid_mesh(10, 9, 8, seed=1)
    assert (mesh.owner < mesh.neighbour).all()
    key = mesh.owner.astype(np.int64) * mesh.n_cells + mesh.neighbour
    assert (np.diff(key) > 0).all()                       # sorted, no duplicate faces
    deg = np.bincount(mesh.owner, minlength=mesh.n_cells) + np.bincount(mesh.neighbour,
                                                                        minlength=mesh.n_cells)
    assert deg.min() >= 3 and deg.max() <= 12
    assert 6.0 < deg.mean() < 7.5


def test_level_sort_keeps_the_gauss_seidel_sweep():
    """Sorting the cells of a block row stably by dependency level (1 + the highest level of
    an earlier-numbered neighbour) keeps the order of every pair of neighbours, so the sweep
    in the sorted numbering is the sweep in the original one, cell by cell."""
    from collections import deque
    mesh = smesh.grid_mesh(9, 8, 7, seed=12)
    n = mesh.n_cells
    rng = np.random.default_rng(7)
    up = -rng.random(mesh.n_faces)
    lo = up * (1.0 + 0.3 * rng.random(mesh.n_faces))
    d = 7.0 + rng.random(n)
    b = rng.normal(size=n)
    nbrs = [[] for _ in range(n)]
    for a, c in zip(mesh.owner.tolist(), mesh.neighbour.tolist()):
        nbrs[a].append(c)
        nbrs[c].append(a)
    # a breadth-first numbering of the whole mesh (one block row)
    seen, order, q = np.zeros(n, bool), [], deque([0])
    seen[0] = True
    while q:
        c = q.popleft()
        order.append(c)
        for v in sorted(nbrs[c]):
            if not seen[v]:
                seen[v] = True
                q.append(v)
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    level = np.zeros(n, np.int64)
    for c in order:
        earlier = [level[v] + 1 for v in nbrs[c] if pos[v] < pos[c]]
        level[c] = max(earlier, default=0)
    sorted_order = sorted(order, key=lambda c: level[c])          # stable
    results = []
    for numbering in (order, sorted_order):
        new = np.empty(n, np.int64)
        new[numbering] = np.arange(n)
        a, c = new[mesh.owner], new[mesh.neighbour]
        flip = a > c
        own, nei = np.where(flip, c, a), np.where(flip, a, c)
        A = osol.ldu_matrix(n, own, nei, np.where(flip, up, lo), d[numbering], np.where(flip, lo, up))
        x = osol.gauss_seidel(A, b[numbering], np.zeros(n), [0, n], 2)
        out = np.empty(n)
        out[numbering] = x
        results.append(out)
    np.testing.assert_allclose(results[1], results[0], rtol=1e-13, atol=1e-15)
    assert not np.array_equal(np.array(order), np.array(sorted_order))
