"""FP64 CPU oracle of the sparse-solver kernels -- TEST INFRASTRUCTURE ONLY.

Plain NumPy/SciPy code that the CUDA sparse kernels are checked against; it shares nothing
with them. What it follows:

  * Sec. 3.2 (many-core PDE solver): the transport equations are discretised by finite
    volumes into sparse systems held by OpenFOAM in LDU form; the paper converts them to a
    t x t block-sparse matrix whose block row I holds the rows of subdomain I, and
    implements SpMV and Gauss-Seidel smoothing on it.
  * Sec. 3.2.3: each thread smooths the rows of its own block row; the couplings through the
    off-diagonal blocks (1.63 % of the nonzeros after reordering) are not waited for. Read
    here as: within a block row the sweep is the sequential Gauss-Seidel of that block (rows
    in ascending order, already-updated values for earlier rows of the block), while every
    coupling to another block uses the value from before the sweep (block-Jacobi between
    blocks). This is the deterministic form of the paper's scheme.
  * Sec. 3.2.4 (matrix construction): the face-to-cell Laplacian, read in its textbook
    finite-volume form with a positive face coefficient g_f (diffusivity x area / distance)
    and a positive diagonal source s_c (e.g. an implicit time term): row c of the matrix is
    s_c x_c + sum over faces f of c of g_f (x_c - x_neighbour).
  * Silent, textbook: LDU addressing (OpenFOAM's lduMatrix): face f couples owner[f] <
    neighbour[f]; A[owner, neighbour] = upper[f], A[neighbour, owner] = lower[f],
    A[c, c] = diag[c].

Functions: ldu_matrix, spmv, residual, gauss_seidel, fv_laplacian.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def ldu_matrix(n_cells, owner, neighbour, lower, diag, upper) -> sp.csr_matrix:
    """The sparse matrix an LDU triple stands for (OpenFOAM addressing, see header)."""
    n = int(n_cells)
    owner = np.asarray(owner, dtype=np.int64)
    neighbour = np.asarray(neighbour, dtype=np.int64)
    cells = np.arange(n, dtype=np.int64)
    rows = np.concatenate([cells, owner, neighbour])
    cols = np.concatenate([cells, neighbour, owner])
    vals = np.concatenate([np.asarray(diag, np.float64), np.asarray(upper, np.float64),
                           np.asarray(lower, np.float64)])
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sort_indices()
    return A


def spmv(A: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """y = A x (Sec. 3.2.3, the SpMV kernel)."""
    return A @ np.asarray(x, np.float64)


def residual(A: sp.csr_matrix, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """r = b - A x."""
    return np.asarray(b, np.float64) - A @ np.asarray(x, np.float64)


def part_of_rows(n: int, part_ptr) -> np.ndarray:
    """Block-row index of every row: rows part_ptr[I] .. part_ptr[I+1]-1 form block row I."""
    part_ptr = np.asarray(part_ptr, dtype=np.int64)
    return np.repeat(np.arange(part_ptr.size - 1), np.diff(part_ptr))


def gauss_seidel(A: sp.csr_matrix, b: np.ndarray, x: np.ndarray, part_ptr,
                 sweeps: int = 1) -> np.ndarray:
    """Block Gauss-Seidel sweeps (Sec. 3.2.3, reading in the header).

    One sweep, written as the linear-algebra statement of the scheme: split A into its
    block-diagonal part B (entries whose row and column lie in the same block row) and the
    rest O; split B into its lower triangle with the diagonal, L, and its strict upper
    triangle U. Then (L) x_new = b - U x_old - O x_old, solved by forward substitution,
    which is exactly the row-by-row update of sequential Gauss-Seidel inside each block.
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    part = part_of_rows(n, part_ptr)
    coo = A.tocoo()
    same = part[coo.row] == part[coo.col]
    B = sp.csr_matrix((coo.data[same], (coo.row[same], coo.col[same])), shape=(n, n))
    O = sp.csr_matrix((coo.data[~same], (coo.row[~same], coo.col[~same])), shape=(n, n))
    L = sp.tril(B, k=0, format="csr")
    U = sp.triu(B, k=1, format="csr")
    b = np.asarray(b, np.float64)
    x = np.array(x, dtype=np.float64)
    for _ in range(int(sweeps)):
        rhs = b - U @ x - O @ x
        x = spla.spsolve_triangular(L, rhs, lower=True)
    return x


def fv_laplacian(n_cells, owner, neighbour, g, s):
    """LDU coefficients of the finite-volume operator s_c x_c + sum_f g_f (x_c - x_nb)
    (Sec. 3.2.4): lower = upper = -g, diag = s + the sum of g over the faces of each cell."""
    g = np.asarray(g, np.float64)
    diag = np.array(s, dtype=np.float64)
    np.add.at(diag, np.asarray(owner, np.int64), g)
    np.add.at(diag, np.asarray(neighbour, np.int64), g)
    return -g.copy(), diag, -g.copy()
