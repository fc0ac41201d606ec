"""Parity of the sparse-solver kernels (Sec. 3.2) with the FP64 oracle, through the C ABI.

Tolerances, derived from the arithmetic: the block format is a copy (bit-exact); SpMV sums at
most 13 FP64 products per row in another order than the oracle, so |y - y_ref| <=
16 eps sum_c |a_rc x_c|; Gauss-Seidel multiplies by the reciprocal of the diagonal instead of
dividing and sums in another order, errors that the forward substitution of a diagonally
dominant matrix does not amplify: |x - x_ref| <= 1e-12 max|x_ref| after a few sweeps.
Double-float arithmetic splits every FP64 operand into two FP32 numbers (48 of its 53 bits)
and forms each product to about 2^-47 and the running sum to about 2^-48 of its size, so a row
of at most 13 terms lands within 2^-42 sum_c |a_rc x_c| (SpMV); the Gauss-Seidel bound above
holds as well.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import mesh as smesh
from oracle import solver as osol

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def mod():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2508_18969_gb300 import solver
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return solver


def _renumbered(nx, ny, nz, parts, seed=7, p_extra=0.15, decompose=True, mod=None):
    """Synthetic mesh renumbered by the decomposition; returns (n, owner, neighbour,
    part_ptr, face coefficients, cell sources) in the new numbering."""
    m = smesh.grid_mesh(nx, ny, nz, seed=seed, p_extra=p_extra)
    if decompose:
        new_of_old, part_ptr = mod.mesh_decompose(m.n_cells, m.owner, m.neighbour, parts)
        own, nei, face_old, _ = mod.mesh_renumber(m.n_cells, m.owner, m.neighbour, new_of_old)
        s = np.empty(m.n_cells)
        s[new_of_old] = m.cell_source
        return m.n_cells, own, nei, part_ptr, m.face_coeff[face_old], s
    part_ptr = np.linspace(0, m.n_cells, parts + 1).round().astype(np.int64)
    return m.n_cells, m.owner, m.neighbour, part_ptr, m.face_coeff, m.cell_source


def _cuda(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _asym_ldu(n, nf, seed):
    rng = np.random.default_rng(seed)
    upper = -rng.random(nf) - 0.1
    lower = upper * (1.0 + 0.5 * rng.random(nf))
    diag = 14.0 + rng.random(n)
    return lower, diag, upper


def _solver(mod, n, own, nei, part_ptr, arith=0):
    return mod.Solver(n, own, nei, part_ptr, arithmetic=arith)


ARITH = [0, 1]                           # DF_SOLVER_FP64, DF_SOLVER_DOUBLE_FLOAT


def _rowtol(arith):
    return 16 * EPS if arith == 0 else 2.0 ** -42


CASES = [
    # (nx, ny, nz, parts, decompose): several block rows with ragged sizes; one block row;
    # a numbering that was not decomposed (short Gauss-Seidel runs)
    (23, 19, 17, 7, True),
    (14, 14, 14, 1, True),
    (17, 13, 11, 5, False),
]


@pytest.mark.parametrize("case", CASES)
def test_block_format_is_exact(mod, case):
    n, own, nei, pp, g, s = _renumbered(*case[:4], decompose=case[4], mod=mod)
    lo, d, up = _asym_ldu(n, own.size, 1)
    S = _solver(mod, n, own, nei, pp)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    rp, col, val = S.export_csr()
    A = osol.ldu_matrix(n, own, nei, lo, d, up)
    assert np.array_equal(rp, A.indptr) and np.array_equal(col, A.indices)
    assert np.array_equal(val, A.data)
    info = S.info()
    assert info["nnz"] == A.nnz and info["max_part"] == np.diff(pp).max()
    S.close()


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("case", CASES)
def test_spmv_and_residual(mod, case, arith):
    n, own, nei, pp, g, s = _renumbered(*case[:4], decompose=case[4], mod=mod)
    lo, d, up = _asym_ldu(n, own.size, 2)
    A = osol.ldu_matrix(n, own, nei, lo, d, up)
    x = np.random.default_rng(3).normal(size=n)
    b = np.random.default_rng(4).normal(size=n)
    S = _solver(mod, n, own, nei, pp, arith)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    y = S.spmv(_cuda(x)).cpu().numpy()
    r = S.residual(_cuda(b), _cuda(x)).cpu().numpy()
    bound = _rowtol(arith) * (abs(A) @ np.abs(x))
    assert (np.abs(y - osol.spmv(A, x)) <= bound).all()
    assert (np.abs(r - osol.residual(A, b, x)) <= bound + 4 * EPS * np.abs(b)).all()
    S.close()


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_gauss_seidel(mod, case, sweeps, arith):
    n, own, nei, pp, g, s = _renumbered(*case[:4], decompose=case[4], mod=mod)
    lo, d, up = _asym_ldu(n, own.size, 5)
    A = osol.ldu_matrix(n, own, nei, lo, d, up)
    b = smesh.rhs_vector(n)
    x0 = np.random.default_rng(6).normal(size=n)
    S = _solver(mod, n, own, nei, pp, arith)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    xd = _cuda(x0)
    S.gauss_seidel(_cuda(b), xd, sweeps)
    got = xd.cpu().numpy()
    want = osol.gauss_seidel(A, b, x0, pp, sweeps)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # deterministic: the same sweep again gives the same bits
    xd2 = _cuda(x0)
    S.gauss_seidel(_cuda(b), xd2, sweeps)
    assert np.array_equal(xd2.cpu().numpy(), got)
    S.close()


@pytest.mark.parametrize("arith", ARITH)
def test_singleton_blocks_and_isolated_cells(mod, arith):
    """Every cell its own block row (block Gauss-Seidel = Jacobi), plus cells with no faces."""
    m = smesh.grid_mesh(6, 5, 4, seed=2)
    n = m.n_cells + 3                                 # three isolated cells at the end
    lo, d, up = _asym_ldu(n, m.n_faces, 7)
    pp = np.arange(n + 1)
    S = _solver(mod, n, m.owner, m.neighbour, pp, arith)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    A = osol.ldu_matrix(n, m.owner, m.neighbour, lo, d, up)
    b = smesh.rhs_vector(n)
    x0 = np.random.default_rng(8).normal(size=n)
    xd = _cuda(x0)
    S.gauss_seidel(_cuda(b), xd, 2)
    want = osol.gauss_seidel(A, b, x0, pp, 2)
    assert np.abs(xd.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    y = S.spmv(_cuda(x0)).cpu().numpy()
    assert (np.abs(y - A @ x0) <= _rowtol(arith) * (abs(A) @ np.abs(x0))).all()
    S.close()


def test_fv_laplacian_then_smoothing(mod):
    """Sec. 3.2.4 assembly on the device, conversion, and Gauss-Seidel smoothing: the LDU
    arrays match the oracle's, and 40 sweeps match the oracle's 40 sweeps."""
    n, own, nei, pp, g, s = _renumbered(24, 22, 20, 6, mod=mod)
    S = _solver(mod, n, own, nei, pp)
    lo, d, up = S.fv_laplacian(_cuda(g), _cuda(s))
    lo_r, d_r, up_r = osol.fv_laplacian(n, own, nei, g, s)
    assert np.array_equal(lo.cpu().numpy(), lo_r) and np.array_equal(up.cpu().numpy(), up_r)
    np.testing.assert_allclose(d.cpu().numpy(), d_r, rtol=16 * EPS, atol=0)
    S.convert(lo, d, up)
    A = osol.ldu_matrix(n, own, nei, lo_r, d_r, up_r)
    b = smesh.rhs_vector(n)
    xd = _cuda(np.zeros(n))
    S.gauss_seidel(_cuda(b), xd, 40)
    want = osol.gauss_seidel(A, b, np.zeros(n), pp, 40)
    assert np.abs(xd.cpu().numpy() - want).max() <= 1e-11 * np.abs(want).max()
    r = S.residual(_cuda(b), xd).cpu().numpy()
    assert np.linalg.norm(r) < 1e-3 * np.linalg.norm(b)
    S.close()


def test_largest_block_row(mod):
    """One block row of 8000 cells (shared memory of a single sweeping warp: 64 KB)."""
    n, own, nei, pp, g, s = _renumbered(20, 20, 20, 1, mod=mod)
    lo, d, up = _asym_ldu(n, own.size, 3)
    A = osol.ldu_matrix(n, own, nei, lo, d, up)
    S = _solver(mod, n, own, nei, pp)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    b = smesh.rhs_vector(n)
    x0 = np.random.default_rng(1).normal(size=n)
    xd = _cuda(x0)
    S.gauss_seidel(_cuda(b), xd, 2)
    want = osol.gauss_seidel(A, b, x0, pp, 2)
    assert np.abs(xd.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    S.close()


def test_argument_errors(mod):
    from paper_2508_18969_gb300 import DFError
    import torch
    m = smesh.grid_mesh(5, 4, 3, seed=1)
    n = m.n_cells
    S = _solver(mod, n, m.owner, m.neighbour, [0, n])
    x = _cuda(np.ones(n))
    with pytest.raises(DFError, match="INVALID_ARG"):
        S.spmv(x)                                     # no matrix converted yet
    lo, d, up = _asym_ldu(n, m.n_faces, 9)
    S.convert(_cuda(lo), _cuda(d), _cuda(up))
    with pytest.raises(DFError, match="INVALID_ARG"):
        S.spmv(x, x)                                  # x aliases y
    with pytest.raises(DFError, match="INVALID_ARG"):
        S.gauss_seidel(x, x, 1)
    S.close()
    big = smesh.grid_mesh(21, 20, 20, seed=1)         # 8400 cells in one block row
    with pytest.raises(DFError, match="INVALID_ARG"):
        mod.Solver(big.n_cells, big.owner, big.neighbour, [0, big.n_cells])
    own = np.concatenate([m.owner, m.owner[:1]])
    nei = np.concatenate([m.neighbour, m.neighbour[:1]])
    with pytest.raises(DFError, match="INVALID_ARG"):
        mod.Solver(n, own, nei, [0, n])               # two faces between one pair of cells
    with pytest.raises(DFError, match="INVALID_ARG"):
        mod.Solver(n, m.neighbour, m.owner, [0, n])   # owner > neighbour
    torch.cuda.synchronize()


SOLVER_WORKLOAD = (256, 256, 128, 16384)  # the bench's mesh-8m workload: 8.4M cells, 512 per row


@pytest.mark.slow
@pytest.mark.parametrize("arith", ARITH)
def test_full_size_sampled_blocks(mod, arith):
    """At the bench's size and launch shape: one SpMV and one Gauss-Seidel sweep, checked on
    sampled block rows. A block row's sweep depends only on its own rows and on the values
    of other blocks before the sweep, so the oracle solves each sampled block alone."""
    import torch
    n, own, nei, pp, g, s = _renumbered(*SOLVER_WORKLOAD, mod=mod)
    S = _solver(mod, n, own, nei, pp, arith)
    lo, d, up = S.fv_laplacian(_cuda(g), _cuda(s))
    S.convert(lo, d, up)
    lo_h, d_h, up_h = lo.cpu().numpy(), d.cpu().numpy(), up.cpu().numpy()
    x0 = np.random.default_rng(12).normal(size=n)
    b = smesh.rhs_vector(n)
    y = S.spmv(_cuda(x0)).cpu().numpy()
    xd = _cuda(x0)
    S.gauss_seidel(_cuda(b), xd, 1)
    x1 = xd.cpu().numpy()
    torch.cuda.synchronize()
    by_nei = np.argsort(nei, kind="stable")
    nei_sorted = nei[by_nei]
    rng = np.random.default_rng(13)
    for I in sorted(rng.choice(len(pp) - 1, 6, replace=False).tolist()) + [len(pp) - 2]:
        r0, r1 = int(pp[I]), int(pp[I + 1])
        fa = np.arange(np.searchsorted(own, r0), np.searchsorted(own, r1))       # owner in block
        fb = by_nei[np.searchsorted(nei_sorted, r0):np.searchsorted(nei_sorted, r1)]
        rows = np.concatenate([np.arange(r0, r1), own[fa], nei[fb]]) - r0
        cols = np.concatenate([np.arange(r0, r1), nei[fa], own[fb]])
        vals = np.concatenate([d_h[r0:r1], up_h[fa], lo_h[fb]])
        Ablk = sp.csr_matrix((vals, (rows, cols)), shape=(r1 - r0, n))
        yb = Ablk @ x0
        assert (np.abs(y[r0:r1] - yb) <= _rowtol(arith) * (abs(Ablk) @ np.abs(x0))).all()
        inside = (cols >= r0) & (cols < r1)
        Aii = sp.csr_matrix((vals[inside], (rows[inside], cols[inside] - r0)), shape=(r1 - r0,) * 2)
        Aio = sp.csr_matrix((vals[~inside], (rows[~inside], cols[~inside])), shape=(r1 - r0, n))
        want = osol.gauss_seidel(Aii, b[r0:r1] - Aio @ x0, x0[r0:r1], [0, r1 - r0], 1)
        assert np.abs(x1[r0:r1] - want).max() <= 1e-12 * np.abs(want).max()
    S.close()
