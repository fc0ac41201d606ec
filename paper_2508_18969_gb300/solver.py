"""Python binding of the sparse-solver module (include/df_solver.h): same names as the C ABI.

Host helpers take and return numpy arrays; the solver's kernels take torch float64 tensors on
the solver's CUDA device. Argument marshalling only: the decomposition runs in the library's
host code, every matrix and vector operation in its CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .api import DFError, _ptr, _stream


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _faces(owner, neighbour):
    o = np.ascontiguousarray(owner, dtype=np.int32)
    n = np.ascontiguousarray(neighbour, dtype=np.int32)
    if o.shape != n.shape or o.ndim != 1:
        raise ValueError("owner and neighbour must be 1-D arrays of one length")
    return o, n


def mesh_decompose(n_cells: int, owner, neighbour, n_parts: int):
    """Sec. 3.2.1 partition + renumbering. Returns (new_of_old int32 [n_cells],
    part_ptr int64 [n_parts + 1])."""
    lib = L.load()
    o, n = _faces(owner, neighbour)
    new_of_old = np.empty(int(n_cells), dtype=np.int32)
    part_ptr = np.empty(int(n_parts) + 1, dtype=np.int64)
    rc = lib.df_mesh_decompose(int(n_cells), o.size, _np_ptr(o), _np_ptr(n), int(n_parts),
                               _np_ptr(new_of_old), _np_ptr(part_ptr))
    if rc != L.DF_OK:
        raise DFError(rc, lib.df_get_last_error(None).decode())
    return new_of_old, part_ptr


def mesh_renumber(n_cells: int, owner, neighbour, new_of_old):
    """The mesh in the numbering new_of_old, LDU face order. Returns (owner, neighbour,
    face_old int64, face_flip uint8)."""
    lib = L.load()
    o, n = _faces(owner, neighbour)
    p = np.ascontiguousarray(new_of_old, dtype=np.int32)
    oo = np.empty_like(o)
    no = np.empty_like(n)
    fo = np.empty(o.size, dtype=np.int64)
    ff = np.empty(o.size, dtype=np.uint8)
    rc = lib.df_mesh_renumber(int(n_cells), o.size, _np_ptr(o), _np_ptr(n), _np_ptr(p),
                              _np_ptr(oo), _np_ptr(no), _np_ptr(fo), _np_ptr(ff))
    if rc != L.DF_OK:
        raise DFError(rc, lib.df_get_last_error(None).decode())
    return oo, no, fo, ff


class Solver:
    """Owns a df_solver: the block-sparse structure of one mesh's matrices on one GPU."""

    def __init__(self, n_cells: int, owner, neighbour, part_ptr, device: int = 0,
                 arithmetic: int = L.DF_SOLVER_FP64):
        self._lib = L.load()
        o, n = _faces(owner, neighbour)
        pp = np.ascontiguousarray(part_ptr, dtype=np.int64)
        h = C.c_void_p()
        rc = self._lib.df_solver_create(int(n_cells), o.size, _np_ptr(o), _np_ptr(n),
                                        pp.size - 1, _np_ptr(pp), int(device), C.byref(h))
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(None).decode())
        self.h = h
        self.n_cells = int(n_cells)
        self.n_faces = int(o.size)
        self.device = torch.device("cuda", device)
        if arithmetic != L.DF_SOLVER_FP64:
            self.set_arithmetic(arithmetic)

    def close(self):
        if getattr(self, "h", None):
            self._lib.df_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_solver_get_last_error(self.h).decode())

    def _vec(self, t, size, name):
        if t is None:
            return None
        if t.dtype != torch.float64 or t.device != self.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor on {self.device}")
        if t.numel() != size:
            raise ValueError(f"{name} must have {size} elements")
        return _ptr(t)

    def info(self):
        i = L.SolverInfo()
        self._check(self._lib.df_solver_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in L.SolverInfo._fields_}

    def set_arithmetic(self, arithmetic: int):
        """L.DF_SOLVER_FP64 (default) or L.DF_SOLVER_DOUBLE_FLOAT."""
        self._check(self._lib.df_solver_set_arithmetic(self.h, int(arithmetic)))

    def convert(self, lower, diag, upper, stream=None):
        nf, n = self.n_faces, self.n_cells
        self._check(self._lib.df_solver_convert(self.h, self._vec(lower, nf, "lower"),
                                                self._vec(diag, n, "diag"),
                                                self._vec(upper, nf, "upper"), _stream(stream)))

    def spmv(self, x, y=None, stream=None):
        if y is None:
            y = torch.empty_like(x)
        n = self.n_cells
        self._check(self._lib.df_solver_spmv(self.h, self._vec(x, n, "x"), self._vec(y, n, "y"),
                                             _stream(stream)))
        return y

    def residual(self, b, x, r=None, stream=None):
        if r is None:
            r = torch.empty_like(x)
        n = self.n_cells
        self._check(self._lib.df_solver_residual(self.h, self._vec(b, n, "b"), self._vec(x, n, "x"),
                                                 self._vec(r, n, "r"), _stream(stream)))
        return r

    def gauss_seidel(self, b, x, sweeps: int = 1, stream=None):
        n = self.n_cells
        self._check(self._lib.df_solver_gauss_seidel(self.h, self._vec(b, n, "b"),
                                                     self._vec(x, n, "x"), int(sweeps),
                                                     _stream(stream)))
        return x

    def fv_laplacian(self, face_coeff, cell_source, out=None, stream=None):
        nf, n = self.n_faces, self.n_cells
        if out is None:
            opts = dict(dtype=torch.float64, device=self.device)
            out = (torch.empty(nf, **opts), torch.empty(n, **opts), torch.empty(nf, **opts))
        lower, diag, upper = out
        self._check(self._lib.df_fv_laplacian(
            self.h, self._vec(face_coeff, nf, "face_coeff"), self._vec(cell_source, n, "cell_source"),
            self._vec(lower, nf, "lower"), self._vec(diag, n, "diag"), self._vec(upper, nf, "upper"),
            _stream(stream)))
        return lower, diag, upper

    def export_csr(self):
        nnz = self.info()["nnz"]
        rp = np.empty(self.n_cells + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.float64)
        self._check(self._lib.df_solver_export_csr(self.h, _np_ptr(rp), _np_ptr(col), _np_ptr(val)))
        return rp, col, val
