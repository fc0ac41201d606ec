"""GB300-native reaction step of the DeepFlame method (arxiv 2508.18969).

The per-cell chemistry step -- real-fluid Peng-Robinson state, Box-Cox/Z-score inputs,
chemistry MLP on tcgen05 tensor cores, Newton recovery of T from conserved enthalpy --
runs in hand-written sm_103a CUDA kernels behind the C ABI of include/df.h (libdfgb.so).
The property network (a PRNet-style surrogate of the real-fluid state) is behind
include/df_propnet.h. The sparse-solver module of the method's PDE side (Sec. 3.2: mesh decomposition, block-sparse
SpMV and Gauss-Seidel, conflict-free assembly) is behind include/df_solver.h. This package is
the thin Python binding of both.
"""
from ._lib import (DF_BF16, DF_FP8_E4M3, DF_FP32, DF_CELL_NO_ROOT, DF_CELL_NONFINITE,  # noqa: F401
                   DF_CELL_NOT_CONVERGED, DF_GELU_TABLE, DF_GELU_TANH, DF_SOLVER_DOUBLE_FLOAT,
                   DF_SOLVER_FP64, DF_TILE_PAIR, DF_HOST_DIRECT, LIB_PATH)
from .api import ChemStepFunction, DFError, MLPEOSFunction, State, version  # noqa: F401
from .solver import Solver, mesh_decompose, mesh_renumber  # noqa: F401
from .propnet import PropNet  # noqa: F401
