"""ctypes declarations of the C ABI in include/df.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfgb.so")

DF_OK = 0
DF_ERR_INVALID_ARG = 1
DF_ERR_CUDA = 2
DF_ERR_NOT_CONVERGED = 3
DF_ERR_NONFINITE_INPUT = 4
DF_ERR_DT_MISMATCH = 5
DF_ERR_UNSUPPORTED = 6
DF_ERR_OOM = 7
DF_ERR_TIMEOUT = 8
STATUS_NAMES = {0: "DF_OK", 1: "DF_ERR_INVALID_ARG", 2: "DF_ERR_CUDA", 3: "DF_ERR_NOT_CONVERGED",
                4: "DF_ERR_NONFINITE_INPUT", 5: "DF_ERR_DT_MISMATCH", 6: "DF_ERR_UNSUPPORTED",
                7: "DF_ERR_OOM", 8: "DF_ERR_TIMEOUT"}

DF_COMPACT_STATIC_MAX_CELLS = 1 << 26

DF_CELL_NOT_CONVERGED = 1
DF_CELL_NO_ROOT = 2
DF_CELL_NONFINITE = 4

DF_FP32, DF_BF16, DF_FP8_E4M3 = 0, 1, 2
DF_GELU_TANH, DF_GELU_TABLE = 0, 1
DF_HOST_DIRECT = -1     # df_chem_step_host: kernels access the host arrays in place
DF_TILE_PAIR = 0x1000   # df_get_tiles: the layer runs on CTA pairs (cta_group::2)

DF_PARAM_WEIGHTS, DF_PARAM_GRADS, DF_PARAM_ADAM_M, DF_PARAM_ADAM_V = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)


class MechDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("W", _dp), ("Tc", _dp), ("pc", _dp), ("omega", _dp),
                ("kij", _dp), ("nasa", _dp)]


class MlpDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.POINTER(C.c_int32)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("lambda_", C.c_double), ("in_mean", _dp), ("in_std", _dp), ("out_mean", _dp),
                ("out_std", _dp), ("dt", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_flagged", C.c_int64), ("newton_iterations", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("T_react", C.c_double), ("newton_tol", C.c_double),
                ("newton_max_iter", C.c_int32), ("device", C.c_int32), ("batch_cells", C.c_int64),
                ("gelu_mode", C.c_int32)]


class Adam(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


class SolverInfo(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_faces", C.c_int64), ("n_parts", C.c_int64),
                ("nnz", C.c_int64), ("nnz_offblock", C.c_int64), ("n_halo", C.c_int64),
                ("n_runs", C.c_int64), ("max_part", C.c_int32), ("max_runs", C.c_int32),
                ("device_bytes", C.c_int64), ("n_chunks", C.c_int64)]


DF_SOLVER_MAX_PART = 8192
DF_SOLVER_FP64, DF_SOLVER_DOUBLE_FLOAT = 0, 1

_VP = C.c_void_p
_I64 = C.c_int64
_ST = C.c_int32

# name -> (restype, argtypes)
SIGNATURES = {
    "df_state_create": (_ST, [C.POINTER(MechDesc), C.POINTER(MlpDesc), C.POINTER(Options),
                              C.POINTER(_VP)]),
    "df_state_destroy": (None, [_VP]),
    "df_real_fluid_props": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    "df_transport_props": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP]),
    "df_chem_step": (_ST, [_VP, _I64, C.c_double, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "df_chem_step_host": (_ST, [_VP, _I64, C.c_double, _VP, _VP, _VP, _I64, _VP, _I64, _VP]),
    "df_chem_source": (_ST, [_VP, _I64, C.c_double, _VP, _VP, _VP, _I64, _VP, _I64, _VP, _VP, _VP,
                             _VP]),
    "df_chem_jacobian": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "df_chem_step_vjp": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP, _I64, _VP, _VP, _I64, _VP]),
    "df_get_step_summary": (_ST, [_VP, _VP, C.POINTER(StepStats)]),
    "df_active_compact": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP]),
    "df_eos_pre": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    "df_mlp_forward": (_ST, [_VP, _I64, _VP, _VP, _VP]),
    "df_eos_post": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _VP]),
    "df_active_compact_static": (_ST, [_I64, C.c_double, _VP, _VP, _VP, _VP]),
    "df_train_step": (_ST, [_VP, _I64, _VP, _VP, _VP, _VP, _I64, C.POINTER(Adam), _VP, _VP]),
    "df_mlp_forward_train": (_ST, [_VP, _I64, _VP, _VP, _VP]),
    "df_mlp_backward": (_ST, [_VP, _I64, _VP, _VP, _VP]),
    "df_adam_step": (_ST, [_VP, C.POINTER(Adam), _VP]),
    "df_get_params": (_ST, [_VP, C.c_int32, C.c_int32, _VP, _VP, _VP]),
    "df_train_get_step": (_ST, [_VP, C.POINTER(_I64)]),
    "df_state_save": (_ST, [_VP, C.c_char_p]),
    "df_state_load": (_ST, [_VP, C.c_char_p]),
    "df_autotune": (_ST, [_VP, _I64, C.c_char_p, _VP]),
    "df_get_tiles": (_ST, [_VP, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
    "df_graph_create": (_ST, [_VP, _I64, C.c_double, _VP, _VP, _VP, _I64, _VP, _VP, C.POINTER(_VP)]),
    "df_graph_launch": (_ST, [_VP, _VP]),
    "df_graph_destroy": (None, [_VP]),
    "df_profile_enable": (_ST, [_VP, C.c_int32]),
    "df_set_wait_limit": (_ST, [_VP, _I64]),
    "df_profile_read": (_ST, [_VP, C.c_int32, C.c_char_p, C.POINTER(_I64), C.POINTER(C.c_double),
                              C.POINTER(C.c_int32)]),
    "df_get_last_error": (C.c_char_p, [_VP]),
    # property network (include/df_propnet.h)
    "df_network_create": (_ST, [C.POINTER(MlpDesc), C.POINTER(Options), C.POINTER(_VP)]),
    "df_propnet_infer": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _I64, _VP]),
    "df_propnet_train_step": (_ST, [_VP, _I64, _VP, _VP, _VP, _I64, _VP, _I64, C.POINTER(Adam), _VP,
                                    _VP]),
    # sparse-solver module (include/df_solver.h)
    "df_mesh_decompose": (_ST, [_I64, _I64, _VP, _VP, C.c_int32, _VP, _VP]),
    "df_mesh_renumber": (_ST, [_I64, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "df_solver_create": (_ST, [_I64, _I64, _VP, _VP, C.c_int32, _VP, C.c_int32, C.POINTER(_VP)]),
    "df_solver_destroy": (None, [_VP]),
    "df_solver_get_info": (_ST, [_VP, C.POINTER(SolverInfo)]),
    "df_solver_set_arithmetic": (_ST, [_VP, C.c_int32]),
    "df_solver_convert": (_ST, [_VP, _VP, _VP, _VP, _VP]),
    "df_solver_spmv": (_ST, [_VP, _VP, _VP, _VP]),
    "df_solver_residual": (_ST, [_VP, _VP, _VP, _VP, _VP]),
    "df_solver_gauss_seidel": (_ST, [_VP, _VP, _VP, C.c_int32, _VP]),
    "df_fv_laplacian": (_ST, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "df_solver_export_csr": (_ST, [_VP, _VP, _VP, _VP]),
    "df_solver_get_last_error": (C.c_char_p, [_VP]),
    "df_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libdfgb.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
