"""C ABI checks that need no GPU: the library loads, exports every entry point the header
declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(df_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2508_18969_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "df_chem_step" in names and "df_state_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_python_binding_covers_the_header(lib):
    from paper_2508_18969_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_version_string(lib):
    assert lib.df_version().decode().startswith("dfgb")


def test_create_rejects_null_arguments(lib):
    from paper_2508_18969_gb300 import _lib
    h = C.c_void_p()
    assert lib.df_state_create(None, None, None, C.byref(h)) == _lib.DF_ERR_INVALID_ARG
    assert h.value is None
    assert b"NULL" in lib.df_get_last_error(None)


def test_create_rejects_bad_lambda_before_device_use(lib):
    import numpy as np
    import synth
    from paper_2508_18969_gb300 import _lib
    mech = synth.make_mechanism(9, 12, 1)
    net = synth.make_network([11, 16, 9], 9, 1)
    keep = []

    def d(a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_double))

    md = _lib.MechDesc(9, d(mech.W), d(mech.Tc), d(mech.pc), d(mech.omega), d(mech.kij), d(mech.nasa))
    widths = (C.c_int32 * 3)(11, 16, 9)
    W = (C.POINTER(C.c_float) * 2)()
    b = (C.POINTER(C.c_float) * 2)()
    for l in range(2):
        w = np.ascontiguousarray(net.W[l], dtype=np.float32).reshape(-1)
        bb = np.ascontiguousarray(net.b[l], dtype=np.float32)
        keep += [w, bb]
        W[l] = w.ctypes.data_as(C.POINTER(C.c_float))
        b[l] = bb.ctypes.data_as(C.POINTER(C.c_float))
    nd = _lib.MlpDesc(2, widths, W, b, 0.3, d(net.in_mean), d(net.in_std), d(net.out_mean),
                      d(net.out_std), 1e-7)
    opt = _lib.Options(0, 600.0, 0.0, 0, 0, 0)
    h = C.c_void_p()
    assert lib.df_state_create(C.byref(md), C.byref(nd), C.byref(opt), C.byref(h)) == _lib.DF_ERR_UNSUPPORTED
    nd.lambda_ = 0.1
    nd.dt = -1.0
    assert lib.df_state_create(C.byref(md), C.byref(nd), C.byref(opt), C.byref(h)) == _lib.DF_ERR_INVALID_ARG
    widths[2] = 8
    nd.dt = 1e-7
    assert lib.df_state_create(C.byref(md), C.byref(nd), C.byref(opt), C.byref(h)) == _lib.DF_ERR_INVALID_ARG


def test_entry_points_reject_null_state(lib):
    from paper_2508_18969_gb300 import _lib
    assert lib.df_chem_step(None, 10, 1e-7, None, None, None, 10, None, None, None) == _lib.DF_ERR_INVALID_ARG
    assert lib.df_real_fluid_props(None, 10, None, None, None, 10, None, None, None, None, None) == _lib.DF_ERR_INVALID_ARG
    assert lib.df_active_compact(None, 10, None, None, None, None) == _lib.DF_ERR_INVALID_ARG
    assert lib.df_chem_step_vjp(None, 10, None, None, None, 10, None, None, 10, None, None, 10,
                                None) == _lib.DF_ERR_INVALID_ARG
    lib.df_state_destroy(None)


def test_static_compaction_rejects_oversize_before_device_use(lib):
    from paper_2508_18969_gb300 import _lib
    big = _lib.DF_COMPACT_STATIC_MAX_CELLS + 1
    rc = lib.df_active_compact_static(big, 600.0, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), None)
    assert rc == _lib.DF_ERR_INVALID_ARG
    assert b"DF_COMPACT_STATIC_MAX_CELLS" in lib.df_get_last_error(None)
    assert lib.df_active_compact_static(10, 600.0, None, None, None, None) == _lib.DF_ERR_INVALID_ARG


def _header_defines():
    """Integer #define constants of include/*.h: name -> value."""
    inc = os.path.join(ROOT, "include")
    out = {}
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        for m in re.finditer(r"^#define\s+(DF_[A-Z0-9_]+)\s+\(?\s*(-?(?:0x[0-9A-Fa-f]+|\d+))\s*\)?",
                             open(os.path.join(inc, f)).read(), flags=re.M):
            out[m.group(1)] = int(m.group(2), 0)
    return out


def test_binding_constants_match_the_headers():
    """Every DF_* integer constant the binding defines has the header's value."""
    from paper_2508_18969_gb300 import _lib
    hdr = _header_defines()
    assert {"DF_OK", "DF_TILE_PAIR", "DF_HOST_DIRECT", "DF_SOLVER_FP64"} <= set(hdr)
    shared = [k for k in hdr if hasattr(_lib, k)]
    assert len(shared) >= 10, shared
    for k in shared:
        assert getattr(_lib, k) == hdr[k], (k, getattr(_lib, k), hdr[k])
