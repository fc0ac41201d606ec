"""Python access to the stiff-chemistry truth integrator of oracle/truth.c.

TEST INFRASTRUCTURE (part of the oracle): plain FP64 C with OpenMP, compiled with gcc into
oracle/_truth.so by build(). Only tests, the smoke check and the bench's CPU leg use it."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "truth.c")
LIB = os.path.join(HERE, "_truth.so")
_lib = None


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed on truth.c:\n{r.stderr}")
    return LIB


_dp = C.POINTER(C.c_double)


class _Mech(C.Structure):
    _fields_ = [("n", C.c_int), ("R", C.c_int), ("W", _dp), ("Tc", _dp), ("pc", _dp),
                ("omega", _dp), ("kij", _dp), ("nasa", _dp), ("nu_f", _dp), ("nu_r", _dp),
                ("A", _dp), ("beta", _dp), ("Ea", _dp)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        lib.truth_state.argtypes = [C.POINTER(_Mech), C.c_long, _dp, _dp, _dp, C.c_long, _dp, _dp,
                                    _dp, C.POINTER(C.c_int)]
        lib.truth_rhs.argtypes = [C.POINTER(_Mech), C.c_double, C.c_double, _dp, _dp, _dp]
        lib.truth_rhs.restype = C.c_int
        lib.truth_advance.argtypes = [C.POINTER(_Mech), C.c_long, _dp, _dp, _dp, C.c_long, C.c_double,
                                      C.c_double, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_long)]
        _lib = lib
    return _lib


class _MechRef:
    """ctypes view of a mechanism, keeping its contiguous arrays alive."""

    def __init__(self, m):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        self.arrs = [f(m.W), f(m.Tc), f(m.pc), f(m.omega), f(m.kij), f(m.nasa), f(m.nu_f),
                     f(m.nu_r), f(m.A), f(m.beta), f(m.Ea)]
        p = [a.ctypes.data_as(_dp) for a in self.arrs]
        self.s = _Mech(int(m.n), int(np.asarray(m.A).shape[0]), *p)


def _d(a):
    return a.ctypes.data_as(_dp)


def state(mech, T, p, Y):
    """(h [J/kg], cp [J/kg/K], rho [kg/m^3], ok) of each cell, C implementation."""
    lib = _load()
    mr = _MechRef(mech)
    T = np.ascontiguousarray(T, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    N = T.shape[0]
    h, cp, rho = np.zeros(N), np.zeros(N), np.zeros(N)
    ok = np.zeros(N, dtype=np.int32)
    lib.truth_state(C.byref(mr.s), N, _d(T), _d(p), _d(Y), Y.shape[1], _d(h), _d(cp), _d(rho),
                    ok.ctypes.data_as(C.POINTER(C.c_int)))
    return h, cp, rho, ok.astype(bool)


def rhs(mech, p, h0, Y, T):
    """(dY/dt, T) of one composition at fixed (p, h0); T is the Newton warm start."""
    lib = _load()
    mr = _MechRef(mech)
    y = np.ascontiguousarray(Y, dtype=np.float64)
    f = np.zeros_like(y)
    t = C.c_double(float(T))
    if not lib.truth_rhs(C.byref(mr.s), float(p), float(h0), _d(y), C.byref(t), _d(f)):
        raise RuntimeError("right-hand side failed (no root or no temperature)")
    return f, t.value


def advance(mech, T, p, Y, dt, rtol=1e-10, atol=1e-14):
    """Integrates every cell over dt with the BDF; returns (T', Y', ok, steps, code) with the
    per-cell codes of truth_advance."""
    lib = _load()
    mr = _MechRef(mech)
    T = np.array(T, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    Y = np.array(Y, dtype=np.float64, order="C")
    N = T.shape[0]
    ok = np.zeros(N, dtype=np.int32)
    steps = np.zeros(N, dtype=np.int64)
    lib.truth_advance(C.byref(mr.s), N, _d(T), _d(p), _d(Y), Y.shape[1], float(dt), float(rtol),
                      float(atol), ok.ctypes.data_as(C.POINTER(C.c_int)),
                      steps.ctypes.data_as(C.POINTER(C.c_long)))
    return T, Y, ok == 1, steps, ok
