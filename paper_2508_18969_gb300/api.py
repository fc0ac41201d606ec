"""Python binding of the reaction-step library: same names as the C ABI, torch tensors in.

Every call marshals pointers and sizes and calls libdfgb.so; no arithmetic of the step
happens here. Tensors must live on the state's CUDA device; fields are float64, the mass
fractions species-major [n, N] (row stride = ldY).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


class DFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_cells(n, T, p=None, Y=None, status=None, n_active=None, device_type="cuda",
                 names=("T", "p", "Y")):
    """Checks the cell arrays a device entry point dereferences, before any library call:
    T and p 1-D float64 of N cells with unit stride, Y float64 [n, N] with unit stride along
    the cells (its row stride is passed as ldY), status int32 and n_active int64 of at least
    N and 1 elements, all on a CUDA device. Any other tensor would be read or written out of
    bounds by the kernels. Returns N."""
    def bad(name, what):
        raise ValueError(f"{name} must be {what}")

    def on_dev(name, t):
        if t.device.type != device_type:
            bad(name, f"on a {device_type} device (got {t.device})")

    nT, np_, nY = names
    on_dev(nT, T)
    if T.dtype != torch.float64 or T.dim() != 1:
        bad(nT, "a 1-D float64 tensor")
    N = T.shape[0]
    if N > 1 and T.stride(0) != 1:
        bad(nT, "contiguous")
    if p is not None:
        on_dev(np_, p)
        if p.dtype != torch.float64 or p.dim() != 1 or p.shape[0] != N or (N > 1 and p.stride(0) != 1):
            bad(np_, f"a contiguous 1-D float64 tensor of {N} cells")
    if Y is not None:
        on_dev(nY, Y)
        if Y.dtype != torch.float64 or Y.dim() != 2 or tuple(Y.shape) != (n, N) or \
                (N > 1 and Y.stride(1) != 1):
            bad(nY, f"a float64 tensor [{n}, {N}] with unit stride along the cells")
    if status is not None:
        on_dev("status", status)
        if status.dtype != torch.int32 or not status.is_contiguous() or status.numel() < N:
            bad("status", f"a contiguous int32 tensor of at least {N} elements")
    if n_active is not None:
        on_dev("n_active", n_active)
        if n_active.dtype != torch.int64 or n_active.numel() < 1:
            bad("n_active", "an int64 tensor of at least one element")
    return N


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class State:
    """Owns a df_state: mechanism constants, network weights and scratch on one GPU.

    mech: object with n, W, Tc, pc, omega, kij [n, n], nasa [n, 7] (numpy float64);
    net: object with widths, W (list of [out, in]), b, lam, in_mean, in_std, out_mean,
    out_std, dt.
    """

    def __init__(self, mech, net, precision: int = L.DF_FP32, T_react: float = 600.0,
                 newton_tol: float = 0.0, newton_max_iter: int = 0, device: int = 0,
                 batch_cells: int = 0, gelu_mode: int = L.DF_GELU_TANH):
        self._lib = L.load()
        self._keep = []
        d = lambda a: self._arr(np.ascontiguousarray(a, dtype=np.float64), C.c_double)
        md = L.MechDesc(int(mech.n), d(mech.W), d(mech.Tc), d(mech.pc), d(mech.omega),
                        d(np.asarray(mech.kij).reshape(-1)), d(np.asarray(mech.nasa).reshape(-1)))
        nl = len(net.W)
        widths = (C.c_int32 * (nl + 1))(*[int(w) for w in net.widths])
        Wp = (C.POINTER(C.c_float) * nl)()
        bp = (C.POINTER(C.c_float) * nl)()
        for l in range(nl):
            Wp[l] = self._arr(np.ascontiguousarray(net.W[l], dtype=np.float32).reshape(-1), C.c_float)
            bp[l] = self._arr(np.ascontiguousarray(net.b[l], dtype=np.float32), C.c_float)
        self._keep += [widths, Wp, bp]
        nd = L.MlpDesc(nl, widths, Wp, bp, float(net.lam), d(net.in_mean), d(net.in_std),
                       d(net.out_mean), d(net.out_std), float(net.dt))
        opt = L.Options(int(precision), float(T_react), float(newton_tol), int(newton_max_iter),
                        int(device), int(batch_cells), int(gelu_mode))
        h = C.c_void_p()
        rc = self._lib.df_state_create(C.byref(md), C.byref(nd), C.byref(opt), C.byref(h))
        self._keep = []
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(None).decode())
        self.h = h
        self.n = int(mech.n)
        self.K0 = self.n + 2
        self.nout = self.n
        self.dt = float(net.dt)
        self.device = torch.device("cuda", device)

    def _arr(self, a, ctype):
        self._keep.append(a)
        return a.ctypes.data_as(C.POINTER(ctype))

    def close(self):
        if getattr(self, "h", None):
            self._lib.df_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(self.h).decode())

    # ---- full step ----
    def chem_step(self, T, p, Y, dt=None, status=None, n_active=None, stream=None):
        N = _check_cells(self.n, T, p, Y, status, n_active)
        self._check(self._lib.df_chem_step(self.h, N, self.dt if dt is None else float(dt),
                                           _ptr(T), _ptr(p), _ptr(Y), Y.stride(0), _ptr(status),
                                           _ptr(n_active), _stream(stream)))

    def chem_step_host(self, T, p, Y, dt=None, status=None, chunk_cells=0, stream=None):
        """df_chem_step_host: one reaction step of cells in host (CPU, ideally pinned) tensors,
        in place on T and Y, pipelined through the device in chunks; stream-ordered on `stream`
        (synchronise it before reading the results)."""
        for t in (T, p, Y):
            if t.device.type != "cpu" or t.dtype != torch.float64:
                raise ValueError("T, p, Y must be float64 CPU tensors")
        if status is not None and (status.device.type != "cpu" or status.dtype != torch.int32):
            raise ValueError("status must be an int32 CPU tensor")
        N = T.shape[0]
        self._check(self._lib.df_chem_step_host(self.h, N, self.dt if dt is None else float(dt),
                                                _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                                _ptr(status), int(chunk_cells), _stream(stream)))

    def chem_source(self, T, p, Y, dt=None, status=None, n_active=None, want_T=True, stream=None):
        """(omega [n, N] FP64 kg/(m^3 s), T' [N] or None): df_chem_source; T, Y unchanged."""
        N = _check_cells(self.n, T, p, Y, status, n_active)
        om = torch.empty(self.n, N, dtype=torch.float64, device=T.device)
        Tn = torch.empty(N, dtype=torch.float64, device=T.device) if want_T else None
        self._check(self._lib.df_chem_source(self.h, N, self.dt if dt is None else float(dt),
                                             _ptr(T), _ptr(p), _ptr(Y), Y.stride(0), _ptr(om),
                                             max(N, 1), _ptr(Tn), _ptr(status), _ptr(n_active),
                                             _stream(stream)))
        return om, Tn

    def chem_jacobian(self, T, p, Y, want_dT=True, stream=None):
        """(J [N, n, n+1] FP32, dTnew [N, n+1] FP64 or None): df_chem_jacobian."""
        N = _check_cells(self.n, T, p, Y)
        J = torch.empty(N, self.n, self.n + 1, dtype=torch.float32, device=T.device)
        dTn = torch.empty(N, self.n + 1, dtype=torch.float64, device=T.device) if want_dT else None
        self._check(self._lib.df_chem_jacobian(self.h, N, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                               _ptr(J), _ptr(dTn), _stream(stream)))
        return J, dTn

    def chem_step_vjp(self, T, p, Y, gT, gY, stream=None):
        """(g_T [N], g_Y [n, N]) FP64: df_chem_step_vjp, the cotangents of (T, Y) from those
        of the step's outputs (T', Y')."""
        N = _check_cells(self.n, T, p, Y)
        gT = gT.to(torch.float64).contiguous()
        gY = gY.to(torch.float64).contiguous()
        if _check_cells(self.n, gT, None, gY) != N:
            raise ValueError(f"gT and gY must hold the {N} cells of T")
        oT = torch.empty(N, dtype=torch.float64, device=T.device)
        oY = torch.empty(self.n, N, dtype=torch.float64, device=T.device)
        self._check(self._lib.df_chem_step_vjp(self.h, N, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                               _ptr(gT), _ptr(gY), max(N, 1), _ptr(oT), _ptr(oY),
                                               max(N, 1), _stream(stream)))
        return oT, oY

    def graph(self, T, p, Y, dt=None, status=None, n_active=None):
        """A Graph replaying df_chem_step on these exact buffers (see df_graph_create)."""
        return Graph(self, T, p, Y, dt, status, n_active)

    def set_wait_limit(self, clocks: int = 0):
        """Clock budget of the tensor-core kernels' pipeline waits (df_set_wait_limit); 0
        restores the default (about one second)."""
        self._check(self._lib.df_set_wait_limit(self.h, int(clocks)))

    def step_summary(self, stream=None):
        """(status code, reacting cells, flagged cells, Newton iterations) of the last step."""
        s = L.StepStats()
        rc = self._lib.df_get_step_summary(self.h, _stream(stream), C.byref(s))
        return rc, s.n_active, s.n_flagged, s.newton_iterations

    def real_fluid_props(self, T, p, Y, stream=None):
        N = _check_cells(self.n, T, p, Y)
        out = [torch.empty(N, dtype=torch.float64, device=T.device) for _ in range(4)]
        self._check(self._lib.df_real_fluid_props(self.h, N, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                                  *[_ptr(o) for o in out], _stream(stream)))
        return tuple(out)

    def transport_props(self, T, p, Y, stream=None):
        """(mu [Pa s], lambda [W/(m K)], alpha [m^2/s]) of every cell (df_transport_props)."""
        N = _check_cells(self.n, T, p, Y)
        out = [torch.empty(N, dtype=torch.float64, device=T.device) for _ in range(3)]
        self._check(self._lib.df_transport_props(self.h, N, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                                 *[_ptr(o) for o in out], _stream(stream)))
        return tuple(out)

    # ---- training ----
    @staticmethod
    def _adam(lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        return L.Adam(float(lr), float(betas[0]), float(betas[1]), float(eps))

    def train_step(self, T, p, Y, Y_target, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, loss=None,
                   stream=None):
        """One Adam step on the states (T, p, Y) with targets Y_target (df_train_step).
        Returns the device FP32 loss tensor (shape [1]) the step writes."""
        _check_cells(self.n, T, p, Y)
        _check_cells(self.n, T, None, Y_target, names=("T", "p", "Y_target"))
        if Y_target.stride(0) != Y.stride(0):
            raise ValueError("Y and Y_target must share their row stride")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=T.device)
        hp = self._adam(lr, betas, eps)
        self._check(self._lib.df_train_step(self.h, T.shape[0], _ptr(T), _ptr(p), _ptr(Y),
                                            _ptr(Y_target), Y.stride(0), C.byref(hp), _ptr(loss),
                                            _stream(stream)))
        return loss

    def mlp_forward_train(self, x, stream=None):
        x = x.contiguous()
        O = torch.empty(x.shape[0], self.nout, dtype=torch.float32, device=x.device)
        self._check(self._lib.df_mlp_forward_train(self.h, x.shape[0], _ptr(x), _ptr(O),
                                                   _stream(stream)))
        return O

    def mlp_backward(self, dO, want_dx=True, stream=None):
        dO = dO.contiguous()
        dX = torch.empty(dO.shape[0], self.K0, dtype=torch.float32, device=dO.device) if want_dx else None
        self._check(self._lib.df_mlp_backward(self.h, dO.shape[0], _ptr(dO), _ptr(dX), _stream(stream)))
        return dX

    def adam_step(self, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, stream=None):
        hp = self._adam(lr, betas, eps)
        self._check(self._lib.df_adam_step(self.h, C.byref(hp), _stream(stream)))

    def params(self, layer, which=L.DF_PARAM_WEIGHTS, widths=None, stream=None):
        """(W [out, in], b [out]) FP32 device tensors of one layer: master weights, last
        gradients or Adam moments (df_get_params)."""
        if widths is None:
            raise ValueError("pass the network widths")
        W = torch.empty(widths[layer + 1], widths[layer], dtype=torch.float32, device=self.device)
        b = torch.empty(widths[layer + 1], dtype=torch.float32, device=self.device)
        self._check(self._lib.df_get_params(self.h, int(layer), int(which), _ptr(W), _ptr(b),
                                            _stream(stream)))
        return W, b

    def train_steps_taken(self):
        v = C.c_int64()
        self._check(self._lib.df_train_get_step(self.h, C.byref(v)))
        return v.value

    def save(self, path):
        self._check(self._lib.df_state_save(self.h, str(path).encode()))

    def load(self, path):
        self._check(self._lib.df_state_load(self.h, str(path).encode()))

    # ---- tile widths of the tensor-core layers ----
    def autotune(self, n_rows=0, cache_path=None, stream=None):
        """Times every compiled tile width per layer and keeps the fastest (df_autotune)."""
        self._check(self._lib.df_autotune(self.h, int(n_rows),
                                          None if cache_path is None else str(cache_path).encode(),
                                          _stream(stream)))
        return self.tiles()

    def tiles(self):
        cap = 8
        bn = (C.c_int32 * cap)()
        nl = C.c_int32()
        self._check(self._lib.df_get_tiles(self.h, bn, cap, C.byref(nl)))
        return [int(bn[i]) for i in range(min(nl.value, cap))]

    # ---- kernel timing ----
    def profile_enable(self, on: bool = True):
        self._check(self._lib.df_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{family: (launches, total_ms)} since the last read; synchronises the device."""
        cap = 32
        names = C.create_string_buffer(32 * cap)
        la = (C.c_int64 * cap)()
        ms = (C.c_double * cap)()
        n = C.c_int32()
        self._check(self._lib.df_profile_read(self.h, cap, names, la, ms, C.byref(n)))
        raw = names.raw
        out = {}
        for i in range(n.value):
            nm = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(la[i]), float(ms[i]))
        return out

    # ---- stages ----
    def active_compact(self, T, stream=None):
        N = _check_cells(self.n, T)
        idx = torch.empty(max(N, 1), dtype=torch.int32, device=T.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=T.device)
        self._check(self._lib.df_active_compact(self.h, N, _ptr(T), _ptr(idx), _ptr(cnt),
                                                _stream(stream)))
        return idx, cnt

    def eos_pre(self, T, p, Y, stream=None):
        N = _check_cells(self.n, T, p, Y)
        h0 = torch.empty(N, dtype=torch.float64, device=T.device)
        Z = torch.empty(N, dtype=torch.float64, device=T.device)
        x = torch.empty(N, self.K0, dtype=torch.float32, device=T.device)
        st = torch.empty(N, dtype=torch.int32, device=T.device)
        self._check(self._lib.df_eos_pre(self.h, N, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                         _ptr(h0), _ptr(Z), _ptr(x), _ptr(st), _stream(stream)))
        return h0, Z, x, st

    def mlp_forward(self, x, stream=None):
        x = x.contiguous()
        O = torch.empty(x.shape[0], self.nout, dtype=torch.float32, device=x.device)
        self._check(self._lib.df_mlp_forward(self.h, x.shape[0], _ptr(x), _ptr(O), _stream(stream)))
        return O

    def eos_post(self, O, h0, T, p, Y, stream=None):
        N = _check_cells(self.n, T, p, Y)
        O = O.contiguous()
        if _check_cells(self.n, h0) != N:
            raise ValueError(f"h0 must hold the {N} cells of T")
        if O.device.type != "cuda" or O.dtype != torch.float32 or tuple(O.shape) != (N, self.n):
            raise ValueError(f"O must be a float32 CUDA tensor [{N}, {self.n}]")
        st = torch.empty(N, dtype=torch.int32, device=T.device)
        self._check(self._lib.df_eos_post(self.h, N, _ptr(O), _ptr(h0), _ptr(T),
                                          _ptr(p), _ptr(Y), Y.stride(0), _ptr(st), _stream(stream)))
        return st


class MLPEOSFunction(torch.autograd.Function):
    """The state's network as a differentiable torch op: forward = df_mlp_forward_train,
    backward = df_mlp_backward (returns dL/dx; dL/dW and dL/db stay in the state for
    State.adam_step). Usage: O = MLPEOSFunction.apply(x, state)."""

    @staticmethod
    def forward(ctx, x, state):
        ctx.state = state
        ctx.rows = x.shape[0]
        return state.mlp_forward_train(x.detach().float())

    @staticmethod
    def backward(ctx, dO):
        dX = ctx.state.mlp_backward(dO.float(), want_dx=ctx.needs_input_grad[0])
        return dX, None


class ChemStepFunction(torch.autograd.Function):
    """The reaction step as a differentiable torch op, (T [N], Y [n, N]) -> (T', Y') at fixed p:
    forward = df_chem_step on copies of T and Y, backward = df_chem_step_vjp (the network's
    tangents and the equation-of-state chain, all in the library's kernels).
    Usage: T1, Y1 = ChemStepFunction.apply(T, Y, p, state)."""

    @staticmethod
    def forward(ctx, T, Y, p, state):
        T0, Y0 = T.detach().contiguous(), Y.detach().contiguous()
        T1, Y1 = T0.clone(), Y0.clone()
        state.chem_step(T1, p, Y1)
        ctx.state = state
        ctx.save_for_backward(T0, Y0, p)
        return T1, Y1

    @staticmethod
    def backward(ctx, gT1, gY1):
        T0, Y0, p = ctx.saved_tensors
        if gT1 is None:
            gT1 = torch.zeros_like(T0)
        if gY1 is None:
            gY1 = torch.zeros_like(Y0)
        gT, gY = ctx.state.chem_step_vjp(T0, p, Y0, gT1, gY1)
        return gT, gY, None, None


class Graph:
    """One captured df_chem_step (df_graph_*); launch() replays it."""

    def __init__(self, state, T, p, Y, dt, status, n_active):
        _check_cells(state.n, T, p, Y, status, n_active)
        self._lib = state._lib
        self._state = state
        self._bufs = (T, p, Y, status, n_active)  # keep the captured buffers alive
        h = C.c_void_p()
        rc = self._lib.df_graph_create(state.h, T.shape[0], state.dt if dt is None else float(dt),
                                       _ptr(T), _ptr(p), _ptr(Y), Y.stride(0), _ptr(status),
                                       _ptr(n_active), C.byref(h))
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(state.h).decode())
        self.h = h

    def launch(self, stream=None):
        rc = self._lib.df_graph_launch(self.h, _stream(stream))
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(self._state.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.df_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def active_compact_static(T, T_react: float, stream=None):
    """Allocation-free a0 (df_active_compact_static): no state, scratch in the library's
    static device array. Returns (idx, count) tensors; the caller allocates them here, the
    library does not."""
    N = _check_cells(0, T)
    lib = L.load()
    idx = torch.empty(max(N, 1), dtype=torch.int32, device=T.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=T.device)
    rc = lib.df_active_compact_static(N, float(T_react), _ptr(T), _ptr(idx), _ptr(cnt), _stream(stream))
    if rc != L.DF_OK:
        raise DFError(rc, lib.df_get_last_error(None).decode())
    return idx, cnt


def version() -> str:
    return L.load().df_version().decode()
