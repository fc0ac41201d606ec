"""Python binding of the property network (include/df_propnet.h): a PRNet-style surrogate of
the real-fluid state, (h, p, Y) -> properties, on a network-only df_state.

Argument marshalling only: inputs, network layers, outputs, loss, backward pass and Adam all
run in libdfgb.so. Tensors live on the network's CUDA device; h, p [N], Y [n, N] species-major
(row stride = ldY), properties [m, N]."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .api import DFError, State, _check_cells, _ptr, _stream


class PropNet(State):
    """Owns a network-only df_state holding a property network.

    net: object with widths ([n+2, ..., m]), W (list of [out, in]), b, lam, in_mean [n+2],
    in_std, out_mean [m], out_std."""

    def __init__(self, net, precision: int = L.DF_BF16, device: int = 0, batch_cells: int = 0):
        self._lib = L.load()
        self._keep = []
        d = lambda a: self._arr(np.ascontiguousarray(a, dtype=np.float64), C.c_double)
        nl = len(net.W)
        widths = (C.c_int32 * (nl + 1))(*[int(w) for w in net.widths])
        Wp = (C.POINTER(C.c_float) * nl)()
        bp = (C.POINTER(C.c_float) * nl)()
        for l in range(nl):
            Wp[l] = self._arr(np.ascontiguousarray(net.W[l], dtype=np.float32).reshape(-1), C.c_float)
            bp[l] = self._arr(np.ascontiguousarray(net.b[l], dtype=np.float32), C.c_float)
        self._keep += [widths, Wp, bp]
        nd = L.MlpDesc(nl, widths, Wp, bp, float(net.lam), d(net.in_mean), d(net.in_std),
                       d(net.out_mean), d(net.out_std), 0.0)
        opt = L.Options(int(precision), 0.0, 0.0, 0, int(device), int(batch_cells), L.DF_GELU_TANH)
        h = C.c_void_p()
        rc = self._lib.df_network_create(C.byref(nd), C.byref(opt), C.byref(h))
        self._keep = []
        if rc != L.DF_OK:
            raise DFError(rc, self._lib.df_get_last_error(None).decode())
        self.h = h
        self.widths = [int(w) for w in net.widths]
        self.n = self.widths[0] - 2
        self.K0 = self.widths[0]
        self.m = self.widths[-1]
        self.nout = self.m
        self.dt = 0.0
        self.device = torch.device("cuda", device)

    def infer(self, h, p, Y, out=None, stream=None):
        """Properties [m, N] (FP64) of the cells (df_propnet_infer)."""
        N = _check_cells(self.n, h, p, Y, names=("h", "p", "Y"))
        if out is None:
            out = torch.empty(self.m, N, dtype=torch.float64, device=h.device)
        _check_cells(self.m, h, None, out, names=("h", "p", "out"))
        self._check(self._lib.df_propnet_infer(self.h, N, _ptr(h), _ptr(p), _ptr(Y), Y.stride(0),
                                               _ptr(out), out.stride(0), _stream(stream)))
        return out

    def fit_step(self, h, p, Y, target, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, loss=None,
                 stream=None):
        """One Adam step towards target properties [m, B] (df_propnet_train_step). Returns the
        device FP32 loss tensor (shape [1]) the step writes."""
        _check_cells(self.n, h, p, Y, names=("h", "p", "Y"))
        _check_cells(self.m, h, None, target, names=("h", "p", "target"))
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=h.device)
        hp = self._adam(lr, betas, eps)
        self._check(self._lib.df_propnet_train_step(self.h, h.shape[0], _ptr(h), _ptr(p), _ptr(Y),
                                                    Y.stride(0), _ptr(target), target.stride(0),
                                                    C.byref(hp), _ptr(loss), _stream(stream)))
        return loss
