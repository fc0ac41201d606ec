"""Training of the chemistry network in FP64 -- TEST INFRASTRUCTURE (part of the oracle).

Loss (this project's reading; the paper trains ODENet offline and prints no loss): the mean
over the batch of the squared error of the normalised network outputs,
  L = (1/B) sum_b sum_k (O_bk - Ohat_bk)^2,  Ohat_k = (BC(Y_target,k) - BC(Y_k) - mean_k) / std_k,
i.e. the network is taught the change of the Box-Cox coordinates that the stiff integration
(oracle/truth.c) produces over dt. Gradients by reverse mode written out layer by layer;
Adam (Kingma & Ba 2015) with bias correction."""
from __future__ import annotations

import numpy as np

from . import network as nw


def targets(net, Y, Y_target):
    """Ohat [N, n] from the mass fractions before (Y [n, N]) and after (Y_target) dt."""
    du = nw.boxcox(Y_target, net.lam) - nw.boxcox(Y, net.lam)
    return ((du - net.out_mean[:, None]) / net.out_std[:, None]).T


def loss_and_grads(net, x, Ohat):
    """(L, [dL/dW_l], [dL/db_l]) for inputs x [B, K0] and targets Ohat [B, n]."""
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    L = net.n_layers
    hs = [x]
    zs = []
    h = x
    for l in range(L):
        z = h @ net.W[l].T + net.b[l][None, :]
        zs.append(z)
        h = nw.gelu_tanh(z) if l < L - 1 else z
        hs.append(h)
    r = hs[-1] - Ohat
    loss = float(np.sum(r * r) / B)
    g = 2.0 * r / B                      # dL/dz of the linear read-out
    dW = [None] * L
    db = [None] * L
    for l in range(L - 1, -1, -1):
        dW[l] = g.T @ hs[l]
        db[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ net.W[l]) * nw.gelu_tanh_grad(zs[l - 1])
    return loss, dW, db


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1) on lists of arrays; returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1.0 - beta1) * g
        vv = beta2 * vv + (1.0 - beta2) * g * g
        mh = mm / (1.0 - beta1 ** t)
        vh = vv / (1.0 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
