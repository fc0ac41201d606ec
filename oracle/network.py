"""Chemistry network side of the step in FP64: Box-Cox, Z-score, MLP, de-normalisation.

  * Inputs (Sec. 2): (T, p, Y_1..Y_n). Species enter through the Box-Cox transform
    BC(y) = (y^lambda - 1) / lambda (Box & Cox 1964; the paper is silent on it, lambda is a
    network parameter, 0.1 here), negative y read as 0. All inputs are then Z-scored
    (Sec. 3.3.1): x = (v - mean) / std.
  * Hidden layers: h_l = GELU(h_{l-1} W_l^T + b_l) with the tanh form of Sec. 3.3.2,
    GELU(x) = 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))); the output layer is linear
    (the paper names GELU as the activation; a linear read-out is this project's reading).
  * Outputs are de-normalised changes of the Box-Cox coordinates over dt:
    du_k = std_k O_k + mean_k, u_k = BC(Y_k) + du_k, Y'_k = max(lambda u_k + 1, 0)^(1/lambda),
    then Y' is divided by its sum.
"""
from __future__ import annotations

import numpy as np


def boxcox(y, lam):
    y = np.maximum(np.asarray(y, dtype=np.float64), 0.0)
    return (y**lam - 1.0) / lam


def boxcox_inverse(u, lam):
    return np.maximum(lam * np.asarray(u, dtype=np.float64) + 1.0, 0.0) ** (1.0 / lam)


def gelu_tanh(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x**3)))


def gelu_tanh_grad(x):
    """d GELU / dx of the tanh form."""
    x = np.asarray(x, dtype=np.float64)
    c = np.sqrt(2.0 / np.pi)
    t = np.tanh(c * (x + 0.044715 * x**3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t**2) * c * (1.0 + 3.0 * 0.044715 * x**2)


def gelu_tanh_grad2(x):
    """d^2 GELU / dx^2 of the tanh form, written out from the first derivative:
    with u = c (x + a x^3), t = tanh u, u' = c (1 + 3 a x^2), u'' = 6 a c x,
    GELU' = (1 + t)/2 + (x/2)(1 - t^2) u', GELU'' = (1 - t^2)(u' - x t u'^2 + x u''/2)."""
    x = np.asarray(x, dtype=np.float64)
    c, a = np.sqrt(2.0 / np.pi), 0.044715
    t = np.tanh(c * (x + a * x**3))
    up = c * (1.0 + 3.0 * a * x**2)
    upp = 6.0 * a * c * x
    return (1.0 - t**2) * (up - x * t * up**2 + 0.5 * x * upp)


GELU_TABLE_LO, GELU_TABLE_HI, GELU_TABLE_H = -3.0, 3.0, 0.01


def gelu_table_coeffs():
    """Second-order table of GELU on [-3, 3] at spacing 0.01 (Sec. 3.3.2): at node
    x_i = -3 + 0.01 i (i = 0..600) the value, slope and half curvature of the tanh form, each
    rounded to binary32 (the precision the GPU tables hold). Returns [601, 3]."""
    n = int(round((GELU_TABLE_HI - GELU_TABLE_LO) / GELU_TABLE_H)) + 1
    xi = GELU_TABLE_LO + GELU_TABLE_H * np.arange(n)
    c = np.stack([gelu_tanh(xi), gelu_tanh_grad(xi), 0.5 * gelu_tanh_grad2(xi)], axis=1)
    return c.astype(np.float32).astype(np.float64)


def gelu_table(x, coeffs=None):
    """The paper's tabulated GELU (Sec. 3.3.2): 0 below -3, x above 3, and in between the
    second-order expansion g + g' d + (g''/2) d^2 about the node at or below x (d = x - x_i).
    The paper gives the range, the spacing and the order; expanding about the lower node is
    this project's reading."""
    x = np.asarray(x, dtype=np.float64)
    if coeffs is None:
        coeffs = gelu_table_coeffs()
    t = (x - GELU_TABLE_LO) / GELU_TABLE_H
    i = np.clip(np.floor(t), 0, coeffs.shape[0] - 2).astype(np.int64)
    d = x - (GELU_TABLE_LO + GELU_TABLE_H * i)
    c = coeffs[i]
    y = c[..., 0] + d * (c[..., 1] + d * c[..., 2])
    return np.where(x <= GELU_TABLE_LO, 0.0, np.where(x >= GELU_TABLE_HI, x, y))


def normalise_inputs(net, T, p, Y):
    """Network input rows x [N, n+2] from the cell states."""
    v = np.concatenate([np.asarray(T, dtype=np.float64)[None, :],
                        np.asarray(p, dtype=np.float64)[None, :],
                        boxcox(Y, net.lam)], axis=0)
    return ((v - net.in_mean[:, None]) / net.in_std[:, None]).T


def mlp_forward(net, x, return_pre=False, act=None):
    """Plain layer-by-layer forward pass; x [N, K0] -> O [N, n]. act replaces the hidden
    activation (default: the tanh-form GELU; gelu_table for the tabulated network)."""
    act = gelu_tanh if act is None else act
    h = np.asarray(x, dtype=np.float64)
    pre = []
    L = net.n_layers
    for l in range(L):
        z = h @ net.W[l].T + net.b[l][None, :]
        pre.append(z)
        h = act(z) if l < L - 1 else z
    return (h, pre) if return_pre else h


def denormalise(net, Y, O):
    """New mass fractions Y' [n, N] from the old Y [n, N] and network outputs O [N, n]."""
    du = O.T * net.out_std[:, None] + net.out_mean[:, None]
    u = boxcox(Y, net.lam) + du
    Yn = boxcox_inverse(u, net.lam)
    return Yn / np.sum(Yn, axis=0, keepdims=True)


def round_to_bf16(a):
    """Round to the nearest bfloat16 (ties to even), via binary32: the value a kernel gets
    when it converts an FP32 number to BF16. Returned as float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def mlp_forward_rounded(net, x, rnd, act=None):
    """MLP forward with the input, the weights and every hidden activation passed through
    the rounding function rnd (e.g. round_to_bf16); sums and GELU stay FP64. This is the
    network as a reduced-precision path stores it, for checking such a path element-wise.
    act replaces the hidden activation as in mlp_forward."""
    act = gelu_tanh if act is None else act
    h = rnd(np.asarray(x, dtype=np.float64))
    L = net.n_layers
    for l in range(L):
        z = h @ rnd(net.W[l]).T + net.b[l][None, :]
        h = rnd(act(z)) if l < L - 1 else z
    return h


E4M3_MAX = 448.0


def round_to_e4m3(a):
    """Round to the nearest FP8 e4m3 value (ties to even, saturating at +-448), via binary32:
    the value a kernel gets when it converts an FP32 number with satfinite rounding.
    e4m3: 3 mantissa bits, exponent bias 7, normals down to 2^-6, subnormals in steps of
    2^-9. Returned as float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)
    mag = np.abs(f)
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.floor(np.log2(np.where(mag > 0, mag, 1.0)))
    e = np.clip(e, -6.0, 8.0)                 # below 2^-6 the quantum stays 2^-9
    q = np.exp2(e - 3.0)
    r = np.round(mag / q) * q                 # numpy rounds half to even
    r = np.minimum(r, E4M3_MAX)
    out = np.copysign(r, f)
    return np.where(np.isnan(f), np.nan, out)


def fp8_weight_rounding(W):
    """Per-output-channel scaled e4m3 weights: row scale s = max|W_row| / 448, stored
    e4m3(W / s), represented value e4m3(W / s) * s (binary32 scale)."""
    W = np.asarray(W, dtype=np.float64)
    amax = np.max(np.abs(W), axis=1, keepdims=True)
    s = np.where(amax > 0, (amax.astype(np.float32) / np.float32(E4M3_MAX)).astype(np.float64), 1.0)
    return round_to_e4m3(W / s) * s


def mlp_forward_fp8(net, x, act_scale):
    """MLP forward as an FP8 path stores it: input and hidden activations as e4m3(v * s) / s
    with a static per-tensor scale s = act_scale, weights with per-output-channel scales;
    sums and GELU in FP64."""
    rq = lambda v: round_to_e4m3(np.asarray(v) * act_scale) / act_scale
    h = rq(np.asarray(x, dtype=np.float64))
    L = net.n_layers
    for l in range(L):
        z = h @ fp8_weight_rounding(net.W[l]).T + net.b[l][None, :]
        h = rq(gelu_tanh(z)) if l < L - 1 else z
    return h


def mlp_jacobian(net, x):
    """dO/dx of the MLP for every row of x, by reverse mode written out layer by layer:
    for a linear layer z = h W^T + b the cotangent maps as g_h = g_z W, through GELU as
    g_z = g_h * GELU'(z). Returns J [N, n_out, K0]."""
    x = np.asarray(x, dtype=np.float64)
    _, pre = mlp_forward(net, x, return_pre=True)
    L = net.n_layers
    n_out = net.W[-1].shape[0]
    N = x.shape[0]
    J = np.zeros((N, n_out, x.shape[1]))
    for k in range(n_out):
        g = np.zeros((N, n_out))
        g[:, k] = 1.0                          # cotangent of output k
        for l in range(L - 1, -1, -1):
            if l < L - 1:
                g = g * gelu_tanh_grad(pre[l])  # through the activation of layer l
            g = g @ net.W[l]                    # through the linear map of layer l
        J[:, k, :] = g
    return J
