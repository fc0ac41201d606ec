"""Seeded synthetic cell states (T, p, Y) standing in for the paper's flow fields.

The paper measures on a supercritical LOX/CH4 Taylor-Green-vortex flame (10 MPa, O2 at
150 K against CH4 at 300 K, Sec. 4.1) and on a rocket engine (above 3000 K, up to 20 MPa,
Sec. 4.1). Neither field is available, so states are drawn along a mixing-plus-burning line:

  * mixture fraction Zf: fuel stream = pure CH4 (species 1), oxidiser = pure O2 (species 0);
  * progress c in [0, 1] burns a fraction c of the limiting reactant along
    CH4 + 2 O2 -> CO2 + 2 H2O (mass is conserved because the molar masses balance);
  * minor species (index >= 4) get seeded log-uniform mass fractions, then all Y are
    divided by their sum.

Layout returned: T [N], p [N], Y [n, N] (species-major, one contiguous row per species).
"""
from __future__ import annotations

import numpy as np

from .mechanism import Mechanism
from .rng import Stream

Z_ST = 0.2  # burning-zone centre in mixture fraction (near the CH4/O2 mass stoichiometry)


def mixing_burning_Y(mech: Mechanism, Zf: np.ndarray, c: np.ndarray, stream: Stream,
                     minor_lo: float, minor_hi: float) -> np.ndarray:
    N = Zf.shape[0]
    n = mech.n
    W = mech.W
    Y = np.zeros((n, N))
    y_ch4 = Zf.copy()
    y_o2 = 1.0 - Zf
    s = 2.0 * W[0] / W[1]                       # kg O2 per kg CH4
    m = c * np.minimum(y_ch4, y_o2 / s)          # kg CH4 burned per kg mixture
    Y[0] = y_o2 - s * m
    Y[1] = y_ch4 - m
    Y[2] = m * 2.0 * W[2] / W[1]
    Y[3] = m * W[3] / W[1]
    if n > 4:
        e = stream.uniform((n - 4) * N, np.log10(minor_lo), np.log10(minor_hi)).reshape(n - 4, N)
        Y[4:] = 10.0 ** e
    Y = np.maximum(Y, 0.0)
    return Y / Y.sum(axis=0, keepdims=True)


def uniform_states(mech: Mechanism, N: int, seed: int):
    """T ~ U[100, 3500] K, p ~ U[5, 20] MPa, Y along the mixing+burning line."""
    s = Stream(seed, "uniform-states")
    T = s.uniform(N, 100.0, 3500.0)
    p = s.uniform(N, 5.0e6, 20.0e6)
    Zf = s.uniform(N)
    c = s.uniform(N)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-2)
    return T, p, Y


def _layer_T(Zf: np.ndarray, c: np.ndarray) -> np.ndarray:
    T_mix = 100.0 * (1.0 - Zf) + 150.0 * Zf
    return T_mix + c * (3500.0 - T_mix)


def mixing_layer_1d(mech: Mechanism, N: int, seed: int, delta: float = 0.1, p: float = 10.0e6):
    """1D supercritical mixing layer on x in [-1, 1]: O2-rich at 100 K, CH4-rich at 150 K,
    Zf(x) = (1 + tanh(x / delta)) / 2, burning zone c = exp(-((Zf - 0.2) / 0.1)^2) lifting T
    towards 3500 K, p = 10 MPa, minor species jittered in [1e-8, 1e-3]."""
    s = Stream(seed, "mixing-layer-1d")
    x = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    Zf = 0.5 * (1.0 + np.tanh(x / delta))
    c = np.exp(-(((Zf - Z_ST) / 0.1) ** 2))
    T = _layer_T(Zf, c)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    return T, np.full(N, p), Y


def reacting_mix(mech: Mechanism, N: int, seed: int, active_fraction: float = 0.3,
                 p: float = 10.0e6):
    """Cells of the 1D mixing layer's two populations, interleaved by a seeded Bernoulli mask:
    reacting cells (probability active_fraction) take Zf ~ U[0.07, 0.33], whose burning
    progress puts T above 727 K; the others are cold unburnt mixing (c = 0, T <= 150 K)."""
    s = Stream(seed, "reacting-mix")
    act = s.uniform(N) < active_fraction
    Zf = np.where(act, s.uniform(N, 0.07, 0.33), s.uniform(N))
    c = np.where(act, np.exp(-(((Zf - Z_ST) / 0.1) ** 2)), 0.0)
    T = _layer_T(Zf, c)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    return T, np.full(N, p), Y


def training_states(mech: Mechanism, N: int, seed: int):
    """Training states: positions x ~ U[-1, 1] across the 1D mixing layer's profile (so cold
    mixing, the burning zone and hot products all appear), p ~ U[5, 20] MPa, minor species
    jittered in [1e-8, 1e-3]."""
    s = Stream(seed, "training-states")
    x = s.uniform(N, -1.0, 1.0)
    Zf = 0.5 * (1.0 + np.tanh(x / 0.1))
    c = np.exp(-(((Zf - Z_ST) / 0.1) ** 2))
    T = _layer_T(Zf, c)
    p = s.uniform(N, 5.0e6, 20.0e6)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    return T, p, Y
