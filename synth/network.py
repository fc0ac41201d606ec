"""Seeded stand-in for the trained chemistry network (ODENet, Sec. 2 and Sec. 4.1).

The paper's trained weights are not available; a seeded, untrained network of the stated
layer widths is drawn instead. Weights are Xavier-uniform, biases ~ U[-0.05, 0.05], both
rounded to binary32 (the precision a trained network is shipped in).

Normalisation constants (Sec. 3.3.1 states Z-score inputs; the Box-Cox step and its lambda
are this project's reading): inputs are (T, p, BC(Y_1..Y_n)); the mean and spread below are
fixed numbers picked to put the synthetic fields' inputs near zero mean and unit spread
(T in 100..3500 K, p in 5..20 MPa, BC(Y) in [-8.4, 0] for Y in [1e-8, 1] at lambda = 0.1).
Outputs are de-normalised with mean 0 and spread 1e-3, so an untrained network moves
the Box-Cox coordinates by O(1e-3) per step, a physically small change of Y.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import Stream


@dataclass
class Network:
    widths: list[int]          # [K0, H1, ..., n]
    W: list[np.ndarray]        # per layer [out, in] float32 values (stored as float64)
    b: list[np.ndarray]        # per layer [out]
    lam: float                 # Box-Cox lambda
    in_mean: np.ndarray        # [K0]
    in_std: np.ndarray         # [K0]
    out_mean: np.ndarray       # [n]
    out_std: np.ndarray        # [n]
    dt: float                  # time step the network advances, s

    @property
    def n_layers(self) -> int:
        return len(self.W)


def make_network(widths: list[int], n_species: int, seed: int, lam: float = 0.1,
                 dt: float = 1e-7, out_std: float = 1e-3) -> Network:
    if widths[0] != n_species + 2 or widths[-1] != n_species:
        raise ValueError("network widths must read (T, p, Y_1..Y_n) and emit n outputs")
    s = Stream(seed, "network")
    Ws, bs = [], []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        w = s.uniform(fan_in * fan_out, -lim, lim).reshape(fan_out, fan_in)
        Ws.append(w.astype(np.float32).astype(np.float64))
        bs.append(s.uniform(fan_out, -0.05, 0.05).astype(np.float32).astype(np.float64))
    in_mean = np.concatenate([[1500.0, 12.5e6], np.full(n_species, -4.0)])
    in_std = np.concatenate([[1000.0, 5.0e6], np.full(n_species, 3.0)])
    return Network(widths=list(widths), W=Ws, b=bs, lam=lam, in_mean=in_mean, in_std=in_std,
                   out_mean=np.zeros(n_species), out_std=np.full(n_species, out_std), dt=dt)


def make_propnet(widths: list[int], n_species: int, seed: int, lam: float = 0.1,
                 in_mean=None, in_std=None, out_mean=None, out_std=None) -> Network:
    """Seeded property network (PRNet-style, Sec. 2): inputs (h, p, BC(Y_1..Y_n)), any number
    of outputs. Weights as make_network. The normalisation constants are network parameters:
    pass the means and spreads of the data the network is meant for, else fixed defaults
    (h ~ 0 +- 2 MJ/kg, p ~ 12.5 +- 5 MPa, BC(Y) ~ -4 +- 3; outputs 0 +- 1)."""
    if widths[0] != n_species + 2:
        raise ValueError("a property network reads (h, p, Y_1..Y_n)")
    s = Stream(seed, "propnet")
    Ws, bs = [], []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        w = s.uniform(fan_in * fan_out, -lim, lim).reshape(fan_out, fan_in)
        Ws.append(w.astype(np.float32).astype(np.float64))
        bs.append(s.uniform(fan_out, -0.05, 0.05).astype(np.float32).astype(np.float64))
    m = widths[-1]
    dflt_mean = np.concatenate([[0.0, 12.5e6], np.full(n_species, -4.0)])
    dflt_std = np.concatenate([[2.0e6, 5.0e6], np.full(n_species, 3.0)])
    return Network(widths=list(widths), W=Ws, b=bs, lam=lam,
                   in_mean=np.asarray(dflt_mean if in_mean is None else in_mean, np.float64),
                   in_std=np.asarray(dflt_std if in_std is None else in_std, np.float64),
                   out_mean=np.asarray(np.zeros(m) if out_mean is None else out_mean, np.float64),
                   out_std=np.asarray(np.ones(m) if out_std is None else out_std, np.float64),
                   dt=0.0)
