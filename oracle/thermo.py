"""NASA-7 ideal-gas thermodynamics on one temperature range (paper silent; textbook form).

Per species, with coefficients a1..a7 and T in K:
  cp/R   = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
  h/(RT) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
  s/R    = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
Mixture values are mass-specific: sum_k Y_k q_k / W_k.
"""
from __future__ import annotations

import numpy as np

R = 8.31446261815324  # J/(mol K)


def species_cp_R(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """cp_k/R, shape [n, N]."""
    a = nasa
    T = np.asarray(T, dtype=np.float64)[None, :]
    return (a[:, 0:1] + a[:, 1:2] * T + a[:, 2:3] * T**2 + a[:, 3:4] * T**3
            + a[:, 4:5] * T**4)


def species_h_RT(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """h_k/(R T), shape [n, N]."""
    a = nasa
    T = np.asarray(T, dtype=np.float64)[None, :]
    return (a[:, 0:1] + a[:, 1:2] * T / 2.0 + a[:, 2:3] * T**2 / 3.0 + a[:, 3:4] * T**3 / 4.0
            + a[:, 4:5] * T**4 / 5.0 + a[:, 5:6] / T)


def species_s_R(nasa: np.ndarray, T: np.ndarray) -> np.ndarray:
    """s_k/R at the reference pressure, shape [n, N]."""
    a = nasa
    T = np.asarray(T, dtype=np.float64)[None, :]
    return (a[:, 0:1] * np.log(T) + a[:, 1:2] * T + a[:, 2:3] * T**2 / 2.0
            + a[:, 3:4] * T**3 / 3.0 + a[:, 4:5] * T**4 / 4.0 + a[:, 6:7])


def species_h_molar(nasa, T):
    """h_k in J/mol, shape [n, N]."""
    return R * np.asarray(T, dtype=np.float64)[None, :] * species_h_RT(nasa, T)


def mixture_h_ig(nasa, W, T, Y):
    """Ideal-gas mass-specific enthalpy sum_k Y_k h_k(T) / W_k, J/kg."""
    return np.sum(Y * species_h_molar(nasa, T) / W[:, None], axis=0)


def mixture_cp_ig(nasa, W, T, Y):
    """Ideal-gas mass-specific heat capacity sum_k Y_k cp_k(T) / W_k, J/(kg K)."""
    return np.sum(Y * R * species_cp_R(nasa, T) / W[:, None], axis=0)
