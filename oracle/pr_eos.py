"""Peng-Robinson real-fluid state of a mixture (FP64). Paper: Sec. 2 names the
Peng-Robinson EoS for the real-fluid properties but prints no equation; these are the
textbook equations of Peng & Robinson (1976) with van der Waals one-fluid mixing.

Pure species i (Tc, pc, omega):
  a_c = 0.45724 R^2 Tc^2 / pc,  b = 0.07780 R Tc / pc,
  kappa = 0.37464 + 1.54226 omega - 0.26992 omega^2,
  sqrt(a(T)) = sqrt(a_c) [1 + kappa (1 - sqrt(T / Tc))].
Mixture (mole fractions X):
  a_m = sum_i sum_j X_i X_j sqrt(a_i a_j) (1 - k_ij),  b_m = sum_i X_i b_i,
  A = a_m p / (R T)^2,  B = b_m p / (R T).
Compressibility: Z^3 - (1 - B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0; among the
real roots with Z > B the one of least departure Gibbs energy
  g/RT = Z - 1 - ln(Z - B) - A / (2 sqrt2 B) ln[(Z + (1 + sqrt2) B) / (Z + (1 - sqrt2) B)]
is taken (ties within 1e-12 go to the larger Z).
Departure enthalpy (J/mol):
  h_dep = R T (Z - 1) + (T da_m/dT - a_m) / (2 sqrt2 b_m) ln[(Z + (1 + sqrt2) B) / (Z + (1 - sqrt2) B)].
Real-fluid mass-specific enthalpy h = h_ig(T, Y) + h_dep / W_mix; density rho = p W_mix / (Z R T).
"""
from __future__ import annotations

import numpy as np

from .thermo import R, mixture_cp_ig, mixture_h_ig

SQ2 = np.sqrt(2.0)
OMEGA_A = 0.45724
OMEGA_B = 0.07780
NO_ROOT = 2  # status bit: no real root with Z > B


def pure_params(Tc, pc, omega):
    a_c = OMEGA_A * R**2 * Tc**2 / pc
    b = OMEGA_B * R * Tc / pc
    kappa = 0.37464 + 1.54226 * omega - 0.26992 * omega**2
    return a_c, b, kappa


def sqrt_a(Tc, pc, omega, T):
    """sqrt(a_i(T)) and its first and second T-derivatives, each [n, N]."""
    a_c, _, kappa = pure_params(Tc, pc, omega)
    T = np.asarray(T, dtype=np.float64)[None, :]
    sac = np.sqrt(a_c)[:, None]
    kap = kappa[:, None]
    tc = Tc[:, None]
    s0 = sac * (1.0 + kap * (1.0 - np.sqrt(T / tc)))
    s1 = -sac * kap / (2.0 * np.sqrt(T * tc))
    s2 = sac * kap / (4.0 * np.sqrt(tc) * T**1.5)
    return s0, s1, s2


def mole_fractions(W, Y):
    """(X [n, N], W_mix [N]) from mass fractions: W_mix = 1 / sum_k Y_k / W_k, X_k = Y_k W_mix / W_k."""
    inv = np.sum(Y / W[:, None], axis=0)
    W_mix = 1.0 / inv
    return Y * W_mix[None, :] / W[:, None], W_mix


def mixture_params(mech, X, T):
    """a_m, da_m/dT, d2a_m/dT2, b_m by the plain double sum over species pairs."""
    s0, s1, s2 = sqrt_a(mech.Tc, mech.pc, mech.omega, T)
    _, b, _ = pure_params(mech.Tc, mech.pc, mech.omega)
    n = mech.n
    a_m = np.zeros_like(X[0])
    da = np.zeros_like(X[0])
    d2a = np.zeros_like(X[0])
    for i in range(n):
        for j in range(n):
            w = X[i] * X[j] * (1.0 - mech.kij[i, j])
            a_m += w * s0[i] * s0[j]
            da += w * (s1[i] * s0[j] + s0[i] * s1[j])
            d2a += w * (s2[i] * s0[j] + 2.0 * s1[i] * s1[j] + s0[i] * s2[j])
    b_m = np.sum(X * b[:, None], axis=0)
    return a_m, da, d2a, b_m


def cubic_coefficients(A, B):
    """(c2, c1, c0) of Z^3 + c2 Z^2 + c1 Z + c0."""
    return -(1.0 - B), A - 3.0 * B**2 - 2.0 * B, -(A * B - B**2 - B**3)


def _cubic_value(Z, c2, c1, c0):
    return ((Z + c2) * Z + c1) * Z + c0


def _polish(Z, c2, c1, c0, iters=8):
    """Newton on the cubic until the residual is within 4 ulp of its term magnitudes."""
    Z = Z.copy()
    for _ in range(iters):
        f = _cubic_value(Z, c2, c1, c0)
        scale = np.abs(Z) ** 3 + np.abs(c2) * Z**2 + np.abs(c1) * np.abs(Z) + np.abs(c0)
        fp = (3.0 * Z + 2.0 * c2) * Z + c1
        go = np.isfinite(Z) & (np.abs(f) > 4.0 * np.finfo(float).eps * scale) & (fp != 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            Zn = Z - f / np.where(fp == 0.0, 1.0, fp)
        better = go & (np.abs(_cubic_value(Zn, c2, c1, c0)) < np.abs(f))
        Z = np.where(better, Zn, Z)
        if not better.any():
            break
    return Z


def cubic_real_roots(c2, c1, c0):
    """Real roots of Z^3 + c2 Z^2 + c1 Z + c0 per cell, [3, N] ascending, NaN where absent.

    Closed form: with Z = t - c2/3 the cubic is t^3 + P t + Q = 0. If
    (Q/2)^2 + (P/3)^3 > 0 there is one real root (Cardano); otherwise three,
    t_k = 2 sqrt(-P/3) cos(phi/3 - 2 pi k/3) with cos(phi) = (3Q / (2P)) sqrt(-3/P).
    Each root is then polished by Newton on the original cubic."""
    c2 = np.asarray(c2, dtype=np.float64)
    N = c2.shape[0]
    P = c1 - c2**2 / 3.0
    Q = 2.0 * c2**3 / 27.0 - c2 * c1 / 3.0 + c0
    disc = (Q / 2.0) ** 2 + (P / 3.0) ** 3
    roots = np.full((3, N), np.nan)
    one = disc > 0.0
    if one.any():
        q = Q[one]
        sq = np.sqrt(disc[one])
        sgn = np.where(q >= 0.0, 1.0, -1.0)
        u = np.cbrt(-q / 2.0 - sgn * sq)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(u != 0.0, u - P[one] / (3.0 * u), 0.0)
        roots[0, one] = t - c2[one] / 3.0
    three = ~one
    if three.any():
        Pm = P[three]
        m = 2.0 * np.sqrt(np.maximum(-Pm / 3.0, 0.0))
        with np.errstate(divide="ignore", invalid="ignore"):
            cphi = np.where(Pm < 0.0, (3.0 * Q[three] / (2.0 * Pm)) * np.sqrt(-3.0 / Pm), 0.0)
        phi = np.arccos(np.clip(cphi, -1.0, 1.0))
        for k in range(3):
            roots[k, three] = m * np.cos(phi / 3.0 - 2.0 * np.pi * k / 3.0) - c2[three] / 3.0
    roots = np.sort(roots, axis=0)  # NaN sorts last
    for k in range(3):
        roots[k] = _polish(roots[k], c2, c1, c0)
    # keep ascending order with NaNs last after polishing
    return np.sort(roots, axis=0)


def log_ratio(Z, B):
    """ln[(Z + (1 + sqrt2) B) / (Z + (1 - sqrt2) B)]."""
    return np.log((Z + (1.0 + SQ2) * B) / (Z + (1.0 - SQ2) * B))


def gibbs_departure(Z, A, B):
    """Dimensionless departure Gibbs energy g/RT of a root."""
    return Z - 1.0 - np.log(Z - B) - A / (2.0 * SQ2 * B) * log_ratio(Z, B)


def select_root(roots, A, B):
    """Z of least g/RT among real roots above B (ties within 1e-12: larger Z); NaN if none."""
    N = A.shape[0]
    Z = np.full(N, np.nan)
    g_best = np.full(N, np.inf)
    for k in (2, 1, 0):  # descending Z, so an exact tie keeps the larger root
        r = roots[k]
        ok = np.isfinite(r) & (r > B)
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(ok, gibbs_departure(np.where(ok, r, 2.0 * B + 1.0), A, B), np.inf)
        take = ok & (g < g_best - 1e-12)
        Z = np.where(take, r, Z)
        g_best = np.where(take, g, g_best)
    return Z


def h_departure(T, Z, A, B, a_m, da, b_m):
    """Molar departure enthalpy, J/mol."""
    return R * T * (Z - 1.0) + (T * da - a_m) / (2.0 * SQ2 * b_m) * log_ratio(Z, B)


def cp_departure(T, p, Z, A, B, a_m, da, d2a, b_m):
    """Molar d(h_dep)/dT at fixed p and composition, with dZ/dT from the implicit cubic."""
    dB = -B / T
    dA = A * (da / a_m - 2.0 / T)
    F_Z = 3.0 * Z**2 - 2.0 * (1.0 - B) * Z + (A - 3.0 * B**2 - 2.0 * B)
    F_A = Z - B
    F_B = Z**2 - (6.0 * B + 2.0) * Z - (A - 2.0 * B - 3.0 * B**2)
    dZ = -(F_A * dA + F_B * dB) / F_Z
    L = log_ratio(Z, B)
    dL = ((dZ + (1.0 + SQ2) * dB) / (Z + (1.0 + SQ2) * B)
          - (dZ + (1.0 - SQ2) * dB) / (Z + (1.0 - SQ2) * B))
    k = 1.0 / (2.0 * SQ2 * b_m)
    return R * (Z - 1.0) + R * T * dZ + k * T * d2a * L + k * (T * da - a_m) * dL


def state(mech, T, p, Y):
    """Real-fluid state of each cell. Returns a dict of [N] arrays (and X [n, N]):
    W_mix, X, a_m, da, d2a, b_m, A, B, Z, status, h_dep (J/mol), h_ig, h (J/kg),
    cp (J/(kg K)), rho (kg/m^3)."""
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    X, W_mix = mole_fractions(mech.W, Y)
    a_m, da, d2a, b_m = mixture_params(mech, X, T)
    A = a_m * p / (R * T) ** 2
    B = b_m * p / (R * T)
    roots = cubic_real_roots(*cubic_coefficients(A, B))
    Z = select_root(roots, A, B)
    status = np.where(np.isfinite(Z), 0, NO_ROOT).astype(np.int32)
    with np.errstate(invalid="ignore", divide="ignore"):
        h_dep = h_departure(T, Z, A, B, a_m, da, b_m)
        cp_dep = cp_departure(T, p, Z, A, B, a_m, da, d2a, b_m)
        h_ig = mixture_h_ig(mech.nasa, mech.W, T, Y)
        h = h_ig + h_dep / W_mix
        cp = mixture_cp_ig(mech.nasa, mech.W, T, Y) + cp_dep / W_mix
        rho = p * W_mix / (Z * R * T)
    return dict(W_mix=W_mix, X=X, a_m=a_m, da=da, d2a=d2a, b_m=b_m, A=A, B=B, roots=roots,
                Z=Z, status=status, h_dep=h_dep, h_ig=h_ig, h=h, cp=cp, rho=rho)
