"""Real-fluid transport properties of a mixture in FP64 -- TEST INFRASTRUCTURE ONLY (part of the
oracle; never imported by the product path).

Sec. 2: under supercritical conditions the paper's property network (PRNet) yields, besides
density and temperature, the transport properties of the mixture -- viscosity mu and thermal
diffusivity alpha among them -- "based on Peng-Robinson EoS". The paper names no transport model.
The reading here is the high-pressure method of Chung, Ajlan, Lee & Starling (Ind. Eng. Chem.
Res. 27, 671, 1988), the usual companion of a cubic EoS in real-fluid combustion codes, as
restated in Poling, Prausnitz & O'Connell, "The Properties of Gases and Liquids" (5th ed.,
Eqs. 9-4.10, 9-5.24..44, 9-6.18..20, 10-3.14, 10-5.5), evaluated at the Peng-Robinson density:

  * species i: Tc, omega, molar mass M (g/mol); critical volume from the Peng-Robinson critical
    compressibility, Vc = Zc R Tc / pc with Zc = 0.307401 (the synthetic mechanism carries no Vc);
    nonpolar, not associating (reduced dipole and association factor 0);
  * mixing (Chung's rules, binary factors 1): sigma_i = 0.809 Vc_i^(1/3), eps_i/k = Tc_i / 1.2593,
    sigma_m^3 = sum_ij x_i x_j sigma_ij^3, (eps/k)_m = sum_ij x_i x_j eps_ij sigma_ij^3 / sigma_m^3,
    omega_m = sum_ij x_i x_j (omega_i + omega_j)/2 sigma_ij^3 / sigma_m^3,
    M_m = [sum_ij x_i x_j eps_ij sigma_ij^2 M_ij^(1/2) / ((eps/k)_m sigma_m^2)]^2 with
    sigma_ij = (sigma_i sigma_j)^(1/2), eps_ij = (eps_i eps_j)^(1/2), M_ij = 2 M_i M_j / (M_i + M_j);
    then Tc_m = 1.2593 (eps/k)_m, Vc_m = (sigma_m / 0.809)^3;
  * viscosity (micropoise): eta = eta* 36.344 (M Tc)^(1/2) / Vc^(2/3),
    eta* = T*^(1/2) / Omega_v F_c (1 / G2 + E6 y) + E7 y^2 G2 exp(E8 + E9 / T* + E10 / T*^2),
    T* = 1.2593 T / Tc, F_c = 1 - 0.2756 omega, y = rho Vc / 6 (rho molar, mol/cm^3),
    G1 = (1 - y/2) / (1 - y)^3,
    G2 = [E1 (1 - exp(-E4 y)) / y + E2 G1 exp(E5 y) + E3 G1] / (E1 E4 + E2 + E3),
    E_i = a_i + b_i omega; Omega_v the collision integral of Neufeld, Janzen & Aziz (1972);
  * thermal conductivity (W/(m K)): lambda = 31.2 eta0 Psi / M' (1 / H2 + B6 y) + q B7 y^2 Tr^(1/2) H2,
    eta0 the dilute viscosity (Pa s; the y -> 0 limit of eta), M' in kg/mol,
    Psi = 1 + a {[0.215 + 0.28288 a - 1.061 b + 0.26665 Z] / [0.6366 + b Z + 1.061 a b]},
    a = Cv/R - 3/2 (ideal-gas Cv of the mixture), b = 0.7862 - 0.7109 omega + 1.3168 omega^2,
    Z = 2 + 10.5 Tr^2, q = 3.586e-3 (Tc / M')^(1/2) / Vc^(2/3), H2 as G2 with B1..B5,
    B_i = a_i + b_i omega;
  * thermal diffusivity alpha = lambda / (rho_mass c_p), c_p the real-fluid (Peng-Robinson)
    mass heat capacity.
"""
from __future__ import annotations

import numpy as np

from . import pr_eos
from .thermo import R, species_cp_R

ZC_PR = 0.307401                 # critical compressibility of the Peng-Robinson EoS
NEUFELD = (1.16145, 0.14874, 0.52487, 0.77320, 2.16178, 2.43787)

# Chung's viscosity coefficients E_i = a_i + b_i omega (+ c_i mu_r^4 + d_i kappa, zero here)
E_AB = np.array([
    [6.324, 50.412], [1.210e-3, -1.154e-3], [5.283, 254.209], [6.623, 38.096],
    [19.745, 7.630], [-1.900, -12.537], [24.275, 3.450], [0.7972, 1.117],
    [-0.2382, 0.06770], [0.06863, 0.3479]])
# Chung's conductivity coefficients B_i = a_i + b_i omega
B_AB = np.array([
    [2.4166, 0.74824], [-0.50924, -1.5094], [6.6107, 5.6207], [14.543, -8.9139],
    [0.79274, 0.82019], [-5.8634, 12.801], [91.089, 128.73]])


def critical_volume(Tc, pc):
    """Vc (cm^3/mol) from the Peng-Robinson critical compressibility."""
    return ZC_PR * R * np.asarray(Tc, np.float64) / np.asarray(pc, np.float64) * 1e6


def collision_integral(Ts):
    """Omega_v(T*) of Neufeld, Janzen & Aziz (1972), valid for 0.3 <= T* <= 100."""
    A, B, C, D, E, F = NEUFELD
    Ts = np.asarray(Ts, np.float64)
    return A * Ts ** (-B) + C * np.exp(-D * Ts) + E * np.exp(-F * Ts)


def mixture_params(mech, X):
    """Chung's pseudo-critical mixture (Tc_m [N], Vc_m [N] cm^3/mol, omega_m [N], M_m [N] g/mol)
    of mole fractions X [n, N], by the plain double sums over species pairs."""
    Vc = critical_volume(mech.Tc, mech.pc)
    sig = 0.809 * Vc ** (1.0 / 3.0)
    eps = mech.Tc / 1.2593
    M = mech.W * 1e3
    n = mech.n
    s3 = np.zeros_like(X[0])
    e3 = np.zeros_like(X[0])
    w3 = np.zeros_like(X[0])
    for i in range(n):
        for j in range(n):
            xx = X[i] * X[j]
            sij3 = (sig[i] * sig[j]) ** 1.5
            s3 += xx * sij3
            e3 += xx * np.sqrt(eps[i] * eps[j]) * sij3
            w3 += xx * 0.5 * (mech.omega[i] + mech.omega[j]) * sij3
    eps_m = e3 / s3
    sig_m2 = s3 ** (2.0 / 3.0)
    mm = np.zeros_like(X[0])
    for i in range(n):
        for j in range(n):
            Mij = 2.0 * M[i] * M[j] / (M[i] + M[j])
            mm += X[i] * X[j] * np.sqrt(eps[i] * eps[j]) * sig[i] * sig[j] * np.sqrt(Mij)
    M_m = (mm / (eps_m * sig_m2)) ** 2
    return 1.2593 * eps_m, s3 / 0.809 ** 3, w3 / s3, M_m


def _g2(C, y):
    """Chung's G2 (or H2) with coefficients C1..C5 at reduced density y > 0."""
    G1 = (1.0 - 0.5 * y) / (1.0 - y) ** 3
    return (C[0] * (1.0 - np.exp(-C[3] * y)) / y + C[1] * G1 * np.exp(C[4] * y) + C[2] * G1) / \
        (C[0] * C[3] + C[1] + C[2])


def viscosity_dilute(T, Tc, Vc, omega, M):
    """Low-pressure viscosity, micropoise (Chung's Eq. 9-4.10 form)."""
    Ts = 1.2593 * np.asarray(T, np.float64) / Tc
    return 40.785 * (1.0 - 0.2756 * omega) * np.sqrt(M * T) / (Vc ** (2.0 / 3.0) * collision_integral(Ts))


def viscosity(T, rho_molar, Tc, Vc, omega, M):
    """Dense-fluid viscosity, micropoise; rho_molar in mol/cm^3."""
    T = np.asarray(T, np.float64)
    Ts = 1.2593 * T / Tc
    E = E_AB[:, 0][:, None] + E_AB[:, 1][:, None] * np.asarray(omega)[None, ...]
    y = rho_molar * Vc / 6.0
    G2 = _g2(E, y)
    eta_k = np.sqrt(Ts) / collision_integral(Ts) * (1.0 - 0.2756 * omega) * (1.0 / G2 + E[5] * y)
    eta_p = E[6] * y ** 2 * G2 * np.exp(E[7] + E[8] / Ts + E[9] / Ts ** 2)
    return (eta_k + eta_p) * 36.344 * np.sqrt(M * Tc) / Vc ** (2.0 / 3.0)


def conductivity(T, rho_molar, Tc, Vc, omega, M, cv_molar):
    """Dense-fluid thermal conductivity, W/(m K); cv_molar the ideal-gas Cv, J/(mol K)."""
    T = np.asarray(T, np.float64)
    Mk = M * 1e-3
    eta0 = viscosity_dilute(T, Tc, Vc, omega, M) * 1e-7          # Pa s
    a = cv_molar / R - 1.5
    b = 0.7862 - 0.7109 * omega + 1.3168 * omega ** 2
    Tr = T / Tc
    Zp = 2.0 + 10.5 * Tr ** 2
    psi = 1.0 + a * (0.215 + 0.28288 * a - 1.061 * b + 0.26665 * Zp) / (0.6366 + b * Zp + 1.061 * a * b)
    Bc = B_AB[:, 0][:, None] + B_AB[:, 1][:, None] * np.asarray(omega)[None, ...]
    y = rho_molar * Vc / 6.0
    H2 = _g2(Bc, y)
    q = 3.586e-3 * np.sqrt(Tc / Mk) / Vc ** (2.0 / 3.0)
    return 31.2 * eta0 * psi / Mk * (1.0 / H2 + Bc[5] * y) + q * Bc[6] * y ** 2 * np.sqrt(Tr) * H2


def state(mech, T, p, Y):
    """Transport properties of cell states: dict of mu (Pa s), lam (W/(m K)), alpha (m^2/s) and
    the intermediate rho_molar (mol/cm^3), Tc_m, Vc_m, omega_m, M_m, cv (J/(mol K)), [N] each."""
    T = np.asarray(T, np.float64)
    s = pr_eos.state(mech, T, p, Y)
    X, W_mix = pr_eos.mole_fractions(mech.W, np.asarray(Y, np.float64))
    Tc, Vc, om, M = mixture_params(mech, X)
    rho_molar = s["rho"] / W_mix * 1e-6                          # mol/cm^3
    cv = R * np.sum(X * species_cp_R(mech.nasa, T), axis=0) - R
    mu = viscosity(T, rho_molar, Tc, Vc, om, M) * 1e-7           # micropoise -> Pa s
    lam = conductivity(T, rho_molar, Tc, Vc, om, M, cv)
    return {"mu": mu, "lam": lam, "alpha": lam / (s["rho"] * s["cp"]), "rho_molar": rho_molar,
            "Tc_m": Tc, "Vc_m": Vc, "omega_m": om, "M_m": M, "cv": cv, "rho": s["rho"],
            "cp": s["cp"], "status": s["status"]}
