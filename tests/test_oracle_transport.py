"""Pins of the transport oracle (oracle/transport.py: Chung et al. 1988 at the Peng-Robinson
density) against facts outside it: tabulated Lennard-Jones collision integrals, the method's own
dilute-gas limit, Eucken's monatomic conductivity, and invariants of the mixing rules."""
from types import SimpleNamespace

import numpy as np
import pytest

import synth
from oracle import transport as tr
from oracle.thermo import R


def test_collision_integral_matches_lennard_jones_table():
    """Neufeld, Janzen & Aziz's fit against the Lennard-Jones 12-6 viscosity collision integral
    Omega(2,2)* tabulated by Hirschfelder, Curtiss & Bird (1954), within 0.5 % on 1 <= T* <= 10."""
    table = {1.0: 1.587, 1.5: 1.314, 2.0: 1.175, 3.0: 1.039, 5.0: 0.9268, 10.0: 0.8242}
    for ts, om in table.items():
        assert tr.collision_integral(ts) == pytest.approx(om, rel=5e-3), ts


def test_dense_viscosity_reduces_to_the_dilute_gas():
    """As the density goes to zero (y -> 0: G2 -> 1, the dense term -> 0) the dense-fluid
    viscosity becomes the low-pressure Chapman-Enskog form 40.785 F_c (M T)^(1/2) /
    (Vc^(2/3) Omega_v): 36.344 * 1.2593^(1/2) = 40.7847."""
    T = np.array([150.0, 400.0, 1500.0, 3000.0])
    Tc, Vc, om, M = 190.6, 99.0, 0.011, 16.04
    dense = tr.viscosity(T, 1e-10, Tc, Vc, om, M)
    np.testing.assert_allclose(dense, tr.viscosity_dilute(T, Tc, Vc, om, M), rtol=2e-5)
    # and the dilute viscosity itself is the hard-sphere-corrected kinetic-theory value:
    # 26.69 (M T)^(1/2) / (sigma^2 Omega_v) micropoise with sigma = 0.809 Vc^(1/3) Angstrom
    sig = 0.809 * Vc ** (1.0 / 3.0)
    ts = 1.2593 * T / Tc
    kt = 26.69 * (1.0 - 0.2756 * om) * np.sqrt(M * T) / (sig ** 2 * tr.collision_integral(ts))
    np.testing.assert_allclose(tr.viscosity_dilute(T, Tc, Vc, om, M), kt, rtol=2e-4)


def test_g2_limits():
    """G2 (and H2) -> 1 at zero density; with only the E3 term it is the Carnahan-Starling
    contact value of the hard-sphere pair distribution, (1 - y/2) / (1 - y)^3."""
    for C in (tr.E_AB[:, 0] + 0.2 * tr.E_AB[:, 1], tr.B_AB[:, 0] + 0.1 * tr.B_AB[:, 1]):
        assert tr._g2(C, 1e-9) == pytest.approx(1.0, rel=1e-6)
    y = np.linspace(0.01, 0.4, 9)
    C = np.array([0.0, 0.0, 3.0, 1.0, 0.0])
    np.testing.assert_allclose(tr._g2(C, y), (1 - y / 2) / (1 - y) ** 3, rtol=1e-14)


def test_monatomic_dilute_conductivity_is_euckens():
    """For Cv = 3R/2 (a = 0, so Psi = 1) the dilute conductivity is Eucken's monatomic value
    lambda = (15/4) R eta / M (31.2 is 15/4 R = 31.18 rounded)."""
    T = np.array([300.0, 900.0, 2500.0])
    Tc, Vc, om, M = 150.7, 75.0, 0.0, 39.95
    lam = tr.conductivity(T, 1e-10, Tc, Vc, om, M, 1.5 * R)
    eta = tr.viscosity_dilute(T, Tc, Vc, om, M) * 1e-7
    np.testing.assert_allclose(lam, 3.75 * R * eta / (M * 1e-3), rtol=1.5e-3)


def _mech(n=3):
    m = synth.make_mechanism(30, 200, 20250820)
    return SimpleNamespace(n=n, W=m.W[:n].copy(), Tc=m.Tc[:n].copy(), pc=m.pc[:n].copy(),
                           omega=m.omega[:n].copy())


def test_mixing_rules_reduce_to_the_pure_fluid_and_ignore_splitting():
    m = _mech(3)
    X = np.zeros((3, 2))
    X[1] = 1.0
    Tc, Vc, om, M = tr.mixture_params(m, X)
    np.testing.assert_allclose(Tc, m.Tc[1], rtol=1e-14)
    np.testing.assert_allclose(Vc, tr.critical_volume(m.Tc[1], m.pc[1]), rtol=1e-13)
    np.testing.assert_allclose(om, m.omega[1], rtol=1e-14)
    np.testing.assert_allclose(M, m.W[1] * 1e3, rtol=1e-13)
    # a species split into two identical halves leaves every mixture parameter unchanged
    Xr = synth.Stream(3, "transport-mix").uniform(3 * 40).reshape(3, 40)
    Xr /= Xr.sum(axis=0)
    m4 = SimpleNamespace(n=4, W=np.append(m.W, m.W[2]), Tc=np.append(m.Tc, m.Tc[2]),
                         pc=np.append(m.pc, m.pc[2]), omega=np.append(m.omega, m.omega[2]))
    X4 = np.vstack([Xr[:2], 0.3 * Xr[2:], 0.7 * Xr[2:]])
    for a, b in zip(tr.mixture_params(m, Xr), tr.mixture_params(m4, X4)):
        np.testing.assert_allclose(a, b, rtol=1e-13)
    # and the order of the species does not matter
    perm = [2, 0, 1]
    mp = SimpleNamespace(n=3, W=m.W[perm], Tc=m.Tc[perm], pc=m.pc[perm], omega=m.omega[perm])
    for a, b in zip(tr.mixture_params(m, Xr), tr.mixture_params(mp, Xr[perm])):
        np.testing.assert_allclose(a, b, rtol=1e-13)


def test_state_properties_are_consistent():
    mech, _, T, p, Y = synth.configs.build("train30-1m", n_cells=400)
    s = tr.state(mech, T, p, Y)
    assert np.all(s["status"] == 0)
    for k in ("mu", "lam", "alpha"):
        assert np.all(np.isfinite(s[k])) and np.all(s[k] > 0), k
    np.testing.assert_allclose(s["alpha"], s["lam"] / (s["rho"] * s["cp"]), rtol=1e-15)
    # at fixed composition and temperature the viscosity rises with the (Peng-Robinson) density
    Tf = np.full(6, 700.0)
    pf = np.linspace(2e6, 20e6, 6)
    Yf = np.repeat(Y[:, :1], 6, axis=1)
    sf = tr.state(mech, Tf, pf, Yf)
    assert np.all(np.diff(sf["rho"]) > 0) and np.all(np.diff(sf["mu"]) > 0)
    assert np.all(np.diff(sf["lam"]) > 0)
