"""Pins of the stiff-chemistry truth (oracle/truth.c): an analytic solution, conservation laws,
chemical equilibrium at long times, the Python oracle's equation of state, an independent
library integrator (scipy's Radau IIA) and self-convergence."""
from types import SimpleNamespace

import numpy as np
import pytest

import synth
from oracle import pr_eos as pe
from oracle import truth
from oracle.thermo import R


@pytest.fixture(scope="module")
def layer():
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=96)
    sel = np.linspace(0, 95, 24).astype(int)
    return mech, T, p, Y, sel


def test_c_equation_of_state_matches_python_oracle():
    for name in ("small-fp32-4k", "layer1d-30sp-1m"):
        mech, _, T, p, Y = synth.configs.build(name, n_cells=200)
        h, cp, rho, ok = truth.state(mech, T, p, Y)
        s = pe.state(mech, T, p, Y)
        assert ok.all()
        np.testing.assert_allclose(h, s["h"], rtol=1e-12, atol=1e-6)
        np.testing.assert_allclose(cp, s["cp"], rtol=1e-11)
        np.testing.assert_allclose(rho, s["rho"], rtol=1e-12)


def _two_species(A=1e7):
    """A <=> B isomers (same W, critical constants, cp and enthalpy), B favoured by entropy
    (s/R offset +50, so Kc = e^50): first order A -> B with constant k = A, isothermal."""
    nasa = np.array([[4.0, 1e-4, 0, 0, 0, -2000.0, 5.0], [4.0, 1e-4, 0, 0, 0, -2000.0, 55.0]])
    return SimpleNamespace(n=2, W=np.array([0.03, 0.03]), Tc=np.array([300.0, 300.0]),
                           pc=np.array([4e6, 4e6]), omega=np.array([0.1, 0.1]), kij=np.zeros((2, 2)),
                           nasa=nasa, nu_f=np.array([[1.0], [0.0]]), nu_r=np.array([[0.0], [1.0]]),
                           A=np.array([A]), beta=np.array([0.0]), Ea=np.array([0.0]))


def test_first_order_decay_is_exponential():
    m = _two_species()
    T = np.array([800.0, 1200.0])
    p = np.array([5e6, 1.5e7])
    Y = np.array([[0.9, 0.6], [0.1, 0.4]])
    for dt in (3e-8, 1e-7, 3e-7):
        T1, Y1, ok, _, _ = truth.advance(m, T, p, Y, dt)
        assert ok.all()
        np.testing.assert_allclose(Y1[0], Y[0] * np.exp(-1e7 * dt), rtol=2e-8)
        np.testing.assert_allclose(T1, T, rtol=1e-10)


def test_mass_elements_and_enthalpy_are_conserved(layer):
    mech, T, p, Y, sel = layer
    T1, Y1, ok, _, _ = truth.advance(mech, T[sel], p[sel], Y[:, sel], 1e-7)
    assert ok.all()
    np.testing.assert_allclose(Y1.sum(axis=0), 1.0, atol=1e-12)
    atoms0 = mech.elements.T @ (Y[:, sel] / mech.W[:, None])
    atoms1 = mech.elements.T @ (Y1 / mech.W[:, None])
    np.testing.assert_allclose(atoms1, atoms0, rtol=1e-11, atol=1e-11)
    h0 = pe.state(mech, T[sel], p[sel], Y[:, sel])["h"]
    h1 = pe.state(mech, T1, p[sel], Y1)["h"]
    np.testing.assert_allclose(h1, h0, rtol=0, atol=1e-6 * np.abs(h0).max() + 1e-3)


def test_reversible_isomerisation_relaxes_to_kc():
    """A <=> B isomers, identical except s/R of B larger by 1: Kc = e, so the forward
    direction carries the Arrhenius constant k and the reverse k / e; Y_A relaxes to
    1 / (1 + e) with rate k (1 + 1/e), exactly."""
    m = _two_species(A=2e6)
    m.nasa = m.nasa.copy()
    m.nasa[1, 6] = m.nasa[0, 6] + 1.0
    T = np.array([900.0])
    p = np.array([8e6])
    Y0 = np.array([[0.8], [0.2]])
    k = 2e6 * (1 + np.exp(-1.0))
    yinf = 1.0 / (1.0 + np.e)
    for dt in (2e-7, 1e-6, 1e-4):
        _, Y1, ok, _, _ = truth.advance(m, T, p, Y0, dt)
        assert ok.all()
        assert Y1[0, 0] == pytest.approx(yinf + (0.8 - yinf) * np.exp(-k * dt), rel=1e-8)


def test_dimerisation_equilibrium_law_of_mass_action():
    """2 A <=> A2 in the ideal-gas limit (pc x 1e12), A2 = two A's in molar thermo except an
    entropy offset, so the reaction is isothermal; at long time c_A2 / c_A^2 must equal
    Kc = exp(ds/R) (R T / p0), in m^3/mol -- the pressure factor of a reaction that changes
    the number of moles. Equilibrium composition from the resulting quadratic."""
    a = np.array([3.5, 5e-4, 0, 0, 0, -1000.0, 8.0])
    nasa = np.vstack([a, 2 * a])
    nasa[1, 6] = 2 * a[6] + 3.0                      # s/R offset of the dimer
    m = SimpleNamespace(n=2, W=np.array([0.016, 0.032]), Tc=np.array([200.0, 300.0]),
                        pc=np.array([4e6, 4e6]) * 1e12, omega=np.array([0.0, 0.0]),
                        kij=np.zeros((2, 2)), nasa=nasa, nu_f=np.array([[2.0], [0.0]]),
                        nu_r=np.array([[0.0], [1.0]]), A=np.array([1e9]), beta=np.array([0.0]),
                        Ea=np.array([0.0]))
    T, p = 1000.0, 2e6
    _, Y1, ok, _, _ = truth.advance(m, np.array([T]), np.array([p]), np.array([[1.0], [0.0]]), 1e-2)
    assert ok.all()
    Kc = np.exp(3.0) * R * T / 101325.0               # m^3/mol
    # mass balance Y_A + Y_A2 = 1, ideal gas rho = p W_mix / (R T):
    # c_A2 / c_A^2 = (Y_A2 / W2) W_A^2 R T / (p W_mix Y_A^2) with 1/W_mix = Y_A/W_A + Y_A2/W2
    from scipy.optimize import brentq

    def resid(yA):
        yA2 = 1 - yA
        Wm = 1.0 / (yA / 0.016 + yA2 / 0.032)
        rho = p * Wm / (R * T)
        return (rho * yA2 / 0.032) / (rho * yA / 0.016) ** 2 - Kc

    yA = brentq(resid, 1e-9, 1 - 1e-12, xtol=1e-15)
    assert Y1[0, 0] == pytest.approx(yA, rel=1e-6)


def test_bdf_agrees_with_scipy_radau(layer):
    from scipy.integrate import solve_ivp
    mech, T, p, Y, sel = layer
    for i in sel[[3, 10, 17]]:
        h0 = pe.state(mech, T[i:i + 1], p[i:i + 1], Y[:, i:i + 1])["h"][0]
        Tw = [T[i]]

        def f(t, y):
            d, Tw[0] = truth.rhs(mech, p[i], h0, y, Tw[0])
            return d

        r = solve_ivp(f, (0.0, 1e-7), Y[:, i], method="Radau", rtol=1e-10, atol=1e-14)
        assert r.success
        _, Y1, ok, _, _ = truth.advance(mech, T[i:i + 1], p[i:i + 1], Y[:, i:i + 1], 1e-7)
        assert ok.all()
        np.testing.assert_allclose(Y1[:, 0], r.y[:, -1], rtol=1e-6, atol=1e-10)


def test_bdf_self_convergence(layer):
    mech, T, p, Y, sel = layer
    a = truth.advance(mech, T[sel], p[sel], Y[:, sel], 1e-7, rtol=1e-9)
    b = truth.advance(mech, T[sel], p[sel], Y[:, sel], 1e-7, rtol=1e-10)
    ok = a[2] & b[2]
    assert ok.all()
    assert np.abs(a[1] - b[1]).max() <= 1e-7
    assert np.abs(a[0] - b[0]).max() <= 1e-4
