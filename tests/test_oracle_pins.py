"""Pins of the FP64 oracle against facts fixed outside the oracle itself: closed forms,
thermodynamic identities, library routines, the Peng-Robinson critical point and the
definition of the acentric factor, brute force on tiny inputs."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import synth
from oracle import network as nw
from oracle import pr_eos as pe
from oracle import step, thermo
from oracle.thermo import R


def _pure(Tc=400.0, pc=5e6, omega=0.2):
    return SimpleNamespace(n=1, Tc=np.array([Tc]), pc=np.array([pc]), omega=np.array([omega]),
                           kij=np.zeros((1, 1)), W=np.array([0.03]), nasa=np.array([[4.0, 1e-3, 0, 0, 0, -1000.0, 5.0]]))


@pytest.fixture(scope="module")
def mech30():
    return synth.make_mechanism(30, 200, 20250820)


# ---------------------------------------------------------------- Peng-Robinson

def test_critical_point_gives_triple_root():
    """At T = Tc, p = pc a pure PR fluid has A = Omega_a, B = Omega_b and a (nearly) triple
    root Z_c = 0.307401 (the constants 0.45724 / 0.07780 are rounded)."""
    m = _pure()
    X = np.ones((1, 1))
    T = np.array([m.Tc[0]])
    a, da, d2a, b = pe.mixture_params(m, X, T)
    A = a * m.pc[0] / (R * T) ** 2
    B = b * m.pc[0] / (R * T)
    assert A[0] == pytest.approx(0.45724, rel=1e-13)
    assert B[0] == pytest.approx(0.07780, rel=1e-13)
    c2, c1, c0 = pe.cubic_coefficients(A, B)
    Zc = 0.307401
    assert c2[0] == pytest.approx(-3 * Zc, abs=2e-5)
    assert c1[0] == pytest.approx(3 * Zc**2, abs=2e-5)
    assert c0[0] == pytest.approx(-Zc**3, abs=2e-5)


def test_cubic_matches_pressure_explicit_form(mech30):
    """Every selected root satisfies the pressure-explicit PR equation
    p = RT/(v - b) - a / (v^2 + 2bv - b^2) with v = Z R T / p."""
    _, _, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=512)
    mech = synth.make_mechanism(9, 12, 20250819)
    s = pe.state(mech, T, p, Y)
    v = s["Z"] * R * T / p
    a, b = s["a_m"], s["b_m"]
    p_back = R * T / (v - b) - a / (v * v + 2 * b * v - b * b)
    np.testing.assert_allclose(p_back, p, rtol=1e-9)


def test_cubic_roots_vs_numpy_roots():
    rs = synth.Stream(7, "cubic")
    for _ in range(200):
        A, B = rs.uniform(1, 0.01, 3.0)[0], rs.uniform(1, 0.005, 0.5)[0]
        c2, c1, c0 = pe.cubic_coefficients(np.array([A]), np.array([B]))
        ours = pe.cubic_real_roots(c2, c1, c0)[:, 0]
        ours = np.sort(ours[np.isfinite(ours)])
        ref = np.roots([1.0, c2[0], c1[0], c0[0]])
        ref = np.sort(ref[np.abs(ref.imag) < 1e-9].real)
        if len(ref) == len(ours):
            np.testing.assert_allclose(ours, ref, rtol=1e-9, atol=1e-12)
        else:  # only near a double root may the count differ
            assert np.min(np.abs(np.diff(np.sort(np.roots([1, c2[0], c1[0], c0[0]]).real)))) < 1e-5


def test_ideal_gas_limit(mech30):
    """a, b -> 0 (pc scaled by 1e12): Z -> 1, h_dep -> 0, rho -> p W / (R T)."""
    m = SimpleNamespace(**vars(mech30))
    m.pc = mech30.pc * 1e12
    _, _, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=256)
    s = pe.state(m, T, p, Y)
    np.testing.assert_allclose(s["Z"], 1.0, atol=1e-10)
    np.testing.assert_allclose(s["h_dep"] / (R * T), 0.0, atol=1e-10)
    np.testing.assert_allclose(s["rho"], p * s["W_mix"] / (R * T), rtol=1e-10)
    np.testing.assert_allclose(s["h"], thermo.mixture_h_ig(m.nasa, m.W, T, Y), rtol=1e-10, atol=1e-6)


@pytest.mark.parametrize("omega", [0.0, 0.15, 0.3, 0.4])
def test_acentric_factor_from_saturation(omega):
    """Definition of the acentric factor: omega = -1 - log10(p_sat(0.7 Tc) / pc). PR's
    kappa(omega) is fitted so the EoS reproduces it; the saturation pressure is where the
    two outer roots have equal departure Gibbs energy."""
    from scipy.optimize import brentq
    m = _pure(omega=omega)
    T = 0.7 * m.Tc[0]
    a, _, _, b = pe.mixture_params(m, np.ones((1, 1)), np.array([T]))

    def dg(p):
        A = a * p / (R * T) ** 2
        B = b * p / (R * T)
        r = pe.cubic_real_roots(*pe.cubic_coefficients(A, B))[:, 0]
        r = r[np.isfinite(r) & (r > B[0])]
        if len(r) < 2:
            return np.nan
        return float(pe.gibbs_departure(r.min(), A, B)[0] - pe.gibbs_departure(r.max(), A, B)[0])

    ps = np.geomspace(1e3, m.pc[0], 300)
    v = np.array([dg(x) for x in ps])
    ok = np.isfinite(v)
    i = np.flatnonzero(np.diff(np.sign(v[ok])) != 0)[0]
    psat = brentq(dg, ps[ok][i], ps[ok][i + 1], xtol=1e-6)
    assert -1.0 - np.log10(psat / m.pc[0]) == pytest.approx(omega, abs=0.01)


def test_root_selection_follows_saturation():
    """Below p_sat the vapour (largest) root is stable, above it the liquid (smallest)."""
    m = _pure(omega=0.2)
    T = 0.7 * m.Tc[0]
    psat = m.pc[0] * 10 ** (-1.2)   # omega = 0.2 reproduced to ~0.002 (previous test)
    for p, want in ((0.8 * psat, "vap"), (1.25 * psat, "liq")):
        Y = np.ones((1, 1))
        s = pe.state(m, np.array([T]), np.array([p]), Y)
        r = s["roots"][:, 0]
        r = r[np.isfinite(r) & (r > s["B"][0])]
        assert len(r) == 3
        assert s["Z"][0] == (r.max() if want == "vap" else r.min())


def test_hdep_is_temperature_derivative_of_gdep(mech30):
    """h_dep = -R T^2 d(g_dep/RT)/dT at fixed p and composition (Gibbs-Helmholtz)."""
    _, _, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=64)
    T = T + 200.0
    s = pe.state(mech30, T, p, Y)

    def g_of(Tt):
        ss = pe.state(mech30, Tt, p, Y)
        return pe.gibbs_departure(ss["Z"], ss["A"], ss["B"])

    dT = 1e-5 * T
    dg = (g_of(T + dT) - g_of(T - dT)) / (2 * dT)
    np.testing.assert_allclose(-R * T**2 * dg, s["h_dep"], rtol=1e-7, atol=1e-4)


def test_cp_is_temperature_derivative_of_h(mech30):
    _, _, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=64)
    T = T + 50.0
    s = pe.state(mech30, T, p, Y)
    dT = 1e-4 * T
    hp = pe.state(mech30, T + dT, p, Y)["h"]
    hm = pe.state(mech30, T - dT, p, Y)["h"]
    np.testing.assert_allclose((hp - hm) / (2 * dT), s["cp"], rtol=1e-5)


def test_mixing_rule_invariants(mech30):
    """k_ij = 0 reduces van der Waals mixing to a_m = (sum_i X_i sqrt(a_i))^2; splitting a
    species into two identical halves (k = 0 between them) leaves a_m unchanged."""
    m = SimpleNamespace(**vars(mech30))
    m.kij = np.zeros_like(mech30.kij)
    _, _, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=32)
    X, _ = pe.mole_fractions(m.W, Y)
    a, _, _, b = pe.mixture_params(m, X, T)
    s0, _, _ = pe.sqrt_a(m.Tc, m.pc, m.omega, T)
    np.testing.assert_allclose(a, np.sum(X * s0, axis=0) ** 2, rtol=1e-13)
    # split species 5 of the real mechanism
    k = 5
    m2 = SimpleNamespace(n=31, Tc=np.append(mech30.Tc, mech30.Tc[k]), pc=np.append(mech30.pc, mech30.pc[k]),
                         omega=np.append(mech30.omega, mech30.omega[k]))
    kij2 = np.zeros((31, 31))
    kij2[:30, :30] = mech30.kij
    kij2[30, :30] = mech30.kij[k]
    kij2[:30, 30] = mech30.kij[:, k]
    kij2[30, k] = kij2[k, 30] = 0.0
    m2.kij = kij2
    X1, _ = pe.mole_fractions(mech30.W, Y)
    X2 = np.vstack([X1, X1[k:k + 1] * 0.4])
    X2[k] *= 0.6
    a1, d1, dd1, b1 = pe.mixture_params(mech30, X1, T)
    a2, d2, dd2, b2 = pe.mixture_params(m2, X2, T)
    np.testing.assert_allclose(a2, a1, rtol=1e-13)
    np.testing.assert_allclose(d2, d1, rtol=1e-12)
    np.testing.assert_allclose(b2, b1, rtol=1e-13)


def test_sqrt_a_derivatives_vs_finite_differences(mech30):
    T = np.linspace(120.0, 3000.0, 16)
    s0, s1, s2 = pe.sqrt_a(mech30.Tc, mech30.pc, mech30.omega, T)
    h = 1e-3
    sp, s1p, _ = pe.sqrt_a(mech30.Tc, mech30.pc, mech30.omega, T + h)
    sm, s1m, _ = pe.sqrt_a(mech30.Tc, mech30.pc, mech30.omega, T - h)
    np.testing.assert_allclose((sp - sm) / (2 * h), s1, rtol=1e-7)
    np.testing.assert_allclose((s1p - s1m) / (2 * h), s2, rtol=1e-6)


# ---------------------------------------------------------------- NASA-7

def test_nasa_cp_h_s_consistency(mech30):
    T = np.linspace(150.0, 3400.0, 40)
    h = thermo.species_h_molar(mech30.nasa, T)
    cp = R * thermo.species_cp_R(mech30.nasa, T)
    s = R * thermo.species_s_R(mech30.nasa, T)
    d = 1e-3
    dh = (thermo.species_h_molar(mech30.nasa, T + d) - thermo.species_h_molar(mech30.nasa, T - d)) / (2 * d)
    ds = R * (thermo.species_s_R(mech30.nasa, T + d) - thermo.species_s_R(mech30.nasa, T - d)) / (2 * d)
    np.testing.assert_allclose(dh, cp, rtol=1e-8)
    np.testing.assert_allclose(ds, cp / T[None, :], rtol=1e-7)
    # h(0 K extrapolated) offset: h/R -> a6 as T -> 0
    assert np.allclose(thermo.species_h_molar(mech30.nasa, np.array([1e-9]))[:, 0] / R,
                       mech30.nasa[:, 5], rtol=1e-9)
    assert np.all(s == s)


# ---------------------------------------------------------------- network side

def test_boxcox_round_trip_and_log_limit():
    y = np.geomspace(1e-12, 1.0, 200)
    for lam in (0.1, 0.25, 0.5):
        # lambda u + 1 = y^lambda carries an absolute rounding error of ~eps, so the
        # relative error of the round trip is ~eps / (lambda y^lambda)
        back = nw.boxcox_inverse(nw.boxcox(y, lam), lam)
        np.testing.assert_array_less(np.abs(back - y), 8 * 2.3e-16 * y ** (1 - lam) / lam + 1e-300)
    np.testing.assert_allclose(nw.boxcox(y, 1e-9), np.log(y), rtol=1e-7, atol=1e-7)
    assert nw.boxcox(0.0, 0.1) == pytest.approx(-10.0)
    assert nw.boxcox(-1e-3, 0.1) == pytest.approx(-10.0)


def test_gelu_matches_torch_tanh_form():
    x = np.linspace(-8, 8, 1001)
    ref = torch.nn.functional.gelu(torch.tensor(x, dtype=torch.float64), approximate="tanh").numpy()
    np.testing.assert_allclose(nw.gelu_tanh(x), ref, rtol=1e-14, atol=1e-15)
    assert nw.gelu_tanh(0.0) == 0.0
    assert nw.gelu_tanh(10.0) == pytest.approx(10.0, rel=1e-15)
    assert abs(nw.gelu_tanh(-10.0)) < 1e-20
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    torch.nn.functional.gelu(xt, approximate="tanh").sum().backward()
    np.testing.assert_allclose(nw.gelu_tanh_grad(x), xt.grad.numpy(), rtol=1e-12, atol=1e-14)


def test_mlp_matches_torch_float64():
    net = synth.make_network([5, 7, 6, 3], 3, 11)
    x = synth.Stream(3, "x").uniform(40 * 5, -2, 2).reshape(40, 5)
    h = torch.tensor(x)
    for l in range(net.n_layers):
        h = torch.nn.functional.linear(h, torch.tensor(net.W[l]), torch.tensor(net.b[l]))
        if l < net.n_layers - 1:
            h = torch.nn.functional.gelu(h, approximate="tanh")
    np.testing.assert_allclose(nw.mlp_forward(net, x), h.numpy(), rtol=1e-13, atol=1e-15)


def test_mlp_brute_force_2_3_1():
    """Hand-set 2-3-1 net: with zero hidden pre-activations GELU(0) = 0 and the output is
    its bias; with hidden pre-activation s on one unit the output is w * GELU(s) + c."""
    net = SimpleNamespace(n_layers=2, W=[np.array([[1.0, -1.0], [0.0, 0.0], [2.0, 0.0]]),
                                         np.array([[0.0, 0.0, 3.0]])],
                          b=[np.zeros(3), np.array([0.5])])
    x = np.array([[1.0, 1.0], [0.0, 5.0]])
    out = nw.mlp_forward(net, x)[:, 0]
    g2 = 0.5 * 2.0 * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (2.0 + 0.044715 * 8.0)))
    assert out[0] == pytest.approx(0.5 + 3.0 * g2, rel=1e-15)
    assert out[1] == pytest.approx(0.5, rel=1e-15)


def _net_2sp(lam=0.5):
    """A two-species network holder with hand-picked normalisation constants (no layers)."""
    return SimpleNamespace(lam=lam, in_mean=np.array([1000.0, 1.0e7, -1.0, 0.5]),
                           in_std=np.array([500.0, 2.0e6, 2.0, 0.25]),
                           out_mean=np.array([0.25, -0.5]), out_std=np.array([2.0, 0.5]))


def test_normalise_inputs_by_hand():
    """Sec. 2 fixes the input order (T, p, Y_1, Y_2) and Sec. 3.3.1 the Z-score
    (v - mean) / std. With lambda = 1/2, BC(y) = 2 (sqrt(y) - 1) is exact on the chosen
    mass fractions: BC(1/4) = -1, BC(1) = 0, BC(9/16) = -1/2, BC(0) = BC(-0.001) = -2.
    Rows and columns written out by hand, one row per cell."""
    net = _net_2sp()
    T = np.array([1500.0, 750.0, 1000.0])
    p = np.array([1.2e7, 8.0e6, 1.0e7])
    Y = np.array([[0.25, 1.0, -0.001],      # species 1 of cells 0, 1, 2
                  [0.5625, 0.0, 1.0]])      # species 2
    x = nw.normalise_inputs(net, T, p, Y)
    want = np.array([
        # (T - 1000)/500, (p - 1e7)/2e6, (BC(Y1) + 1)/2, (BC(Y2) - 0.5)/0.25
        [1.0, 1.0, 0.0, -4.0],              # BC = (-1, -1/2)
        [-0.5, -1.0, 0.5, -10.0],           # BC = (0, -2)
        [0.0, 0.0, -0.5, -2.0],             # BC = (-2, 0)
    ])
    assert x.shape == (3, 4)
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-15)


def test_denormalise_by_hand():
    """The read-out de-normalisation: du = out_std O + out_mean, u = BC(Y) + du,
    Y' = max(lambda u + 1, 0)^(1/lambda), then Y' / sum Y'. With lambda = 1/2 every value is
    exact: cell 0 has du = (2 * 0.5 + 0.25, 0.5 * 1 - 0.5) = (1.25, 0), u = (0.25, -0.5),
    Y' = (1.125^2, 0.75^2) = (81/64, 36/64), renormalised (9/13, 4/13); cell 1 has
    du = (-2.75, 0.5), u = (-2.75, -0.5), lambda u_1 + 1 < 0 clips species 1 to 0, so
    Y' = (0, 1). A swapped mean and spread, a missing renormalisation or a forward instead of
    an inverse transform all move these values."""
    net = _net_2sp()
    Y = np.array([[0.25, 1.0],
                  [0.5625, 0.25]])
    O = np.array([[0.5, 1.0],              # cell 0 (rows are cells)
                  [-1.5, 2.0]])            # cell 1
    Yn = nw.denormalise(net, Y, O)
    want = np.array([[9.0 / 13.0, 0.0],
                     [4.0 / 13.0, 1.0]])
    np.testing.assert_allclose(Yn, want, rtol=1e-15, atol=1e-16)


def test_mole_fractions_by_hand_and_sum():
    """X_k = Y_k W_mix / W_k with W_mix = 1 / sum Y_k / W_k. Equal masses of species of
    2 g/mol and 32 g/mol: 1 / W_mix = 250 + 15.625 = 265.625 mol/kg, X = (16/17, 1/17).
    On a 30-species field: sum X = 1 and X_k W_k / W_mix gives back Y_k."""
    X, Wm = pe.mole_fractions(np.array([0.002, 0.032]), np.array([[0.5], [0.5]]))
    np.testing.assert_allclose(X[:, 0], [16.0 / 17.0, 1.0 / 17.0], rtol=1e-15)
    assert Wm[0] == pytest.approx(1.0 / 265.625, rel=1e-15)
    mech = synth.make_mechanism(30, 200, 20250820)
    _, _, _, _, Y = synth.configs.build("layer1d-30sp-1m", n_cells=500)
    X, Wm = pe.mole_fractions(mech.W, Y)
    np.testing.assert_allclose(X.sum(axis=0), 1.0, rtol=1e-14)
    np.testing.assert_allclose(X * mech.W[:, None] / Wm[None, :], Y, rtol=1e-14, atol=1e-300)
    # heavier species have smaller mole fractions than mass fractions, and conversely
    heavy = mech.W[:, None] > Wm[None, :]
    assert np.all((X <= Y * (1 + 1e-14))[heavy]) and np.all((X >= Y * (1 - 1e-14))[~heavy])


# ---------------------------------------------------------------- step level

def test_newton_round_trip(mech30):
    _, _, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=128)
    h0 = pe.state(mech30, T, p, Y)["h"]
    T0 = np.clip(T + np.where(np.arange(128) % 2 == 0, 300.0, -40.0), 60.0, 4000.0)
    Ts, st = step.solve_T(mech30, p, Y, h0, T0)
    assert np.all(st == 0)
    np.testing.assert_allclose(Ts, T, atol=1e-8, rtol=0)


def test_newton_started_at_the_root_stops_at_once(mech30):
    """h(T0) = h0 exactly gives a zero Newton step, which must end the iteration (and not
    be mistaken for a step that leaves the bracket); from a nearby start the count stays
    small for every cell of the uniform workload."""
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=1024)
    h0 = pe.state(mech, T, p, Y)["h"]
    Ts, st, it = step.solve_T(mech, p, Y, h0, T, return_iters=True)
    assert np.all(st == 0) and np.all(it <= 2)
    np.testing.assert_allclose(Ts, T, rtol=1e-14)
    x = nw.normalise_inputs(net, T, p, Y)
    Yn = nw.denormalise(net, Y, nw.mlp_forward(net, x))
    Ts, st, it = step.solve_T(mech, p, Yn, h0, T, tol=1e-10, return_iters=True)
    assert np.all(st == 0) and it.max() <= 8, np.bincount(it)


def test_zero_network_output_leaves_state():
    """A network whose read-out is identically zero (and zero output mean) predicts no
    change: Y' = Y to round-off and, by enthalpy conservation, T' = T."""
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=256)
    net.W[-1] = np.zeros_like(net.W[-1])
    net.b[-1] = np.zeros_like(net.b[-1])
    To, Yo, st = step.chem_step(mech, net, T, p, Y, net.dt, T_react=0.0)
    assert np.all(st == 0)
    np.testing.assert_allclose(Yo, Y, atol=1e-15)
    np.testing.assert_allclose(To, T, atol=1e-8)


def test_step_mass_and_inactive_cells():
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=512)
    To, Yo, st = step.chem_step(mech, net, T, p, Y, net.dt, T_react=600.0)
    act = T > 600.0
    np.testing.assert_allclose(Yo.sum(axis=0), 1.0, atol=1e-14)
    assert np.array_equal(To[~act], T[~act]) and np.array_equal(Yo[:, ~act], Y[:, ~act])
    assert np.all(st == 0)
    # enthalpy of the new state equals the old one
    h_old = pe.state(mech, T[act], p[act], Y[:, act])["h"]
    h_new = pe.state(mech, To[act], p[act], Yo[:, act])["h"]
    # Newton stops at |dT| <= 1e-12 T, i.e. |dh| <~ cp * 1e-12 * T ~ 1e-5 J/kg
    np.testing.assert_allclose(h_new, h_old, rtol=0, atol=1e-4)


def test_dt_mismatch_raises():
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=8)
    with pytest.raises(ValueError):
        step.chem_step(mech, net, T, p, Y, 2e-7)


def test_active_cells_brute_force():
    T = synth.Stream(5, "T").uniform(1000, 100.0, 1200.0)
    T[::7] = 600.0  # ties at the threshold are inactive
    want = [i for i in range(T.shape[0]) if T[i] > 600.0]
    assert step.active_cells(T, 600.0).tolist() == want


def test_nonfinite_cells_are_flagged_and_untouched():
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=16)
    T = T.copy(); p = p.copy(); Y = Y.copy()
    T[3] = np.nan
    p[5] = np.inf
    Y[2, 7] = np.nan
    To, Yo, st = step.chem_step(mech, net, T, p, Y, net.dt, T_react=0.0)
    for i in (3, 5, 7):
        assert st[i] & step.NONFINITE
    assert To[5] == T[5] and np.array_equal(Yo[:, 7], Y[:, 7], equal_nan=True)


def test_oracle_is_independent_of_the_cuda_package():
    """The oracle never imports the CUDA library package, and vice versa."""
    import pathlib
    root = pathlib.Path(__file__).resolve().parents[1]
    for f in (root / "oracle").rglob("*.py"):
        assert "paper_2508_18969_gb300" not in f.read_text(), f
    pkg = root / "paper_2508_18969_gb300"
    if pkg.exists():
        for f in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")):
            txt = f.read_text()
            assert "import oracle" not in txt and "from oracle" not in txt, f


def test_round_to_bf16_matches_torch():
    x = synth.Stream(9, "bf16").normal(4000) * 10.0 ** synth.Stream(9, "e").uniform(4000, -6, 6)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nw.round_to_bf16(x), ref)


def test_rounded_mlp_with_identity_rounding_is_the_mlp():
    net = synth.make_network([5, 7, 6, 3], 3, 11)
    x = synth.Stream(3, "x").uniform(40 * 5, -2, 2).reshape(40, 5)
    np.testing.assert_array_equal(nw.mlp_forward_rounded(net, x, lambda a: a), nw.mlp_forward(net, x))


def test_round_to_e4m3_matches_torch():
    x = synth.Stream(10, "fp8").normal(6000) * 10.0 ** synth.Stream(10, "e").uniform(6000, -4, 2.3)
    x = x[np.abs(x) <= 440.0]
    ref = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(nw.round_to_e4m3(x), ref)
    # saturation and the representable extremes
    assert nw.round_to_e4m3(1e6) == 448.0 and nw.round_to_e4m3(-500.0) == -448.0
    assert nw.round_to_e4m3(2.0 ** -9) == 2.0 ** -9 and nw.round_to_e4m3(2.0 ** -11) == 0.0


def test_mlp_jacobian_matches_torch_autograd():
    net = synth.make_network([5, 7, 6, 3], 3, 11)
    x = synth.Stream(4, "xj").uniform(6 * 5, -2, 2).reshape(6, 5)
    J = nw.mlp_jacobian(net, x)

    def f(v):
        h = v
        for l in range(net.n_layers):
            h = torch.nn.functional.linear(h, torch.tensor(net.W[l]), torch.tensor(net.b[l]))
            if l < net.n_layers - 1:
                h = torch.nn.functional.gelu(h, approximate="tanh")
        return h

    for i in range(x.shape[0]):
        ref = torch.autograd.functional.jacobian(f, torch.tensor(x[i])).numpy()
        np.testing.assert_allclose(J[i], ref, rtol=1e-12, atol=1e-14)


def test_step_jacobian_zero_network_closed_form():
    """With an identically zero read-out, Y' = Y / sum(Y), so d(dY_k)/dY_j = -Y_k and
    d(dY)/dT = 0; h is homogeneous of degree one in Y, which makes dT'/dY_j = h / cp and
    dT'/dT = 1."""
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=24)
    net.W[-1] = np.zeros_like(net.W[-1])
    net.b[-1] = np.zeros_like(net.b[-1])
    J, dTn = step.chem_step_jacobian_fd(mech, net, T, p, Y, dY_min=1e-4)
    s = pe.state(mech, T, p, Y)
    for i in range(24):
        cols = [c for c in range(1, mech.n + 1) if np.isfinite(J[i, 0, c])]
        np.testing.assert_allclose(J[i][:, cols], np.repeat(-Y[:, i:i + 1], len(cols), axis=1),
                                   atol=2e-8)
        np.testing.assert_allclose(J[i][:, 0], 0.0, atol=1e-10)
        np.testing.assert_allclose(dTn[i, cols], s["h"][i] / s["cp"][i], rtol=1e-5, atol=1e-3)
        assert dTn[i, 0] == pytest.approx(1.0, rel=1e-6)


def test_step_jacobian_columns_conserve_mass():
    """sum_k Y'_k = 1 for any input, so sum_k d(dY_k)/dT = 0 and sum_k d(dY_k)/dY_j = -1."""
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=16)
    J, _ = step.chem_step_jacobian_fd(mech, net, T, p, Y, dY_min=1e-4)
    colsum = np.nansum(J, axis=1)
    fin = np.isfinite(J[:, 0, :])
    np.testing.assert_allclose(colsum[:, 0], 0.0, atol=1e-9)
    np.testing.assert_allclose(colsum[:, 1:][fin[:, 1:]], -1.0, atol=1e-7)


def test_training_gradients_match_torch_autograd():
    from oracle import train
    net = synth.make_network([5, 9, 7, 3], 3, 21)
    x = synth.Stream(5, "tx").uniform(12 * 5, -2, 2).reshape(12, 5)
    Oh = synth.Stream(5, "to").normal(12 * 3).reshape(12, 3)
    loss, dW, db = train.loss_and_grads(net, x, Oh)
    Wt = [torch.tensor(w, requires_grad=True) for w in net.W]
    bt = [torch.tensor(b, requires_grad=True) for b in net.b]
    h = torch.tensor(x)
    for l in range(net.n_layers):
        h = torch.nn.functional.linear(h, Wt[l], bt[l])
        if l < net.n_layers - 1:
            h = torch.nn.functional.gelu(h, approximate="tanh")
    lt = ((h - torch.tensor(Oh)) ** 2).sum() / x.shape[0]
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    for l in range(net.n_layers):
        np.testing.assert_allclose(dW[l], Wt[l].grad.numpy(), rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(db[l], bt[l].grad.numpy(), rtol=1e-11, atol=1e-14)


def test_adam_matches_torch_optim():
    from oracle import train
    rs = synth.Stream(6, "adam")
    p0 = [rs.normal(12).reshape(3, 4), rs.normal(3)]
    gs = [[rs.normal(12).reshape(3, 4), rs.normal(3)] for _ in range(3)]
    pt = [torch.tensor(a, requires_grad=True) for a in p0]
    opt = torch.optim.Adam(pt, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = [a.copy() for a in p0], [np.zeros_like(a) for a in p0], [np.zeros_like(a) for a in p0]
    for t, g in enumerate(gs, start=1):
        for a, gg in zip(pt, g):
            a.grad = torch.tensor(gg)
        opt.step()
        p, m, v = train.adam_step(p, g, m, v, t, lr=1e-2)
    for a, b in zip(p, pt):
        np.testing.assert_allclose(a, b.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_source_terms_conserve_mass_and_vanish_without_chemistry():
    """omega = rho (Y' - Y) / dt: sums to zero over species (Y' is renormalised), is zero for
    cells that do not react, and is zero everywhere for a network whose read-out is zero."""
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=300)
    om, Tn, st = step.chem_source(mech, net, T, p, Y, net.dt, T_react=600.0)
    rho = pe.state(mech, T, p, Y)["rho"]
    assert np.all(np.abs(om.sum(axis=0)) <= 1e-12 * rho / net.dt)
    cold = T <= 600.0
    assert np.all(om[:, cold] == 0.0) and np.array_equal(Tn[cold], T[cold])
    hot = ~cold & (st == 0)
    assert np.abs(om[:, hot]).max() > 0.0
    net.W[-1] = np.zeros_like(net.W[-1])
    net.b[-1] = np.zeros_like(net.b[-1])
    om0, Tn0, st0 = step.chem_source(mech, net, T, p, Y, net.dt, T_react=0.0)
    ok = st0 == 0
    assert np.abs(om0[:, ok]).max() <= 1e-9 * (rho[ok] / net.dt).max()


def test_gelu_second_derivative_vs_finite_differences():
    x = np.linspace(-6, 6, 241)
    h = 1e-4
    fd = (nw.gelu_tanh_grad(x + h) - nw.gelu_tanh_grad(x - h)) / (2 * h)
    np.testing.assert_allclose(nw.gelu_tanh_grad2(x), fd, atol=1e-7)


def test_tabulated_gelu_follows_its_definition_and_error_bound():
    """The tabulated GELU (Sec. 3.3.2): exactly 0 below -3 and x above 3; inside, within the
    remainder of a second-order expansion over one interval (largest third derivative times
    h^3 / 6) plus the binary32 rounding of the coefficients; equal to the tanh form at the
    nodes."""
    x = np.linspace(-8, 8, 200001)
    y = nw.gelu_table(x)
    assert np.all(y[x <= -3] == 0.0) and np.array_equal(y[x >= 3], x[x >= 3])
    inside = (x > -3) & (x < 3)
    g3 = np.abs(np.diff(nw.gelu_tanh_grad2(np.linspace(-3, 3, 60001)))).max() / 1e-4
    bound = g3 * 0.01**3 / 6 + 4e-7
    assert np.abs(y[inside] - nw.gelu_tanh(x[inside])).max() <= bound
    nodes = -3 + 0.01 * np.arange(1, 600)
    np.testing.assert_allclose(nw.gelu_table(nodes), nw.gelu_tanh(nodes), atol=4e-7)
    # the jumps at the ends of the table are the paper's approximation: GELU(3) - 3, GELU(-3)
    assert abs(nw.gelu_tanh(3.0) - 3.0) > 1e-3 and abs(nw.gelu_tanh(-3.0)) > 1e-3


def _vjp_case(n_cells, T_react):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=n_cells)
    # keep every temperature clear of the reaction threshold, so that no difference crosses it
    T = np.where(np.abs(T - T_react) < 0.02 * T_react, T_react + 0.05 * T_react, T)
    rng = np.random.default_rng(7)
    gT = rng.uniform(-1e-3, 1e-3, n_cells)
    gY = rng.uniform(-1.0, 1.0, Y.shape)
    return mech, net, T, p, Y, gT, gY, rng


def test_step_vjp_adjoint_identity_with_directional_differences():
    """<g, S'(x) v> = <S'(x)^T g, v>: the directional difference of the whole step along a
    random direction v (one perturbation of T and every Y_j at once) against the reverse-mode
    product dotted with v, on reacting and non-reacting cells (which pass the cotangents)."""
    T_react = 600.0
    mech, net, T, p, Y, gT, gY, rng = _vjp_case(20, T_react)
    assert np.any(T <= T_react) and np.any(T > T_react)
    floor = 1e-4
    vT = rng.uniform(-1.0, 1.0, T.shape) * T
    vY = np.where(Y >= floor, rng.uniform(-1.0, 1.0, Y.shape) * Y, 0.0)
    gvT, gvY = step.chem_step_vjp(mech, net, T, p, Y, gT, gY, T_react=T_react,
                                  dY_rel=1e-4, dY_min=floor)
    eps = 1e-4
    Tp, Yp, sp = step.chem_step(mech, net, T + eps * vT, p, Y + eps * vY, net.dt, T_react)
    Tm, Ym, sm = step.chem_step(mech, net, T - eps * vT, p, Y - eps * vY, net.dt, T_react)
    assert np.all(sp == 0) and np.all(sm == 0)
    lhs = gT * (Tp - Tm) / (2 * eps) + np.sum(gY * (Yp - Ym), axis=0) / (2 * eps)
    rhs = gvT * vT + np.sum(np.where(vY != 0.0, gvY * vY, 0.0), axis=0)
    scale = np.abs(gT * vT) + np.sum(np.abs(gY * vY), axis=0)
    np.testing.assert_allclose(lhs, rhs, atol=1e-6 * scale.max())
    off = ~(T > T_react)
    np.testing.assert_array_equal(gvT[off], gT[off])
    np.testing.assert_array_equal(gvY[:, off], gY[:, off])
    # a non-finite temperature is left as it was by the step: its cotangents pass through too
    Tn = T.copy()
    Tn[0] = np.nan
    gvT, gvY = step.chem_step_vjp(mech, net, Tn, p, Y, gT, gY, T_react=T_react, dY_min=floor)
    assert gvT[0] == gT[0] and np.array_equal(gvY[:, 0], gY[:, 0])


def test_step_vjp_zero_network_closed_form():
    """With a zero read-out Y' = Y / sum(Y) (sum 1 here) and T' keeps h: dY'_k/dY_j =
    [k = j] - Y_k, dY'/dT = 0, dT'/dT = 1 and dT'/dY_j = h / cp, so the product is
    g_T = gT and g_Y_j = gT h / cp + gY_j - sum_k gY_k Y_k."""
    mech, net, T, p, Y, gT, gY, _ = _vjp_case(12, 0.0)
    net.W[-1] = np.zeros_like(net.W[-1])
    net.b[-1] = np.zeros_like(net.b[-1])
    gvT, gvY = step.chem_step_vjp(mech, net, T, p, Y, gT, gY, T_react=0.0, dY_min=1e-4)
    s = pe.state(mech, T, p, Y)
    want = gT[None, :] * (s["h"] / s["cp"])[None, :] + gY - np.sum(gY * Y, axis=0)[None, :]
    fin = np.isfinite(gvY)
    assert fin.sum() > 0.5 * fin.size
    np.testing.assert_allclose(gvY[fin], want[fin], rtol=1e-5, atol=1e-3 * np.abs(gT).max() + 1e-7)
    np.testing.assert_allclose(gvT, gT, rtol=1e-6)
