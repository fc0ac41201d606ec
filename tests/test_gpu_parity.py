"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and for the
whole reaction step. Tolerances: integer work (the reacting-cell list, status bits) is
bit-exact; EoS outputs (Z, rho, h, cp, h0) within 1e-10 relative; the FP32 network path
within |dY| <= 1e-6 absolute of the FP64 network; recovered T within 1e-3 K of the oracle's
Newton fed with the GPU's own Y' (every precision).

BF16 and FP8 networks have no fixed accuracy bar: their error against the FP64 oracle is a
stated result. Their bounds here are regression bounds, about ten times the largest error
measured on GB300 for the same case (the measured value is given beside each), so a loss of
an order of magnitude in accuracy fails. The whole-step T error of a BF16/FP8 step against the
FP64 oracle comes from the network's dY (T' follows Y' through h(T', p, Y') = h0), so it is
bounded the same way and not by the 1e-3 K Newton bar."""
import numpy as np
import pytest

import synth
from oracle import network as onw
from oracle import pr_eos as ope
from oracle import step as ostep

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EOS_RTOL = 1e-10


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    assert torch.cuda.is_available()
    return m


DEV = "cuda:0"


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def host(t):
    return t.detach().cpu().numpy()


def _h_scale(mech, T, p, Y):
    """Magnitude of the terms summed into h (for a relative tolerance on a signed sum)."""
    from oracle.thermo import species_h_molar
    s = ope.state(mech, T, p, Y)
    return np.sum(np.abs(Y * species_h_molar(mech.nasa, T) / mech.W[:, None]), axis=0) + \
        np.abs(s["h_dep"] / s["W_mix"])


WORKLOADS = [("small-fp32-4k", 4096), ("layer1d-30sp-1m", 6000), ("react30-16m", 5000),
             ("mix3d-30sp-64m", 5000)]


# ---------------------------------------------------------------- a0

@pytest.mark.parametrize("N", [0, 1, 77, 4096, 3 * 4096 + 5, 100003])
def test_compaction_bit_exact(df, N):
    mech, net, _, _, _ = synth.configs.build("small-fp32-4k", n_cells=8)
    st = df.State(mech, net, T_react=600.0, batch_cells=256)
    T = synth.Stream(N, "compact").uniform(N, 100.0, 1200.0)
    if N > 10:
        T[3] = np.nan
        T[5] = 600.0
        T[7] = np.inf
    idx, cnt = st.active_compact(dev(T))
    torch.cuda.synchronize()
    want = ostep.active_cells(T, 600.0)
    c = int(host(cnt)[0])
    assert c == want.shape[0]
    assert np.array_equal(host(idx)[:c].astype(np.int64), want)
    T2 = np.nan_to_num(T, nan=500.0, posinf=700.0)
    for thr, expect in ((-1.0, N), (1e9, 0)):
        st2 = df.State(mech, net, T_react=thr, batch_cells=256)
        _, cnt2 = st2.active_compact(dev(T2))
        assert int(host(cnt2)[0]) == expect


def test_compaction_rejects_more_cells_than_int32_indices(df):
    """The list holds int32 indices, so df_active_compact refuses more than INT32_MAX cells on
    the host, before any launch (small buffers suffice: nothing is read)."""
    import ctypes
    mech, net, _, _, _ = synth.configs.build("small-fp32-4k", n_cells=8)
    st = df.State(mech, net, T_react=600.0, batch_cells=256)
    T = torch.zeros(8, dtype=torch.float64, device=DEV)
    idx = torch.zeros(8, dtype=torch.int32, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    lib = df._lib.load()
    rc = lib.df_active_compact(st.h, (1 << 31), ctypes.c_void_p(T.data_ptr()),
                               ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == df._lib.DF_ERR_INVALID_ARG
    assert b"INT32_MAX" in lib.df_get_last_error(st.h)
    st.close()


# ---------------------------------------------------------------- a1-a5 and properties

@pytest.mark.parametrize("name,N", WORKLOADS)
def test_eos_pre_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    st = df.State(mech, net, batch_cells=1024)
    h0, Z, x, s = st.eos_pre(dev(T), dev(p), dev(Y))
    torch.cuda.synchronize()
    o = ope.state(mech, T, p, Y)
    assert np.array_equal(host(s), o["status"])
    np.testing.assert_allclose(host(Z), o["Z"], rtol=EOS_RTOL)
    scale = _h_scale(mech, T, p, Y)
    eh = np.max(np.abs(host(h0) - o["h"]) / scale)
    assert eh <= EOS_RTOL
    xo = onw.normalise_inputs(net, T, p, Y)
    ex = np.abs(host(x) - xo).max()
    print(f"ERR eos_pre {name}: Z rel {np.max(np.abs(host(Z) / o['Z'] - 1)):.3e} "
          f"h0 rel {eh:.3e} x abs {ex:.3e}")
    np.testing.assert_allclose(host(x), xo, atol=2e-6, rtol=1e-6)


@pytest.mark.parametrize("name,N", WORKLOADS[:2])
def test_real_fluid_props_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    st = df.State(mech, net, batch_cells=1024)
    rho, h, cp, Z = st.real_fluid_props(dev(T), dev(p), dev(Y))
    torch.cuda.synchronize()
    o = ope.state(mech, T, p, Y)
    np.testing.assert_allclose(host(Z), o["Z"], rtol=EOS_RTOL)
    np.testing.assert_allclose(host(rho), o["rho"], rtol=EOS_RTOL)
    assert np.max(np.abs(host(h) - o["h"]) / _h_scale(mech, T, p, Y)) <= EOS_RTOL
    np.testing.assert_allclose(host(cp), o["cp"], rtol=1e-9)


# ---------------------------------------------------------------- a6-a7

@pytest.mark.parametrize("name,N", WORKLOADS[:2])
def test_mlp_fp32_vs_fp64(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y)
    st = df.State(mech, net, precision=df.DF_FP32, batch_cells=1024)
    O = st.mlp_forward(dev(x.astype(np.float32)))
    torch.cuda.synchronize()
    Oo = onw.mlp_forward(net, x.astype(np.float32).astype(np.float64))
    print(f"ERR mlp_fp32 {name}: max |dO| {np.abs(host(O) - Oo).max():.3e}")
    # |dY| <= out_std * |dO| <= 1e-3 * |dO|; measured max |dO| 2.8e-7
    np.testing.assert_allclose(host(O), Oo, atol=3e-6, rtol=0)


@pytest.mark.parametrize("name,N,bn", [("small-fp32-4k", 1000, None), ("layer1d-30sp-1m", 3000, None),
                                        ("layer1d-30sp-1m", 777, "160"), ("layer1d-30sp-1m", 777, "256"),
                                        ("layer1d-30sp-1m", 777, "128"), ("layer1d-30sp-1m", 777, "192")])
def test_mlp_bf16_vs_rounded_oracle(df, name, N, bn, monkeypatch):
    """tcgen05 BF16 path against the FP64 network with BF16 rounding at the same points
    (input, weights, hidden activations); differences come only from FP32 accumulation
    order and the tanh approximation, which can move a hidden activation by one BF16 ulp."""
    if bn:
        monkeypatch.setenv("DFGB_BN", bn)
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32).astype(np.float64)
    st = df.State(mech, net, precision=df.DF_BF16, batch_cells=512)
    O = host(st.mlp_forward(dev(x.astype(np.float32))))
    torch.cuda.synchronize()
    Oq = onw.mlp_forward_rounded(net, x, onw.round_to_bf16)
    err = np.abs(O - Oq)
    Oe = onw.mlp_forward(net, x)
    print(f"ERR mlp_bf16 {name} {N} {bn}: rounded max {err.max():.3e} mean {err.mean():.3e}; "
          f"exact max {np.abs(O - Oe).max():.3e}")
    # measured: max 5.4e-4, mean 1.35e-5 (rounded oracle); max 1.23e-3 (exact network)
    assert err.max() <= 5e-3, err.max()
    assert err.mean() <= 1.5e-4, err.mean()
    # and against the exact FP64 network: BF16 storage error only
    assert np.abs(O - Oe).max() <= 1.5e-2


# ---------------------------------------------------------------- a8-a10

@pytest.mark.parametrize("name,N", WORKLOADS[:2])
def test_eos_post_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    o = ope.state(mech, T, p, Y)
    x = onw.normalise_inputs(net, T, p, Y)
    O = onw.mlp_forward(net, x).astype(np.float32)
    st = df.State(mech, net, batch_cells=1024)
    Td, Yd = dev(T), dev(Y)
    s = st.eos_post(dev(O), dev(o["h"]), Td, dev(p), Yd)
    torch.cuda.synchronize()
    Yn = onw.denormalise(net, Y, O.astype(np.float64))
    Tn, so = ostep.solve_T(mech, p, Yn, o["h"], T)
    assert np.array_equal(host(s), so)
    # the kernel forms Y' = Y (1 + lambda du Y^-lambda)^(1/lambda) with Y^-lambda in FP32
    # (relative error ~2e-7), which only scales the raw increment Y' - Y before the
    # renormalisation; renormalisation spreads it over the species of a cell (and may cancel
    # most of the increment itself). On top, the kernel carries Y (1 + delta), the sum and
    # the renormalisation in double-float (48-bit significands: below 2^-44 relative after
    # the four operations), the oracle in FP64.
    du = O.astype(np.float64).T * net.out_std[:, None] + net.out_mean[:, None]
    raw = np.abs(onw.boxcox_inverse(onw.boxcox(Y, net.lam) + du, net.lam) - Y)
    tol = 1e-6 * (raw + raw.sum(axis=0, keepdims=True)) + 1e-13 * np.abs(Yn) + 1e-300
    print(f"ERR eos_post {name}: max |dY| {np.abs(host(Yd) - Yn).max():.3e} "
          f"max |dT| {np.abs(host(Td) - Tn).max():.3e}")
    assert np.all(np.abs(host(Yd) - Yn) <= tol)
    np.testing.assert_allclose(host(Td), Tn, rtol=0, atol=1e-3)


# ---------------------------------------------------------------- whole step

def _step_check(df, mech, net, T, p, Y, prec, T_react, batch, dY_tol, dT_tol=1e-3):
    st = df.State(mech, net, precision=prec, T_react=T_react, batch_cells=batch)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    status = torch.full((T.shape[0],), -1, dtype=torch.int32, device=DEV)
    nact = torch.zeros(1, dtype=torch.int64, device=DEV)
    st.chem_step(Td, pd, Yd, status=status, n_active=nact)
    rc, a, f, _ = st.step_summary()
    To, Yo, so = ostep.chem_step(mech, net, T, p, Y, net.dt, T_react=T_react)
    Tg, Yg, sg = host(Td), host(Yd), host(status)
    assert np.array_equal(sg, so)
    act = ostep.active_cells(T, T_react)
    assert a == act.shape[0] == int(host(nact)[0])
    inact = np.setdiff1d(np.arange(T.shape[0]), act)
    assert np.array_equal(Tg[inact], T[inact]) and np.array_equal(Yg[:, inact], Y[:, inact])
    dY = np.abs(Yg - Yo).max()
    # T recovery with the GPU's own Y' (network error kept out of the Newton check)
    ok = act[so[act] == 0]
    h0 = ope.state(mech, T[ok], p[ok], Y[:, ok])["h"]
    Tr, sr = ostep.solve_T(mech, p[ok], Yg[:, ok], h0, T[ok])
    dTn = np.abs(Tg[ok] - Tr).max() if ok.size else 0.0
    dT = np.abs(Tg - To).max()
    print(f"ERR step prec={prec} n={mech.n} N={T.shape[0]}: max |dY| {dY:.3e} "
          f"max |dT| step {dT:.3e} Newton {dTn:.3e}")
    assert dY <= dY_tol, dY
    assert dT <= dT_tol, dT
    assert np.all(sr == 0)
    assert dTn <= 1e-3
    return dY


@pytest.mark.parametrize("name,N,T_react,batch", [("small-fp32-4k", 4096, 0.0, 1024),
                                                  ("small-fp32-4k", 4096, 600.0, 1000),
                                                  ("layer1d-30sp-1m", 6000, 0.0, 2048),
                                                  ("react30-16m", 5000, 600.0, 700)])
def test_chem_step_fp32(df, name, N, T_react, batch):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    _step_check(df, mech, net, T, p, Y, df.DF_FP32, T_react, batch, 1e-6)


@pytest.mark.parametrize("name,N,T_react,batch", [("small-fp32-4k", 4096, 600.0, 1024),
                                                  ("layer1d-30sp-1m", 6000, 0.0, 2048),
                                                  ("react30-16m", 5000, 600.0, 700)])
def test_chem_step_bf16(df, name, N, T_react, batch):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    # measured: max |dY| 3.3e-7 .. 3.6e-7, whole-step max |dT| 7.5e-4 .. 1.4e-3 K
    dY = _step_check(df, mech, net, T, p, Y, df.DF_BF16, T_react, batch, 4e-6, 1.5e-2)
    print(f"BF16 {name}: max |dY| vs FP64 = {dY:.3e}")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_full_size_sampled(df, prec):
    """The 2^20-cell mixing-layer workload in the bench's launch configuration; 2048 sampled
    cells are recomputed by the oracle (cells are independent)."""
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m")
    N = T.shape[0]
    st = df.State(mech, net, precision=df.DF_FP32 if prec == "fp32" else df.DF_BF16, T_react=0.0)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    status = torch.empty(N, dtype=torch.int32, device=DEV)
    st.chem_step(Td, pd, Yd, status=status)
    torch.cuda.synchronize()
    sel = np.sort(synth.Stream(1, "sample").integers(2048, N))
    To, Yo, so = ostep.chem_step(mech, net, T[sel], p[sel], Y[:, sel], net.dt, T_react=0.0)
    assert np.array_equal(host(status)[sel], so)
    dY = np.abs(host(Yd)[:, sel] - Yo).max()
    h0 = ope.state(mech, T[sel], p[sel], Y[:, sel])["h"]
    Tr, _ = ostep.solve_T(mech, p[sel], host(Yd)[:, sel], h0, T[sel])
    print(f"ERR full_size {prec}: max |dY| {dY:.3e} max |dT| step "
          f"{np.abs(host(Td)[sel] - To).max():.3e} Newton {np.abs(host(Td)[sel] - Tr).max():.3e}")
    # measured (BF16): max |dY| 3.0e-7, whole-step max |dT| 7.7e-4 K
    assert dY <= (1e-6 if prec == "fp32" else 4e-6), dY
    assert np.abs(host(Td)[sel] - To).max() <= (1e-3 if prec == "fp32" else 1e-2)
    assert np.abs(host(Td)[sel] - Tr).max() <= 1e-3


def test_repeated_steps_converge_everywhere(df):
    """Twenty-six BF16 steps over the 2^20-cell mixing layer, the bench's sequence: every
    T-from-h solve converges and no cell is flagged (the FP64 oracle flags none of these states).
    A Newton step smaller than one FP32 ulp of T once failed the double-float bracket test,
    which compared a truncated and a rounded split by their high parts, and sent the chord
    iteration to bisection and past its iteration budget in about ten cells per million."""
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m")
    N = T.shape[0]
    st = df.State(mech, net, precision=df.DF_BF16, T_react=0.0)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    status = torch.empty(N, dtype=torch.int32, device=DEV)
    flagged = []
    for _ in range(26):
        st.chem_step(Td, pd, Yd, status=status)
        flagged.append(int(torch.count_nonzero(status).item()))
    rc, n_act, n_flag, iters = st.step_summary()
    print(f"ERR repeated steps: flagged per step {flagged}, Newton iterations per cell "
          f"{iters / n_act:.4f}")
    assert max(flagged) == 0 and n_flag == 0
    assert iters / n_act < 2.05


def test_nonfinite_cells_and_empty_call(df):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=300)
    T = T.copy(); p = p.copy(); Y = Y.copy()
    T[3] = np.nan
    p[5] = np.inf
    Y[2, 7] = np.nan
    p[9] = -1.0
    st = df.State(mech, net, T_react=0.0, batch_cells=128)
    Td, Yd = dev(T), dev(Y)
    status = torch.empty(300, dtype=torch.int32, device=DEV)
    st.chem_step(Td, dev(p), Yd, status=status)
    rc, a, f, _ = st.step_summary()
    To, Yo, so = ostep.chem_step(mech, net, T, p, Y, net.dt, T_react=0.0)
    assert np.array_equal(host(status), so)
    assert f == int(np.count_nonzero(so[ostep.active_cells(T, 0.0)]))
    assert rc == 3  # DF_ERR_NOT_CONVERGED: flagged cells were reported
    empty = torch.empty(0, dtype=torch.float64, device=DEV)
    st.chem_step(empty, empty, torch.empty(9, 0, dtype=torch.float64, device=DEV))


def test_dt_mismatch_is_rejected(df):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=16)
    st = df.State(mech, net)
    with pytest.raises(df.DFError) as e:
        st.chem_step(dev(T), dev(p), dev(Y), dt=2e-7)
    assert e.value.code == 5


# ---------------------------------------------------------------- FP8 e4m3

@pytest.mark.parametrize("name,N,bn", [("small-fp32-4k", 1000, None), ("layer1d-30sp-1m", 3000, None),
                                        ("layer1d-30sp-1m", 777, "256"), ("layer1d-30sp-1m", 777, "192")])
def test_mlp_fp8_vs_rounded_oracle(df, name, N, bn, monkeypatch):
    """tcgen05 FP8 path against the FP64 network with e4m3 rounding at the same points
    (input and hidden activations x32, per-output-channel weight scales). A hidden
    activation whose FP32 accumulation lands on the other side of an e4m3 rounding boundary
    differs by one e4m3 step (6-12 %), so the bound is on the maximum and the mean."""
    if bn:
        monkeypatch.setenv("DFGB_BN", bn)
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32).astype(np.float64)
    st = df.State(mech, net, precision=df.DF_FP8_E4M3, batch_cells=512)
    O = host(st.mlp_forward(dev(x.astype(np.float32))))
    torch.cuda.synchronize()
    Oq = onw.mlp_forward_fp8(net, x, 32.0)
    err = np.abs(O - Oq)
    print(f"FP8 {name}: max {err.max():.3e} mean {err.mean():.3e} vs rounded oracle; "
          f"max {np.abs(O - onw.mlp_forward(net, x)).max():.3e} vs exact")
    # measured: max 5.1e-3, mean 1.5e-5 (rounded oracle)
    assert err.max() <= 5e-2, err.max()
    assert err.mean() <= 1.5e-4, err.mean()


@pytest.mark.parametrize("name,N,T_react,batch", [("layer1d-30sp-1m", 6000, 0.0, 2048),
                                                  ("react30-16m", 5000, 600.0, 700)])
def test_chem_step_fp8(df, name, N, T_react, batch):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    # measured: max |dY| 3.6e-6 .. 4.1e-6, whole-step max |dT| 1.3e-2 .. 1.4e-2 K
    dY = _step_check(df, mech, net, T, p, Y, df.DF_FP8_E4M3, T_react, batch, 4e-5, 0.15)
    print(f"FP8 {name}: max |dY| vs FP64 = {dY:.3e}")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_replay_matches_direct_steps(df, prec):
    """Two replays of a captured step give bit-identical fields and status to two direct
    df_chem_step calls (same kernels, fixed tile order, no atomics on the data path)."""
    mech, net, T, p, Y = synth.configs.build("react30-16m", n_cells=5000)
    st = df.State(mech, net, precision=df.DF_FP32 if prec == "fp32" else df.DF_BF16,
                  T_react=600.0, batch_cells=2048)
    Ta, Ya, Tb, Yb, pd = dev(T), dev(Y), dev(T), dev(Y), dev(p)
    sa = torch.empty(T.shape[0], dtype=torch.int32, device=DEV)
    sb = torch.empty_like(sa)
    g = st.graph(Tb, pd, Yb, status=sb)
    for _ in range(2):
        st.chem_step(Ta, pd, Ya, status=sa)
        g.launch()
    torch.cuda.synchronize()
    assert torch.equal(Ta, Tb) and torch.equal(Ya, Yb) and torch.equal(sa, sb)
    assert not torch.equal(Ta, dev(T))   # the steps did change the field
    g.close()


# ---------------------------------------------------------------- Jacobians

@pytest.mark.parametrize("name,N,prec", [("small-fp32-4k", 400, "fp32"), ("layer1d-30sp-1m", 160, "fp32"),
                                         ("small-fp32-4k", 400, "bf16"), ("layer1d-30sp-1m", 160, "fp8")])
def test_chem_jacobian_vs_finite_differences(df, name, N, prec):
    """df_chem_jacobian against central differences of the oracle's step (every cell taken as
    reacting). Columns of species below 1e-4 are excluded (the Box-Cox slope is singular at 0,
    so differences there carry no information)."""
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    pr = {"fp32": df.DF_FP32, "bf16": df.DF_BF16, "fp8": df.DF_FP8_E4M3}[prec]
    st = df.State(mech, net, precision=pr, T_react=0.0, batch_cells=256)
    J, dTn = st.chem_jacobian(dev(T), dev(p), dev(Y))
    torch.cuda.synchronize()
    J, dTn = host(J).astype(np.float64), host(dTn)
    # step 1e-4 Y_j: the oracle's Newton stops at 1e-12 T, which a smaller step would amplify
    # into the differences of T'; the truncation error stays O(1e-8) relative
    Jf, dTf = ostep.chem_step_jacobian_fd(mech, net, T, p, Y, dY_rel=1e-4, dY_min=1e-4)
    mask = np.isfinite(Jf)
    assert np.all(np.isfinite(J)), "flagged cells in the Jacobian"
    # the network part of J is ~out_std * dO/dv ~ 1e-3; BF16 tangents carry ~1 % of it
    atol = 2e-6 if prec == "fp32" else 5e-5
    err = np.abs(J - Jf)[mask]
    print(f"Jacobian {name} {prec}: max |dJ| {err.max():.3e}")
    assert err.max() <= atol + 1e-4 * np.abs(Jf[mask]).max()
    tm = np.isfinite(dTf)
    rel = np.abs(dTn - dTf)[tm] / (np.abs(dTf[tm]) + 1.0)
    print(f"dTnew {name} {prec}: max rel {rel.max():.3e}")
    assert rel.max() <= (1e-4 if prec == "fp32" else 5e-2)


# ---------------------------------------------------------------- source terms

@pytest.mark.parametrize("name,N,T_react,prec", [("small-fp32-4k", 4096, 600.0, "fp32"),
                                                 ("layer1d-30sp-1m", 3000, 0.0, "fp32"),
                                                 ("react30-16m", 3000, 600.0, "bf16")])
def test_chem_source_matches_step_and_oracle(df, name, N, T_react, prec):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    P = df.DF_FP32 if prec == "fp32" else df.DF_BF16
    st = df.State(mech, net, precision=P, T_react=T_react, batch_cells=1024)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    status = torch.full((N,), -1, dtype=torch.int32, device=DEV)
    om, Tn = st.chem_source(Td, pd, Yd, status=status)
    torch.cuda.synchronize()
    assert np.array_equal(host(Td), T) and np.array_equal(host(Yd), Y)   # inputs untouched
    # the same step in place
    T2, Y2 = dev(T), dev(Y)
    st.chem_step(T2, pd, Y2)
    torch.cuda.synchronize()
    Ts, Ys = host(T2), host(Y2)
    om, Tn, sg = host(om), host(Tn), host(status)
    assert np.array_equal(Tn, Ts)
    rho = ope.state(mech, T, p, Y)["rho"]
    back = Y + om * net.dt / rho[None, :]
    assert np.all(np.abs(back - Ys) <= 1e-12 * np.abs(Ys) + 1e-16)
    inact = np.setdiff1d(np.arange(N), ostep.active_cells(T, T_react))
    assert np.all(om[:, inact] == 0.0) and np.all(om[:, sg != 0] == 0.0)
    # against the oracle's source terms: the step's dY bar scaled by rho / dt
    om_o, Tn_o, so = ostep.chem_source(mech, net, T, p, Y, net.dt, T_react=T_react)
    assert np.array_equal(sg, so)
    dY_tol = 1e-6 if prec == "fp32" else 4e-6   # BF16 measured 3.1e-7
    print(f"ERR source {name} {prec}: max |dw| dt/rho {np.max(np.abs(om - om_o) * net.dt / rho[None, :]):.3e}")
    assert np.all(np.abs(om - om_o) <= dY_tol * rho[None, :] / net.dt)
    assert np.all(np.abs(om.sum(axis=0)) <= 1e-11 * rho / net.dt)


# ---------------------------------------------------------------- tile autotuning

@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_autotune_keeps_results_and_caches(df, prec, tmp_path):
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=5000)
    P = df.DF_BF16 if prec == "bf16" else df.DF_FP8_E4M3
    st = df.State(mech, net, precision=P, T_react=0.0, batch_cells=4096)
    before = st.tiles()
    T1, Y1 = dev(T), dev(Y)
    st.chem_step(T1, dev(p), Y1)
    cache = tmp_path / "tiles.txt"
    after = st.autotune(n_rows=4096, cache_path=cache)
    assert len(after) == net.n_layers
    paired = [b & ~df.DF_TILE_PAIR for b in after[:-1] if b & df.DF_TILE_PAIR]
    single = [b for b in after[:-1] if not b & df.DF_TILE_PAIR]
    assert all(b in (160, 224, 256) for b in paired) and after[-1] in (32, 64)
    assert all(b in (64, 128, 160, 192, 224, 256) for b in single)
    T2, Y2 = dev(T), dev(Y)
    st.chem_step(T2, dev(p), Y2)
    torch.cuda.synchronize()
    # the tiling changes neither the arithmetic nor its order
    assert np.array_equal(host(T1), host(T2)) and np.array_equal(host(Y1), host(Y2))
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == net.n_layers
    st2 = df.State(mech, net, precision=P, T_react=0.0, batch_cells=4096)
    assert st2.autotune(n_rows=4096, cache_path=cache) == after
    assert cache.read_text().strip().splitlines() == lines
    print(f"{prec}: tiles {before} -> {after}")


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_every_tile_width_gives_the_same_outputs(df, prec, monkeypatch):
    """Every single-CTA tile width gives the network outputs of the cost model's tiles bit for
    bit. With widths 1600, 800 and 400 the last n tile of a layer is narrowed to the columns
    left (rounded up to 16): 64 columns at 192 and 256, 32 at 224, 16 for the 400-wide layer at
    192, none at 160 and 64; 1100 rows leave a ragged last row tile."""
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=1100)
    P = df.DF_FP8_E4M3 if prec == "fp8" else df.DF_BF16
    x = dev(onw.normalise_inputs(net, T, p, Y).astype(np.float32))
    st = df.State(mech, net, precision=P, batch_cells=1100)
    O_ref = host(st.mlp_forward(x))
    st.close()
    for bn in ("64", "128", "160", "192", "224", "256"):
        monkeypatch.setenv("DFGB_BN", bn)
        st = df.State(mech, net, precision=P, batch_cells=1100)
        assert all(t & ~df.DF_TILE_PAIR == int(bn) for t in st.tiles()[:-1]), st.tiles()
        O = host(st.mlp_forward(x))
        torch.cuda.synchronize()
        assert np.array_equal(O, O_ref), (bn, np.abs(O - O_ref).max())
        st.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16-table"])
def test_cta_pair_tiles_match_single_cta_tiles(df, prec, monkeypatch):
    """Hidden layers on CTA pairs (cta_group::2 MMAs on 256-row tiles, each CTA holding half
    of the tile's weight rows) give the same network outputs, bit for bit, as the same layers
    on single CTAs. Batches of 1408 and 592 rows: 11 and 5 row tiles, so the last pair of each
    batch has its second row tile past the rows. The cost model puts the 1600 -> 800 and
    800 -> 400 layers of this network on pairs."""
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=2000)
    P = df.DF_FP8_E4M3 if prec == "fp8" else df.DF_BF16
    gm = df.DF_GELU_TABLE if prec == "bf16-table" else df.DF_GELU_TANH
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32)
    st = df.State(mech, net, precision=P, batch_cells=1408, gelu_mode=gm)
    tiles = st.tiles()
    assert tiles[1] & df.DF_TILE_PAIR and tiles[2] & df.DF_TILE_PAIR, tiles
    O_pair = host(st.mlp_forward(dev(x)))
    monkeypatch.setenv("DFGB_BN", "224")
    st1 = df.State(mech, net, precision=P, batch_cells=1408, gelu_mode=gm)
    assert not any(t & df.DF_TILE_PAIR for t in st1.tiles())
    O_single = host(st1.mlp_forward(dev(x)))
    torch.cuda.synchronize()
    assert np.array_equal(O_pair, O_single), np.abs(O_pair - O_single).max()
    # and the pair path against the oracle with the same rounding points
    xr = x.astype(np.float64)
    Oq = (onw.mlp_forward_fp8(net, xr, 32.0) if prec == "fp8"
          else onw.mlp_forward_rounded(net, xr, onw.round_to_bf16))
    err = np.abs(O_pair - Oq)
    print(f"ERR cta_pair {prec}: max {err.max():.3e} mean {err.mean():.3e}")
    # measured: max 4.9e-3 (FP8), 3.8e-4 (BF16), 3.4e-4 (BF16, table)
    assert err.max() <= (5e-2 if prec == "fp8" else 4e-3), err.max()
    st.close()
    st1.close()


@pytest.mark.parametrize("N,batch", [(1, 256), (300, 512), (1300, 1408), (4097, 2048), (65613, 65536)])
def test_fused_layers_match_separate_layers(df, N, batch, monkeypatch):
    """Layers 0 and 1 of the 32-1600-800-400-30 network fused into one kernel (the layer-0
    activations produced on chip, block by block, and consumed there by layer 1's MMAs; enabled
    with DFGB_FUSE01=1) give the network outputs of the two layers run separately, bit for bit:
    the same K=16 MMAs in the same order, the same bias, GELU and BF16 rounding. Row counts
    cover a single row, a ragged row tile, several batches and a ragged last batch."""
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32)
    monkeypatch.setenv("DFGB_FUSE01", "1")
    st = df.State(mech, net, precision=df.DF_BF16, batch_cells=batch)
    st.profile_enable(True)
    O_fused = host(st.mlp_forward(dev(x)))
    fams = st.profile_read()
    assert "layer0+1" in fams and "layer0" not in fams, fams
    monkeypatch.setenv("DFGB_FUSE01", "0")
    st1 = df.State(mech, net, precision=df.DF_BF16, batch_cells=batch)
    st1.profile_enable(True)
    O_sep = host(st1.mlp_forward(dev(x)))
    assert "layer0" in st1.profile_read()
    torch.cuda.synchronize()
    assert np.array_equal(O_fused, O_sep), np.abs(O_fused - O_sep).max()
    st.close()
    st1.close()


def test_autotune_is_a_no_op_for_fp32(df):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=64)
    st = df.State(mech, net, precision=df.DF_FP32)
    assert st.autotune() == [0] * net.n_layers


# ---------------------------------------------------------------- tabulated GELU (Sec. 3.3.2)

@pytest.mark.parametrize("name,N", WORKLOADS[:2])
def test_tabulated_gelu_mlp_fp32_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32).astype(np.float64)
    st = df.State(mech, net, precision=df.DF_FP32, batch_cells=1024, gelu_mode=df.DF_GELU_TABLE)
    O = host(st.mlp_forward(dev(x.astype(np.float32))))
    torch.cuda.synchronize()
    Oo = onw.mlp_forward(net, x, act=onw.gelu_table)
    # as the tanh-form FP32 path; the table is evaluated in FP32 (an interval index may fall
    # on the neighbouring node, which moves the value by at most the expansion remainder)
    print(f"ERR table_fp32 {name}: max {np.abs(O - Oo).max():.3e}")
    np.testing.assert_allclose(O, Oo, atol=4e-6, rtol=0)   # measured max 3.8e-7
    # the tabulation is a different activation: against the tanh-form network the outputs move
    Ot = onw.mlp_forward(net, x)
    print(f"{name}: max |O_table - O_tanh| (FP64 oracle) = {np.abs(Oo - Ot).max():.3e}")


@pytest.mark.parametrize("name,N", WORKLOADS[:2])
def test_tabulated_gelu_mlp_bf16_vs_rounded_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    x = onw.normalise_inputs(net, T, p, Y).astype(np.float32).astype(np.float64)
    st = df.State(mech, net, precision=df.DF_BF16, batch_cells=512, gelu_mode=df.DF_GELU_TABLE)
    O = host(st.mlp_forward(dev(x.astype(np.float32))))
    torch.cuda.synchronize()
    Oq = onw.mlp_forward_rounded(net, x, onw.round_to_bf16, act=onw.gelu_table)
    err = np.abs(O - Oq)
    print(f"ERR table_bf16 {name}: max {err.max():.3e} mean {err.mean():.3e}")
    # measured: max 4.8e-4, mean 1.7e-5
    assert err.max() <= 5e-3 and err.mean() <= 2e-4, (err.max(), err.mean())


def test_tabulated_gelu_step_accuracy_and_unsupported_calls(df):
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=6000)
    res = {}
    for mode in (df.DF_GELU_TANH, df.DF_GELU_TABLE):
        st = df.State(mech, net, precision=df.DF_FP32, T_react=0.0, gelu_mode=mode)
        Td, Yd = dev(T), dev(Y)
        st.chem_step(Td, dev(p), Yd)
        torch.cuda.synchronize()
        res[mode] = (host(Td), host(Yd))
    To, Yo, _ = ostep.chem_step(mech, net, T, p, Y, net.dt, T_react=0.0)
    dtab = np.abs(res[df.DF_GELU_TABLE][1] - Yo).max()
    dtanh = np.abs(res[df.DF_GELU_TANH][1] - Yo).max()
    print(f"max |dY| vs the FP64 tanh-form oracle: tanh {dtanh:.3e}, table {dtab:.3e}")
    assert dtanh <= 1e-6 and dtab <= 1e-4
    st = df.State(mech, net, precision=df.DF_BF16, gelu_mode=df.DF_GELU_TABLE)
    with pytest.raises(df.DFError) as e:
        st.chem_jacobian(dev(T[:10]), dev(p[:10]), dev(Y[:, :10]))
    assert e.value.code == df._lib.DF_ERR_UNSUPPORTED
    with pytest.raises(df.DFError) as e:
        st.train_step(dev(T[:10]), dev(p[:10]), dev(Y[:, :10]), dev(Y[:, :10]))
    assert e.value.code == df._lib.DF_ERR_UNSUPPORTED


# ---------------------------------------------------------------- species-count extremes

def _extreme_case(n, N, seed):
    """n species (1: a hand-made pure fluid; otherwise a generated mechanism), a random
    network n+2 -> 48 -> 32 -> n, uniform states T in [300, 2500] K, p in [5, 20] MPa and
    mass fractions on the simplex."""
    from types import SimpleNamespace
    if n == 1:
        mech = SimpleNamespace(n=1, W=np.array([0.032]), Tc=np.array([154.6]), pc=np.array([5.04e6]),
                               omega=np.array([0.022]), kij=np.zeros((1, 1)),
                               nasa=np.array([[3.5, 5e-4, -1e-8, 0.0, 0.0, -1050.0, 4.0]]))
    else:
        mech = synth.mechanism.make_mechanism(n, 1 if n < 6 else 200, 41)
    net = synth.network.make_network([n + 2, 48, 32, n], n, seed)
    s = synth.Stream(seed, "extreme-states")
    T = s.uniform(N, 300.0, 2500.0)
    p = s.uniform(N, 5e6, 20e6)
    Y = s.uniform(n * N, 0.0, 1.0).reshape(n, N) + 1e-6
    return mech, net, T, p, Y / Y.sum(axis=0, keepdims=True)


@pytest.mark.parametrize("n", [1, 5, 32])
def test_species_count_extremes(df, n):
    mech, net, T, p, Y = _extreme_case(n, 3001, 40 + n)
    st = df.State(mech, net, precision=df.DF_FP32, T_react=0.0, batch_cells=1024)
    rho, h, cp, Z = (host(a) for a in st.real_fluid_props(dev(T), dev(p), dev(Y)))
    o = ope.state(mech, T, p, Y)
    np.testing.assert_allclose(Z, o["Z"], rtol=EOS_RTOL)
    assert np.all(np.abs(h - o["h"]) <= EOS_RTOL * (np.abs(o["h"]) + _h_scale(mech, T, p, Y)))
    np.testing.assert_allclose(rho, o["rho"], rtol=EOS_RTOL)
    _step_check(df, mech, net, T, p, Y, df.DF_FP32, 0.0, 1024, 1e-6)
    # measured (BF16): max |dY| up to 1.2e-6 (n = 5), whole-step max |dT| up to 4.7e-3 K
    _step_check(df, mech, net, T, p, Y, df.DF_BF16, 0.0, 1024, 1.5e-5, 5e-2)
