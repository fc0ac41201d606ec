"""The reverse-mode product of the reaction step (df_chem_step_vjp) and the differentiable step
built on it (ChemStepFunction), through the C ABI.

Against the oracle: the FP64 product from central differences of the oracle's step, with the
tolerance of the Jacobian parity test carried through the contraction (per entry,
sum_k |gY_k| (2e-6 + 1e-4 max|J|) + |gT| 1e-4 (|dT'/dv| + 1) for an FP32 network; BF16
tangents 5e-5 and 5e-2). Against the library's own Jacobian: the contraction written out in
FP64, to 1e-12 of the magnitudes summed. Non-reacting cells copy the cotangents bit for bit."""
import numpy as np
import pytest

import synth
from oracle import step as ostep

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
T_REACT = 600.0


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    assert torch.cuda.is_available()
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def host(t):
    return t.detach().cpu().numpy()


def _case(name, N, seed=11):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    rng = np.random.default_rng(seed)
    gT = rng.uniform(-1e-3, 1e-3, N)
    gY = rng.uniform(-1.0, 1.0, Y.shape)
    return mech, net, T, p, Y, gT, gY


@pytest.mark.parametrize("name,N,batch,prec", [("small-fp32-4k", 300, 128, "fp32"),
                                               ("react30-16m", 200, 64, "fp32"),
                                               ("small-fp32-4k", 300, 128, "bf16")])
def test_step_vjp_vs_oracle(df, name, N, batch, prec):
    """Reacting and non-reacting cells, several batches and a ragged last one."""
    mech, net, T, p, Y, gT, gY = _case(name, N)
    react = T > T_REACT
    assert react.any() and (~react).any()
    pr = {"fp32": df.DF_FP32, "bf16": df.DF_BF16}[prec]
    st = df.State(mech, net, precision=pr, T_react=T_REACT, batch_cells=batch)
    oT, oY = st.chem_step_vjp(dev(T), dev(p), dev(Y), dev(gT), dev(gY))
    torch.cuda.synchronize()
    oT, oY = host(oT), host(oY)
    kw = dict(dY_rel=1e-4, dY_min=1e-4)
    rT, rY = ostep.chem_step_vjp(mech, net, T, p, Y, gT, gY, T_react=T_REACT, **kw)
    Jf, dTf = ostep.chem_step_jacobian_fd(mech, net, T, p, Y, **kw)
    # non-reacting cells: the cotangents themselves, exactly
    np.testing.assert_array_equal(oT[~react], gT[~react])
    np.testing.assert_array_equal(oY[:, ~react], gY[:, ~react])
    assert np.all(np.isfinite(oT)) and np.all(np.isfinite(oY)), "flagged cells"
    atolJ, rJ, rT_ = (2e-6, 1e-4, 1e-4) if prec == "fp32" else (5e-5, 1e-4, 5e-2)
    Jmax = np.nanmax(np.abs(Jf))
    sg = np.abs(gY).sum(axis=0)                                   # [N]
    tol = sg[:, None] * (atolJ + rJ * Jmax) + np.abs(gT)[:, None] * rT_ * (np.abs(dTf) + 1.0)
    got = np.concatenate([oT[:, None], oY.T], axis=1)
    ref = np.concatenate([rT[:, None], rY.T], axis=1)
    m = react[:, None] & np.isfinite(ref)
    err = np.abs(got - ref)
    print(f"vjp {name} {prec}: max err {err[m].max():.3e}, max err / tol {(err / tol)[m].max():.3f}")
    # species below the difference floor (1e-4) have no oracle column; T always has one
    assert np.all(m[react, 0]) and m.sum() > 0.25 * react.sum() * (mech.n + 1)
    assert np.all(err[m] <= tol[m])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_step_vjp_is_the_contraction_of_the_jacobian(df, prec):
    """The product equals sum_k gY_k (J[k][t] + [t = k + 1]) + gT dT'/dv_t over the library's
    own Jacobian, and repeats bit for bit."""
    mech, net, T, p, Y, gT, gY = _case("react30-16m", 1000, seed=5)
    pr = {"fp32": df.DF_FP32, "bf16": df.DF_BF16}[prec]
    st = df.State(mech, net, precision=pr, T_react=T_REACT, batch_cells=256)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    J, dTn = st.chem_jacobian(Td, pd, Yd)
    o1 = st.chem_step_vjp(Td, pd, Yd, dev(gT), dev(gY))
    o2 = st.chem_step_vjp(Td, pd, Yd, dev(gT), dev(gY))
    torch.cuda.synchronize()
    J, dTn = host(J).astype(np.float64), host(dTn)
    n = mech.n
    eye = np.hstack([np.zeros((n, 1)), np.eye(n)])
    ref = gT[:, None] * dTn + np.einsum("kc,ckt->ct", gY, J + eye[None])
    mag = np.abs(gT)[:, None] * np.abs(dTn) + np.einsum("kc,ckt->ct", np.abs(gY), np.abs(J + eye[None]))
    got = np.concatenate([host(o1[0])[:, None], host(o1[1]).T], axis=1)
    react = T > T_REACT
    fin = np.all(np.isfinite(J.reshape(len(T), -1)), axis=1) & react
    assert fin.sum() > 0.9 * react.sum()
    assert np.all(np.abs(got - ref)[fin] <= 1e-12 * mag[fin] + 1e-300)
    assert np.all(np.isnan(got[react & ~fin]))
    assert np.array_equal(host(o1[0]), host(o2[0])) and np.array_equal(host(o1[1]), host(o2[1]))


def test_chem_step_function_forward_and_backward(df):
    """ChemStepFunction: forward is df_chem_step on copies, backward is df_chem_step_vjp."""
    mech, net, T, p, Y, gT, gY = _case("small-fp32-4k", 500, seed=3)
    st = df.State(mech, net, precision=df.DF_BF16, T_react=T_REACT, batch_cells=256)
    Td = dev(T).requires_grad_(True)
    Yd = dev(Y).requires_grad_(True)
    pd = dev(p)
    T1, Y1 = df.ChemStepFunction.apply(Td, Yd, pd, st)
    Tr, Yr = dev(T), dev(Y)
    st.chem_step(Tr, pd, Yr)
    assert torch.equal(T1, Tr) and torch.equal(Y1, Yr)
    assert torch.equal(Td.detach(), dev(T)), "the inputs are not modified"
    wT, wY = dev(gT), dev(gY)
    loss = (wT * T1).sum() + (wY * Y1).sum()
    gTd, gYd = torch.autograd.grad(loss, (Td, Yd))
    vT, vY = st.chem_step_vjp(dev(T), pd, dev(Y), wT, wY)
    assert torch.equal(gTd, vT) and torch.equal(gYd, vY)
    # a loss of Y' alone: T' gets no cotangent
    T1, Y1 = df.ChemStepFunction.apply(Td, Yd, pd, st)
    (gY_only,) = torch.autograd.grad((wY * Y1).sum(), (Yd,))
    _, vY0 = st.chem_step_vjp(dev(T), pd, dev(Y), torch.zeros_like(wT), wY)
    assert torch.equal(gY_only, vY0)


def test_step_vjp_empty_and_argument_errors(df):
    from paper_2508_18969_gb300 import _lib
    mech, net, T, p, Y, gT, gY = _case("small-fp32-4k", 64)
    st = df.State(mech, net, T_react=T_REACT, batch_cells=64)
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    oT, oY = st.chem_step_vjp(e, e, torch.empty(mech.n, 0, dtype=torch.float64, device=DEV), e,
                              torch.empty(mech.n, 0, dtype=torch.float64, device=DEV))
    assert oT.numel() == 0 and oY.numel() == 0
    lib = st._lib
    N = len(T)
    Td, pd, Yd = dev(T), dev(p), dev(Y)
    rc = lib.df_chem_step_vjp(st.h, N, Td.data_ptr(), pd.data_ptr(), Yd.data_ptr(), N, None, None,
                              N, None, None, N, None)
    assert rc == _lib.DF_ERR_INVALID_ARG
    g = dev(gY)
    rc = lib.df_chem_step_vjp(st.h, N, Td.data_ptr(), pd.data_ptr(), Yd.data_ptr(), N,
                              Td.data_ptr(), g.data_ptr(), N - 1, Td.data_ptr(), g.data_ptr(), N,
                              None)
    assert rc == _lib.DF_ERR_INVALID_ARG
