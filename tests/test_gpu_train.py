"""Training through the C ABI against the FP64 oracle (oracle/train.py): loss, gradients of
every layer, input gradients (the torch.autograd.Function), Adam updates over several
steps, save/load, and that the reaction step, its CUDA graph and its Jacobian see the
trained weights. FP32 states are held to FP32 accumulation error; BF16 states, whose
activations and output gradients are stored in BF16, to a relative Frobenius error."""
import copy

import numpy as np
import pytest

import synth
from oracle import network as onw
from oracle import step as ostep
from oracle import train as otr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


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


def _targets(Y, seed):
    """Valid perturbed mass fractions (any target exercises the gradients)."""
    u = synth.Stream(seed, "train-target").uniform(Y.size, -0.05, 0.05).reshape(Y.shape)
    Yt = Y * (1.0 + u) + 1e-6
    return Yt / Yt.sum(axis=0, keepdims=True)


def _grads(df, st, net):
    out = []
    for l in range(net.n_layers):
        W, b = st.params(l, df._lib.DF_PARAM_GRADS, widths=net.widths)
        out.append((host(W).astype(np.float64), host(b).astype(np.float64)))
    return out


def _weights(df, st, net):
    out = []
    for l in range(net.n_layers):
        W, b = st.params(l, df._lib.DF_PARAM_WEIGHTS, widths=net.widths)
        out.append((host(W).astype(np.float64), host(b).astype(np.float64)))
    return out


def _net_with(net, params):
    n2 = copy.copy(net)
    n2.W = [w.astype(np.float32) for w, _ in params]
    n2.b = [b.astype(np.float32) for _, b in params]
    return n2


def _f64(net):
    n2 = copy.copy(net)
    n2.W = [np.asarray(w, dtype=np.float64) for w in net.W]
    n2.b = [np.asarray(b, dtype=np.float64) for b in net.b]
    return n2


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _moments(df, st, net, which):
    out = []
    for l in range(net.n_layers):
        W, b = st.params(l, which, widths=net.widths)
        out.append((host(W).astype(np.float64), host(b).astype(np.float64)))
    return out


@pytest.mark.parametrize("name,N", [("small-fp32-4k", 1000), ("layer1d-30sp-1m", 700),
                                    ("train30-1m", 333)])
def test_fp32_gradients_and_adam_match_oracle(df, name, N):
    """Three steps. Each step: the oracle's loss and gradients at the state's current master
    weights; then the oracle's Adam step from the state's own gradients and moments."""
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    Yt = _targets(Y, N)
    st = df.State(mech, net, precision=df.DF_FP32, T_react=0.0)
    lr = 1e-3
    x = onw.normalise_inputs(net, T, p, Y)
    Oh = otr.targets(net, Y, Yt)
    L = net.n_layers
    lib = df._lib
    args = (dev(T), dev(p), dev(Y), dev(Yt))
    for step in range(1, 4):
        w0 = _weights(df, st, net)
        m0 = _moments(df, st, net, lib.DF_PARAM_ADAM_M) if step > 1 else None
        v0 = _moments(df, st, net, lib.DF_PARAM_ADAM_V) if step > 1 else None
        loss = host(st.train_step(*args, lr=lr))[0]
        torch.cuda.synchronize()
        ref = _f64(net)
        ref.W, ref.b = [w for w, _ in w0], [b for _, b in w0]
        loss_o, dW, db = otr.loss_and_grads(ref, x, Oh)
        assert loss == pytest.approx(loss_o, rel=2e-5)
        g = _grads(df, st, net)
        for l in range(L):
            assert np.abs(g[l][0] - dW[l]).max() <= 2e-4 * np.abs(dW[l]).max(), (step, l)
            assert np.abs(g[l][1] - db[l]).max() <= 2e-4 * np.abs(db[l]).max(), (step, l)
        params = [w for w, _ in w0] + [b for _, b in w0]
        grads = [a for a, _ in g] + [b for _, b in g]
        if m0 is None:
            m = [np.zeros_like(a) for a in params]
            v = [np.zeros_like(a) for a in params]
        else:
            m = [a for a, _ in m0] + [b for _, b in m0]
            v = [a for a, _ in v0] + [b for _, b in v0]
        want, _, _ = otr.adam_step(params, grads, m, v, step, lr=lr)
        w1 = _weights(df, st, net)
        got = [a for a, _ in w1] + [b for _, b in w1]
        for a, b in zip(got, want):
            # FP32 Adam arithmetic: a few ulp of the update (~lr) and of the weight
            assert np.abs(a - b).max() <= 1e-5 * lr + 2e-7 * np.abs(b).max(), step
    assert st.train_steps_taken() == 3


@pytest.mark.parametrize("name,N", [("small-fp32-4k", 1000), ("layer1d-30sp-1m", 1500)])
def test_bf16_gradients_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    Yt = _targets(Y, N + 1)
    st = df.State(mech, net, precision=df.DF_BF16, T_react=0.0)
    loss = host(st.train_step(dev(T), dev(p), dev(Y), dev(Yt), lr=1e-4))[0]
    torch.cuda.synchronize()
    # oracle on the BF16 working weights (the storage precision of the forward pass)
    nq = _f64(net)
    nq.W = [onw.round_to_bf16(np.asarray(w, np.float64)) for w in net.W]
    x = onw.round_to_bf16(onw.normalise_inputs(net, T, p, Y))
    loss_o, dW, db = otr.loss_and_grads(nq, x, otr.targets(net, Y, Yt))
    assert loss == pytest.approx(loss_o, rel=2e-2)
    g = _grads(df, st, net)
    for l in range(net.n_layers):
        assert _rel(g[l][0], dW[l]) <= 3e-2, l
        assert _rel(g[l][1], db[l]) <= 3e-2, l


@pytest.mark.parametrize("prec,name,N", [("fp32", "small-fp32-4k", 777), ("bf16", "small-fp32-4k", 777),
                                         ("fp32", "layer1d-30sp-1m", 300), ("bf16", "layer1d-30sp-1m", 300)])
def test_autograd_function_gradients(df, prec, name, N):
    """MLPEOSFunction: O = net(x); L = sum(O * C) for a fixed C, so dL/dO = C; dL/dx against
    the oracle's reverse-mode Jacobian, dL/dW against the oracle's gradients."""
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    st = df.State(mech, net, precision=df.DF_FP32 if prec == "fp32" else df.DF_BF16)
    x = onw.normalise_inputs(net, T, p, Y)
    Cw = synth.Stream(N, "cotangent").uniform(N * mech.n, -1.0, 1.0).reshape(N, mech.n)
    xt = dev(x.astype(np.float32)).requires_grad_(True)
    O = df.MLPEOSFunction.apply(xt, st)
    (O * dev(Cw.astype(np.float32))).sum().backward()
    dX = host(xt.grad).astype(np.float64)
    ref = _f64(net)
    if prec == "bf16":
        ref.W = [onw.round_to_bf16(w) for w in ref.W]
        x = onw.round_to_bf16(x)
    J = onw.mlp_jacobian(ref, x)
    dX_o = np.einsum("bk,bkj->bj", Cw, J)
    # a target with O - Ohat = C B / 2 makes the oracle's dL/dz of the read-out equal C
    O_o = onw.mlp_forward(ref, x)
    _, dW, db = otr.loss_and_grads(ref, x, O_o - Cw * N / 2.0)
    g = _grads(df, st, net)
    if prec == "fp32":
        np.testing.assert_allclose(dX, dX_o, rtol=0, atol=2e-4 * np.abs(dX_o).max())
        for l in range(net.n_layers):
            assert np.abs(g[l][0] - dW[l]).max() <= 2e-4 * np.abs(dW[l]).max(), l
    else:
        assert _rel(dX, dX_o) <= 3e-2
        for l in range(net.n_layers):
            assert _rel(g[l][0], dW[l]) <= 3e-2, l


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_training_on_stiff_targets_reduces_loss(df, prec):
    """Targets from the BDF integration of the cell chemistry over the network's dt, outputs
    normalised by the targets' own mean and spread (as for a trained network); 120 full-batch
    Adam steps must cut the loss by 5x, decreasing from each block of 20 steps to the next."""
    from oracle import truth
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=512)
    T1, Y1, ok, _, _ = truth.advance(mech, T, p, Y, net.dt)
    T, p, Y, Y1 = T[ok], p[ok], Y[:, ok], Y1[:, ok]
    du = onw.boxcox(Y1, net.lam) - onw.boxcox(Y, net.lam)
    net = copy.copy(net)
    net.out_mean = du.mean(axis=1)
    net.out_std = du.std(axis=1) + 1e-12
    st = df.State(mech, net, precision=df.DF_FP32 if prec == "fp32" else df.DF_BF16)
    args = (dev(T), dev(p), dev(Y), dev(Y1))
    losses = []
    for _ in range(120):
        losses.append(float(host(st.train_step(*args, lr=1e-2))[0]))
    assert np.all(np.isfinite(losses))
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    assert last < 0.2 * first, (first, last)
    blocks = np.array(losses).reshape(6, 20).mean(axis=1)
    assert np.all(np.diff(blocks) < 0), blocks


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_trained_weights_reach_step_graph_and_jacobian(df, prec, tmp_path):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=600)
    P = df.DF_FP32 if prec == "fp32" else df.DF_BF16
    st = df.State(mech, net, precision=P, T_react=0.0)
    Yt = _targets(Y, 5)
    # graph and Jacobian context made before training
    Tg, Yg = dev(T), dev(Y)
    pd = dev(p)
    g = st.graph(Tg, pd, Yg)
    J0, _ = st.chem_jacobian(dev(T), pd, dev(Y))
    for _ in range(5):
        st.train_step(dev(T), pd, dev(Y), dev(Yt), lr=1e-2)
    torch.cuda.synchronize()
    trained = _weights(df, st, net)
    assert max(np.abs(trained[l][0] - net.W[l]).max() for l in range(net.n_layers)) > 1e-2
    # a fresh state built from the trained weights is the reference
    net2 = _net_with(net, trained)
    st2 = df.State(mech, net2, precision=P, T_react=0.0)
    g.launch()
    Td, Yd = dev(T), dev(Y)
    st2.chem_step(Td, pd, Yd)
    torch.cuda.synchronize()
    assert np.array_equal(host(Tg), host(Td)) and np.array_equal(host(Yg), host(Yd))
    J1, d1 = st.chem_jacobian(dev(T), pd, dev(Y))
    J2, d2 = st2.chem_jacobian(dev(T), pd, dev(Y))
    torch.cuda.synchronize()
    assert np.array_equal(host(J1), host(J2))
    assert not np.array_equal(host(J0), host(J1))
    # save / load: a third state loads the trained parameters and continues identically
    path = tmp_path / "params.bin"
    st.save(path)
    st3 = df.State(mech, net, precision=P, T_react=0.0)
    st3.load(path)
    assert st3.train_steps_taken() == 5
    w3 = _weights(df, st3, net)
    for l in range(net.n_layers):
        assert np.array_equal(w3[l][0], trained[l][0]) and np.array_equal(w3[l][1], trained[l][1])
    l1 = host(st.train_step(dev(T), pd, dev(Y), dev(Yt), lr=1e-2))
    l3 = host(st3.train_step(dev(T), pd, dev(Y), dev(Yt), lr=1e-2))
    assert l1[0] == l3[0]
    wa, wb = _weights(df, st, net), _weights(df, st3, net)
    for l in range(net.n_layers):
        assert np.array_equal(wa[l][0], wb[l][0])


def test_training_argument_errors(df):
    mech, net, T, p, Y = synth.configs.build("small-fp32-4k", n_cells=64)
    st = df.State(mech, net, precision=df.DF_FP32)
    with pytest.raises(df.DFError) as e:
        st.train_step(dev(T), dev(p), dev(Y), dev(Y), lr=-1.0)
    assert e.value.code == df._lib.DF_ERR_INVALID_ARG
    with pytest.raises(df.DFError) as e:
        st.mlp_backward(torch.zeros(64, mech.n, device=DEV))
    assert e.value.code == df._lib.DF_ERR_INVALID_ARG
    st.mlp_forward_train(torch.zeros(64, mech.n + 2, device=DEV))
    with pytest.raises(df.DFError):
        st.mlp_backward(torch.zeros(63, mech.n, device=DEV))
    # empty batch: no update, zero loss
    e0 = torch.empty(0, dtype=torch.float64, device=DEV)
    loss = st.train_step(e0, e0, torch.empty(mech.n, 0, dtype=torch.float64, device=DEV),
                         torch.empty(mech.n, 0, dtype=torch.float64, device=DEV))
    assert float(host(loss)[0]) == 0.0 and st.train_steps_taken() == 0
    st8 = df.State(mech, net, precision=df.DF_FP8_E4M3)
    with pytest.raises(df.DFError) as e:
        st8.train_step(dev(T), dev(p), dev(Y), dev(Y))
    assert e.value.code == df._lib.DF_ERR_UNSUPPORTED
    with pytest.raises(df.DFError):
        st.load("/nonexistent/params.bin")
