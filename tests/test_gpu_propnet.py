"""The property network (PRNet-style surrogate, include/df_propnet.h) through the C ABI against
the FP64 oracle (oracle/propnet.py): inference in FP32 and BF16, training steps (loss,
gradients, Adam) in FP32, BF16 training that learns, the paper's layer sizes on tcgen05, and
the separation of network-only and reaction-step states."""
import copy

import numpy as np
import pytest

import synth
from oracle import network as onw
from oracle import propnet as opn
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


def _case(n_species, N, widths, seed=5, transport=False):
    """Mechanism, states, exact properties (with transport: rho, T, ln mu, ln lambda,
    ln alpha), and a property network whose normalisation matches the states."""
    mech = synth.make_mechanism(n_species, 12 if n_species < 20 else 200, 1)
    T, p, Y = synth.fields.uniform_states(mech, N, seed=seed)
    h, props = (opn.exact_with_transport if transport else opn.exact)(mech, T, p, Y)
    bc = onw.boxcox(Y, 0.1)
    v = np.concatenate([h[None, :], p[None, :], bc], axis=0)
    net = synth.make_propnet(widths, n_species, seed=seed + 1, lam=0.1,
                             in_mean=v.mean(axis=1), in_std=v.std(axis=1) + 1e-3,
                             out_mean=props.mean(axis=1), out_std=props.std(axis=1))
    return mech, net, h, p, Y, props


def _f64(net):
    n2 = copy.copy(net)
    n2.W = [np.asarray(w, np.float64) for w in net.W]
    n2.b = [np.asarray(b, np.float64) for b in net.b]
    return n2


def test_infer_fp32_vs_oracle(df):
    mech, net, h, p, Y, props = _case(9, 3000, [11, 64, 32, 2])
    pn = df.PropNet(net, precision=df.DF_FP32, batch_cells=1024)   # several batches
    got = host(pn.infer(dev(h), dev(p), dev(Y)))
    torch.cuda.synchronize()
    want = opn.infer(net, h, p, Y)
    # FP32 inputs (Box-Cox by exp2/log2) and FP32 accumulation: ~1e-6 of a normalised output
    tol = 2e-5 * net.out_std[:, None]
    assert (np.abs(got - want) <= tol).all(), np.abs((got - want) / net.out_std[:, None]).max()
    pn.close()


def test_infer_bf16_vs_rounded_oracle(df):
    mech, net, h, p, Y, props = _case(30, 2000, [32, 256, 128, 2])
    pn = df.PropNet(net, precision=df.DF_BF16)
    got = host(pn.infer(dev(h), dev(p), dev(Y)))
    torch.cuda.synchronize()
    x = opn.inputs(net, h, p, Y).astype(np.float32).astype(np.float64)
    want = opn.outputs(net, onw.mlp_forward_rounded(net, x, onw.round_to_bf16))
    err = np.abs(got - want) / net.out_std[:, None]
    assert err.max() <= 2e-2 and err.mean() <= 1e-3, (err.max(), err.mean())
    pn.close()


def test_paper_sizes_on_tensor_cores(df):
    """Sec. 4.1's layer widths (hidden 1024-512-256 for density, 2048-1024-512 for temperature
    and transport) on 30 species: density alone, and T with the logarithms of viscosity, thermal
    conductivity and thermal diffusivity (4 outputs, as the paper's second network); BF16
    tcgen05 against the BF16-rounded oracle on a strided sample."""
    for widths in ([32, 1024, 512, 256, 1], [32, 2048, 1024, 512, 4]):
        mech, net, h, p, Y, props = _case(30, 5000, widths, seed=11, transport=True)
        rows = [0] if widths[-1] == 1 else [1, 2, 3, 4]
        net.out_mean, net.out_std = net.out_mean[rows], net.out_std[rows]
        pn = df.PropNet(net, precision=df.DF_BF16)
        got = host(pn.infer(dev(h), dev(p), dev(Y)))
        torch.cuda.synchronize()
        sel = np.arange(0, 5000, 37)
        x = opn.inputs(net, h[sel], p[sel], Y[:, sel]).astype(np.float32).astype(np.float64)
        want = opn.outputs(net, onw.mlp_forward_rounded(net, x, onw.round_to_bf16))
        err = np.abs(got[:, sel] - want) / net.out_std[:, None]
        assert err.max() <= 3e-2 and err.mean() <= 2e-3, (widths, err.max(), err.mean())
        pn.close()


def test_fp32_training_steps_match_oracle(df):
    """Three Adam steps: the loss and gradients at the current master weights, and the
    update, against the oracle."""
    mech, net, h, p, Y, props = _case(9, 700, [11, 48, 24, 2])
    pn = df.PropNet(net, precision=df.DF_FP32)
    lib = df._lib
    x = opn.inputs(net, h, p, Y).astype(np.float32).astype(np.float64)
    Oh = opn.targets(net, props)
    args = (dev(h), dev(p), dev(Y), dev(props))
    lr = 1e-3
    for step in range(1, 4):
        w0 = [tuple(host(t).astype(np.float64) for t in pn.params(l, lib.DF_PARAM_WEIGHTS,
                                                               widths=net.widths))
              for l in range(net.n_layers)]
        loss = host(pn.fit_step(*args, lr=lr))[0]
        torch.cuda.synchronize()
        ref = _f64(net)
        ref.W, ref.b = [w for w, _ in w0], [b for _, b in w0]
        loss_o, dW, db = otr.loss_and_grads(ref, x, Oh)
        assert loss == pytest.approx(loss_o, rel=2e-5)
        for l in range(net.n_layers):
            gW, gb = (host(t).astype(np.float64) for t in pn.params(l, lib.DF_PARAM_GRADS,
                                                                     widths=net.widths))
            assert np.abs(gW - dW[l]).max() <= 2e-4 * np.abs(dW[l]).max(), (step, l)
            assert np.abs(gb - db[l]).max() <= 2e-4 * np.abs(db[l]).max(), (step, l)
    assert pn.train_steps_taken() == 3
    pn.close()


def test_bf16_training_learns_the_eos(df):
    """300 BF16 Adam steps on 8192 states cut the loss by more than 10x and bring the density
    and temperature of held-out states within a few percent of the equation of state."""
    mech, net, h, p, Y, props = _case(9, 12000, [11, 128, 64, 2], seed=21)
    pn = df.PropNet(net, precision=df.DF_BF16)
    tr = slice(0, 8192)
    args = (dev(h[tr]), dev(p[tr]), dev(Y[:, tr].copy()), dev(props[:, tr].copy()))
    first = None
    for step in range(300):
        loss = pn.fit_step(*args, lr=2e-3)
        if step == 0:
            first = float(host(loss)[0])
    last = float(host(loss)[0])
    assert last < first / 10.0, (first, last)
    te = slice(8192, 12000)
    got = host(pn.infer(dev(h[te]), dev(p[te]), dev(Y[:, te].copy())))
    rel = np.abs(got - props[:, te]) / net.out_std[:, None]
    assert np.median(rel) < 0.1, np.median(rel)
    pn.close()


def test_state_kinds_are_separate(df):
    from paper_2508_18969_gb300 import DFError
    mech, net, h, p, Y, props = _case(9, 64, [11, 16, 2])
    pn = df.PropNet(net, precision=df.DF_FP32)
    with pytest.raises(DFError, match="UNSUPPORTED"):
        pn.chem_step(dev(props[1]), dev(p), dev(Y))
    with pytest.raises(DFError, match="UNSUPPORTED"):
        df.PropNet(net, precision=df.DF_FP8_E4M3)
    chem = df.State(mech, synth.make_network([11, 16, 9], 9, 1), precision=df.DF_FP32)
    with pytest.raises(DFError, match="UNSUPPORTED"):
        chem._check(chem._lib.df_propnet_infer(chem.h, 64, None, None, None, 64, None, 64, None))
    chem.close()
    # the generic network calls work on the network-only state
    x = opn.inputs(net, h, p, Y).astype(np.float32)
    O = host(pn.mlp_forward(dev(x)))
    torch.cuda.synchronize()
    assert np.abs(O - onw.mlp_forward(net, x.astype(np.float64))).max() <= 1e-5
    pn.close()
