"""Pins of the property-network oracle: inputs and outputs of hand-set cases whose Box-Cox
values are exact, the exact properties against the equation-of-state oracle they wrap, and
the regression gradients of a narrow-output network against finite differences."""
import copy

import numpy as np

import synth
from oracle import network as onw
from oracle import pr_eos
from oracle import propnet as opn
from oracle import train as otr


def _tiny(widths, lam=0.5):
    net = synth.make_propnet(widths, widths[0] - 2, seed=3, lam=lam)
    net.in_mean = np.array([1.0e5, 1.0e7] + [0.0] * (widths[0] - 2))
    net.in_std = np.array([2.0e5, 5.0e6] + [1.0] * (widths[0] - 2))
    return net


def test_inputs_by_hand():
    """lambda = 1/2: BC(1/4) = (1/2 - 1) / (1/2) = -1, BC(1) = 0, BC(0) = -2 exactly."""
    net = _tiny([5, 2])
    h = np.array([3.0e5, 1.0e5])
    p = np.array([2.0e7, 1.0e7])
    Y = np.array([[0.25, 1.0], [1.0, 0.0], [0.0, -0.1]])
    x = opn.inputs(net, h, p, Y)
    assert np.array_equal(x, np.array([[1.0, 2.0, -1.0, 0.0, -2.0],
                                       [0.0, 0.0, 0.0, -2.0, -2.0]]))


def test_outputs_of_a_linear_read_out_by_hand():
    """One linear layer that copies inputs 0 and 1 (h and p Z-scores) to outputs 0 and 1."""
    net = _tiny([4, 2])
    net.W = [np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 1.0, 0.0, 0.0]])]
    net.b = [np.array([0.5, -1.0])]
    net.out_mean = np.array([300.0, 1500.0])
    net.out_std = np.array([100.0, 1000.0])
    h = np.array([3.0e5])
    p = np.array([2.0e7])
    Y = np.array([[0.25], [1.0]])
    props = opn.infer(net, h, p, Y)
    # O = (1 + 0.5, 2 - 1) -> (300 + 100 * 1.5, 1500 + 1000 * 1)
    assert np.array_equal(props, np.array([[450.0], [2500.0]]))
    assert np.array_equal(opn.targets(net, props), np.array([[1.5, 1.0]]))


def test_exact_properties_wrap_the_eos():
    mech = synth.make_mechanism(9, 12, 1)
    T, p, Y = synth.fields.uniform_states(mech, 50, seed=4)
    h, props = opn.exact(mech, T, p, Y)
    s = pr_eos.state(mech, T, p, Y)
    assert np.array_equal(h, s["h"]) and np.array_equal(props[0], s["rho"])
    assert np.array_equal(props[1], T)


def test_exact_transport_properties_wrap_the_transport_oracle():
    from oracle import transport
    mech = synth.make_mechanism(9, 12, 1)
    T, p, Y = synth.fields.uniform_states(mech, 50, seed=4)
    h, props = opn.exact_with_transport(mech, T, p, Y)
    s = transport.state(mech, T, p, Y)
    assert np.array_equal(h, pr_eos.state(mech, T, p, Y)["h"])
    assert np.array_equal(props[0], s["rho"]) and np.array_equal(props[1], T)
    for r, k in ((2, "mu"), (3, "lam"), (4, "alpha")):
        assert np.array_equal(props[r], np.log(s[k]))


def test_regression_gradients_by_finite_differences():
    """loss_and_grads on a 6 -> 5 -> 2 network with two outputs, against central differences
    of the loss in every weight and bias."""
    net = synth.make_propnet([6, 5, 2], 4, seed=9, lam=0.1)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, 6))
    Oh = rng.normal(size=(7, 2))
    loss, dW, db = otr.loss_and_grads(net, x, Oh)
    eps = 1e-6
    for l in range(net.n_layers):
        for arr, g in ((net.W[l], dW[l]), (net.b[l], db[l])):
            for idx in np.ndindex(arr.shape):
                n2 = copy.deepcopy(net)
                tgt = n2.W[l] if arr is net.W[l] else n2.b[l]
                tgt[idx] += eps
                lp = otr.loss_and_grads(n2, x, Oh)[0]
                tgt[idx] -= 2 * eps
                lm = otr.loss_and_grads(n2, x, Oh)[0]
                assert abs((lp - lm) / (2 * eps) - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
    assert loss > 0
