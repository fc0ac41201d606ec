"""FP64 property network (PRNet-style surrogate of the real-fluid state) -- TEST
INFRASTRUCTURE ONLY (part of the oracle; never imported by the product path).

  * Sec. 2: for supercritical flames a second network, PRNet, reads the flow state -- energy
    E, pressure p and composition Y -- and yields the real-fluid properties (density rho,
    temperature T, viscosity, thermal diffusivity) that the Peng-Robinson EoS fixes. Sec. 4.1
    gives its sizes: (3, 1024, 512, 256, 1) for rho, (3, 2048, 1024, 512, 4) for T and the
    transport properties.
  * Reading here: the energy input is the conserved mass-specific enthalpy h of the reaction
    step (the quantity this project's step conserves, Newton on h(T)); composition enters
    through the Box-Cox coordinates of all n species (the chemistry network's inputs), so a
    network reads n + 2 inputs, Z-scored (Sec. 3.3.1); outputs are de-normalised properties:
    rho for the density network; T and the logarithms of viscosity, thermal conductivity and
    thermal diffusivity for the 4-output temperature-and-transport network (the transport
    properties span decades, so the network regresses their logarithms).
  * The exact properties a surrogate is trained on and compared with are the oracle's own
    Peng-Robinson state (pr_eos.state): h, rho and T of a cell state (T, p, Y); and the
    transport oracle (transport.state: Chung et al. 1988 at the Peng-Robinson density).

Training uses oracle.train.loss_and_grads (the mean squared error of the normalised outputs,
reverse mode written out) and oracle.train.adam_step.
"""
from __future__ import annotations

import numpy as np

from . import network as nw
from . import pr_eos
from . import transport


def inputs(net, h, p, Y):
    """Network input rows x [N, n+2]: (h, p, BC(Y_1..Y_n)) Z-scored."""
    v = np.concatenate([np.asarray(h, np.float64)[None, :], np.asarray(p, np.float64)[None, :],
                        nw.boxcox(Y, net.lam)], axis=0)
    return ((v - net.in_mean[:, None]) / net.in_std[:, None]).T


def outputs(net, O):
    """Properties [m, N] from network outputs O [N, m]: mean + spread * O."""
    return (np.asarray(O, np.float64) * net.out_std[None, :] + net.out_mean[None, :]).T


def infer(net, h, p, Y, act=None):
    """The surrogate's properties [m, N] of cells (h, p, Y)."""
    return outputs(net, nw.mlp_forward(net, inputs(net, h, p, Y), act=act))


def exact(mech, T, p, Y):
    """(h [N], properties [2, N] = (rho, T)) of cell states from the Peng-Robinson oracle."""
    s = pr_eos.state(mech, T, p, Y)
    return s["h"], np.stack([s["rho"], np.asarray(T, np.float64)])


def exact_with_transport(mech, T, p, Y):
    """(h [N], properties [5, N] = (rho, T, ln mu, ln lambda, ln alpha)) of cell states from the
    Peng-Robinson and transport oracles (mu Pa s, lambda W/(m K), alpha m^2/s)."""
    s = transport.state(mech, T, p, Y)
    h = pr_eos.state(mech, T, p, Y)["h"]
    return h, np.stack([s["rho"], np.asarray(T, np.float64), np.log(s["mu"]), np.log(s["lam"]),
                        np.log(s["alpha"])])


def targets(net, props):
    """Normalised regression targets [N, m] of properties [m, N]."""
    return ((np.asarray(props, np.float64) - net.out_mean[:, None]) / net.out_std[:, None]).T
