"""Named workloads: mechanism size, network widths, cell count and field recipe.

  small-fp32-4k     9 species, 12 reactions, network 11-256-128-64-9, 4096 cells, uniform states
  layer1d-30sp-1m   30 species, 200 reactions, network 32-1600-800-400-30, 2**20 cells,
                    1D supercritical mixing layer (every cell goes through the network)
  react30-16m       same mechanism and network, 2**24 cells of which ~30 % react (T > 600 K)
  train30-1m        same mechanism and network, 2**20 training states across the mixing layer
                    with p ~ U[5, 20] MPa (targets come from the stiff integration)
  mix3d-30sp-64m    same mechanism and network, 400^3 cells of a 3D mixing layer displaced by
                    gradient noise, p 5-20 MPa, every cell through the network
Seeds are 20250818 + workload number; the 16M-cell workload reuses the 30-species
mechanism and network.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import fields
from .mechanism import make_mechanism
from .network import make_network


@dataclass(frozen=True)
class Workload:
    name: str
    n_species: int
    n_reactions: int
    widths: tuple
    n_cells: int
    field: str
    seed: int
    T_react: float        # cells with T above this react; 0 lets every cell through


WORKLOADS = {
    "small-fp32-4k": Workload("small-fp32-4k", 9, 12, (11, 256, 128, 64, 9), 4096, "uniform",
                              20250819, 0.0),
    "layer1d-30sp-1m": Workload("layer1d-30sp-1m", 30, 200, (32, 1600, 800, 400, 30), 1 << 20,
                                "layer1d", 20250820, 0.0),
    "react30-16m": Workload("react30-16m", 30, 200, (32, 1600, 800, 400, 30), 1 << 24,
                            "reacting", 20250820, 600.0),
    "train30-1m": Workload("train30-1m", 30, 200, (32, 1600, 800, 400, 30), 1 << 20,
                           "training", 20250820, 0.0),
    "mix3d-30sp-64m": Workload("mix3d-30sp-64m", 30, 200, (32, 1600, 800, 400, 30), 400 ** 3,
                               "mixing3d", 20250820, 0.0),
}


def build(name: str, n_cells: int | None = None, field_seed: int | None = None):
    """(mechanism, network, T, p, Y) of a workload; n_cells overrides the cell count."""
    w = WORKLOADS[name]
    mech = make_mechanism(w.n_species, w.n_reactions, w.seed)
    net = make_network(list(w.widths), w.n_species, w.seed)
    N = w.n_cells if n_cells is None else n_cells
    fs = w.seed if field_seed is None else field_seed
    if w.field == "uniform":
        T, p, Y = fields.uniform_states(mech, N, fs)
    elif w.field == "layer1d":
        T, p, Y = fields.mixing_layer_1d(mech, N, fs)
    elif w.field == "reacting":
        T, p, Y = fields.reacting_mix(mech, N, fs)
    elif w.field == "training":
        T, p, Y = fields.training_states(mech, N, fs + 4)
    elif w.field == "mixing3d":
        T, p, Y = fields.mixing_layer_3d(mech, N, fs + 5)
    else:
        raise KeyError(w.field)
    return mech, net, T, p, Y
