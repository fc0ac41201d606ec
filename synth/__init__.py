"""Seeded synthetic inputs (mechanism, network parameters, cell states).

Holds none of the method's arithmetic: it draws numbers. Both the oracle side and the
CUDA side of the tests and the bench take their inputs from here.
"""
from .rng import Stream
from .mechanism import Mechanism, make_mechanism
from .network import Network, make_network, make_propnet
from . import fields, configs, mesh
