"""Seeded synthetic C/H/O mechanism: species, real-fluid constants, thermo coefficients, reactions.

This module only DRAWS data. It evaluates none of the method's formulas (no equation of
state, no thermodynamic polynomial, no rate expression): every range below is chosen so
that the drawn numbers are valid by construction.

Draw recipe (the paper's 17-species LOX/CH4 mechanism of Sec. 4.1 is not available, so a
seeded stand-in of the same kind is drawn):
  * species: formulas C_x H_y O_z with x in 0..2, y in 0..4, z in 0..2 (not all zero);
    index 0 = O2, 1 = CH4, 2 = H2O, 3 = CO2, the others drawn without replacement;
  * molar masses from C 12.011, H 1.008, O 15.999 g/mol (stored in kg/mol);
  * Peng-Robinson constants: Tc ~ U[100, 800] K, pc ~ U[2, 10] MPa, omega ~ U[0, 0.4],
    binary interaction k_ij = k_ji ~ U[0, 0.1] rounded to binary32, k_ii = 0;
  * NASA-7 style coefficients on one range: a1 ~ U[3.5, 6], a2 ~ U[0, 2e-3],
    |a3| <= 4e-8, |a4| <= 4e-12, |a5| <= 4e-16, which bounds cp/R to [2.78, 13.7] on
    100..3500 K; a6 (enthalpy offset, in K) biased so that O2 and CH4 sit near their real
    values and H2O, CO2 are strongly negative (an exothermic CH4 + 2 O2 -> CO2 + 2 H2O);
    a7 ~ U[-5, 12];
  * reactions: all element-balanced reversible reactions A <=> B + C and A + B <=> C + D,
    shuffled by seed, first R kept, each written in a seeded direction; Arrhenius
    log10 A ~ U[6, 14] (cm3/mol)^(order-1)/s, beta ~ U[-1, 2], Ea ~ U[0, 250] kJ/mol.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import Stream

ATOMIC_MASS = np.array([12.011, 1.008, 15.999])  # g/mol of C, H, O
FIXED = [(0, 0, 2), (1, 4, 0), (0, 2, 1), (1, 0, 2)]  # O2, CH4, H2O, CO2


def formula_name(c: tuple[int, int, int]) -> str:
    out = ""
    for sym, k in zip("CHO", c):
        if k:
            out += sym + (str(k) if k > 1 else "")
    return out


@dataclass
class Mechanism:
    n: int
    names: list[str]
    elements: np.ndarray      # [n, 3] atoms of C, H, O
    W: np.ndarray             # [n] kg/mol
    Tc: np.ndarray            # [n] K
    pc: np.ndarray            # [n] Pa
    omega: np.ndarray         # [n]
    kij: np.ndarray           # [n, n] symmetric, zero diagonal, binary32-exact
    nasa: np.ndarray          # [n, 7] a1..a7
    nu_f: np.ndarray          # [n, R] reactant stoichiometric coefficients
    nu_r: np.ndarray          # [n, R] product stoichiometric coefficients
    A: np.ndarray             # [R] pre-exponential, CGS-molar units
    beta: np.ndarray          # [R]
    Ea: np.ndarray            # [R] J/mol
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_reactions(self) -> int:
        return self.nu_f.shape[1]


def _pool():
    return [(x, y, z) for x in range(3) for y in range(5) for z in range(3) if (x, y, z) != (0, 0, 0)]


def _balanced_reactions(comp: np.ndarray):
    """All unordered element-balanced reactions (one <=> two) and (two <=> two)."""
    n = comp.shape[0]
    pairs = {}
    for i in range(n):
        for j in range(i, n):
            key = tuple(comp[i] + comp[j])
            pairs.setdefault(key, []).append((i, j))
    out = []
    for a in range(n):  # A <=> B + C
        for (i, j) in pairs.get(tuple(comp[a]), []):
            out.append(((a,), (i, j)))
    for key in sorted(pairs):  # A + B <=> C + D
        group = pairs[key]
        for u in range(len(group)):
            for v in range(u + 1, len(group)):
                out.append((group[u], group[v]))
    return out


def make_mechanism(n_species: int, n_reactions: int, seed: int) -> Mechanism:
    if n_species < 4 or n_species > len(_pool()):
        raise ValueError("n_species must be in [4, 44]")
    pool = [c for c in _pool() if c not in FIXED]
    rs = Stream(seed, "species")
    for attempt in range(64):
        perm = rs.permutation(len(pool))
        comps = FIXED + [pool[i] for i in perm[: n_species - 4]]
        comp = np.array(comps, dtype=np.int64)
        cand = _balanced_reactions(comp)
        if len(cand) >= n_reactions:
            break
    else:
        raise RuntimeError("could not draw a species set with enough balanced reactions")
    n = n_species
    W = comp.astype(np.float64) @ ATOMIC_MASS * 1e-3

    s = Stream(seed, "real-fluid")
    Tc = s.uniform(n, 100.0, 800.0)
    pc = s.uniform(n, 2.0e6, 10.0e6)
    omega = s.uniform(n, 0.0, 0.4)
    kij = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    kv = s.uniform(len(iu[0]), 0.0, 0.1).astype(np.float32).astype(np.float64)
    kij[iu] = kv
    kij = kij + kij.T

    t = Stream(seed, "thermo")
    nasa = np.zeros((n, 7))
    nasa[:, 0] = t.uniform(n, 3.5, 6.0)
    nasa[:, 1] = t.uniform(n, 0.0, 2.0e-3)
    nasa[:, 2] = t.uniform(n, -4.0e-8, 4.0e-8)
    nasa[:, 3] = t.uniform(n, -4.0e-12, 4.0e-12)
    nasa[:, 4] = t.uniform(n, -4.0e-16, 4.0e-16)
    a6 = t.uniform(n, -20000.0, 30000.0)
    fixed_a6 = [(-1500.0, -500.0), (-11000.0, -9000.0), (-31000.0, -29000.0), (-49000.0, -47000.0)]
    u6 = t.uniform(4)
    for k, (lo, hi) in enumerate(fixed_a6):
        a6[k] = lo + (hi - lo) * u6[k]
    nasa[:, 5] = a6
    nasa[:, 6] = t.uniform(n, -5.0, 12.0)

    r = Stream(seed, "reactions")
    order = r.permutation(len(cand))[:n_reactions]
    flip = r.uniform(n_reactions) < 0.5
    nu_f = np.zeros((n, n_reactions))
    nu_r = np.zeros((n, n_reactions))
    for col, (ci, fl) in enumerate(zip(order, flip)):
        lhs, rhs = cand[ci]
        if fl:
            lhs, rhs = rhs, lhs
        for k in lhs:
            nu_f[k, col] += 1.0
        for k in rhs:
            nu_r[k, col] += 1.0
    A = 10.0 ** r.uniform(n_reactions, 6.0, 14.0)
    beta = r.uniform(n_reactions, -1.0, 2.0)
    Ea = r.uniform(n_reactions, 0.0, 250.0e3)

    return Mechanism(n=n, names=[formula_name(tuple(c)) for c in comps], elements=comp, W=W,
                     Tc=Tc, pc=pc, omega=omega, kij=kij, nasa=nasa, nu_f=nu_f, nu_r=nu_r,
                     A=A, beta=beta, Ea=Ea, seed=seed)
