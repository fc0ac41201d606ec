"""Seeded synthetic cell states (T, p, Y) standing in for the paper's flow fields.

The paper measures on a supercritical LOX/CH4 Taylor-Green-vortex flame (10 MPa, O2 at
150 K against CH4 at 300 K, Sec. 4.1) and on a rocket engine (above 3000 K, up to 20 MPa,
Sec. 4.1). Neither field is available, so states are drawn along a mixing-plus-burning line:

  * mixture fraction Zf: fuel stream = pure CH4 (species 1), oxidiser = pure O2 (species 0);
  * progress c in [0, 1] burns a fraction c of the limiting reactant along
    CH4 + 2 O2 -> CO2 + 2 H2O (mass is conserved because the molar masses balance);
  * minor species (index >= 4) get seeded log-uniform mass fractions, then all Y are
    divided by their sum.

Layout returned: T [N], p [N], Y [n, N] (species-major, one contiguous row per species).
"""
from __future__ import annotations

import numpy as np

from .mechanism import Mechanism
from .rng import Stream

Z_ST = 0.2  # burning-zone centre in mixture fraction (near the CH4/O2 mass stoichiometry)


def mixing_burning_Y(mech: Mechanism, Zf: np.ndarray, c: np.ndarray, stream: Stream,
                     minor_lo: float, minor_hi: float, minor_u: np.ndarray | None = None) -> np.ndarray:
    """minor_u (optional, [n - 4, N] in [0, 1)) replaces the stream's draws for the minor
    species."""
    N = Zf.shape[0]
    n = mech.n
    W = mech.W
    Y = np.zeros((n, N))
    y_ch4 = Zf.copy()
    y_o2 = 1.0 - Zf
    s = 2.0 * W[0] / W[1]                       # kg O2 per kg CH4
    m = c * np.minimum(y_ch4, y_o2 / s)          # kg CH4 burned per kg mixture
    Y[0] = y_o2 - s * m
    Y[1] = y_ch4 - m
    Y[2] = m * 2.0 * W[2] / W[1]
    Y[3] = m * W[3] / W[1]
    if n > 4:
        lo, hi = np.log10(minor_lo), np.log10(minor_hi)
        if minor_u is None:
            e = stream.uniform((n - 4) * N, lo, hi).reshape(n - 4, N)
        else:
            e = lo + (hi - lo) * minor_u
        Y[4:] = 10.0 ** e
    Y = np.maximum(Y, 0.0)
    return Y / Y.sum(axis=0, keepdims=True)


def uniform_states(mech: Mechanism, N: int, seed: int):
    """T ~ U[100, 3500] K, p ~ U[5, 20] MPa, Y along the mixing+burning line."""
    s = Stream(seed, "uniform-states")
    T = s.uniform(N, 100.0, 3500.0)
    p = s.uniform(N, 5.0e6, 20.0e6)
    Zf = s.uniform(N)
    c = s.uniform(N)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-2)
    return T, p, Y


def _layer_T(Zf: np.ndarray, c: np.ndarray) -> np.ndarray:
    T_mix = 100.0 * (1.0 - Zf) + 150.0 * Zf
    return T_mix + c * (3500.0 - T_mix)


def mixing_layer_1d(mech: Mechanism, N: int, seed: int, delta: float = 0.1, p: float = 10.0e6):
    """1D supercritical mixing layer on x in [-1, 1]: O2-rich at 100 K, CH4-rich at 150 K,
    Zf(x) = (1 + tanh(x / delta)) / 2, burning zone c = exp(-((Zf - 0.2) / 0.1)^2) lifting T
    towards 3500 K, p = 10 MPa, minor species jittered in [1e-8, 1e-3]."""
    s = Stream(seed, "mixing-layer-1d")
    x = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
    Zf = 0.5 * (1.0 + np.tanh(x / delta))
    c = np.exp(-(((Zf - Z_ST) / 0.1) ** 2))
    T = _layer_T(Zf, c)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    return T, np.full(N, p), Y


def _reacting_chunk(mech: Mechanism, N: int, seed: int, active_fraction: float, p: float,
                    j0: int, j1: int):
    """(T, p, Y) of cells j0..j1-1 of the reacting-mix field of N cells. Every draw is indexed
    by its position in the field's one stream (mask [0, N), reacting Zf [N, 2N), cold Zf
    [2N, 3N), minor species k at [3N + k N, 3N + (k + 1) N)), so any chunking gives the values
    of the serial draw."""
    s = Stream(seed, "reacting-mix")
    j = np.arange(j0, j1, dtype=np.uint64)
    N64 = np.uint64(N)
    act = s.uniform_at(j) < active_fraction
    Zf = np.where(act, s.uniform_at(N64 + j, 0.07, 0.33), s.uniform_at(2 * N64 + j))
    c = np.where(act, np.exp(-(((Zf - Z_ST) / 0.1) ** 2)), 0.0)
    T = _layer_T(Zf, c)
    nm = mech.n - 4
    mu = None
    if nm > 0:
        k = np.arange(nm, dtype=np.uint64)[:, None]
        mu = s.uniform_at(3 * N64 + k * N64 + j[None, :])
    return T, np.full(j1 - j0, p), mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3, minor_u=mu)


def reacting_mix(mech: Mechanism, N: int, seed: int, active_fraction: float = 0.3,
                 p: float = 10.0e6, chunk: int = 1 << 16, workers: int | None = None):
    """Cells of the 1D mixing layer's two populations, interleaved by a seeded Bernoulli mask:
    reacting cells (probability active_fraction) take Zf ~ U[0.07, 0.33], whose burning
    progress puts T above 727 K; the others are cold unburnt mixing (c = 0, T <= 150 K),
    minor species jittered in [1e-8, 1e-3]. Large fields are generated in chunks by a pool of
    processes as the 3D layer is; the values do not depend on the chunking."""
    return _generate(_reacting_chunk, (mech, N, seed, active_fraction, p), mech.n, N, chunk, workers)


def training_states(mech: Mechanism, N: int, seed: int):
    """Training states: positions x ~ U[-1, 1] across the 1D mixing layer's profile (so cold
    mixing, the burning zone and hot products all appear), p ~ U[5, 20] MPa, minor species
    jittered in [1e-8, 1e-3]."""
    s = Stream(seed, "training-states")
    x = s.uniform(N, -1.0, 1.0)
    Zf = 0.5 * (1.0 + np.tanh(x / 0.1))
    c = np.exp(-(((Zf - Z_ST) / 0.1) ** 2))
    T = _layer_T(Zf, c)
    p = s.uniform(N, 5.0e6, 20.0e6)
    Y = mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    return T, p, Y


def _layer3d_chunk(mech: Mechanism, N: int, seed: int, side: int, delta: float, j0: int, j1: int):
    """(T, p, Y) of cells j0..j1-1 of the 3D mixing layer of N cells."""
    from .noise import fractal3, permutation_table
    G = side ** 3
    s = Stream(seed, "mixing-layer-3d")
    j = np.arange(j0, j1, dtype=np.int64)
    g = (j * G) // N if N != G else j
    ix, iy, iz = g % side, (g // side) % side, g // (side * side)
    x = -1.0 + (ix + 0.5) * (2.0 / side)
    y = (iy + 0.5) / side
    z = (iz + 0.5) / side
    nz = fractal3(3.0 * (x + 1.0), 3.0 * y, 3.0 * z, permutation_table(seed), octaves=2)
    Zf = 0.5 * (1.0 + np.tanh((x + 0.15 * nz) / delta))
    c = np.exp(-(((Zf - Z_ST) / 0.1) ** 2))
    T = _layer_T(Zf, c)
    npv = fractal3(1.5 * (x + 1.0) + 17.0, 1.5 * y + 5.0, 1.5 * z + 11.0, permutation_table(seed + 1),
                   octaves=1)
    p = 12.5e6 + 7.5e6 * np.clip(2.5 * npv, -1.0, 1.0)
    nm = mech.n - 4
    mu = None
    if nm > 0:
        k = np.arange(nm, dtype=np.int64)[:, None]
        mu = s.uniform_at((k * G + g[None, :]).astype(np.uint64))
    return T, p, mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3, minor_u=mu)


_SHM = {}


def _worker_init(names, N, n):
    from multiprocessing import shared_memory
    for key, shape in (("T", (N,)), ("p", (N,)), ("Y", (n, N))):
        shm = shared_memory.SharedMemory(name=names[key])
        _SHM[key] = (shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf))


def _worker(args):
    fn, fargs, j0, j1 = args
    T, p, Y = fn(*fargs, j0, j1)
    _SHM["T"][1][j0:j1] = T
    _SHM["p"][1][j0:j1] = p
    _SHM["Y"][1][:, j0:j1] = Y
    return j1 - j0


def _generate(fn, fargs, n: int, N: int, chunk: int, workers: int | None):
    """(T, p, Y) of N cells from fn(*fargs, j0, j1), which returns the cells j0..j1-1; chunks of
    `chunk` cells, by a pool of processes writing into shared memory when the field is large
    (spawned, so it is safe after CUDA has been initialised)."""
    import os
    if workers is None:
        workers = min(len(os.sched_getaffinity(0)), 32) if N >= (1 << 23) else 1
    ranges = [(j0, min(N, j0 + chunk)) for j0 in range(0, N, chunk)]
    if workers <= 1 or len(ranges) <= 1:
        T, p, Y = np.empty(N), np.empty(N), np.empty((n, N))
        for j0, j1 in ranges:
            T[j0:j1], p[j0:j1], Y[:, j0:j1] = fn(*fargs, j0, j1)
        return T, p, Y
    import multiprocessing as mp
    from multiprocessing import shared_memory
    blocks = {k: shared_memory.SharedMemory(create=True, size=8 * sz)
              for k, sz in (("T", N), ("p", N), ("Y", n * N))}
    try:
        names = {k: b.name for k, b in blocks.items()}
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_worker_init, initargs=(names, N, n)) as pool:
            done = sum(pool.imap_unordered(_worker, [(fn, fargs, j0, j1) for j0, j1 in ranges]))
        assert done == N
        T = np.ndarray((N,), np.float64, blocks["T"].buf).copy()
        p = np.ndarray((N,), np.float64, blocks["p"].buf).copy()
        Y = np.ndarray((n, N), np.float64, blocks["Y"].buf).copy()
        return T, p, Y
    finally:
        for b in blocks.values():
            b.close()
            b.unlink()


def mixing_layer_3d(mech: Mechanism, N: int, seed: int, side: int = 400, delta: float = 0.1,
                    chunk: int = 1 << 16, workers: int | None = None):
    """3D supercritical mixing layer on a side^3 grid over [-1, 1] x [0, 1] x [0, 1], cells
    numbered x fastest. The 1D layer's mixture fraction Zf(x) = (1 + tanh(x / delta)) / 2 is
    displaced by improved gradient noise (two octaves, amplitude 0.15 in x), the burning zone
    and T follow the 1D layer, p = 12.5 MPa + 7.5 MPa * clip(2.5 n_p, -1, 1) with a second,
    single-octave noise field n_p (so p spans 5-20 MPa), minor species jittered in [1e-8, 1e-3].
    N < side^3 takes the evenly strided grid cells floor(j side^3 / N) with the draws those
    cells have in the full field (every draw is indexed by the global cell number); values
    agree up to the last-bit rounding of numpy's vectorised transcendental functions. Large
    fields are generated by a pool of processes."""
    return _generate(_layer3d_chunk, (mech, N, seed, side, delta), mech.n, N, chunk, workers)
