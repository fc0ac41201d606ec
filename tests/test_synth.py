"""Checks of the seeded input generators (synth/): the counter-based stream, the gradient
noise of the 3D field and the field recipes' invariants. CPU only."""
import numpy as np

import synth
from synth import fields, noise
from synth.rng import Stream


def test_stream_indexed_draws_equal_sequential_draws():
    a = Stream(3, "x").uniform(1000)
    s = Stream(3, "x")
    b = s.uniform_at(np.arange(1000))
    assert np.array_equal(a, b)
    s.uniform(10)
    assert np.array_equal(s.uniform(5), Stream(3, "x").uniform_at(np.arange(10, 15)))


def test_noise_zero_on_lattice_bounded_and_continuous():
    perm = noise.permutation_table(11)
    assert sorted(perm[:256].tolist()) == list(range(256))
    assert np.array_equal(perm[:256], perm[256:])
    g = np.arange(-3.0, 7.0)
    assert np.abs(noise.noise3(g, 2 * g, -g, perm)).max() == 0.0
    s = Stream(5, "pts")
    r = np.stack([s.uniform(50000, -40, 40) for _ in range(3)])
    v = noise.noise3(r[0], r[1], r[2], perm)
    assert np.abs(v).max() <= 1.05 and 0.15 < v.std() < 0.4 and abs(v.mean()) < 0.02
    h = 1e-7
    for ax in range(3):
        d = r.copy()
        d[ax] += h
        assert np.abs(noise.noise3(*d, perm) - v).max() < 10 * h
    # the lattice repeats every 256 units
    assert np.allclose(noise.noise3(r[0] + 256.0, r[1], r[2], perm), v, atol=1e-9)


def test_mixing_layer_3d_invariants_and_subsampling():
    mech = synth.mechanism.make_mechanism(30, 200, 20250820)
    side, Nfull = 40, 40 ** 3
    T, p, Y = fields.mixing_layer_3d(mech, Nfull, 9, side=side, chunk=9000)
    assert np.abs(Y.sum(axis=0) - 1.0).max() < 1e-13 and Y.min() >= 0.0
    assert 5e6 <= p.min() and p.max() <= 20e6 and p.max() - p.min() > 5e6
    assert 100.0 <= T.min() and T.max() <= 3500.0
    # cells numbered x fastest: the mixing layer runs along x
    Tg = T.reshape(side, side, side)
    assert Tg[:, :, : side // 4].mean() < 200.0
    # the noise displaces the layer across y and z
    assert np.std(Tg[:, :, side // 2 - 1]) > 0.0
    # a strided sample takes the full field's draws at those cells (numpy's vectorised powers
    # may round the last bit differently by array position)
    N = 1000
    Ts, ps, Ys = fields.mixing_layer_3d(mech, N, 9, side=side, chunk=333)
    g = (np.arange(N) * Nfull) // N
    assert np.array_equal(Ts, T[g]) and np.array_equal(ps, p[g])
    np.testing.assert_allclose(Ys, Y[:, g], rtol=1e-14, atol=0)


def test_mixing_layer_3d_parallel_equals_serial():
    mech = synth.mechanism.make_mechanism(9, 12, 20250819)
    a = fields.mixing_layer_3d(mech, 60000, 4, side=50, chunk=7000, workers=1)
    b = fields.mixing_layer_3d(mech, 60000, 4, side=50, chunk=7000, workers=3)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_reacting_mix_chunked_and_parallel_equal_the_sequential_draw():
    """The reacting-mix field drawn in chunks (serially or by a pool) takes the values of one
    sequential pass over its stream: mask, reacting Zf, cold Zf, then the minor species."""
    from synth.rng import Stream
    mech = synth.make_mechanism(30, 200, 20250820)
    N, seed = 50000, 7
    s = Stream(seed, "reacting-mix")
    act = s.uniform(N) < 0.3
    Zf = np.where(act, s.uniform(N, 0.07, 0.33), s.uniform(N))
    c = np.where(act, np.exp(-(((Zf - fields.Z_ST) / 0.1) ** 2)), 0.0)
    Y = fields.mixing_burning_Y(mech, Zf, c, s, 1e-8, 1e-3)
    a = fields.reacting_mix(mech, N, seed, chunk=7000, workers=1)
    b = fields.reacting_mix(mech, N, seed, chunk=6000, workers=3)
    assert np.array_equal(a[2], Y) and np.array_equal(b[2], Y)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], fields._layer_T(Zf, c))
    assert abs(np.mean(a[0] > 600.0) - 0.3) < 0.01
