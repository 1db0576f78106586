"""The seeded input generators shared by the CUDA path's tests and the oracle's: the
splitmix64 stream against the test vector published with the generator, and the spin,
flip and proposal recipes against the properties they promise."""
import numpy as np

import synth


def test_splitmix64_published_vector():
    # first outputs of splitmix64 seeded with 1234567, as published with the generator
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    got = synth.SplitMix64(1234567).next_u64_array(5)
    assert [int(x) for x in got] == ref
    # the stream continues where it stopped
    g = synth.SplitMix64(1234567)
    assert [int(x) for x in np.concatenate([g.next_u64_array(2), g.next_u64_array(3)])] == ref


def test_uniform_and_normal_ranges():
    u = synth.SplitMix64(9).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    z = synth.SplitMix64(9).normal(100001)
    assert z.shape == (100001,) and abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_spin_recipes():
    s = synth.spins_uniform(64, 37, 3)
    assert s.dtype == np.int8 and s.shape == (64, 37) and set(np.unique(s)) == {-1, 1}
    assert np.array_equal(s, synth.spins_uniform(64, 37, 3))          # seeded
    assert not np.array_equal(s, synth.spins_uniform(64, 37, 4))
    z = synth.spins_zero_magnetisation(50, 256, 2003)
    assert z.dtype == np.int8 and np.all(z.sum(axis=1) == 0) and set(np.unique(z)) == {-1, 1}
    assert len({r.tobytes() for r in z}) == 50                           # distinct permutations


def test_flip_lists():
    sample, sites = synth.single_flips(3, 5)
    assert sample.tolist() == [0] * 5 + [1] * 5 + [2] * 5
    assert sites[:, 0].tolist() == list(range(5)) * 3 and np.all(sites[:, 1] == -1)
    for periodic in (False, True):
        smp, st = synth.random_flips(7, 20, 500, 11, pair_frac=0.5, max_sep=3, periodic=periodic)
        assert smp.min() >= 0 and smp.max() < 7
        assert st[:, 0].min() >= 0 and st[:, 0].max() < 20
        pair = st[:, 1] >= 0
        assert 0.3 < pair.mean() < 0.7 and st[pair, 1].max() < 20
        sep = np.abs(st[pair, 1] - st[pair, 0])
        if periodic:
            sep = np.minimum(sep, 20 - sep)
        assert sep.min() >= 1 and sep.max() <= 3


def test_typewriter_blocks():
    N, s = 37, 8                       # blocks 0..4, the last one 5 sites wide
    for parity in (0, 1):
        t = synth.typewriter_sites(200, N, s, parity, 5)
        blocks = [b for b in range(5) if b % 2 == parity]
        assert t.shape == (200, len(blocks))
        for j, b in enumerate(blocks):
            lo, hi = b * s, min(N, (b + 1) * s)
            assert t[:, j].min() >= lo and t[:, j].max() < hi
            assert len(np.unique(t[:, j])) == hi - lo                  # every site of the block drawn
    u = synth.uniforms(4, 6, 1)
    assert u.shape == (4, 6) and np.array_equal(u, synth.uniforms(4, 6, 1))
