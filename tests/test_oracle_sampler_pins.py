"""Pins of the oracle's screened typewriter sampler (Alg. 2) against exact Metropolis.

  * with a window covering every proposal (eps >= 1) every decision is taken from exact
    amplitudes and each is followed by a refresh: the batch must reproduce sequential
    exact Metropolis (same proposals, same uniforms) configuration for configuration;
  * the screened acceptance rule is exact whenever the window bounds the error of the
    scattering approximation (App. "Screened Metropolis sampler is exact"): when a run's
    largest |min(1, R~) - min(1, R)| over the proposals it decided approximately is at most
    eps, its decisions are the exact Metropolis decisions;
  * the typewriter proposals of one half-sweep are spaced by more than the block width.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import ModelDesc


def _setup(seed=3, N=24, C=4, s=4, parity=0, L=3):
    desc = ModelDesc(L=L, d=6, s=4, w=1, dh=6, dout=2, periodic=0)
    p = synth.init_params(desc, seed, a_scale=2.0)
    sl = synth.param_slices(desc)
    rng = synth.SplitMix64(seed + 7)
    for l in [f"l{i}" for i in range(1, L + 1)] + ["f"]:
        u = rng.uniform(desc.d)
        p[sl[f"{l}.log_dt"]] = np.log(0.05) + u * (np.log(0.5) - np.log(0.05))
    spins = synth.spins_uniform(C, N, seed + 11)
    sites = synth.typewriter_sites(C, N, s, parity, seed + 13)
    u = synth.uniforms(C, sites.shape[1], seed + 17)
    return desc, p, spins, sites, u


def test_typewriter_spacing():
    sites = synth.typewriter_sites(5, 37, 4, 1, 1)
    assert sites.shape[1] == len([b for b in range(10) if b % 2 == 1])
    d = np.diff(sites, axis=1)
    assert np.all(d > 4) and np.all(sites >= 0) and np.all(sites < 37)
    for j, b in enumerate([b for b in range(10) if b % 2 == 1]):
        assert np.all((sites[:, j] >= 4 * b) & (sites[:, j] < min(37, 4 * b + 4)))


@pytest.mark.parametrize("parity", [0, 1])
def test_full_window_equals_exact_metropolis(parity):
    desc, p, spins, sites, u = _setup(parity=parity)
    ref_s, ref_a = oracle.metropolis_exact(desc, p, spins, sites, u)
    s2, a2, refreshes, _ = oracle.sampler_batch(desc, p, spins, sites, u, eps=2.0)
    assert np.array_equal(s2, ref_s) and np.array_equal(a2, ref_a)
    assert refreshes == np.count_nonzero(sites >= 0)
    assert 0 < ref_a.sum() < ref_a.size      # both outcomes occur


def test_screened_rule_is_exact_when_window_bounds_error():
    desc, p, spins, sites, u = _setup(seed=5, C=6, s=3)
    ref_s, ref_a = oracle.metropolis_exact(desc, p, spins, sites, u)
    eps = 0.0
    for _ in range(6):
        s2, a2, refreshes, err = oracle.sampler_batch(desc, p, spins, sites, u, eps=eps)
        if err <= eps:
            break
        eps = err
    assert err <= eps
    assert np.array_equal(s2, ref_s) and np.array_equal(a2, ref_a)
    assert refreshes < np.count_nonzero(sites >= 0)   # not every decision needed the exact ratio
