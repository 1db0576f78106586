"""Theorem 1 on the CPU: the ABACUS recurrence with the library's readings of
Alg. 1 (embedding source term, pre-gate slice activations, no double-counted
P_M term) reproduces the oracle's full recompute to rounding."""
import numpy as np
import pytest

import oracle
import synth
from synth import ModelDesc
from tests import abacus_ref


@pytest.mark.parametrize("L,periodic,w,N", [(1, 0, 1, 7), (2, 0, 2, 9), (3, 1, 1, 8), (4, 0, 1, 9), (4, 1, 2, 11)])
def test_abacus_recurrence_equals_full_recompute(L, periodic, w, N):
    desc = ModelDesc(L=L, d=3, s=3, w=w, dh=4, dout=2, periodic=periodic)
    p = synth.init_params(desc, 500 + L + 10 * periodic, a_scale=6.0)
    spins = synth.spins_uniform(2, N, 3 + L)
    sample, sites = synth.random_flips(2, N, 16, seed=L, pair_frac=0.5, max_sep=2, periodic=bool(periodic))
    # Always include the chain ends.
    sample = np.concatenate([sample, [0, 1, 0]]).astype(np.int32)
    sites = np.concatenate([sites, [[0, -1], [N - 1, -1], [N - 2, N - 1]]]).astype(np.int32)
    ref = oracle.dlogpsi(desc, p, spins, sample, sites)
    model = abacus_ref.Model(desc, p, N)
    caches = [abacus_ref.build_caches(model, spins[b]) for b in range(2)]
    lp, om = oracle.logpsi(desc, p, spins)
    for b in range(2):
        np.testing.assert_allclose(caches[b]["Omega"], om[b], rtol=1e-12, atol=1e-13)
    got = np.array([abacus_ref.flip_ratio(model, spins[sample[f]], caches[sample[f]], sites[f])
                    for f in range(len(sample))])
    assert np.abs(ref).max() > 1e-5
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)
