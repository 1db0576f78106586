"""Screened typewriter sampler on the GPU (dn_sampler_batch through the C ABI) against the
oracle's Alg. 2 (pinned to exact Metropolis in the CPU tests): same proposals and uniforms,
FP64 - configurations, accept flags and the number of exact (refresh) decisions equal."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import ModelDesc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    return dysonnet


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _model(seed, L=3, d=8, periodic=0):
    desc = ModelDesc(L=L, d=d, s=4, w=1, dh=8, dout=2, periodic=periodic)
    p = synth.init_params(desc, seed, a_scale=2.0)
    sl = synth.param_slices(desc)
    rng = synth.SplitMix64(seed + 7)
    for l in [f"l{i}" for i in range(1, L + 1)] + ["f"]:
        u = rng.uniform(desc.d)
        p[sl[f"{l}.log_dt"]] = np.log(0.05) + u * (np.log(0.5) - np.log(0.05))
    return desc, p


@pytest.mark.parametrize("eps", [0.0, 0.02, 2.0])
@pytest.mark.parametrize("periodic", [0, 1])
def test_sampler_batch_matches_oracle_fp64(dn, eps, periodic):
    desc, p = _model(21 + periodic, periodic=periodic)
    C, N, s = 7, 26, 4
    spins = synth.spins_uniform(C, N, 5 + periodic)
    model = dn.Model(desc, p)
    sp = cuda(spins)
    for parity in (0, 1):
        sites = synth.typewriter_sites(C, N, s, parity, 40 + parity)
        u = synth.uniforms(C, sites.shape[1], 60 + parity)
        ref_s, ref_a, ref_r, _ = oracle.sampler_batch(desc, p, spins, sites, u, eps)
        acc, st = model.sampler_batch(sp, cuda(sites), cuda(u), eps, prec="fp64")
        got = sp.cpu().numpy()
        assert np.array_equal(acc.cpu().numpy(), ref_a), f"parity {parity}"
        assert np.array_equal(got, ref_s)
        assert st["refreshes"] == ref_r
        assert st["proposals"] == np.count_nonzero(sites >= 0)
        assert st["accepted"] == int(ref_a.sum())
        spins = ref_s
    model.close()


def test_sampler_fp32_and_empty_proposals(dn):
    desc, p = _model(33, L=4, d=16)
    C, N, s = 5, 40, 5
    spins = synth.spins_uniform(C, N, 8)
    sites = synth.typewriter_sites(C, N, s, 0, 9)
    sites[1, :] = -1                       # a chain without proposals
    sites[3, 1] = -1
    u = synth.uniforms(C, sites.shape[1], 10)
    eps = 0.05
    ref_s, ref_a, _, err = oracle.sampler_batch(desc, p, spins, sites, u, eps)
    model = dn.Model(desc, p)
    sp = cuda(spins)
    acc, st = model.sampler_batch(sp, cuda(sites), cuda(u), eps, prec="fp32")
    assert np.array_equal(sp.cpu()[1].numpy(), spins[1])
    assert st["proposals"] == np.count_nonzero(sites >= 0)
    assert np.array_equal(acc.cpu().numpy(), ref_a)
    assert np.array_equal(sp.cpu().numpy(), ref_s)
    model.close()


def test_sampler_rejects_bad_input(dn):
    desc, p = _model(3)
    model = dn.Model(desc, p)
    spins = synth.spins_uniform(2, 12, 1)
    spins[0, 4] = 3
    sites = synth.typewriter_sites(2, 12, 4, 0, 2)
    u = synth.uniforms(2, sites.shape[1], 3)
    with pytest.raises(dn.DysonNetError):
        model.sampler_batch(cuda(spins), cuda(sites), cuda(u), 0.0, prec="fp64")
    with pytest.raises(dn.DysonNetError):
        model.sampler_batch(cuda(synth.spins_uniform(2, 12, 1)), cuda(sites), cuda(u), -1.0, prec="fp64")
    model.close()
