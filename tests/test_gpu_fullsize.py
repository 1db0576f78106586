"""Full-size parity: the N=128, 4 x 32 x 32 FP32 workload at the bench's size
(4096 configurations, all 128 single flips each, through the same calls the
bench times), with sampled outputs checked one by one against the FP64 oracle,
and properties that hold at any size checked on all outputs."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    return dysonnet


def test_bench_workload_sampled_against_oracle(dn):
    cfg = synth.CONFIGS["lrtfim_n128"]
    desc, params = cfg["desc"], synth.make_params(cfg)
    B, N = cfg["B"], cfg["N"]
    spins_np = synth.make_spins(cfg)
    spins = torch.from_numpy(spins_np).cuda()
    model = dn.Model(desc, params)
    eloc = model.local_energy(cfg["ham"], spins, prec="fp32").cpu().numpy()
    assert np.all(np.isfinite(eloc))
    rng = np.random.default_rng(5)
    # Local energies of 6 sampled configurations (each: 129 full forward passes in the oracle).
    bs = np.sort(rng.choice(B, 6, replace=False))
    ref = oracle.eloc(desc, params, cfg["ham"], spins_np[bs])
    e_eloc = np.max(np.abs(eloc[bs] - ref) / np.maximum(1.0, np.abs(ref)))
    print(f"N=128 sampled local energies rel err {e_eloc:.3e}")
    assert e_eloc <= 1e-4
    # All single-flip ratios of a 512-configuration slice, 96 sampled flips against the oracle.
    lo = int(rng.integers(0, B - 512))
    cache = model.forward_cache(spins[lo:lo + 512].contiguous(), prec="fp32")
    r = cache.single_flip_ratios().cpu().numpy()
    assert cache.check() == dn.DN_OK
    cache.destroy()
    assert np.all(np.isfinite(r))
    pick = rng.choice(512 * N, 96, replace=False)
    sample = (pick // N).astype(np.int32)
    sites = np.stack([pick % N, -np.ones_like(pick)], axis=1).astype(np.int32)
    ref = oracle.dlogpsi(desc, params, spins_np[lo:lo + 512], sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np[lo + np.unique(sample)][:1])
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp[0])))
    e_r = np.max(np.abs(r.reshape(-1)[pick] - ref) / den)
    print(f"N=128 sampled flip ratios rel err {e_r:.3e}")
    assert e_r <= 1e-4
    model.close()


def test_bench_workload_flip_list_matches_grouped(dn):
    """The general flip-list kernel and the all-single-flips kernel agree on 64
    configurations of the workload (same caches, different kernels)."""
    cfg = synth.CONFIGS["lrtfim_n128"]
    desc, params = cfg["desc"], synth.make_params(cfg)
    spins_np = synth.make_spins(cfg, B=64)
    model = dn.Model(desc, params)
    cache = model.forward_cache(torch.from_numpy(spins_np).cuda(), prec="fp32")
    grouped = cache.single_flip_ratios().cpu().numpy().reshape(-1)
    sample, sites = synth.single_flips(64, cfg["N"])
    listed = cache.flip_ratios(torch.from_numpy(sample).cuda(), torch.from_numpy(sites).cuda()).cpu().numpy()
    cache.destroy()
    model.close()
    # Both run in FP32 with different summation orders: compare at the FP32 bar, with
    # the error metric used against the oracle.
    den = np.maximum(np.abs(listed), 1e-3 * (1.0 + np.abs(oracle.logpsi(desc, params, spins_np)[0][sample])))
    assert np.max(np.abs(grouped - listed) / den) <= 1e-4


def _c3_model(N):
    cfg = synth.CONFIGS["j1j2_n256"]
    return cfg, cfg["desc"], synth.make_params(cfg)


def test_j1j2_workload_model_pair_flips(dn):
    """The N=256 J1-J2 ring model (6 x 64 x 64, periodic) on one zero-magnetisation
    configuration: 32 sampled antialigned NN/NNN pair flips against the oracle (FP32)."""
    cfg, desc, params = _c3_model(256)
    N = 256
    spins_np = synth.spins_zero_magnetisation(1, N, cfg["spins_seed"])
    s = spins_np[0]
    cand = [(i, (i + b) % N) for b in (1, 2) for i in range(N) if s[i] != s[(i + b) % N]]
    rng = np.random.default_rng(9)
    pick = [cand[k] for k in rng.choice(len(cand), 32, replace=False)]
    sample = np.zeros(len(pick), dtype=np.int32)
    sites = np.array(pick, dtype=np.int32)
    model = dn.Model(desc, params)
    cache = model.forward_cache(torch.from_numpy(spins_np).cuda(), prec="fp32", max_cluster=3)
    got = cache.flip_ratios(torch.from_numpy(sample).cuda(), torch.from_numpy(sites).cuda()).cpu().numpy()
    assert cache.check() == dn.DN_OK
    cache.destroy()
    model.close()
    ref = oracle.dlogpsi(desc, params, spins_np, sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np)
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp[0])))
    assert np.max(np.abs(got - ref) / den) <= 1e-4


def test_j1j2_local_energy_workload_architecture(dn):
    """Local energy of the J1-J2 chain with the 6 x 64 x 64 periodic model on a
    shorter ring (N = 48, 3 configurations) against the oracle, FP32."""
    cfg, desc, params = _c3_model(48)
    spins_np = synth.spins_zero_magnetisation(3, 48, 77)
    model = dn.Model(desc, params)
    got = model.local_energy(cfg["ham"], torch.from_numpy(spins_np).cuda(), prec="fp32").cpu().numpy()
    model.close()
    ref = oracle.eloc(desc, params, cfg["ham"], spins_np)
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-4


def test_n1024_cooperative_kernel_sampled_against_oracle(dn):
    """The bench's long-chain line: N = 1024, 6 x 64 x 64 FP32 model, 4 chains with all
    1024 single flips each through the grouped call (cooperative d = 64 layer kernel with
    swizzled link chunks); 6 sampled flips checked one by one against the oracle's full
    recompute (about 4 s of host time per flip), all outputs finite."""
    N = 1024
    desc = synth.ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    params = synth.init_params(desc, 1005, a_scale=10.0)
    spins_np = synth.spins_uniform(4, N, 2005)
    model = dn.Model(desc, params)
    cache = model.forward_cache(torch.from_numpy(spins_np).cuda(), prec="fp32")
    r = cache.single_flip_ratios().cpu().numpy().reshape(-1)
    assert cache.check() == dn.DN_OK
    cache.destroy()
    model.close()
    assert r.shape == (4 * N,) and np.all(np.isfinite(r))
    rng = np.random.default_rng(11)
    # sites near both ends and in the bulk of the chain
    pick = np.concatenate([rng.choice(4 * N, 3, replace=False), [0, 2 * N + 1, 4 * N - 2]])
    sample = (pick // N).astype(np.int32)
    sites = np.stack([pick % N, -np.ones_like(pick)], axis=1).astype(np.int32)
    ref = oracle.dlogpsi(desc, params, spins_np, sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np)
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp[sample])))
    err = np.max(np.abs(r[pick] - ref) / den)
    print(f"N=1024 coop sampled rel err {err:.3e}")
    assert err <= 1e-4
