"""BF16 precision (tensor-core forward) against the FP64 oracle, and FP32 at the same
tensor-core shapes (d a multiple of 16: link hops on tcgen05).

FP32 keeps the FP32 bars of the other parity tests (1e-4 on log psi and on log-amplitude
ratios).  BF16 carries every operand of the forward pass's S4 convolutions and channel
mixing as two BF16 terms (hi + lo, 8 mantissa bits each; products hi*hi + hi*lo + lo*hi
with FP32 accumulation, about 2^-17 relative per product); the link tensors, the adjoint
and the ABACUS contractions stay at FP32 accuracy.  (With one BF16 term per operand,
2^-9 per product, the same J1-J2 test measured 0.11 on ratios and 6.9e-4 on log psi.)
The bounds below are the library's stated BF16 bounds, above the largest errors
measured on these workloads on a GB300 (printed by the tests).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import ModelDesc

pytestmark = pytest.mark.gpu

BF16_TOL_LOGPSI = 2e-5     # |log psi - ref| / max(1, |ref|); measured <= 4.8e-6
BF16_TOL_RATIO = 1e-3      # rel on log-amplitude ratios (denominator as in the FP32 tests); measured <= 3.7e-4


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    return dysonnet


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(got, ref, lp_ref):
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp_ref)))
    return np.abs(got - ref) / den


def errors(dn, desc, params, spins, sample, sites, prec, mc=1):
    model = dn.Model(desc, params)
    lp = torch.empty(spins.shape[0], dtype=torch.float64, device="cuda")
    cache = model.forward_cache(cuda(spins), prec=prec, max_cluster=mc, logpsi=lp)
    got = cache.flip_ratios(cuda(sample), cuda(sites)).cpu().numpy()
    assert cache.check() == dn.DN_OK
    cache.destroy()
    model.close()
    lp_ref, _ = oracle.logpsi(desc, params, spins)
    ref = oracle.dlogpsi(desc, params, spins, sample, sites)
    e_lp = np.abs(lp.cpu().numpy() - lp_ref) / np.maximum(1.0, np.abs(lp_ref))
    return e_lp.max(), rel_err(got, ref, lp_ref[sample]).max()


TC_CASES = [
    # L, d, s, w, dh, dout, periodic, N, B, max_cluster
    (3, 16, 8, 1, 16, 2, 0, 40, 3, 1),
    (4, 32, 8, 2, 32, 2, 1, 61, 3, 2),
    (3, 64, 8, 2, 32, 2, 0, 130, 2, 1),    # two site tiles, ragged
]


@pytest.mark.parametrize("case", TC_CASES)
def test_fp32_at_tensor_core_shapes(dn, case):
    L, d, s, w, dh, dout, periodic, N, B, mc = case
    desc = ModelDesc(L=L, d=d, s=s, w=w, dh=dh, dout=dout, periodic=periodic)
    params = synth.init_params(desc, 700 + d + L, a_scale=8.0)
    spins = synth.spins_uniform(B, N, 77 + N)
    sample, sites = synth.random_flips(B, N, 48, seed=d, pair_frac=0.5 if mc > 1 else 0.0,
                                       max_sep=max(1, mc - 1), periodic=bool(periodic))
    e_lp, e = errors(dn, desc, params, spins, sample, sites, "fp32", mc)
    assert e_lp <= 1e-4, f"log psi {e_lp:.3e}"
    assert e <= 1e-4, f"ratios {e:.3e}"


@pytest.mark.parametrize("case", TC_CASES[:2])
def test_bf16_forward_and_ratios(dn, case):
    L, d, s, w, dh, dout, periodic, N, B, mc = case
    desc = ModelDesc(L=L, d=d, s=s, w=w, dh=dh, dout=dout, periodic=periodic)
    params = synth.init_params(desc, 700 + d + L, a_scale=8.0)
    spins = synth.spins_uniform(B, N, 77 + N)
    sample, sites = synth.random_flips(B, N, 48, seed=d, pair_frac=0.5 if mc > 1 else 0.0,
                                       max_sep=max(1, mc - 1), periodic=bool(periodic))
    e_lp, e = errors(dn, desc, params, spins, sample, sites, "bf16", mc)
    print(f"bf16 d={d}: log psi {e_lp:.3e}, ratios {e:.3e}")
    assert e_lp <= BF16_TOL_LOGPSI, f"log psi {e_lp:.3e}"
    assert e <= BF16_TOL_RATIO, f"ratios {e:.3e}"


def test_bf16_workload_model_local_energy(dn):
    """BF16 local energy of the N=128, 4 x 32 workload model on 6 configurations."""
    cfg = synth.CONFIGS["lrtfim_n128"]
    desc, N = cfg["desc"], cfg["N"]
    params = synth.make_params(cfg)
    spins = synth.make_spins(cfg, 6)
    model = dn.Model(desc, params)
    e32 = model.local_energy(cfg["ham"], cuda(spins), prec="fp32").cpu().numpy()
    e16 = model.local_energy(cfg["ham"], cuda(spins), prec="bf16").cpu().numpy()
    model.close()
    ref = oracle.eloc(desc, params, cfg["ham"], spins)
    scale = np.maximum(1.0, np.abs(ref))
    err32 = np.max(np.abs(e32 - ref) / scale)
    err16 = np.max(np.abs(e16 - ref) / scale)
    print(f"local energy rel err: fp32 {err32:.3e}, bf16 {err16:.3e}")
    assert err32 <= 1e-4
    assert err16 <= BF16_TOL_RATIO


def test_bf16_recompute_baseline(dn):
    desc = ModelDesc(L=3, d=32, s=8, w=2, dh=32, dout=2, periodic=0)
    params = synth.init_params(desc, 91, a_scale=6.0)
    spins = synth.spins_uniform(3, 33, 5)
    sample, sites = synth.random_flips(3, 33, 30, seed=4, pair_frac=0.3)
    model = dn.Model(desc, params)
    lp_ref, _ = oracle.logpsi(desc, params, spins)
    lp = model.full_forward(cuda(spins), prec="bf16").cpu().numpy()
    assert np.max(np.abs(lp - lp_ref) / np.maximum(1, np.abs(lp_ref))) <= BF16_TOL_LOGPSI
    got = model.recompute_flip_ratios(cuda(spins), cuda(sample), cuda(sites), prec="fp32").cpu().numpy()
    ref = oracle.dlogpsi(desc, params, spins, sample, sites)
    assert rel_err(got, ref, lp_ref[sample]).max() <= 1e-4
    model.close()


def test_bf16_needs_tensor_core_shapes(dn):
    desc = ModelDesc(L=2, d=12, s=4, w=1, dh=8, dout=2, periodic=0)
    params = synth.init_params(desc, 5, a_scale=2.0)
    spins = synth.spins_uniform(2, 10, 1)
    model = dn.Model(desc, params)
    with pytest.raises(Exception) as ei:
        model.forward_cache(cuda(spins), prec="bf16")
    assert "UNSUPPORTED" in str(ei.value).upper() or str(dn.DN_EUNSUPPORTED) in str(ei.value)
    model.close()


def test_bf16_j1j2_workload_model_pair_flips(dn):
    """The model the BF16 precision is specified for: the N = 256 J1-J2 ring, 6 x 64 x 64,
    zero-magnetisation configurations, connected configurations from antialigned NN and
    NNN pairs.  A stratified subset against the FP64 oracle: 2 configurations, 16 NN and
    16 NNN pairs each (the oracle recomputes the whole network per pair)."""
    cfg = synth.CONFIGS["j1j2_n256"]
    desc, params, N = cfg["desc"], synth.make_params(cfg), cfg["N"]
    spins = synth.make_spins(cfg, 2)
    rng = np.random.default_rng(17)
    sample, sites = [], []
    for b in range(spins.shape[0]):
        s = spins[b]
        for sep in (1, 2):
            cand = [(i, (i + sep) % N) for i in range(N) if s[i] != s[(i + sep) % N]]
            for k in rng.choice(len(cand), 16, replace=False):
                sample.append(b)
                sites.append(cand[k])
    sample, sites = np.array(sample, dtype=np.int32), np.array(sites, dtype=np.int32)
    e_lp, e = errors(dn, desc, params, spins, sample, sites, "bf16", mc=3)
    e_lp32, e32 = errors(dn, desc, params, spins, sample, sites, "fp32", mc=3)
    print(f"bf16 J1-J2 N=256 6x64x64 pair flips: log psi {e_lp:.3e}, ratios {e:.3e} "
          f"(fp32: {e_lp32:.3e}, {e32:.3e})")
    assert e32 <= 1e-4 and e_lp32 <= 1e-4
    assert e_lp <= BF16_TOL_LOGPSI, f"log psi {e_lp:.3e}"
    assert e <= BF16_TOL_RATIO, f"ratios {e:.3e}"
