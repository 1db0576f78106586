"""Link-construction kernels (App. "Exact algorithm to construct link tensors",
Eqs. X_def, L_def) through the C ABI.

The last vertex hop of a chain and the band of G^(L) run either fused in one kernel
(`k_dband_tc`) or as two kernels with the hop output in device memory.  Both are
exact; the fused one forms every sum in the same order, so the interlayer link
tensors K must agree to the last bit (checked to 1e-6 of the tensor's largest entry,
with the bit-exact outcome printed), and the flip ratios built on them must match the
FP64 oracle within the FP32 bar (1e-4).
"""
import ctypes

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


def _traced_kernels(lib, fn):
    lib.dn_profile_enable(1)
    try:
        fn()
        torch.cuda.synchronize()
        names = []
        lib.dn_profile_count.restype = ctypes.c_int
        buf = ctypes.create_string_buffer(256)
        n_l, ms = ctypes.c_longlong(), ctypes.c_double()
        for i in range(lib.dn_profile_count()):
            if lib.dn_profile_get(i, buf, 256, ctypes.byref(n_l), ctypes.byref(ms)) == 0 and n_l.value > 0:
                names.append(buf.value.decode())
        return names
    finally:
        lib.dn_profile_enable(0)


def _rel(got, ref, lp):
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp)))
    return np.max(np.abs(got - ref) / den)


CASES = [
    # L, N, w, periodic, max_cluster, B
    (4, 24, 2, 0, 1, 3),     # band half-width 4 (9 offsets), one full column tile per site group
    (4, 37, 2, 0, 1, 2),     # ragged last column tile (one source site)
    (5, 40, 2, 1, 1, 2),     # ring, two chains ending in the fused kernel
    (4, 33, 1, 0, 2, 2),     # w = 1, pairs: half-width 3 (7 offsets)
    (4, 20, 1, 1, 1, 2),     # ring, half-width 2 (5 offsets)
]


@pytest.mark.parametrize("case", CASES)
def test_fused_chain_end_equals_two_kernels_and_oracle(dn, case):
    L, N, w, periodic, mc, B = case
    desc = ModelDesc(L=L, d=32, s=8, w=w, dh=32, dout=2, periodic=periodic)
    params = synth.init_params(desc, 900 + N, a_scale=8.0)
    spins_np = synth.spins_uniform(B, N, 31 + N)
    spins = torch.from_numpy(spins_np).cuda()
    model = dn.Model(desc, params)
    lib = dn._lib()
    caches = {}
    try:
        for fused in (False, True):
            dn.set_fused_links(fused)
            names = _traced_kernels(lib, lambda: caches.__setitem__(fused, model.forward_cache(spins, prec="fp32",
                                                                                               max_cluster=mc)))
            assert any(n.endswith("k_dband") for n in names) == fused, names
    finally:
        dn.set_fused_links(True)
    K0, K1 = caches[False].tensor("K").cpu().numpy(), caches[True].tensor("K").cpu().numpy()
    # Band entries whose partner site is off an open chain are unspecified: compare the rest.
    nR = 2 * (desc.W + mc - 1 - 1) + 1
    Kv0 = K0.reshape(B, -1, N, nR, 32, 32)
    Kv1 = K1.reshape(B, -1, N, nR, 32, 32)
    R = (nR - 1) // 2
    mask = np.ones((N, nR), bool)
    if not periodic:
        for i in range(N):
            for o in range(nR):
                k = i + o - R
                mask[i, o] = 0 <= k < N
    a, b = Kv0[:, :, mask], Kv1[:, :, mask]
    diff = np.max(np.abs(a - b)) / np.abs(a).max()
    print(f"{case}: fused vs two-kernel K max diff / max |K| = {diff:.3e} (bit-identical: {np.array_equal(a, b)})")
    assert diff <= 1e-6
    # Flip ratios on the fused caches against the oracle.
    if mc == 1:
        sample, sites = synth.single_flips(B, N)
    else:
        sample, sites = synth.random_flips(B, N, 24, seed=N, pair_frac=0.5, max_sep=mc - 1)
    got = caches[True].flip_ratios(torch.from_numpy(sample).cuda(), torch.from_numpy(sites).cuda()).cpu().numpy()
    for c in caches.values():
        assert c.check() == dn.DN_OK
        c.destroy()
    ref = oracle.dlogpsi(desc, params, spins_np, sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np)
    e = _rel(got, ref, lp[sample])
    print(f"{case}: ratios vs oracle rel err {e:.3e}")
    assert e <= 1e-4
    model.close()


def test_fused_chain_end_bench_model(dn):
    """The N = 128, 4 x 32 x 32 workload model: fused and two-kernel link tensors of 8
    configurations agree, and 64 sampled ratios match the oracle."""
    cfg = synth.CONFIGS["lrtfim_n128"]
    desc, params = cfg["desc"], synth.make_params(cfg)
    spins_np = synth.make_spins(cfg, B=8)
    spins = torch.from_numpy(spins_np).cuda()
    model = dn.Model(desc, params)
    Ks = {}
    try:
        for fused in (False, True):
            dn.set_fused_links(fused)
            c = model.forward_cache(spins, prec="fp32")
            Ks[fused] = c.tensor("K").cpu().numpy()
            if fused:
                rng = np.random.default_rng(3)
                pick = rng.choice(8 * 128, 64, replace=False)
                sample = (pick // 128).astype(np.int32)
                sites = np.stack([pick % 128, -np.ones_like(pick)], axis=1).astype(np.int32)
                got = c.flip_ratios(torch.from_numpy(sample).cuda(), torch.from_numpy(sites).cuda()).cpu().numpy()
            assert c.check() == dn.DN_OK
            c.destroy()
    finally:
        dn.set_fused_links(True)
    Kv0, Kv1 = (K.reshape(8, 3, 128, 9, 32, 32) for K in (Ks[False], Ks[True]))
    inner = slice(4, 124)     # rows whose whole band lies on the chain
    diff = np.max(np.abs(Kv0[:, :, inner] - Kv1[:, :, inner])) / np.abs(Kv0[:, :, inner]).max()
    print(f"bench model: fused vs two-kernel K max diff / max |K| = {diff:.3e}")
    assert diff <= 1e-6
    ref = oracle.dlogpsi(desc, params, spins_np, sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np)
    e = _rel(got, ref, lp[sample])
    print(f"bench model: ratios vs oracle rel err {e:.3e}")
    assert e <= 1e-4
    model.close()


FFT_CASES = [
    # L, N, d, w, periodic, max_cluster, B, prec
    (3, 24, 8, 2, 0, 1, 3, "fp64"),     # the only pair (3, 1); M = 64
    (4, 37, 8, 1, 0, 2, 2, "fp64"),     # pair (4, 2) of the last chain; ragged N, pairs; M = 128
    (3, 16, 8, 2, 1, 1, 2, "fp64"),     # ring: circular correlation of length N
    (3, 40, 32, 2, 0, 1, 2, "fp32"),
    (4, 32, 32, 2, 1, 2, 2, "fp32"),    # ring, pairs
]


@pytest.mark.parametrize("case", FFT_CASES)
def test_fft_links_equal_direct_band_and_oracle(dn, case):
    """The band links of the one-intermediate pair (l, m) = (L, L - 2) by FFT (the
    two-layer link of App. "Efficient construction of link tensors") equal the direct band
    sum to rounding, and the ratios built on them match the FP64 oracle."""
    L, N, d, w, periodic, mc, B, prec = case
    desc = ModelDesc(L=L, d=d, s=6, w=w, dh=d, dout=2, periodic=periodic)
    params = synth.init_params(desc, 300 + N + d, a_scale=8.0)
    spins_np = synth.spins_uniform(B, N, 61 + N)
    spins = torch.from_numpy(spins_np).cuda()
    model = dn.Model(desc, params)
    lib = dn._lib()
    caches = {}
    try:
        for fft in (False, True):
            dn.set_fft_links(2 if fft else 0)
            names = _traced_kernels(lib, lambda: caches.__setitem__(fft, model.forward_cache(spins, prec=prec,
                                                                                             max_cluster=mc)))
            assert any(n.endswith("k_link_fft") for n in names) == fft, names
    finally:
        dn.set_fft_links(1)
    nR = 2 * (desc.W + mc - 1 - 1) + 1
    R = (nR - 1) // 2
    pair = (L - 3) * (L - 2) // 2 + (L - 3)            # index of (L, L - 2)
    Kd, Kf = (caches[f].tensor("K").cpu().numpy().reshape(B, -1, N, nR, d, d)[:, pair] for f in (False, True))
    mask = np.ones((N, nR), bool)
    if not periodic:
        for i in range(N):
            for o in range(nR):
                mask[i, o] = 0 <= i + o - R < N
    a, b = Kd[:, mask], Kf[:, mask]
    diff = np.max(np.abs(a - b)) / np.abs(a).max()
    print(f"{case}: FFT vs direct band links max diff / max |K| = {diff:.3e}")
    assert diff <= (1e-12 if prec == "fp64" else 1e-5)
    if mc == 1:
        sample, sites = synth.single_flips(B, N)
    else:
        sample, sites = synth.random_flips(B, N, 24, seed=N, pair_frac=0.5, max_sep=mc - 1, periodic=bool(periodic))
    got = caches[True].flip_ratios(torch.from_numpy(sample).cuda(), torch.from_numpy(sites).cuda()).cpu().numpy()
    for c in caches.values():
        assert c.check() == dn.DN_OK
        c.destroy()
    ref = oracle.dlogpsi(desc, params, spins_np, sample, sites)
    lp, _ = oracle.logpsi(desc, params, spins_np)
    e = _rel(got, ref, lp[sample])
    print(f"{case}: ratios vs oracle rel err {e:.3e}")
    assert e <= (1e-10 if prec == "fp64" else 1e-4)
    model.close()
