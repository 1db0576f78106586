"""Per-configuration log-derivatives O_b = d log psi(sigma_b) / d theta on the GPU
(dn_logpsi_grad through the C ABI) against the oracle's reverse pass, which the CPU tests
pin to central differences and to the network's homogeneity.

Bars: FP64 1e-10 and FP32 1e-4 on every element, relative to
max(|O_ref[b, k]|, 1e-2 max(1, max_k |O_ref[b, k]|)): entries down to one percent of their
sample's largest log-derivative are held to the bar relative to themselves; smaller ones,
whose FP32 value is set by cancellation between much larger terms, to the bar relative to
that floor.
"""
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


def _params(desc, seed):
    p = synth.init_params(desc, seed, a_scale=6.0)
    sl = synth.param_slices(desc)
    rng = synth.SplitMix64(seed + 500)
    for l in [f"l{i}" for i in range(1, desc.L + 1)] + ["f"]:
        u = rng.uniform(desc.d)
        p[sl[f"{l}.log_dt"]] = np.log(0.02) + u * (np.log(0.5) - np.log(0.02))
    for l in range(1, desc.L + 1):
        for nm in ("beta", "b1", "b2"):
            s = sl[f"l{l}.{nm}"]
            p[s] = 0.3 * rng.normal(s.stop - s.start)
    return p


FLOOR = 1e-2


def _err(got, ref, floor=FLOOR):
    """Largest element-wise error relative to max(|ref|, floor * max(1, row maximum))."""
    row = np.maximum(1.0, np.abs(ref).max(axis=1, keepdims=True))
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor * row))


CASES = [
    # L, d, s, w, dh, dout, periodic, fkind, N, B
    (2, 4, 3, 1, 5, 2, 0, 0, 9, 3),
    (3, 6, 4, 2, 7, 2, 1, 0, 13, 2),
    (3, 8, 5, 1, 8, 1, 0, 1, 37, 2),      # several site tiles, ragged outer-product tiles
    (4, 33, 4, 2, 35, 2, 0, 0, 40, 2),    # channel and MLP widths past one 32-wide tile
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grad_matches_oracle(dn, case, prec):
    L, d, s, w, dh, dout, periodic, fkind, N, B = case
    desc = ModelDesc(L=L, d=d, s=s, w=w, dh=dh, dout=dout, periodic=periodic, fkind=fkind)
    p = _params(desc, 40 + L + d)
    spins = synth.spins_uniform(B, N, 7 + N)
    model = dn.Model(desc, p)
    lp, O, _ = model.logpsi_grad(cuda(spins), prec=prec)
    lp_ref, O_ref = oracle.grad_logpsi(desc, p, spins)
    got = O.double().cpu().numpy()
    bar = 1e-10 if prec == "fp64" else 1e-4
    e = _err(got, O_ref)
    print(f"{prec} {case}: O element-wise rel err {e:.3e} (floor 1e-2); "
          f"floor 1e-4: {_err(got, O_ref, 1e-4):.3e}; row-max normalised: {_err(got, O_ref, 1.0):.3e}")
    assert e <= bar
    assert np.max(np.abs(lp.cpu().numpy() - lp_ref) / np.maximum(1.0, np.abs(lp_ref))) <= bar
    model.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vjp_and_autograd(dn, prec):
    desc = ModelDesc(L=3, d=8, s=4, w=1, dh=8, dout=2, periodic=0)
    p = _params(desc, 77)
    spins = synth.spins_uniform(4, 21, 3)
    wts = np.array([0.5, -1.25, 2.0, 0.75])
    _, O_ref = oracle.grad_logpsi(desc, p, spins)
    ref = wts @ O_ref
    model = dn.Model(desc, p)
    _, _, vjp = model.logpsi_grad(cuda(spins), prec=prec, weights=cuda(wts), with_O=False)
    model.close()
    bar = 1e-10 if prec == "fp64" else 1e-4
    scale = max(1.0, np.abs(ref).max())
    assert np.max(np.abs(vjp.cpu().numpy() - ref)) / scale <= bar
    theta = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    lp = dn.LogPsi.apply(theta, desc, cuda(spins), prec)
    (g,) = torch.autograd.grad((lp * torch.tensor(wts, device=lp.device)).sum(), theta)
    assert g.shape == theta.shape
    assert np.max(np.abs(g.numpy() - ref)) / scale <= bar


def test_grad_rejects_bad_input(dn):
    desc = ModelDesc(L=2, d=4, s=3, w=1, dh=4, dout=2, periodic=0)
    p = _params(desc, 3)
    model = dn.Model(desc, p)
    spins = synth.spins_uniform(2, 8, 1)
    spins[1, 3] = 0
    with pytest.raises(dn.DysonNetError):
        model.logpsi_grad(cuda(spins), prec="fp64")
    with pytest.raises(dn.DysonNetError):
        model.logpsi_grad(cuda(synth.spins_uniform(2, 8, 1)), prec="bf16")
    model.close()


def test_grad_lrtfim_n256_workload_sampled(dn):
    """Forward + backward of 4096 configurations of the N = 256, 6 x 64 x 64 long-range
    TFIM model in FP32; two configurations checked against the oracle."""
    desc = ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    p = synth.init_params(desc, 1004, a_scale=10.0)
    spins = synth.spins_uniform(4096, 256, 2004)
    model = dn.Model(desc, p)
    lp, O, _ = model.logpsi_grad(cuda(spins), prec="fp32")
    assert O.shape == (4096, model.nparams)
    assert torch.isfinite(O).all()
    pick = [0, 4095]
    lp_ref, O_ref = oracle.grad_logpsi(desc, p, spins[pick])
    got = O[pick].double().cpu().numpy()
    e = _err(got, O_ref)
    print(f"N=256 workload sampled O element-wise rel err {e:.3e} (floor 1e-2); "
          f"floor 1e-4: {_err(got, O_ref, 1e-4):.3e}")
    assert e <= 1e-4
    model.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sr_matrices(dn, prec):
    desc = ModelDesc(L=2, d=8, s=4, w=1, dh=8, dout=2, periodic=0)
    p = _params(desc, 5)
    spins = synth.spins_uniform(70, 12, 9)           # two 64-sample tiles, ragged
    _, O = oracle.grad_logpsi(desc, p, spins)
    P = O.shape[1]
    blk = (3, 100)
    G_ref, S_ref = oracle.sr_matrices(O, block=blk)
    Od = cuda(O if prec == "fp64" else O.astype(np.float32))
    G, S = dn.sr_matrices(Od, gram=True, block=blk)
    bar = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(G.cpu().numpy() - G_ref)) <= bar * np.abs(G_ref).max()
    assert np.max(np.abs(S.cpu().numpy() - S_ref)) <= bar * np.abs(S_ref).max()
    assert P > 100


def test_sr_gram_many_k_splits(dn):
    """FP32 Gram over 700,000 parameters: the tensor-core Gram accumulates at most 16384
    terms per split in FP32 and sums the 43 splits in FP64; checked against an FP64
    product of the same (FP32) values, with ragged 128-sample tiles."""
    B, P = 600, 700_000
    rng = np.random.default_rng(11)
    O = (rng.standard_normal((B, P)) * rng.uniform(0.1, 3.0, size=P)).astype(np.float32)
    O[:, :5000] += 0.7                      # columns with a mean, removed by the centring
    G, _ = dn.sr_matrices(cuda(O), gram=True)
    Oc = O.astype(np.float64) - O.astype(np.float64).mean(axis=0)
    G_ref = Oc @ Oc.T / B
    err = np.max(np.abs(G.cpu().numpy() - G_ref)) / np.abs(G_ref).max()
    print(f"SR Gram B={B} P={P}: max error / max |G| = {err:.3e}")
    assert err <= 1e-5
