"""The forward pass's S4 convolution by FFT (dn_set_fft_conv) against the direct sum and
the FP64 oracle: log-amplitudes of the full forward pass and the ABACUS ratios built on
its caches, open chains (transform length the power of two >= 2N - 1) and rings of
power-of-two length (circular transform), FP64 and FP32; and the N = 1024, 6 x 64 x 64
model of the bench's long-chain line, where FP32 takes the FFT by default."""
import numpy as np
import pytest
import torch

import oracle
import synth
from synth import ModelDesc

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.fixture(scope="module")
def dn():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_11189_gb300 import dysonnet
    yield dysonnet
    dysonnet.set_fft_conv(1)


def rel_err(got, ref, lp_ref):
    den = np.maximum(np.abs(ref), 1e-3 * (1.0 + np.abs(lp_ref)))
    return np.abs(got - ref) / den


def run(dn, desc, params, spins_np, prec, mode):
    dn.set_fft_conv(mode)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(spins_np).cuda()
    lp = model.full_forward(spins, prec=prec).cpu().numpy()
    lpc = torch.empty(spins_np.shape[0], dtype=torch.float64, device="cuda")
    cache = model.forward_cache(spins, prec=prec, logpsi=lpc)
    r = cache.single_flip_ratios().cpu().numpy().reshape(-1)
    assert cache.check() == dn.DN_OK
    cache.destroy()
    model.close()
    dn.set_fft_conv(1)
    return lp, lpc.cpu().numpy(), r


CASES = [
    # L, d, s, w, dh, dout, periodic, N, B
    (3, 8, 4, 1, 8, 2, 0, 37, 3),     # open, M = 128
    (2, 16, 8, 2, 16, 1, 0, 64, 2),   # open, M = 128, N a power of two
    (3, 8, 4, 1, 8, 2, 1, 32, 3),     # ring, circular M = 32
    (4, 6, 3, 2, 6, 2, 0, 19, 2),     # open, d = 6: three channel pairs per field
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fft_conv_matches_direct_and_oracle(dn, case, prec):
    L, d, s, w, dh, dout, periodic, N, B = case
    desc = ModelDesc(L=L, d=d, s=s, w=w, dh=dh, dout=dout, periodic=periodic)
    params = synth.init_params(desc, 700 + N + d, a_scale=6.0)
    spins = synth.spins_uniform(B, N, 71 + N)
    lp_f, lpc_f, r_f = run(dn, desc, params, spins, prec, 2)
    lp_d, lpc_d, r_d = run(dn, desc, params, spins, prec, 0)
    lp_ref, _ = oracle.logpsi(desc, params, spins)
    sample, sites = synth.single_flips(B, N)
    ref = oracle.dlogpsi(desc, params, spins, sample, sites)
    for lp in (lp_f, lpc_f, lp_d):
        assert np.max(np.abs(lp - lp_ref) / np.maximum(1.0, np.abs(lp_ref))) <= TOL[prec]
    assert rel_err(r_f, ref, lp_ref[sample]).max() <= TOL[prec]
    # FFT and direct sum agree to rounding
    assert rel_err(r_f, r_d, lp_ref[sample]).max() <= (1e-12 if prec == "fp64" else 2e-5)


def test_fft_conv_n1024_default(dn):
    """FP32 forward of the N = 1024, 6 x 64 x 64 model (FFT by default at this size) against
    the oracle's log-amplitudes and the direct sum, two configurations."""
    N = 1024
    desc = synth.ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    params = synth.init_params(desc, 1005, a_scale=10.0)
    spins = synth.spins_uniform(2, N, 2005)
    model = dn.Model(desc, params)
    dn.set_fft_conv(1)
    lp_f = model.full_forward(torch.from_numpy(spins).cuda(), prec="fp32").cpu().numpy()
    dn.set_fft_conv(0)
    lp_d = model.full_forward(torch.from_numpy(spins).cuda(), prec="fp32").cpu().numpy()
    dn.set_fft_conv(1)
    model.close()
    lp_ref, _ = oracle.logpsi(desc, params, spins)
    e_f = np.max(np.abs(lp_f - lp_ref) / np.maximum(1.0, np.abs(lp_ref)))
    e_d = np.max(np.abs(lp_d - lp_ref) / np.maximum(1.0, np.abs(lp_ref)))
    print(f"N=1024 log psi rel err: FFT {e_f:.3e}, direct {e_d:.3e}")
    assert e_f <= 1e-4 and e_d <= 1e-4
