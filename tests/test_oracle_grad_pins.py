"""Pins of the oracle's parameter derivatives d log psi / d theta (the per-configuration
log-derivatives O_k of Sec. "Variational Monte Carlo").

  * central finite differences (h = 1e-6, FP64) of the oracle's own forward pass, for
    every parameter, on open and periodic chains and both readouts: a dropped term, a
    sign, a transposed weight or a wrong tap index in the reverse pass fails here;
  * homogeneity (Euler's theorem), exact and independent of any difference quotient:
    the network is linear in the embedding e, in the C and B of each S4 kernel and in
    the readout kernel, so with the identity readout
      sum_c e_c dlogpsi/de_c = log psi,
      sum over the final kernel's C (or B) of theta dlogpsi/dtheta = log psi,
      sum over layer 1's C (or B) of theta dlogpsi/dtheta = log psi - A^T pool(e sigma).
"""
import numpy as np
import pytest

import oracle
import synth
from synth import ModelDesc


def _desc_params(periodic, fkind, L=2, seed=5):
    desc = ModelDesc(L=L, d=3, s=3, w=1, dh=4, dout=2, periodic=periodic, fkind=fkind)
    p = synth.init_params(desc, seed, a_scale=20.0)
    sl = synth.param_slices(desc)
    rng = synth.SplitMix64(seed + 1000)
    # step sizes in [0.1, 0.5] so that the kernels reach across the chain
    for l in [f"l{i}" for i in range(1, L + 1)] + ["f"]:
        u = rng.uniform(desc.d)
        p[sl[f"{l}.log_dt"]] = np.log(0.1) + u * (np.log(0.5) - np.log(0.1))
    # non-zero biases so that every term of the MLP derivative is exercised
    for l in range(1, L + 1):
        for nm in ("beta", "b1", "b2"):
            s = sl[f"l{l}.{nm}"]
            p[s] = 0.3 * rng.normal(s.stop - s.start)
    return desc, p, sl


@pytest.mark.parametrize("periodic,fkind,L", [(0, 0, 2), (1, 0, 2), (0, 1, 3), (1, 1, 3)])
def test_grad_matches_central_differences(periodic, fkind, L):
    desc, p, _ = _desc_params(periodic, fkind, L)
    spins = synth.spins_uniform(2, 7, 11 + periodic)
    lp, g = oracle.grad_logpsi(desc, p, spins)
    lp_ref, _ = oracle.logpsi(desc, p, spins)
    assert np.array_equal(lp, lp_ref) or np.max(np.abs(lp - lp_ref)) <= 1e-13 * np.max(np.abs(lp_ref))
    h = 1e-6
    fd = np.zeros_like(g)
    for k in range(p.size):
        pp = p.copy()
        pp[k] += h
        a, _ = oracle.logpsi(desc, pp, spins)
        pp[k] -= 2 * h
        b, _ = oracle.logpsi(desc, pp, spins)
        fd[:, k] = (a - b) / (2 * h)
    # central differences: truncation O(h^2), rounding ~ eps |log psi| / h
    tol = 1e-8 * np.maximum(1.0, np.abs(lp_ref))[:, None] + 1e-6 * np.abs(fd)
    bad = np.abs(g - fd) > tol
    assert not bad.any(), f"{bad.sum()} entries, worst {np.max(np.abs(g - fd)):.3e} at {np.argmax(np.abs(g - fd).max(0))}"
    assert np.abs(fd).max() > 1e-2   # the check is not vacuous


@pytest.mark.parametrize("periodic", [0, 1])
def test_grad_homogeneity(periodic):
    desc, p, sl = _desc_params(periodic, fkind=1, L=3, seed=9)
    spins = synth.spins_uniform(3, 9, 21)
    lp, g = oracle.grad_logpsi(desc, p, spins)

    def euler(names):
        return sum(g[:, sl[n]] @ p[sl[n]] for n in names)

    tol = 1e-11 * np.maximum(1.0, np.abs(lp))
    assert np.all(np.abs(euler(["e"]) - lp) <= tol)
    assert np.all(np.abs(euler(["A"]) - lp) <= tol)
    assert np.all(np.abs(euler(["f.cf_re", "f.cf_im", "f.cb_re", "f.cb_im"]) - lp) <= tol)
    assert np.all(np.abs(euler(["f.b_re", "f.b_im"]) - lp) <= tol)
    # layer 1: everything but the pooled embedding term scales with its C (or B)
    _, omega = oracle.plan(desc, p, spins.shape[1])
    A = p[sl["A"]].reshape(desc.d, desc.dout)
    e = p[sl["e"]]
    pool0 = (omega.T @ spins.T.astype(np.float64)).T * e          # [B][d]
    rest = lp - (pool0 @ A).sum(axis=1)
    assert np.all(np.abs(euler(["l1.cf_re", "l1.cf_im", "l1.cb_re", "l1.cb_im"]) - rest) <= tol)
    assert np.all(np.abs(euler(["l1.b_re", "l1.b_im"]) - rest) <= tol)


def test_sr_matrices_spectra_and_trace():
    """The sample-space Gram Oc Oc^T / B and the parameter-space S = Oc^T Oc / B share their
    non-zero eigenvalues (both are squares of the singular values of Oc / sqrt(B)); both are
    symmetric positive semi-definite, the Gram annihilates the all-ones vector (centring), and
    trace = sum_b |Oc_b|^2 / B."""
    desc, p, sl = _desc_params(0, 0, L=2, seed=13)
    spins = synth.spins_uniform(6, 8, 5)
    _, O = oracle.grad_logpsi(desc, p, spins)
    P = O.shape[1]
    G, S = oracle.sr_matrices(O, block=(0, P))
    B = O.shape[0]
    assert np.allclose(G, G.T, atol=0) and np.allclose(S, S.T, rtol=1e-13, atol=1e-13 * np.abs(S).max())
    eg = np.sort(np.linalg.eigvalsh(G))[::-1]
    es = np.sort(np.linalg.eigvalsh(S))[::-1][:B]
    assert eg.min() >= -1e-10 * eg.max()
    assert np.allclose(eg[:B - 1], es[:B - 1], rtol=1e-9, atol=1e-10 * eg.max())
    assert abs(eg[-1]) <= 1e-10 * eg.max()
    assert np.abs(G @ np.ones(B)).max() <= 1e-10 * np.abs(G).max()
    Oc = O - O.mean(axis=0)
    assert np.isclose(np.trace(G), (Oc * Oc).sum() / B, rtol=1e-12)
    _, Sb = oracle.sr_matrices(O, block=(5, 7))
    assert np.allclose(Sb, S[5:12, 5:12], rtol=1e-12, atol=1e-14 * np.abs(S).max())
