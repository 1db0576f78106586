"""Pins of the CPU FP64 oracle against what the paper and mathematics fix.

Each test targets a different plausible mistake:
  * taps vs an independent state-space scan (direction, index, discretisation);
  * periodic closed form vs the explicit sum over periodic images;
  * the forward circulant's DFT vs the Cauchy-kernel resolvent (Eq. resolvent);
  * Jastrow limit (App. "DysonNet can exactly represent power law decay",
    Eqs. jastrow_short, Jij_short): with one layer, one channel and a one-site
    window the log-amplitude is exactly quadratic in the spins, with couplings
    set by the convolution taps; a shifted window pins the window orientation;
  * a linear network (constant vertex) has a closed-form pooled output that
    fixes the order and orientation of U, V and of the layers;
  * log cosh readout against numpy's log(cosh);
  * exact diagonalisation against Jordan-Wigner (nearest-neighbour TFIM,
    Sec. "Benchmarking") and the Majumdar-Ghosh energy (App. j1j2);
  * exact enumeration: sum psi^2 E_loc / sum psi^2 = <psi|H|psi>/<psi|psi>,
    and the variational principle (Eq. local-estimator).
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla
import torch

import oracle
import synth
from synth import ModelDesc


def _s4block(desc, params, prefix):
    sl = synth.param_slices(desc)
    start = sl[f"{prefix}.lam_re"].start
    stop = sl[f"{prefix}.cb_im"].stop
    return params[start:stop]


def _fast_desc_params(seed=7, periodic=0, L=2, d=3, s=4, w=1, dh=3, dout=2, dt_range=None, fkind=0):
    desc = ModelDesc(L=L, d=d, s=s, w=w, dh=dh, dout=dout, periodic=periodic, fkind=fkind)
    p = synth.init_params(desc, seed, a_scale=3.0)
    if dt_range is not None:
        sl = synth.param_slices(desc)
        rng = synth.SplitMix64(seed + 99)
        for l in [f"l{i}" for i in range(1, L + 1)] + ["f"]:
            u = rng.uniform(d)
            p[sl[f"{l}.log_dt"]] = np.log(dt_range[0]) + u * (np.log(dt_range[1]) - np.log(dt_range[0]))
    return desc, p


def _conv_open(g, h):
    """u_i = sum_j g[i-j] h_j with g indexed r + N - 1 (library convolution, per channel)."""
    N, d = h.shape
    u = np.zeros_like(h)
    for c in range(d):
        full = np.convolve(h[:, c], g[:, c])      # full[k] = sum_j h[j] g[k - j]
        u[:, c] = full[N - 1:2 * N - 1]
    return u


# ------------------------------------------------------------------ taps --

@pytest.mark.parametrize("N", [1, 2, 7, 33])
def test_taps_equal_state_space_scan(N):
    desc, p = _fast_desc_params(seed=11, d=4, s=5)
    blk = _s4block(desc, p, "l1")
    g = oracle.s4_taps(desc, blk, N, periodic=False)
    rng = np.random.default_rng(N)
    h = rng.standard_normal((N, desc.d))
    u_scan = oracle.s4_scan(desc, blk, h)
    u_conv = _conv_open(g, h)
    np.testing.assert_allclose(u_conv, u_scan, rtol=1e-12, atol=1e-13)


def test_periodic_taps_equal_image_sum():
    # Large steps so that the images decay within K windows.
    desc, p = _fast_desc_params(seed=5, d=3, s=4, dt_range=(0.3, 0.9))
    blk = _s4block(desc, p, "l2")
    N, K = 6, 400
    gper = oracle.s4_taps(desc, blk, N, periodic=True)
    gopen = oracle.s4_taps(desc, blk, N * K, periodic=False)   # r in (-NK, NK)
    img = np.zeros_like(gper)
    for r in range(N):
        for m in range(-K + 1, K):
            rr = r + m * N
            if -N * K < rr < N * K:
                img[r] += gopen[rr + N * K - 1]
    np.testing.assert_allclose(gper, img, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("N", [4, 9, 64])
def test_circulant_dft_equals_resolvent(N):
    desc, p = _fast_desc_params(seed=3, d=3, s=6)
    blk = _s4block(desc, p, "f")
    gc = oracle.s4_circulant_fwd_complex(desc, blk, N)            # [N][d] complex
    dft = np.fft.ifft(gc, axis=0) * N                             # sum_r g_r exp(+2 pi i k r / N)
    res = oracle.s4_resolvent(desc, blk, N)
    np.testing.assert_allclose(dft, res, rtol=1e-10, atol=1e-12)
    # The real periodic taps with the backward output zeroed are Re of the complex circulant.
    q = p.copy()
    sl = synth.param_slices(desc)
    q[sl["f.cb_re"]] = 0.0
    q[sl["f.cb_im"]] = 0.0
    g_real = oracle.s4_taps(desc, _s4block(desc, q, "f"), N, periodic=True)
    np.testing.assert_allclose(g_real, gc.real, rtol=1e-12, atol=1e-14)


def test_discretised_modes_inside_unit_disk():
    # Re(Lambda) < 0 => |lam_bar| < 1: open taps decay with distance.
    desc, p = _fast_desc_params(seed=21, d=2, s=3, dt_range=(0.5, 1.0))
    g = oracle.s4_taps(desc, _s4block(desc, p, "l1"), 200, periodic=False)
    assert np.abs(g[199 + 150]).max() < 1e-4 * np.abs(g[199:199 + 5]).max()


# --------------------------------------------------------------- Jastrow --

def _quadratic_fit(N, values):
    """Exact fit of values(sigma) on {1, sigma_i, sigma_i sigma_j}; returns (c, h, J, resid)."""
    confs = np.array(list(itertools.product([1, -1], repeat=N)), dtype=np.int8)
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    X = np.concatenate([np.ones((len(confs), 1)), confs.astype(float),
                        np.stack([confs[:, i] * confs[:, j] for i, j in pairs], axis=1).astype(float)], axis=1)
    y = values(confs)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    resid = np.abs(X @ coef - y).max()
    J = np.zeros((N, N))
    for k, (i, j) in enumerate(pairs):
        J[i, j] = J[j, i] = coef[1 + N + k]
    return coef[0], coef[1:1 + N], J, resid


def _jastrow_model(periodic, r0, seed):
    """L=1, d=1, dh=1, dout=1, f=identity; window weight only at offset r0 (w=1)."""
    desc = ModelDesc(L=1, d=1, s=3, w=1, dh=1, dout=1, periodic=periodic, fkind=1)
    p = synth.init_params(desc, seed, a_scale=1.0)
    sl = synth.param_slices(desc)
    kap = np.zeros(3)
    kap[r0 + 1] = 1.3
    p[sl["l1.kappa"]] = kap
    p[sl["l1.beta"]] = 0.2
    p[sl["l1.W1"]] = 0.9
    p[sl["l1.b1"]] = -0.1
    p[sl["l1.W2"]] = 1.7
    p[sl["l1.b2"]] = 0.3
    p[sl["l1.U"]] = 0.8
    p[sl["l1.V"]] = -1.1
    p[sl["e"]] = 0.7
    p[sl["A"]] = 1.5
    return desc, p, sl


def _chi(p, sl, s):
    """chi(sigma) of the one-channel MLP, GELU from torch (exact erf form)."""
    a = float(p[sl["l1.W1"]][0]) * (float(p[sl["l1.kappa"]][np.nonzero(p[sl["l1.kappa"]])[0][0]]) * s
                                    + float(p[sl["l1.beta"]][0])) + float(p[sl["l1.b1"]][0])
    ga = torch.nn.functional.gelu(torch.tensor(a, dtype=torch.float64)).item()
    return float(p[sl["l1.W2"]][0]) * ga + float(p[sl["l1.b2"]][0])


@pytest.mark.parametrize("periodic", [1, 0])
@pytest.mark.parametrize("r0", [0, 1, -1])
def test_jastrow_limit_couplings(periodic, r0):
    N = 8
    desc, p, sl = _jastrow_model(periodic, r0, seed=40 + r0 + 3 * periodic)
    taps, omega = oracle.plan(desc, p, N)
    g = taps[0][:, 0]
    om = omega[:, 0]
    c, h, J, resid = _quadratic_fit(N, lambda conf: oracle.logpsi(desc, p, conf)[0])
    assert resid < 1e-12                     # exactly quadratic in sigma

    UV = float(p[sl["l1.U"]][0]) * float(p[sl["l1.V"]][0])
    D1 = UV * (_chi(p, sl, 1) - _chi(p, sl, -1)) / 2
    A, e = float(p[sl["A"]][0]), float(p[sl["e"]][0])

    def gt(r):                                 # tap at offset r = i - j
        return g[r % N] if periodic else (g[r + N - 1] if -N < r < N else 0.0)

    # log psi = A sum_i omega_i [e s_i + D(s_{i+r0}) sum_j g_{i-j} e s_j]; the coupling
    # of (a, b) collects i = a - r0 with j = b, and i = b - r0 with j = a.
    Jpred = np.zeros((N, N))
    for a in range(N):
        for b in range(N):
            if a == b:
                continue
            acc = 0.0
            for (x, y) in ((a, b), (b, a)):
                i = x - r0
                if periodic:
                    i %= N
                elif not 0 <= i < N:
                    continue
                acc += om[i] * gt(i - y)
            Jpred[a, b] = A * e * D1 * acc
    np.testing.assert_allclose(J, Jpred, rtol=1e-9, atol=1e-12)
    if periodic and r0 == 0:
        # Paper's form for an even kernel: J_ij proportional to G_|i-j| (Eq. Jij_short).
        sym = np.array([[gt(i - j) + gt(j - i) for j in range(N)] for i in range(N)])
        ratio = J[~np.eye(N, dtype=bool)] / sym[~np.eye(N, dtype=bool)]
        np.testing.assert_allclose(ratio, ratio[0], rtol=1e-8)


def test_even_kernel_matches_paper_jastrow_formula():
    """With C_bwd = C_fwd the taps are even and J_ij = 2 A' D_1 G_|i-j| (Eq. Jij_short),
    A' = A * omega * e absorbing the embedding and the pooled readout kernel."""
    N = 7
    desc, p, sl = _jastrow_model(1, 0, seed=77)
    p[sl["l1.cb_re"]] = p[sl["l1.cf_re"]]
    p[sl["l1.cb_im"]] = p[sl["l1.cf_im"]]
    taps, omega = oracle.plan(desc, p, N)
    g = taps[0][:, 0]
    c, h, J, resid = _quadratic_fit(N, lambda conf: oracle.logpsi(desc, p, conf)[0])
    UV = float(p[sl["l1.U"]][0]) * float(p[sl["l1.V"]][0])
    D1 = UV * (_chi(p, sl, 1) - _chi(p, sl, -1)) / 2
    Aeff = float(p[sl["A"]][0]) * float(p[sl["e"]][0]) * omega[0, 0]
    for i in range(N):
        for j in range(i + 1, N):
            r = min(j - i, N - (j - i))
            assert abs(J[i, j] - 2 * Aeff * D1 * g[r]) < 1e-11


# ------------------------------------------------------ linear network ----

@pytest.mark.parametrize("L", [1, 3])
def test_constant_vertex_closed_form(L):
    """chi = const => D_j = c U V for every site; on a ring the pooled output is
    Omega = A^T omega_bar sum_l (prod_{n<=l} c_n U_n V_n diag(Gamma_n)) e * M,
    M = sum_i sigma_i, Gamma_n = column sum of the circulant taps."""
    N, d = 9, 4
    desc = ModelDesc(L=L, d=d, s=3, w=1, dh=2, dout=2, periodic=1, fkind=1)
    p = synth.init_params(desc, 123, a_scale=1.0)
    sl = synth.param_slices(desc)
    cs = []
    for l in range(1, L + 1):
        p[sl[f"l{l}.W2"]] = 0.0
        cl = 0.5 + 0.3 * l
        p[sl[f"l{l}.b2"]] = cl
        cs.append(cl)
    taps, omega = oracle.plan(desc, p, N)
    spins = synth.spins_uniform(5, N, 9)
    _, Om = oracle.logpsi(desc, p, spins)
    A = p[sl["A"]].reshape(d, 2)
    e = p[sl["e"]]
    vec = e.copy()
    tot = e.copy()
    for l in range(1, L + 1):
        U = p[sl[f"l{l}.U"]].reshape(d, d)
        V = p[sl[f"l{l}.V"]].reshape(d, d)
        Gam = taps[l - 1].sum(axis=0)
        vec = cs[l - 1] * U @ (V @ (Gam * vec))
        tot = tot + vec
    wbar = omega[0]
    for b in range(5):
        M = float(spins[b].sum())
        pred = A.T @ (wbar * tot) * M
        np.testing.assert_allclose(Om[b], pred, rtol=1e-10, atol=1e-12)


def test_logcosh_readout():
    desc1, p = _fast_desc_params(seed=8, dout=1, fkind=1)
    desc0 = ModelDesc(**{**desc1.as_dict(), "fkind": 0})
    spins = synth.spins_uniform(6, 11, 5)
    lp1, _ = oracle.logpsi(desc1, p, spins)
    lp0, _ = oracle.logpsi(desc0, p, spins)
    np.testing.assert_allclose(lp0, np.log(np.cosh(lp1)), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------- Hamiltonians -----

def _all_confs(N):
    idx = np.arange(2 ** N, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)) & 1
    return (1 - 2 * bits).astype(np.int8)


def _sparse_H(N, ham):
    """Sparse H in the sigma^z basis, built from the Pauli/spin algebra directly.
    Basis index x: sigma_i = 1 - 2 * bit_i(x)."""
    confs = _all_confs(N)
    dim = 2 ** N
    rows, cols, vals = [], [], []
    diag = np.zeros(dim)
    if ham["kind"] == 0:
        norm = 1.0
        if ham.get("kac", 0):
            norm = sum(2.0 * r ** (-ham["alpha"]) for r in range(1, N // 2 + 1))
        for i in range(N):
            for j in range(i + 1, N):
                r = j - i
                if ham.get("periodic", 0):
                    r = min(r, N - r)
                diag += ham["J"] * r ** (-ham["alpha"]) / norm * confs[:, i] * confs[:, j]
            rows.append(np.arange(dim))
            cols.append(np.arange(dim) ^ (1 << i))
            vals.append(np.full(dim, ham["h"]))
    else:
        for b, Jb in ((1, ham["J1"]), (2, ham["J2"])):
            imax = N if ham.get("periodic", 1) else N - b
            for i in range(imax):
                j = (i + b) % N
                diag += Jb * 0.25 * confs[:, i] * confs[:, j]
                anti = confs[:, i] != confs[:, j]
                x = np.arange(dim)[anti]
                rows.append(x)
                cols.append(x ^ (1 << i) ^ (1 << j))
                vals.append(np.full(x.shape[0], 0.5 * Jb))
    rows.append(np.arange(dim))
    cols.append(np.arange(dim))
    vals.append(diag)
    H = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim))
    return H


def _ground(H):
    return spla.eigsh(H, k=1, which="SA", tol=1e-12)[0][0]


@pytest.mark.parametrize("N,J,h", [(6, 1.0, 1.0), (9, -0.7, 1.3), (10, 1.0, 0.4)])
def test_ed_nearest_neighbour_tfim_matches_jordan_wigner(N, J, h):
    ham = dict(kind=0, J=J, alpha=80.0, h=h, periodic=0, kac=0)
    E0 = _ground(_sparse_H(N, ham))
    # Open-chain free fermions: E0 = -sum of singular values of the bidiagonal
    # matrix with h on the diagonal and J on the superdiagonal.
    M = np.diag(np.full(N, h)) + np.diag(np.full(N - 1, J), 1)
    Ejw = -np.linalg.svd(M, compute_uv=False).sum()
    assert abs(E0 - Ejw) < 1e-9


@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_ed_majumdar_ghosh(N):
    ham = dict(kind=1, J1=1.0, J2=0.5, periodic=1)
    E0 = _ground(_sparse_H(N, ham))
    assert abs(E0 - (-3.0 * N / 8.0)) < 1e-9


def test_oracle_diagonal_matches_sparse_H():
    N = 9
    for ham in (dict(kind=0, J=1.0, alpha=3.0, h=1.0, periodic=0, kac=0),
                dict(kind=0, J=-2.0, alpha=1.5, h=0.3, periodic=1, kac=1),
                dict(kind=1, J1=1.0, J2=0.5, periodic=1)):
        H = _sparse_H(N, ham)
        confs = _all_confs(N)
        idx = np.random.default_rng(1).integers(0, 2 ** N, 40)
        np.testing.assert_allclose(oracle.diag(ham, confs[idx]), H.diagonal()[idx], rtol=1e-13, atol=1e-13)


def _enumeration_check(desc, params, ham, N, ground_check=True):
    confs = _all_confs(N)
    lp, _ = oracle.logpsi(desc, params, confs)
    el = oracle.eloc(desc, params, ham, confs)
    w = np.exp(2 * (lp - lp.max()))
    E_mc = (w * el).sum() / w.sum()
    psi = np.exp(lp - lp.max())
    H = _sparse_H(N, ham)
    E_ray = psi @ (H @ psi) / (psi @ psi)
    assert abs(E_mc - E_ray) < 1e-11 * max(1.0, abs(E_ray))
    if ground_check:
        assert E_ray >= _ground(H) - 1e-10
    return E_mc


@pytest.mark.parametrize("case", ["tfim_open", "tfim_ring_kac", "j1j2"])
def test_exact_enumeration_rayleigh_quotient(case):
    if case == "j1j2":
        desc, p = _fast_desc_params(seed=31, periodic=1, L=2, d=3)
        ham = dict(kind=1, J1=1.0, J2=0.5, periodic=1)
        N = 10
    elif case == "tfim_ring_kac":
        desc, p = _fast_desc_params(seed=32, periodic=1, L=3, d=2)
        ham = dict(kind=0, J=-1.5, alpha=2.0, h=0.8, periodic=1, kac=1)
        N = 9
    else:
        desc, p = _fast_desc_params(seed=33, periodic=0, L=2, d=3)
        ham = dict(kind=0, J=1.0, alpha=3.0, h=1.0, periodic=0, kac=0)
        N = 10
    _enumeration_check(desc, p, ham, N)


@pytest.mark.slow
def test_exact_enumeration_lrtfim_n16_workload():
    """The N=16 workload: all 2^16 amplitudes, E_var = Rayleigh quotient >= E_0."""
    cfg = synth.CONFIGS["lrtfim_n16"]
    _enumeration_check(cfg["desc"], synth.make_params(cfg), cfg["ham"], cfg["N"])


def test_dlogpsi_is_difference_of_forward_passes():
    desc, p = _fast_desc_params(seed=4, L=3)
    spins = synth.spins_uniform(3, 12, 8)
    sample, sites = synth.random_flips(3, 12, 20, seed=2, pair_frac=0.5)
    dl = oracle.dlogpsi(desc, p, spins, sample, sites)
    for f in range(20):
        q = spins[sample[f]].copy()
        for j in sites[f]:
            if j >= 0:
                q[j] = -q[j]
        a, _ = oracle.logpsi(desc, p, q[None])
        b, _ = oracle.logpsi(desc, p, spins[sample[f]][None])
        assert abs(dl[f] - (a[0] - b[0])) < 1e-13
