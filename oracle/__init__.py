"""CPU FP64 oracle for the DysonNet local estimator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path never
does.  The C source ``oracle.c`` is a plain, slow, direct transcription of the
definitions (see its header for the equations it follows) and shares no code
with the CUDA library.

Every function here is pinned by ``tests/test_oracle_pins.py`` against what
the paper and mathematics fix (resolvent closed form, state-space scan,
periodic image sums, the Jastrow limit, exact enumeration, exact
diagonalisation, Jordan-Wigner and Majumdar-Ghosh energies).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Desc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("L", "d", "s", "w", "dh", "dout", "periodic", "fkind")]


class Ham(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("J", ctypes.c_double), ("alpha", ctypes.c_double),
                ("h", ctypes.c_double), ("J1", ctypes.c_double), ("J2", ctypes.c_double),
                ("periodic", ctypes.c_int), ("kac", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.or_nparams.argtypes = [P(Desc)]
        _lib.or_nparams.restype = ctypes.c_int
    return _lib


def _desc(desc) -> Desc:
    return Desc(desc.L, desc.d, desc.s, desc.w, desc.dh, desc.dout, desc.periodic, desc.fkind)


def _ham(ham: dict) -> Ham:
    return Ham(int(ham.get("kind", 0)), float(ham.get("J", 0.0)), float(ham.get("alpha", 0.0)),
               float(ham.get("h", 0.0)), float(ham.get("J1", 0.0)), float(ham.get("J2", 0.0)),
               int(ham.get("periodic", 0)), int(ham.get("kac", 0)))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def nparams(desc) -> int:
    d = _desc(desc)
    return _load().or_nparams(ctypes.byref(d))


def _p(params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    return p


def s4_taps(desc, s4block: np.ndarray, N: int, periodic: bool) -> np.ndarray:
    """Taps of one S4 block: open -> [2N-1][d] (row r+N-1), periodic -> [N][d]."""
    lib = _load()
    R = N if periodic else 2 * N - 1
    out = np.zeros((R, desc.d))
    blk = _p(s4block)
    lib.or_s4_taps(ctypes.byref(_desc(desc)), _ptr(blk), ctypes.c_int(N), ctypes.c_int(int(periodic)), _ptr(out))
    return out


def s4_resolvent(desc, s4block, N: int) -> np.ndarray:
    """Cauchy-kernel resolvent G_c(z_k), forward direction: complex [N][d]."""
    out = np.zeros((N, desc.d, 2))
    blk = _p(s4block)
    _load().or_s4_resolvent(ctypes.byref(_desc(desc)), _ptr(blk), ctypes.c_int(N), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def s4_circulant_fwd_complex(desc, s4block, N: int) -> np.ndarray:
    out = np.zeros((N, desc.d, 2))
    blk = _p(s4block)
    _load().or_s4_circulant_fwd_complex(ctypes.byref(_desc(desc)), _ptr(blk), ctypes.c_int(N), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def s4_scan(desc, s4block, h: np.ndarray) -> np.ndarray:
    """Open-chain state-space scan of h [N][d]."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    N = h.shape[0]
    u = np.zeros_like(h)
    blk = _p(s4block)
    _load().or_s4_scan(ctypes.byref(_desc(desc)), _ptr(blk), ctypes.c_int(N), _ptr(h), _ptr(u))
    return u


def plan(desc, params, N: int):
    """(taps [L][R][d], omega [N][d]) as used by the oracle's forward."""
    R = N if desc.periodic else 2 * N - 1
    taps = np.zeros((desc.L, R, desc.d))
    omega = np.zeros((N, desc.d))
    p = _p(params)
    _load().or_plan_export(ctypes.byref(_desc(desc)), _ptr(p), ctypes.c_int(N), _ptr(taps), _ptr(omega))
    return taps, omega


def logpsi(desc, params, spins: np.ndarray):
    """(log psi [B], Omega [B][dout]) by the full forward pass."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    B, N = spins.shape
    lp = np.zeros(B)
    om = np.zeros((B, desc.dout))
    p = _p(params)
    _load().or_logpsi(ctypes.byref(_desc(desc)), _ptr(p), ctypes.c_int(N), _ptr(spins), ctypes.c_int(B),
                      _ptr(lp), _ptr(om))
    return lp, om


def grad_logpsi(desc, params, spins: np.ndarray):
    """(log psi [B], d log psi / d theta [B][nparams]) by hand-written reverse mode."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    B, N = spins.shape
    lp = np.zeros(B)
    g = np.zeros((B, nparams(desc)))
    p = _p(params)
    _load().or_grad_logpsi(ctypes.byref(_desc(desc)), _ptr(p), ctypes.c_int(N), _ptr(spins), ctypes.c_int(B),
                           _ptr(lp), _ptr(g))
    return lp, g


def sr_matrices(O: np.ndarray, block=None):
    """Stochastic-reconfiguration matrices of log-derivatives O [B][P] (Sec. "Variational Monte
    Carlo"), centred over the samples, Oc = O - mean_b O: (Oc Oc^T / B, and for block = (k0, nk)
    Oc[:, k0:k0+nk]^T Oc[:, k0:k0+nk] / B or None).  Plain FP64 matrix products."""
    O = np.asarray(O, dtype=np.float64)
    B = O.shape[0]
    Oc = O - O.mean(axis=0, keepdims=True)
    G = Oc @ Oc.T / B
    S = None
    if block is not None:
        k0, nk = block
        Ob = Oc[:, k0:k0 + nk]
        S = Ob.T @ Ob / B
    return G, S


def _flipped(sigma: np.ndarray, site: int) -> np.ndarray:
    s = sigma.copy()
    s[site] = -s[site]
    return s


def _f(desc, om):
    """log of the amplitude function of the readout: sum_k log cosh(Omega_k) (or the identity)."""
    om = np.asarray(om, dtype=np.float64)
    if desc.fkind == 0:
        a = np.abs(om)
        return np.sum(a + np.log1p(np.exp(-2.0 * a)) - np.log(2.0), axis=-1)
    return np.sum(om, axis=-1)


def metropolis_exact(desc, params, spins: np.ndarray, sites: np.ndarray, u: np.ndarray):
    """Sequential Metropolis with exact amplitudes: for each chain and each proposal in order,
    accept iff u < min(1, |psi(sigma')|^2 / |psi(sigma)|^2).  Returns (spins, accepted)."""
    spins = np.array(spins, dtype=np.int8)
    C, K = sites.shape
    acc = np.zeros((C, K), dtype=np.int8)
    for c in range(C):
        sigma = spins[c].copy()
        for k in range(K):
            site = int(sites[c, k])
            if site < 0:
                continue
            s2 = _flipped(sigma, site)
            lp, _ = logpsi(desc, params, np.stack([sigma, s2]))
            if u[c, k] < min(1.0, np.exp(2.0 * (lp[1] - lp[0]))):
                sigma = s2
                acc[c, k] = 1
        spins[c] = sigma
    return spins, acc


def sampler_batch(desc, params, spins: np.ndarray, sites: np.ndarray, u: np.ndarray, eps: float):
    """One batch of the screened typewriter sampler (Alg. 2) in the algorithm's order.  The
    update vector of a proposal is Omega(sigma0 with the flip) - Omega(sigma0) by two full
    forward passes (what ABACUS computes exactly, Theorem 1).  Returns (spins, accepted,
    refreshes, max_err) with max_err the largest |min(1, R~) - min(1, R)| over the proposals
    decided from the scattering approximation."""
    spins = np.array(spins, dtype=np.int8)
    C, K = sites.shape
    acc = np.zeros((C, K), dtype=np.int8)
    refreshes, max_err = 0, 0.0

    def updates(ref, c):
        cfgs = [ref] + [(_flipped(ref, int(sites[c, k])) if sites[c, k] >= 0 else ref) for k in range(K)]
        _, om = logpsi(desc, params, np.stack(cfgs))
        return om[0], om[1:] - om[0]

    for c in range(C):
        sigma = spins[c].copy()
        Om, dOm = updates(sigma, c)
        for k in range(K):
            site = int(sites[c, k])
            if site < 0:
                continue
            p = min(1.0, float(np.exp(2.0 * (_f(desc, Om + dOm[k]) - _f(desc, Om)))))
            s2 = _flipped(sigma, site)
            lp, _ = logpsi(desc, params, np.stack([sigma, s2]))
            p_exact = min(1.0, float(np.exp(2.0 * (lp[1] - lp[0]))))
            if abs(u[c, k] - p) <= eps:
                take = u[c, k] < p_exact
                if take:
                    sigma = s2
                refreshes += 1
                Om, dOm = updates(sigma, c)
            else:
                max_err = max(max_err, abs(p - p_exact))
                take = u[c, k] < p
                if take:
                    sigma = s2
                    Om = Om + dOm[k]
            acc[c, k] = 1 if take else 0
        spins[c] = sigma
    return spins, acc, refreshes, max_err


def dlogpsi(desc, params, spins: np.ndarray, sample: np.ndarray, sites: np.ndarray) -> np.ndarray:
    """log psi(sigma') - log psi(sigma) for each flip set, by full recompute."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    B, N = spins.shape
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    sites = np.ascontiguousarray(sites, dtype=np.int32).reshape(-1, 2)
    F = sample.shape[0]
    out = np.zeros(F)
    p = _p(params)
    _load().or_dlogpsi(ctypes.byref(_desc(desc)), _ptr(p), ctypes.c_int(N), _ptr(spins), ctypes.c_int(B),
                       _ptr(sample), _ptr(sites), ctypes.c_int(F), _ptr(out))
    return out


def diag(ham: dict, spins: np.ndarray) -> np.ndarray:
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    lib = _load()
    lib.or_diag.restype = ctypes.c_double
    H = _ham(ham)
    return np.array([lib.or_diag(ctypes.byref(H), ctypes.c_int(spins.shape[1]), _ptr(np.ascontiguousarray(s)))
                     for s in spins])


def eloc(desc, params, ham: dict, spins: np.ndarray) -> np.ndarray:
    """Local energy per configuration, every ratio by full recompute."""
    spins = np.ascontiguousarray(spins, dtype=np.int8)
    B, N = spins.shape
    if ham.get("kind", 0) == 1 and N < 3:
        raise ValueError("J1-J2 chain needs N >= 3")
    out = np.zeros(B)
    p = _p(params)
    H = _ham(ham)
    _load().or_eloc(ctypes.byref(_desc(desc)), _ptr(p), ctypes.byref(H), ctypes.c_int(N), _ptr(spins),
                    ctypes.c_int(B), _ptr(out))
    return out
