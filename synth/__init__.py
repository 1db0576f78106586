"""Seeded synthetic inputs for the DysonNet local estimator.

This module is the only code shared by the CPU oracle and the CUDA path.  It
draws random numbers and lays them out; it performs none of the method's
arithmetic (no kernels, no activations, no energies).

Random source: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written out here from its published
definition.  Uniform doubles take the top 53 bits; normals use Box-Muller.

Parameter vector layout (float64, flat).  ``W = 2w+1``, ``dh`` = MLP width.
An *S4 block* holds one diagonal S4 kernel (Sec. "Implementation of
DysonNet", Eqs. resolvent and discretization):

    lam_re[d][s] lam_im[d][s]   continuous-time diagonal state matrix (Re < 0)
    log_dt[d]                   log of the step size Delta per channel
    b_re[d][s]  b_im[d][s]      input vector B
    cf_re[d][s] cf_im[d][s]     output vector C for the forward direction
    cb_re[d][s] cb_im[d][s]     output vector C for the backward direction

The full vector is ``L`` layer blocks followed by the final block:

    layer l:  S4 block | kappa[W][dh] | beta[dh] | W1[dh][dh] | b1[dh]
              | W2[d][dh] | b2[d] | U[d][d] | V[d][d]
    final:    S4 block (readout kernel G^f) | A[d][dout] | e[d]

Matrices are row-major with the output index first (``y = M x`` reads
``M[out][in]``).  ``kappa[r + w]`` is the window weight at offset ``r``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream; ``next_u64`` follows the published reference steps."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64_array(self, n: int) -> np.ndarray:
        # state_k = seed + k*GAMMA (mod 2^64), then the three mixing rounds.
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(self.GAMMA)
            self.state = int(z[-1]) if n > 0 else self.state
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64_array(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller on pairs of uniforms."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[0::2]                      # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
        out = np.empty(2 * m)
        out[0::2] = z[:m]
        out[1::2] = z[m:]
        return out[:n]


@dataclass(frozen=True)
class ModelDesc:
    """N-agnostic DysonNet hyper-parameters."""
    L: int
    d: int
    s: int
    w: int
    dh: int
    dout: int = 2
    periodic: int = 0
    fkind: int = 0          # 0: log cosh readout, 1: identity (Jastrow test limit)

    @property
    def W(self) -> int:
        return 2 * self.w + 1

    def as_dict(self):
        return asdict(self)


def s4_block_size(desc: ModelDesc) -> int:
    return 8 * desc.d * desc.s + desc.d


def layer_block_size(desc: ModelDesc) -> int:
    d, dh, W = desc.d, desc.dh, desc.W
    return s4_block_size(desc) + W * dh + dh + dh * dh + dh + d * dh + d + 2 * d * d


def n_params(desc: ModelDesc) -> int:
    return desc.L * layer_block_size(desc) + s4_block_size(desc) + desc.d * desc.dout + desc.d


def param_slices(desc: ModelDesc) -> dict:
    """Named slices into the flat vector (for tests that need to edit weights)."""
    d, s, dh, W = desc.d, desc.s, desc.dh, desc.W
    out = {}
    off = 0

    def take(name, n):
        nonlocal off
        out[name] = slice(off, off + n)
        off += n

    def s4(prefix):
        for nm in ("lam_re", "lam_im"):
            take(f"{prefix}.{nm}", d * s)
        take(f"{prefix}.log_dt", d)
        for nm in ("b_re", "b_im", "cf_re", "cf_im", "cb_re", "cb_im"):
            take(f"{prefix}.{nm}", d * s)

    for l in range(1, desc.L + 1):
        s4(f"l{l}")
        take(f"l{l}.kappa", W * dh)
        take(f"l{l}.beta", dh)
        take(f"l{l}.W1", dh * dh)
        take(f"l{l}.b1", dh)
        take(f"l{l}.W2", d * dh)
        take(f"l{l}.b2", d)
        take(f"l{l}.U", d * d)
        take(f"l{l}.V", d * d)
    s4("f")
    take("A", d * desc.dout)
    take("e", d)
    assert off == n_params(desc)
    return out


def init_params(desc: ModelDesc, seed: int, a_scale: float = 1.0) -> np.ndarray:
    """Random-init weights (no training; synthetic).

    S4D-Lin init: Lambda_n = -1/2 + i*pi*n; Delta log-uniform in [1e-3, 1e-1];
    B ~ CN(0, 1); C ~ CN(0, 1/s).  U, V, W1, W2 ~ N(0, 1/fan_in); kappa, e ~
    N(0, 1); A ~ N(0, a_scale^2); biases 0.
    """
    rng = SplitMix64(seed)
    p = np.zeros(n_params(desc))
    sl = param_slices(desc)
    d, s, dh, W = desc.d, desc.s, desc.dh, desc.W

    def s4(prefix):
        p[sl[f"{prefix}.lam_re"]] = -0.5
        p[sl[f"{prefix}.lam_im"]] = np.tile(math.pi * np.arange(s, dtype=np.float64), d)
        u = rng.uniform(d)
        p[sl[f"{prefix}.log_dt"]] = math.log(1e-3) + u * (math.log(1e-1) - math.log(1e-3))
        p[sl[f"{prefix}.b_re"]] = rng.normal(d * s) * math.sqrt(0.5)
        p[sl[f"{prefix}.b_im"]] = rng.normal(d * s) * math.sqrt(0.5)
        for nm in ("cf_re", "cf_im", "cb_re", "cb_im"):
            p[sl[f"{prefix}.{nm}"]] = rng.normal(d * s) * math.sqrt(0.5 / s)

    for l in range(1, desc.L + 1):
        s4(f"l{l}")
        p[sl[f"l{l}.kappa"]] = rng.normal(W * dh)
        p[sl[f"l{l}.W1"]] = rng.normal(dh * dh) / math.sqrt(dh)
        p[sl[f"l{l}.W2"]] = rng.normal(d * dh) / math.sqrt(dh)
        p[sl[f"l{l}.U"]] = rng.normal(d * d) / math.sqrt(d)
        p[sl[f"l{l}.V"]] = rng.normal(d * d) / math.sqrt(d)
    s4("f")
    p[sl["A"]] = rng.normal(d * desc.dout) * a_scale
    p[sl["e"]] = rng.normal(d)
    return p


def spins_uniform(B: int, N: int, seed: int) -> np.ndarray:
    """B uniform random +-1 configurations, int8 [B][N]."""
    u = SplitMix64(seed).uniform(B * N)
    return np.where(u < 0.5, 1, -1).astype(np.int8).reshape(B, N)


def spins_zero_magnetisation(B: int, N: int, seed: int) -> np.ndarray:
    """B configurations with N/2 up spins at random positions (Fisher-Yates)."""
    assert N % 2 == 0
    rng = SplitMix64(seed)
    out = np.empty((B, N), dtype=np.int8)
    base = np.array([1] * (N // 2) + [-1] * (N // 2), dtype=np.int8)
    for b in range(B):
        x = base.copy()
        u = rng.uniform(N)
        for i in range(N - 1, 0, -1):
            j = int(u[i] * (i + 1))
            x[i], x[j] = x[j], x[i]
        out[b] = x
    return out


def single_flips(B: int, N: int):
    """Every single flip of every sample: (sample[F], sites[F][2]) int32."""
    sample = np.repeat(np.arange(B, dtype=np.int32), N)
    sites = np.full((B * N, 2), -1, dtype=np.int32)
    sites[:, 0] = np.tile(np.arange(N, dtype=np.int32), B)
    return sample, sites


def random_flips(B: int, N: int, F: int, seed: int, pair_frac: float = 0.0,
                 max_sep: int = 2, periodic: bool = False):
    """F random flip sets: single sites, or pairs at separation 1..max_sep."""
    rng = SplitMix64(seed)
    u = rng.uniform(4 * F).reshape(F, 4)
    sample = np.minimum((u[:, 0] * B).astype(np.int32), B - 1)
    sites = np.full((F, 2), -1, dtype=np.int32)
    j = np.minimum((u[:, 1] * N).astype(np.int32), N - 1)
    sites[:, 0] = j
    is_pair = u[:, 2] < pair_frac
    sep = 1 + np.minimum((u[:, 3] * max_sep).astype(np.int32), max_sep - 1)
    if periodic:
        j2 = (j + sep) % N
    else:
        j2 = j + sep
        over = j2 >= N
        j2 = np.where(over, j - sep, j2)
    sites[is_pair, 1] = j2[is_pair]
    return sample, sites


# Named workloads (sizes, seeds and spin recipe): long-range TFIM chains of 16 and 128
# sites, the J1-J2 ring of 256 sites.
CONFIGS = {
    "lrtfim_n16": dict(desc=ModelDesc(L=2, d=8, s=8, w=2, dh=8, dout=2, periodic=0), N=16, B=64,
               weights_seed=1001, spins_seed=2001, spins="uniform", a_scale=10.0,
               ham=dict(kind=0, J=1.0, alpha=3.0, h=1.0, periodic=0, kac=0)),
    "lrtfim_n128": dict(desc=ModelDesc(L=4, d=32, s=32, w=2, dh=32, dout=2, periodic=0), N=128, B=4096,
               weights_seed=1002, spins_seed=2002, spins="uniform", a_scale=10.0,
               ham=dict(kind=0, J=1.0, alpha=3.0, h=1.0, periodic=0, kac=0)),
    "j1j2_n256": dict(desc=ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=1), N=256, B=8192,
               weights_seed=1003, spins_seed=2003, spins="zero_mag", a_scale=10.0,
               ham=dict(kind=1, J1=1.0, J2=0.5, periodic=1)),
}


def make_params(cfg: dict) -> np.ndarray:
    return init_params(cfg["desc"], cfg["weights_seed"], a_scale=cfg["a_scale"])


def make_spins(cfg: dict, B: int | None = None) -> np.ndarray:
    B = cfg["B"] if B is None else B
    if cfg["spins"] == "uniform":
        return spins_uniform(B, cfg["N"], cfg["spins_seed"])
    return spins_zero_magnetisation(B, cfg["N"], cfg["spins_seed"])


def typewriter_sites(C: int, N: int, s: int, parity: int, seed: int) -> np.ndarray:
    """Proposal sites of one typewriter half-sweep for C chains: the chain is cut into blocks
    of width s; every block of the given parity (0: even, 1: odd) gets one uniformly drawn
    site.  int32 [C][K], K = number of such blocks."""
    blocks = [b for b in range((N + s - 1) // s) if b % 2 == parity]
    u = SplitMix64(seed).uniform(C * len(blocks)).reshape(C, len(blocks))
    out = np.empty((C, len(blocks)), dtype=np.int32)
    for j, b in enumerate(blocks):
        width = min(s, N - b * s)
        out[:, j] = b * s + np.minimum((u[:, j] * width).astype(np.int64), width - 1)
    return out


def uniforms(C: int, K: int, seed: int) -> np.ndarray:
    """Uniform [0, 1) float64 [C][K] (the Metropolis test draws)."""
    return SplitMix64(seed).uniform(C * K).reshape(C, K)
