"""Dense CPU FP64 restatement of ABACUS (test tool, not the oracle).

Builds the per-sample caches with dense (N*d x N*d) propagators, then runs the
slice-local recurrence of Alg. 1 / Eqs. recur_step and recur_out with the
readings used by the library:

  * s^(0)_j = e * dsigma_j on the flipped sites F (embedding difference);
  * p^(l)_i = sum_{k in S} g^(l)_{i-k} s^(l-1)_k            (slice Toeplitz, M~)
            + sum_{j in F} dsigma_j  ell^(l)_{i,j}           (background-propagated
                                                              embedding, l >= 2)
            + sum_{m=1}^{l-2} sum_{k in S} K^(l,m)_{i,k} s^(m)_k   (links, Eq. Lmn)
    on the slice S = union_{j in F} [j-w, j+w];
  * s^(l)_i = U (dchi^(l)_i * (y^(l)_i + V p^(l)_i)),  y = V u_0 (pre-gate input);
  * dOmega_k = sum_{j in F} t_{k,j} dsigma_j + sum_l sum_{i in S} rho^(l)_{k,i} . s^(l)_i,
    rho from the adjoint of the frozen network (Eq. Tl with A folded in).

Its only job is to show, on the CPU, that these readings reproduce the
oracle's full recompute exactly (Theorem 1) and to give intermediate caches
to compare against when debugging.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

import oracle
import synth


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


class Model:
    def __init__(self, desc, params, N):
        self.desc, self.N = desc, N
        self.p = np.asarray(params, dtype=np.float64)
        sl = synth.param_slices(desc)
        d, dh, W = desc.d, desc.dh, desc.W
        self.layers = []
        for l in range(1, desc.L + 1):
            self.layers.append(dict(
                kappa=self.p[sl[f"l{l}.kappa"]].reshape(W, dh), beta=self.p[sl[f"l{l}.beta"]],
                W1=self.p[sl[f"l{l}.W1"]].reshape(dh, dh), b1=self.p[sl[f"l{l}.b1"]],
                W2=self.p[sl[f"l{l}.W2"]].reshape(d, dh), b2=self.p[sl[f"l{l}.b2"]],
                U=self.p[sl[f"l{l}.U"]].reshape(d, d), V=self.p[sl[f"l{l}.V"]].reshape(d, d)))
        self.A = self.p[sl["A"]].reshape(d, desc.dout)
        self.e = self.p[sl["e"]]
        self.taps, self.omega = oracle.plan(desc, params, N)
        # Dense per-channel Toeplitz/circulant matrices T[l][c][i, j] = g_{i-j}.
        ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        if desc.periodic:
            idx = (ii - jj) % N
        else:
            idx = ii - jj + N - 1
        self.T = [np.stack([self.taps[l][idx, c] for c in range(d)]) for l in range(desc.L)]

    def tap(self, l, r):
        """g^(l)_r (l 1-based), zero outside the open chain's range."""
        N = self.N
        if self.desc.periodic:
            return self.taps[l - 1][r % N]
        if -N < r < N:
            return self.taps[l - 1][r + N - 1]
        return np.zeros(self.desc.d)

    def spin_at(self, sp, i):
        N = self.N
        if self.desc.periodic:
            return float(sp[i % N])
        return float(sp[i]) if 0 <= i < N else 0.0

    def chi(self, l, sp, i):
        lay = self.layers[l - 1]
        w = self.desc.w
        phi = lay["beta"].copy()
        for r in range(-w, w + 1):
            phi = phi + lay["kappa"][r + w] * self.spin_at(sp, i + r)
        a = _gelu(lay["W1"] @ phi + lay["b1"])
        return lay["W2"] @ a + lay["b2"]

    def conv(self, l, v):           # v [N][d] -> G^(l) v
        return np.einsum("cij,jc->ic", self.T[l - 1], v)

    def conv_T(self, l, v):         # G^(l)^T v
        return np.einsum("cij,ic->jc", self.T[l - 1], v)

    def Dmat(self, l, chi_i):       # D_i = U diag(chi_i) V
        lay = self.layers[l - 1]
        return lay["U"] @ (chi_i[:, None] * lay["V"])


def build_caches(model: Model, sp):
    """Per-sample caches for one configuration sp[N]."""
    desc, N, d = model.desc, model.N, model.desc.d
    L = desc.L
    chi = np.stack([[model.chi(l, sp, i) for i in range(N)] for l in range(1, L + 1)])   # [L][N][d]
    h = model.e[None, :] * sp[:, None].astype(float)
    pooled = (model.omega * h).sum(0)
    u_all, y_all = [], []
    for l in range(1, L + 1):
        u = model.conv(l, h)
        y = u @ model.layers[l - 1]["V"].T
        h = (chi[l - 1] * y) @ model.layers[l - 1]["U"].T
        pooled = pooled + (model.omega * h).sum(0)
        u_all.append(u)
        y_all.append(y)
    Omega = model.A.T @ pooled
    # Adjoint: rho^(L)_k = A_k * omega ; rho^(l-1) = A_k*omega + G^(l)T D0^(l)T rho^(l).
    rho = np.zeros((L + 1, desc.dout, N, d))
    for k in range(desc.dout):
        r = model.A[:, k][None, :] * model.omega
        rho[L, k] = r
        for l in range(L, 0, -1):
            lay = model.layers[l - 1]
            z = ((r @ lay["U"]) * chi[l - 1]) @ lay["V"]        # D0^T r per site
            r = model.A[:, k][None, :] * model.omega + model.conv_T(l, z)
            rho[l - 1, k] = r
    t = np.einsum("knc,c->kn", rho[0], model.e)              # [dout][N]
    # Dense propagators on the flattened (site, channel) space.
    G = []
    Bm = []
    for l in range(1, L + 1):
        Gd = np.zeros((N * d, N * d))
        for c in range(d):
            Gd[c::d, c::d] = model.T[l - 1][c]
        Dd = np.zeros((N * d, N * d))
        for i in range(N):
            Dd[i * d:(i + 1) * d, i * d:(i + 1) * d] = model.Dmat(l, chi[l - 1][i])
        G.append(Gd)
        Bm.append(Dd @ Gd)
    # links[(l, m)] = G^(l) B^(l-1) ... B^(m+1) (full matrix), 0 <= m <= l-2.
    links = {}
    for l in range(2, L + 1):
        for m in range(0, l - 1):
            X = np.eye(N * d)
            for n in range(m + 1, l):           # apply B^(m+1) first
                X = Bm[n - 1] @ X
            links[(l, m)] = G[l - 1] @ X
    return dict(chi=chi, u=np.stack(u_all), y=np.stack(y_all), Omega=Omega, rho=rho, t=t, links=links)


def logcosh(x):
    a = np.abs(x)
    return a + np.log1p(np.exp(-2 * a)) - np.log(2.0)


def flip_ratio(model: Model, sp, cache, sites):
    """Delta log psi for flipping the given sites of sp (ABACUS recurrence)."""
    desc, N, d, L, w = model.desc, model.N, model.desc.d, model.desc.L, model.desc.w
    F = [j for j in sites if j >= 0]
    spn = sp.copy()
    for j in F:
        spn[j] = -spn[j]
    dsig = {j: float(spn[j] - sp[j]) for j in F}
    S = sorted({(j + r) % N if desc.periodic else j + r for j in F for r in range(-w, w + 1)
                if desc.periodic or 0 <= j + r < N})
    s = {0: {j: model.e * dsig[j] for j in F}}
    dOm = np.zeros(desc.dout)
    for k in range(desc.dout):
        dOm[k] = sum(cache["t"][k, j] * dsig[j] for j in F)
    for l in range(1, L + 1):
        lay = model.layers[l - 1]
        p = {}
        for i in S:
            acc = np.zeros(d)
            for k_, v in s[l - 1].items():
                acc = acc + model.tap(l, i - k_) * v
            if l >= 2:
                P = cache["links"][(l, 0)]
                for j in F:
                    col = P[:, j * d:(j + 1) * d] @ model.e
                    acc = acc + dsig[j] * col[i * d:(i + 1) * d]
            for m in range(1, l - 1):
                P = cache["links"][(l, m)]
                for k_, v in s[m].items():
                    acc = acc + P[i * d:(i + 1) * d, k_ * d:(k_ + 1) * d] @ v
            p[i] = acc
        s[l] = {}
        for i in S:
            dchi = model.chi(l, spn, i) - cache["chi"][l - 1][i]
            s[l][i] = lay["U"] @ (dchi * (cache["y"][l - 1][i] + lay["V"] @ p[i]))
            for k in range(desc.dout):
                dOm[k] += cache["rho"][l, k, i] @ s[l][i]
    Om = cache["Omega"]
    if desc.fkind == 0:
        return float(np.sum(logcosh(Om + dOm) - logcosh(Om)))
    return float(np.sum(dOm))
