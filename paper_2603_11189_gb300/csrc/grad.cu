// Per-configuration log-derivatives O_b = d log psi(sigma_b) / d theta of the DysonNet
// (the quantities of the energy gradient and of stochastic reconfiguration, Sec.
// "Variational Monte Carlo"), by a reverse pass over the activations of the forward.
//
// With a_c = sum_k A_ck f'(Omega_k) the readout seeds dh^(l)_i = omega_i . a at every
// layer; a layer h = U (chi . V u), u = G h^(l-1), chi = W2 GELU(W1 phi + b1) + b2,
// phi = sum_r kappa_r sigma_{i+r} + beta is reversed as
//   dt = U^T dh, dy = chi . dt, dchi = y . dt, du = V^T dy,       (k_mix, adjoint)
//   dU = sum_i dh_i (chi . y)_i^T, dV = sum_i dy_i u_i^T, MLP terms (k_outer),
//   dg_r = sum_i du_i h^(l-1)_{i-r}                               (k_dtaps)
//   dh^(l-1) = G^T du + omega . a                                  (k_conv, transpose)
// and the S4 parameters follow from dg through the bilinear discretisation
// (k_s4_grad): the taps are the real part of analytic functions of each complex
// parameter z, so dJ/dRe z = Re F'(z) and dJ/dIm z = -Im F'(z).
#include <math.h>

#include "dn_internal.cuh"

namespace dn {

namespace {

template <typename T>
__device__ __forceinline__ T gelu_t(T x);
template <>
__device__ __forceinline__ double gelu_t<double>(double x) {
    return 0.5 * x * (1.0 + erf(x * 0.70710678118654752440));
}
template <>
__device__ __forceinline__ float gelu_t<float>(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678f));
}
// d/dx [x Phi(x)] = Phi(x) + x phi(x)
template <typename T>
__device__ __forceinline__ T gelu_prime_t(T x);
template <>
__device__ __forceinline__ double gelu_prime_t<double>(double x) {
    return 0.5 * (1.0 + erf(x * 0.70710678118654752440)) + x * exp(-0.5 * x * x) * 0.39894228040143267794;
}
template <>
__device__ __forceinline__ float gelu_prime_t<float>(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678f)) + x * expf(-0.5f * x * x) * 0.39894228f;
}

}  // namespace

// h0[b][i][c] = e_c sigma_{b,i}
template <typename T>
__global__ void k_h0(int N, int d, long long B, const int8_t *__restrict__ spins, const T *__restrict__ e,
                     T *__restrict__ h) {
    const long long n = B * N * d;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(x % d);
        h[x] = e[c] * (T)spins[x / d];
    }
}

// Readout: f'(Omega_k), a_c = sum_k A_ck f'(Omega_k), dA_ck = pool_c f'(Omega_k).
template <typename T>
__global__ void k_grad_readout(int d, int dout, int f_kind, int npool, int B, const double *__restrict__ A64,
                               const double *__restrict__ pooled, const double *__restrict__ Omega,
                               double *__restrict__ acoef, T *__restrict__ O, long long P, long long offA) {
    const int b = blockIdx.x, c = threadIdx.x;
    if (b >= B || c >= d) return;
    double pc = 0.0;
    for (int q = 0; q < npool; ++q) pc += pooled[((long long)b * npool + q) * d + c];
    double a = 0.0;
    for (int k = 0; k < dout; ++k) {
        const double om = Omega[(long long)b * dout + k];
        const double fp = f_kind == 0 ? tanh(om) : 1.0;
        O[(long long)b * P + offA + c * dout + k] = (T)(pc * fp);
        a += A64[c * dout + k] * fp;
    }
    acoef[(long long)b * d + c] = a;
}

// dst[b][i][c] (+)= omega_{i,c} a_{b,c}
template <typename T>
__global__ void k_add_omega(int N, int d, long long B, const T *__restrict__ omega, const double *__restrict__ acoef,
                            T *__restrict__ dst, int add) {
    const long long n = B * N * d;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(x % d);
        const long long bi = x / d;
        const int i = (int)(bi % N);
        const long long b = bi / N;
        const T v = omega[(long long)i * d + c] * (T)acoef[b * d + c];
        dst[x] = add ? dst[x] + v : v;
    }
}

// Per (sample, site) of layer l: the MLP of the vertex recomputed from the spins and its
// reverse, plus the operands of the per-sample outer-product sums.
//   in:  dtv = U^T dh, y, chi (layer l)
//   out: tY = chi . y, dy = chi . dt, dchi = y . dt  [B][N][d];
//        a1 = GELU(z), phi, dz = (W2^T dchi) . GELU'(z), dphi = W1^T dz  [B][N][dh];
//        win[B][N][W] = sigma_{i+r}, r = -w..w.
// One CTA per (sample, tile of kMbTile sites).  W1^T and W2^T of the layer are staged in
// shared memory once per CTA; the site-major operands are kept transposed ([k][site]) so
// that a thread (output e, group of 8 sites) reads its 8 sites with two 16-byte loads
// (the same address for the whole warp) and its weight row without bank conflicts.
constexpr int kMbTile = 32, kMbSub = 8, kMbTPB = 4;   // sites per tile, per thread group, tiles per CTA

template <typename T>
__global__ void __launch_bounds__(256) k_mlp_back(Geom g, int l, Weights<T> w, const int8_t *__restrict__ spins,
                                                  const T *__restrict__ chi, const T *__restrict__ y,
                                                  const T *__restrict__ dtv, T *__restrict__ tY, T *__restrict__ dy,
                                                  T *__restrict__ dchi, T *__restrict__ a1, T *__restrict__ phi,
                                                  T *__restrict__ dz, T *__restrict__ dphi, T *__restrict__ win,
                                                  int nb) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, dh = g.dh, L = g.L, wd = g.w, W = g.W;
    // Row strides dh+1 and d+1: a warp reading along either index of the weights hits
    // distinct banks.
    T *W1s = reinterpret_cast<T *>(smraw);     // [f][e] = W1[e][f], row stride dh + 1
    T *W2s = W1s + dh * (dh + 1);              // [e][c] = W2[c][e], row stride d + 1
    T *phT = W2s + dh * (d + 1);               // [f][tile]
    T *zT = phT + dh * kMbTile;                // [e][tile]  z, then dz
    T *dcT = zT + dh * kMbTile;                // [c][tile]  dchi
    const int ntile = (N + kMbTile - 1) / kMbTile;
    const T *kap = w.kappa + (long long)(l - 1) * W * dh;
    const T *beta = w.beta + (long long)(l - 1) * dh;
    const T *b1 = w.b1 + (long long)(l - 1) * dh;
    for (int q = threadIdx.x; q < dh * dh; q += blockDim.x)
        W1s[(q / dh) * (dh + 1) + q % dh] = w.W1T[(long long)(l - 1) * dh * dh + q];
    for (int q = threadIdx.x; q < dh * d; q += blockDim.x)
        W2s[(q / d) * (d + 1) + q % d] = w.W2T[(long long)(l - 1) * dh * d + q];
    for (int it = 0; it < kMbTPB; ++it) {
        const long long item = (long long)blockIdx.x * kMbTPB + it;
        if (item >= (long long)nb * ntile) break;
        __syncthreads();   // the previous tile's reads of the staged activations (and the weight staging) are done
        const long long b = item / ntile;
        const int i0 = (int)(item % ntile) * kMbTile;
        const int ns = min(kMbTile, N - i0);
        const int8_t *sp = spins + b * N;
        const long long fb = (b * N + i0);          // first row of the tile in [B][N][.] arrays
        const T *chib = chi + ((b * L + (l - 1)) * N + i0) * d;
        auto spin = [&](int j) -> T {
            if (g.periodic) return (T)sp[((j % N) + N) % N];
            return (j >= 0 && j < N) ? (T)sp[j] : (T)0;
        };
        for (int idx = threadIdx.x; idx < kMbTile * dh; idx += blockDim.x) {
            const int t = idx / dh, e = idx % dh, i = i0 + t;
            T acc = 0;
            if (t < ns) {
                acc = beta[e];
                for (int r = -wd; r <= wd; ++r) acc += kap[(r + wd) * dh + e] * spin(i + r);
                phi[(fb + t) * dh + e] = acc;
            }
            phT[e * kMbTile + t] = acc;
        }
        for (int idx = threadIdx.x; idx < ns * W; idx += blockDim.x) {
            const int t = idx / W, r = idx % W;
            win[(fb + t) * W + r] = spin(i0 + t + r - wd);
        }
        for (int idx = threadIdx.x; idx < kMbTile * d; idx += blockDim.x) {
            const int t = idx / d, c = idx % d;
            T v = 0;
            if (t < ns) {
                const long long o = (fb + t) * d + c;
                const T yv = y[o], dv = dtv[o], xv = chib[(long long)t * d + c];
                tY[o] = xv * yv;
                dy[o] = xv * dv;
                v = yv * dv;
                dchi[o] = v;
            }
            dcT[c * kMbTile + t] = v;
        }
        __syncthreads();
        constexpr int nsub = kMbTile / kMbSub;
        // z = W1 phi + b1 (into zT), a1 = GELU(z)
        for (int q = threadIdx.x; q < dh * nsub; q += blockDim.x) {
            const int e = q % dh, t0 = (q / dh) * kMbSub;
            T acc[kMbSub];
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) acc[u] = b1[e];
            for (int f = 0; f < dh; ++f) {
                const T wv = W1s[f * (dh + 1) + e];
                const T *pp = phT + f * kMbTile + t0;
    #pragma unroll
                for (int u = 0; u < kMbSub; ++u) acc[u] += wv * pp[u];
            }
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) {
                zT[e * kMbTile + t0 + u] = acc[u];
                if (t0 + u < ns) a1[(fb + t0 + u) * dh + e] = gelu_t<T>(acc[u]);
            }
        }
        __syncthreads();
        // dz = (W2^T dchi) . GELU'(z) (in place of z)
        for (int q = threadIdx.x; q < dh * nsub; q += blockDim.x) {
            const int e = q % dh, t0 = (q / dh) * kMbSub;
            T acc[kMbSub];
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) acc[u] = 0;
            for (int c = 0; c < d; ++c) {
                const T wv = W2s[e * (d + 1) + c];
                const T *pp = dcT + c * kMbTile + t0;
    #pragma unroll
                for (int u = 0; u < kMbSub; ++u) acc[u] += wv * pp[u];
            }
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) {
                const T v = acc[u] * gelu_prime_t<T>(zT[e * kMbTile + t0 + u]);
                acc[u] = v;
                if (t0 + u < ns) dz[(fb + t0 + u) * dh + e] = v;
            }
            // (e, t0) belongs to this thread alone: overwrite z with dz in place.
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) zT[e * kMbTile + t0 + u] = acc[u];
        }
        __syncthreads();
        // dphi = W1^T dz
        for (int q = threadIdx.x; q < dh * nsub; q += blockDim.x) {
            const int f = q % dh, t0 = (q / dh) * kMbSub;
            T acc[kMbSub];
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u) acc[u] = 0;
            for (int e = 0; e < dh; ++e) {
                const T wv = W1s[f * (dh + 1) + e];
                const T *pp = zT + e * kMbTile + t0;
    #pragma unroll
                for (int u = 0; u < kMbSub; ++u) acc[u] += wv * pp[u];
            }
    #pragma unroll
            for (int u = 0; u < kMbSub; ++u)
                if (t0 + u < ns) dphi[(fb + t0 + u) * dh + f] = acc[u];
        }
    }
}

// Per-sample sums of outer products over the sites:
//   O[b][off + a ldo + c] = sum_i X[b][i][a] Y[b][i][c]   (Y null: Y = 1, one column)
// X, Y rows of length dx, dy (row stride = length, sample stride N rows).  One CTA per
// (sample, 32 x 32 output tile); the sites stream through shared memory 32 at a time.
constexpr int kOpT = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_outer(int N, int dx, int dyc, const T *__restrict__ X,
                                               const T *__restrict__ Y, T *__restrict__ O, long long P, long long off,
                                               int ldo) {
    __shared__ T xs[kOpT][kOpT + 1], ys[kOpT][kOpT + 1];
    const int ta = (dx + kOpT - 1) / kOpT, tc = (dyc + kOpT - 1) / kOpT;
    const long long b = blockIdx.x / ((long long)ta * tc);
    const int rem = (int)(blockIdx.x % ((long long)ta * tc));
    const int a0 = (rem / tc) * kOpT, c0 = (rem % tc) * kOpT;
    const int tx = threadIdx.x % kOpT, ty = threadIdx.x / kOpT;   // ty in [0, 8): 4 rows each
    T acc[4] = {0, 0, 0, 0};
    const T *Xb = X + b * (long long)N * dx;
    const T *Yb = Y ? Y + b * (long long)N * dyc : nullptr;
    for (int i0 = 0; i0 < N; i0 += kOpT) {
        for (int q = threadIdx.x; q < kOpT * kOpT; q += blockDim.x) {
            const int ii = q / kOpT, jj = q % kOpT, i = i0 + ii;
            xs[ii][jj] = (i < N && a0 + jj < dx) ? Xb[(long long)i * dx + a0 + jj] : (T)0;
            ys[ii][jj] = (i < N && c0 + jj < dyc) ? (Yb ? Yb[(long long)i * dyc + c0 + jj] : (T)1) : (T)0;
        }
        __syncthreads();
#pragma unroll 4
        for (int ii = 0; ii < kOpT; ++ii) {
            const T yv = ys[ii][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += xs[ii][ty * 4 + q] * yv;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = a0 + ty * 4 + q, c = c0 + tx;
        if (a < dx && c < dyc) O[b * P + off + (long long)a * ldo + c] = acc[q];
    }
}

// dg[b][r][c] = sum_i du[b][i][c] h[b][i - r][c]  (taps layout: row r + N - 1 open, r periodic)
constexpr int kDtCt = 8;

template <typename T>
__global__ void k_dtaps(int N, int d, int periodic, int R, const T *__restrict__ du, const T *__restrict__ h,
                        T *__restrict__ dg) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *su = reinterpret_cast<T *>(smraw);   // [N][CT]
    T *sh = su + (size_t)N * kDtCt;         // [N][CT]
    const int nct = (d + kDtCt - 1) / kDtCt;
    const long long b = blockIdx.x / nct;
    const int c0 = (int)(blockIdx.x % nct) * kDtCt;
    for (int q = threadIdx.x; q < N * kDtCt; q += blockDim.x) {
        const int i = q / kDtCt, c = q % kDtCt;
        const bool ok = c0 + c < d;
        su[q] = ok ? du[(b * N + i) * d + c0 + c] : (T)0;
        sh[q] = ok ? h[(b * N + i) * d + c0 + c] : (T)0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < R * kDtCt; q += blockDim.x) {
        const int row = q / kDtCt, c = q % kDtCt;
        if (c0 + c >= d) continue;
        T acc = 0;
        if (!periodic) {
            const int r = row - (N - 1);
            const int lo = r > 0 ? r : 0, hi = r < 0 ? N - 1 + r : N - 1;   // 0 <= i - r < N
            for (int i = lo; i <= hi; ++i) acc += su[i * kDtCt + c] * sh[(i - r) * kDtCt + c];
        } else {
            const int r = row;
            for (int i = 0; i < N; ++i) {
                int j = i - r;
                if (j < 0) j += N;
                acc += su[i * kDtCt + c] * sh[j * kDtCt + c];
            }
        }
        dg[((long long)b * R + row) * d + c0 + c] = acc;
    }
}

// de[b][c] = sum_i dh0[b][i][c] sigma_{b,i}
template <typename T>
__global__ void k_grad_e(int N, int d, int B, const T *__restrict__ dh0, const int8_t *__restrict__ spins,
                         T *__restrict__ O, long long P, long long off) {
    const int b = blockIdx.x, c = threadIdx.x;
    if (b >= B || c >= d) return;
    T acc = 0;
    for (int i = 0; i < N; ++i) acc += dh0[((long long)b * N + i) * d + c] * (T)spins[(long long)b * N + i];
    O[(long long)b * P + off + c] = acc;
}

// Readout kernel: d omega_{i,c} = a_c sum_l h^(l)_{i,c}; omega_{i,c} = (1/N) sum_k g^f_{k-i,c}, so
// open: dg^f_r = (1/N) sum over i with 0 <= i + r < N; periodic: dg^f_r = (1/N) sum_i for every r.
template <typename T>
__global__ void k_grad_gf(int N, int d, int L, int periodic, int R, long long B, const T *__restrict__ h,
                          long long lstride, const double *__restrict__ acoef, T *__restrict__ dgf) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= B * d) return;
    const long long b = x / d;
    const int c = (int)(x % d);
    const double a = acoef[b * d + c];
    auto domega = [&](int i) -> double {
        double s = 0.0;
        for (int l = 0; l <= L; ++l) s += (double)h[l * lstride + (b * N + i) * d + c];
        return a * s;
    };
    double total = 0.0;
    for (int i = 0; i < N; ++i) total += domega(i);
    T *out = dgf + b * (long long)R * d + c;
    if (periodic) {
        for (int r = 0; r < N; ++r) out[(long long)r * d] = (T)(total / N);
        return;
    }
    double S = 0.0;
    for (int k = 0; k < N; ++k) {
        S += domega(k);
        out[(long long)(N - 1 - k + N - 1) * d] = (T)(S / N);            // r = N-1-k >= 0: i in [0, k]
        if (k + 1 <= N - 1) out[(long long)(-(k + 1) + N - 1) * d] = (T)((total - S) / N);   // r = -(k+1)
    }
}

// Powers lam_bar^q, q = 0..N, of every mode of the S4 blocks (complex, interleaved re/im):
// pw[blk][c][n][q][2], blocks 0..L-1 the layers, L the readout kernel.
template <typename T>
__global__ void k_s4_pow(const double *__restrict__ params, int L, int d, int s, long long layer_size,
                         long long final_off, int N, T *__restrict__ pw) {
    const long long n_all = (long long)(L + 1) * d * s * (N + 1);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n_all; x += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(x % (N + 1));
        const long long cn = x / (N + 1);
        const int n = (int)(cn % s);
        const long long bc = cn / s;
        const int c = (int)(bc % d), blk = (int)(bc / d);
        const double *p = params + (blk < L ? (long long)blk * layer_size : final_off);
        const long long ds = (long long)d * s, k = (long long)c * s + n;
        const double dt = exp(p[2 * ds + c]);
        const double ar = 0.5 * dt * p[k], ai = 0.5 * dt * p[ds + k];
        const double dr = 1.0 - ar, di = -ai, dd = dr * dr + di * di;
        const double lr = ((1.0 + ar) * dr + ai * di) / dd, li = (ai * dr - (1.0 + ar) * di) / dd;
        const double lnrho = 0.5 * log(lr * lr + li * li), th = atan2(li, lr);
        double sn, cs;
        sincos(q * th, &sn, &cs);
        const double mag = exp(q * lnrho);
        pw[2 * x] = (T)(mag * cs);
        pw[2 * x + 1] = (T)(mag * sn);
    }
}

// S4 parameters of one block from J = sum_r dg_r g_r (per sample).  One CTA per (channel c,
// tile of kSgB samples); thread (sample, mode) accumulates the power sums over the taps,
// then forms the parameter derivatives in FP64.
constexpr int kSgB = 16, kSgN = 16;

template <typename T>
__global__ void __launch_bounds__(kSgB * kSgN) k_s4_grad(const double *__restrict__ blk, int d, int s, int N,
                                                        int periodic, int R, int B, const T *__restrict__ dg,
                                                        const T *__restrict__ pw, T *__restrict__ O, long long P,
                                                        long long off) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sdg = reinterpret_cast<T *>(smraw);              // [kSgB][R]
    T *spw = sdg + (size_t)kSgB * R;                    // [kSgN][N+1][2]
    double *sdt = reinterpret_cast<double *>(spw + (size_t)kSgN * (N + 1) * 2);   // [kSgB][kSgN]
    const int nbt = (B + kSgB - 1) / kSgB;
    const int c = blockIdx.x / nbt, b0 = (blockIdx.x % nbt) * kSgB;
    const int tb = threadIdx.x / kSgN, tn = threadIdx.x % kSgN;
    const int b = b0 + tb;
    for (int q = threadIdx.x; q < kSgB * R; q += blockDim.x) {
        const int bb = q / R, r = q % R;
        sdg[q] = (b0 + bb < B) ? dg[((long long)(b0 + bb) * R + r) * d + c] : (T)0;
    }
    const long long ds = (long long)d * s;
    const double *lre = blk, *lim = blk + ds, *logdt = blk + 2 * ds;
    const double *bre = logdt + d, *bim = bre + ds, *cfre = bim + ds, *cfim = cfre + ds, *cbre = cfim + ds,
                 *cbim = cbre + ds;
    const double dt = exp(logdt[c]);
    double gdt = 0.0;
    const T *dgb = sdg + (size_t)tb * R;
    for (int n0 = 0; n0 < s; n0 += kSgN) {
        __syncthreads();
        for (int q = threadIdx.x; q < kSgN * (N + 1) * 2; q += blockDim.x) {
            const int nn = q / ((N + 1) * 2), rest = q % ((N + 1) * 2);
            spw[q] = (n0 + nn < s) ? pw[(((long long)c * s + n0 + nn) * (N + 1)) * 2 + rest] : (T)0;
        }
        __syncthreads();
        const int n = n0 + tn;
        if (n >= s || b >= B) continue;
        const T *p = spw + (size_t)tn * (N + 1) * 2;
        // power sums (T accumulation), see the oracle's derivation
        T a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0, a3r = 0, a3i = 0;
        if (!periodic) {
            for (int q = 0; q <= N - 1; ++q) {           // r = q >= 0: Gp, Hp
                const T x = dgb[q + N - 1];
                a0r += x * p[2 * q];
                a0i += x * p[2 * q + 1];
                if (q > 0) {
                    a2r += x * (T)q * p[2 * (q - 1)];
                    a2i += x * (T)q * p[2 * (q - 1) + 1];
                }
            }
            for (int q = 1; q <= N - 1; ++q) {           // r = -q: Gm, Hm
                const T x = dgb[N - 1 - q];
                a1r += x * p[2 * q];
                a1i += x * p[2 * q + 1];
                a3r += x * (T)q * p[2 * (q - 1)];
                a3i += x * (T)q * p[2 * (q - 1) + 1];
            }
        } else {
            for (int r = 0; r < N; ++r) {                // Sf, Sb, Sf1, Sb1
                const T x = dgb[r];
                a0r += x * p[2 * r];
                a0i += x * p[2 * r + 1];
                a1r += x * p[2 * (N - r)];
                a1i += x * p[2 * (N - r) + 1];
                if (r > 0) {
                    a2r += x * (T)r * p[2 * (r - 1)];
                    a2i += x * (T)r * p[2 * (r - 1) + 1];
                }
                a3r += x * (T)(N - r) * p[2 * (N - r - 1)];
                a3i += x * (T)(N - r) * p[2 * (N - r - 1) + 1];
            }
        }
        // FP64 epilogue: complex arithmetic by hand (re, im pairs)
        const long long k = (long long)c * s + n;
        const double Lr = lre[k], Li = lim[k], Br = bre[k], Bi = bim[k];
        const double Cfr = cfre[k], Cfi = cfim[k], Cbr = cbre[k], Cbi = cbim[k];
        // den = 1 - dt Lam / 2, lam_bar = (1 + dt Lam/2)/den, B_bar = dt B/den
        const double denr = 1.0 - 0.5 * dt * Lr, deni = -0.5 * dt * Li, dd = denr * denr + deni * deni;
        const double idr = denr / dd, idi = -deni / dd;                        // 1/den
        const double bbr = dt * (Br * idr - Bi * idi), bbi = dt * (Br * idi + Bi * idr);
        auto cmul = [](double xr, double xi, double yr, double yi, double &zr, double &zi) {
            zr = xr * yr - xi * yi;
            zi = xr * yi + xi * yr;
        };
        double wfr, wfi, wbr, wbi, Qr, Qi, Er, Ei;
        if (!periodic) {
            // wf = B_bar Gp, wb = B_bar Gm, Q = Cf Gp + Cb Gm, E = B_bar (Cf Hp + Cb Hm)
            cmul(bbr, bbi, a0r, a0i, wfr, wfi);
            cmul(bbr, bbi, a1r, a1i, wbr, wbi);
            double t1r, t1i, t2r, t2i;
            cmul(Cfr, Cfi, a0r, a0i, t1r, t1i);
            cmul(Cbr, Cbi, a1r, a1i, t2r, t2i);
            Qr = t1r + t2r;
            Qi = t1i + t2i;
            cmul(Cfr, Cfi, a2r, a2i, t1r, t1i);
            cmul(Cbr, Cbi, a3r, a3i, t2r, t2i);
            cmul(bbr, bbi, t1r + t2r, t1i + t2i, Er, Ei);
        } else {
            // inv = 1/(1 - lam^N); S = Cf Sf + Cb Sb, S1 = Cf Sf1 + Cb Sb1
            const double lNr = (double)p[2 * N], lNi = (double)p[2 * N + 1];
            const double onr = 1.0 - lNr, oni = -lNi, oo = onr * onr + oni * oni;
            const double ivr = onr / oo, ivi = -oni / oo;
            double t1r, t1i, t2r, t2i, Sr, Si, S1r, S1i;
            cmul(Cfr, Cfi, a0r, a0i, t1r, t1i);
            cmul(Cbr, Cbi, a1r, a1i, t2r, t2i);
            Sr = t1r + t2r;
            Si = t1i + t2i;
            cmul(Cfr, Cfi, a2r, a2i, t1r, t1i);
            cmul(Cbr, Cbi, a3r, a3i, t2r, t2i);
            S1r = t1r + t2r;
            S1i = t1i + t2i;
            double ur, ui;
            cmul(bbr, bbi, ivr, ivi, ur, ui);           // B_bar / (1 - lam^N)
            cmul(ur, ui, a0r, a0i, wfr, wfi);
            cmul(ur, ui, a1r, a1i, wbr, wbi);
            cmul(Sr, Si, ivr, ivi, Qr, Qi);
            // E = B_bar [S1 inv + S N lam^(N-1) inv^2]
            const double lN1r = (double)p[2 * (N - 1)], lN1i = (double)p[2 * (N - 1) + 1];
            double v1r, v1i, v2r, v2i, iv2r, iv2i;
            cmul(S1r, S1i, ivr, ivi, v1r, v1i);
            cmul(ivr, ivi, ivr, ivi, iv2r, iv2i);
            cmul(Sr, Si, lN1r, lN1i, v2r, v2i);
            cmul(v2r * N, v2i * N, iv2r, iv2i, v2r, v2i);
            cmul(bbr, bbi, v1r + v2r, v1i + v2i, Er, Ei);
        }
        // den^2, then dLam = E dt/den^2 + Q dt^2 B / (2 den^2), dB = Q dt/den, dDt = (E Lam + Q B)/den^2
        double i2r, i2i;
        cmul(idr, idi, idr, idi, i2r, i2i);
        double t1r, t1i, t2r, t2i, dLr, dLi, dBr, dBi, dDr, dDi;
        cmul(Er, Ei, i2r * dt, i2i * dt, t1r, t1i);
        cmul(Qr, Qi, Br, Bi, t2r, t2i);
        cmul(t2r, t2i, i2r * 0.5 * dt * dt, i2i * 0.5 * dt * dt, t2r, t2i);
        dLr = t1r + t2r;
        dLi = t1i + t2i;
        cmul(Qr, Qi, idr * dt, idi * dt, dBr, dBi);
        cmul(Er, Ei, Lr, Li, t1r, t1i);
        cmul(Qr, Qi, Br, Bi, t2r, t2i);
        cmul(t1r + t2r, t1i + t2i, i2r, i2i, dDr, dDi);
        gdt += dDr;
        T *Ob = O + (long long)b * P + off;
        Ob[k] = (T)dLr;
        Ob[ds + k] = (T)(-dLi);
        Ob[2 * ds + d + k] = (T)dBr;
        Ob[3 * ds + d + k] = (T)(-dBi);
        Ob[4 * ds + d + k] = (T)wfr;
        Ob[5 * ds + d + k] = (T)(-wfi);
        Ob[6 * ds + d + k] = (T)wbr;
        Ob[7 * ds + d + k] = (T)(-wbi);
    }
    // log_dt: sum over the modes (threads tn of the sample, in a fixed order)
    sdt[tb * kSgN + tn] = gdt;
    __syncthreads();
    if (tn == 0 && b < B) {
        double acc = 0.0;
        for (int q = 0; q < kSgN; ++q) acc += sdt[tb * kSgN + q];
        O[(long long)b * P + off + 2 * ds + c] = (T)(acc * dt);
    }
}

// vjp[k] += sum_b w_b O[b][k] (FP64 accumulation, samples in order)
template <typename T>
__global__ void k_vjp(const T *__restrict__ O, const double *__restrict__ wts, int B, long long P,
                      double *__restrict__ vjp) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b) acc += wts[b] * (double)O[(long long)b * P + k];
        vjp[k] += acc;
    }
}

// Stochastic-reconfiguration matrices from the log-derivatives, centred over the samples.
// Column means m[k] = (1/B) sum_b O[b][k] (FP64).
template <typename T>
__global__ void k_colmean(const T *__restrict__ O, int B, long long P, T *__restrict__ m) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b) acc += (double)O[(long long)b * P + k];
        m[k] = (T)(acc / B);
    }
}

// S[a][c] = scale sum_k (X[a][k] - m_a|k) (X[c][k] - m_a|k) for a, c < n, with X[a][k] at
// X + a sa + k sk; the mean (in the precision of X) is m[k] (mean_by_k) or m[a].  One CTA per
// 128 x 128 tile with c0 >= a0 (the other half is mirrored); K streams through shared
// memory 16 at a time, the next slice's loads in flight while the current one is used.
// Each thread keeps an 8 x 8 block in registers; in FP32 the block is added every kGrFold
// terms into a second FP32 sum held in shared memory (two-level summation: the error grows
// with sqrt(kGrFold) + sqrt(K / kGrFold) instead of sqrt(K)).
constexpr int kGrT = 128, kGrK = 16, kGrFold = 512, kGrPad = kGrT + 4;
constexpr int kGrLd = kGrK * kGrT / 256;   // elements of each operand a thread stages per slice

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T *__restrict__ X, long long sa, long long sk, int n, long long K,
                                              const T *__restrict__ m, int mean_by_k, double scale,
                                              double *__restrict__ S) {
    __shared__ __align__(16) T xa[kGrK][kGrPad];
    __shared__ __align__(16) T xc[kGrK][kGrPad];
    extern __shared__ __align__(16) unsigned char smfold[];
    T *fold = reinterpret_cast<T *>(smfold);     // [64][blockDim]: thread-private second-level sums
    const int nt = (n + kGrT - 1) / kGrT;
    int t = blockIdx.x, ta = 0;
    while (t >= nt - ta) {
        t -= nt - ta;
        ++ta;
    }
    const int tc = ta + t;
    const int a0 = ta * kGrT, c0 = tc * kGrT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    constexpr bool kFold = sizeof(T) == 4;
    // This thread's staging slots: (kk, r) for q = threadIdx.x + 256 u.
    int skk[kGrLd], sr[kGrLd];
#pragma unroll
    for (int u = 0; u < kGrLd; ++u) {
        const int q = threadIdx.x + 256 * u;
        if (sk == 1) {           // K contiguous in memory: 16 threads read one row's slice
            sr[u] = q / kGrK;
            skk[u] = q % kGrK;
        } else {
            skk[u] = q / kGrT;
            sr[u] = q % kGrT;
        }
    }
    T pa[kGrLd], pc[kGrLd];
    auto fetch = [&](long long k0) {
#pragma unroll
        for (int u = 0; u < kGrLd; ++u) {
            const long long k = k0 + skk[u];
            const int a = a0 + sr[u], c = c0 + sr[u];
            T va = 0, vc = 0;
            if (k < K) {
                if (a < n) va = X[a * sa + k * sk] - (mean_by_k ? m[k] : m[a]);
                if (c < n) vc = X[c * sa + k * sk] - (mean_by_k ? m[k] : m[c]);
            }
            pa[u] = va;
            pc[u] = vc;
        }
    };
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0;
    if constexpr (kFold) {
        for (int q = 0; q < 64; ++q) fold[q * blockDim.x + threadIdx.x] = 0;
    }
    int since = 0;
    fetch(0);
    for (long long k0 = 0; k0 < K; k0 += kGrK) {
#pragma unroll
        for (int u = 0; u < kGrLd; ++u) {
            xa[skk[u]][sr[u]] = pa[u];
            xc[skk[u]][sr[u]] = pc[u];
        }
        __syncthreads();
        if (k0 + kGrK < K) fetch(k0 + kGrK);
#pragma unroll 2
        for (int kk = 0; kk < kGrK; ++kk) {
            T av[8], cv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                av[i] = xa[kk][ty * 8 + i];
                cv[i] = xc[kk][tx * 8 + i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * cv[j];
        }
        __syncthreads();
        if constexpr (kFold) {
            since += kGrK;
            if (since >= kGrFold) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        fold[(i * 8 + j) * blockDim.x + threadIdx.x] += acc[i][j];
                        acc[i][j] = 0;
                    }
                since = 0;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int a = a0 + ty * 8 + i, c = c0 + tx * 8 + j;
            if (a < n && c < n) {
                double v = (double)acc[i][j];
                if constexpr (kFold) v += (double)fold[(i * 8 + j) * blockDim.x + threadIdx.x];
                v *= scale;
                S[(long long)a * n + c] = v;
                S[(long long)c * n + a] = v;
            }
        }
}

// ------------------------------------------------------------------ host --
static unsigned grid_of(long long n) {
    long long g = (n + 255) / 256;
    if (g > 65535LL * 8) g = 65535LL * 8;
    return (unsigned)(g > 0 ? g : 1);
}

template <typename T>
cudaError_t launch_h0(int N, int d, int B, const int8_t *spins, const T *e, T *h, cudaStream_t st) {
    ProfScope _ps("k_h0", st);
    k_h0<T><<<grid_of((long long)B * N * d), 256, 0, st>>>(N, d, B, spins, e, h);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_readout(const Geom &g, int f_kind, int npool, int B, const double *A64, const double *pooled,
                                const double *Omega, double *acoef, T *O, long long P, long long offA,
                                cudaStream_t st) {
    ProfScope _ps("k_grad_readout", st);
    k_grad_readout<T><<<B, ((g.d + 31) / 32) * 32, 0, st>>>(g.d, g.dout, f_kind, npool, B, A64, pooled, Omega, acoef,
                                                            O, P, offA);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_omega(const Geom &g, int B, const T *omega, const double *acoef, T *dst, bool add,
                             cudaStream_t st) {
    ProfScope _ps("k_add_omega", st);
    k_add_omega<T><<<grid_of((long long)B * g.N * g.d), 256, 0, st>>>(g.N, g.d, B, omega, acoef, dst, add ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mlp_back(const Geom &g, int l, const Weights<T> &w, const int8_t *spins, int B, const T *chi,
                            const T *y, const T *dtv, const GradScratch<T> &s, cudaStream_t st) {
    const int ntile = (g.N + kMbTile - 1) / kMbTile;
    const size_t smem =
        ((size_t)g.dh * (g.dh + 1) + (size_t)g.dh * (g.d + 1) + (size_t)kMbTile * (2 * g.dh + g.d)) * sizeof(T);
    if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(k_mlp_back<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    ProfScope _ps("k_mlp_back", st);
    const long long groups = ((long long)B * ntile + kMbTPB - 1) / kMbTPB;
    k_mlp_back<T><<<(unsigned)groups, 256, smem, st>>>(g, l, w, spins, chi, y, dtv, s.tY, s.dy, s.dchi, s.a1, s.phi,
                                                       s.dz, s.dphi, s.win, B);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_outer(int N, int B, int dx, int dyc, const T *X, const T *Y, T *O, long long P, long long off,
                         int ldo, cudaStream_t st) {
    const long long tiles = (long long)((dx + kOpT - 1) / kOpT) * ((dyc + kOpT - 1) / kOpT);
    ProfScope _ps("k_outer", st);
    k_outer<T><<<(unsigned)(B * tiles), 256, 0, st>>>(N, dx, dyc, X, Y, O, P, off, ldo);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dtaps(const Geom &g, int B, const T *du, const T *h, T *dg, cudaStream_t st) {
    const size_t smem = 2 * (size_t)g.N * kDtCt * sizeof(T);
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(k_dtaps<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int nct = (g.d + kDtCt - 1) / kDtCt;
    ProfScope _ps("k_dtaps", st);
    k_dtaps<T><<<(unsigned)((long long)B * nct), 256, smem, st>>>(g.N, g.d, g.periodic, g.R, du, h, dg);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_e(const Geom &g, int B, const T *dh0, const int8_t *spins, T *O, long long P, long long off,
                          cudaStream_t st) {
    ProfScope _ps("k_grad_e", st);
    k_grad_e<T><<<B, ((g.d + 31) / 32) * 32, 0, st>>>(g.N, g.d, B, dh0, spins, O, P, off);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_gf(const Geom &g, int B, const T *h, long long lstride, const double *acoef, T *dgf,
                           cudaStream_t st) {
    ProfScope _ps("k_grad_gf", st);
    k_grad_gf<T><<<(unsigned)(((long long)B * g.d + 127) / 128), 128, 0, st>>>(g.N, g.d, g.L, g.periodic, g.R, B, h,
                                                                              lstride, acoef, dgf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_s4_pow(const dn_model *m, int N, T *pw, cudaStream_t st) {
    const dn_model_desc &D = m->desc;
    ProfScope _ps("k_s4_pow", st);
    k_s4_pow<T><<<grid_of((long long)(D.L + 1) * D.d * D.s * (N + 1)), 256, 0, st>>>(
        m->params_dev, D.L, D.d, D.s, m->layer_size, (long long)D.L * m->layer_size, N, pw);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_s4_grad(const dn_model *m, int blk, int N, int B, const T *dg, const T *pw, T *O, long long P,
                           cudaStream_t st) {
    const dn_model_desc &D = m->desc;
    const int R = D.periodic ? N : 2 * N - 1;
    const long long boff = blk < D.L ? (long long)blk * m->layer_size : (long long)D.L * m->layer_size;
    const size_t smem = ((size_t)kSgB * R + (size_t)kSgN * (N + 1) * 2) * sizeof(T) + 8 + kSgB * kSgN * sizeof(double);
    const size_t smem_al = (smem + 15) & ~size_t(15);
    if (smem_al > 220 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(k_s4_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_al);
    if (err != cudaSuccess) return err;
    const int nbt = (B + kSgB - 1) / kSgB;
    const T *pwb = pw + (long long)blk * D.d * D.s * (N + 1) * 2;
    ProfScope _ps("k_s4_grad", st);
    k_s4_grad<T><<<(unsigned)((long long)D.d * nbt), kSgB * kSgN, smem_al, st>>>(
        m->params_dev + boff, D.d, D.s, N, D.periodic, R, B, dg, pwb, O, P, boff);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vjp(const T *O, const double *wts, int B, long long P, double *vjp, cudaStream_t st) {
    ProfScope _ps("k_vjp", st);
    k_vjp<T><<<grid_of(P), 256, 0, st>>>(O, wts, B, P, vjp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sr_matrices(const T *O, int B, long long P, double *gram, long long k0, int nk, double *Ssub,
                               T *mean, float *part, int nsplit, cudaStream_t st) {
    {
        ProfScope _ps("k_colmean", st);
        k_colmean<T><<<grid_of(P), 256, 0, st>>>(O, B, P, mean);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const size_t gfold = sizeof(T) == 4 ? 64 * 256 * sizeof(T) : 0;
    if ((err = cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gfold)) != cudaSuccess)
        return err;
    if (gram && part) {
        // FP32: tensor cores (BF16 planes, FP32-grade products), K split, splits summed in FP64
        if ((err = launch_gram_tc(reinterpret_cast<const float *>(O), B, P, reinterpret_cast<const float *>(mean),
                                  1.0 / B, gram, part, nsplit, nullptr, st)) != cudaSuccess)
            return err;
    } else if (gram) {
        const long long nt = (B + kGrT - 1) / kGrT;
        ProfScope _ps("k_gram", st);
        k_gram<T><<<(unsigned)(nt * (nt + 1) / 2), 256, gfold, st>>>(O, P, 1, B, P, mean, 1, 1.0 / B, gram);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (Ssub && nk > 0) {
        const long long nt = (nk + kGrT - 1) / kGrT;
        ProfScope _ps("k_gram", st);
        k_gram<T><<<(unsigned)(nt * (nt + 1) / 2), 256, gfold, st>>>(O + k0, 1, P, nk, B, mean + k0, 0, 1.0 / B, Ssub);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

#define DN_GRAD_INST(T)                                                                                              \
    template cudaError_t launch_h0<T>(int, int, int, const int8_t *, const T *, T *, cudaStream_t);                   \
    template cudaError_t launch_grad_readout<T>(const Geom &, int, int, int, const double *, const double *,         \
                                                const double *, double *, T *, long long, long long, cudaStream_t);  \
    template cudaError_t launch_add_omega<T>(const Geom &, int, const T *, const double *, T *, bool, cudaStream_t); \
    template cudaError_t launch_mlp_back<T>(const Geom &, int, const Weights<T> &, const int8_t *, int, const T *,   \
                                            const T *, const T *, const GradScratch<T> &, cudaStream_t);             \
    template cudaError_t launch_outer<T>(int, int, int, int, const T *, const T *, T *, long long, long long, int,   \
                                         cudaStream_t);                                                              \
    template cudaError_t launch_dtaps<T>(const Geom &, int, const T *, const T *, T *, cudaStream_t);                 \
    template cudaError_t launch_grad_e<T>(const Geom &, int, const T *, const int8_t *, T *, long long, long long,    \
                                          cudaStream_t);                                                             \
    template cudaError_t launch_grad_gf<T>(const Geom &, int, const T *, long long, const double *, T *,             \
                                           cudaStream_t);                                                            \
    template cudaError_t launch_s4_pow<T>(const dn_model *, int, T *, cudaStream_t);                                  \
    template cudaError_t launch_vjp<T>(const T *, const double *, int, long long, double *, cudaStream_t);            \
    template cudaError_t launch_sr_matrices<T>(const T *, int, long long, double *, long long, int, double *, T *,     \
                                               float *, int, cudaStream_t);                                            \
    template cudaError_t launch_s4_grad<T>(const dn_model *, int, int, int, const T *, const T *, T *, long long,     \
                                           cudaStream_t);

DN_GRAD_INST(double)
DN_GRAD_INST(float)

}  // namespace dn
