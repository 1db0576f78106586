// DysonNet forward pass and adjoint (output links) on sm_103a.
//
//  k_taps     S4 kernel generation in FP64 (App. "Details on the implementation
//             of the DysonNet block", Eq. discretization; periodic chains use
//             the closed-form circulant sum of the open kernel's images).
//  k_omega    pooling weights of P_M G^f (Eq. wavefunc): omega_i = (1/N) sum_k g^f_{k-i}.
//  k_chi      chi^(l)_i = W2 GELU(W1 phi^(l)_i + b1) + b2, phi from the spin window
//             (Eq. Dpractical, local vertex of width W = 2w+1).
//  k_conv     u = G x, channel-diagonal Toeplitz/circulant convolution (the
//             Green's-function mixer of the DysonNet block definition), or its
//             transpose for the adjoint.
//  k_mix      h = U (chi * (V u)) per site (D_j = U diag(chi_j) V), with the
//             pooled readout accumulated in FP64; or the adjoint V^T chi U^T.
//  k_readout  Omega = A^T sum_l pooled_l, log psi = sum_k f(Omega_k).
#include <math.h>

#include <type_traits>

#include "dn_internal.cuh"

namespace dn {

template <typename T>
__device__ __forceinline__ T gelu(T x);
template <>
__device__ __forceinline__ double gelu<double>(double x) {
    return 0.5 * x * (1.0 + erf(x * 0.70710678118654752440));
}
template <>
__device__ __forceinline__ float gelu<float>(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678f));
}

// ------------------------------------------------------------------ taps --
__global__ void k_taps(const double *__restrict__ params, int L, int d, int s, long long layer_size,
                       long long final_off, int N, int periodic, int R, double *__restrict__ out) {
    const int ri = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y, blk = blockIdx.z;
    if (ri >= R) return;
    const double *p = params + (blk < L ? (long long)blk * layer_size : final_off);
    const long long ds = (long long)d * s;
    const double *lre = p, *lim = p + ds, *logdt = p + 2 * ds;
    const double *bre = logdt + d, *bim = bre + ds;
    const double *cfre = bim + ds, *cfim = cfre + ds, *cbre = cfim + ds, *cbim = cbre + ds;
    const double dt = exp(logdt[c]);
    double acc = 0.0;
    for (int n = 0; n < s; ++n) {
        const long long k = (long long)c * s + n;
        // lam_bar = (1 + dt/2 Lam) / (1 - dt/2 Lam), B_bar = dt B / (1 - dt/2 Lam)
        const double ar = 0.5 * dt * lre[k], ai = 0.5 * dt * lim[k];
        const double dr = 1.0 - ar, di = -ai, dd = dr * dr + di * di;
        const double lr = ((1.0 + ar) * dr + ai * di) / dd;
        const double li = (ai * dr - (1.0 + ar) * di) / dd;
        const double br = dt * bre[k], bi = dt * bim[k];
        const double bbr = (br * dr + bi * di) / dd, bbi = (bi * dr - br * di) / dd;
        const double lnrho = 0.5 * log(lr * lr + li * li), th = atan2(li, lr);
        if (!periodic) {
            const int r = ri - (N - 1);
            const int q = r < 0 ? -r : r;
            double sn, cs;
            sincos(q * th, &sn, &cs);
            const double mag = exp(q * lnrho);
            const double cr = r >= 0 ? cfre[k] : cbre[k], ci = r >= 0 ? cfim[k] : cbim[k];
            const double tr = cr * bbr - ci * bbi, ti = cr * bbi + ci * bbr;   // C B_bar
            acc += tr * (mag * cs) - ti * (mag * sn);                         // Re(C B_bar lam^q)
        } else {
            const int r = ri;
            double s1, c1, s2, c2, sN, cN;
            sincos(r * th, &s1, &c1);
            sincos((N - r) * th, &s2, &c2);
            sincos(N * th, &sN, &cN);
            const double m1 = exp(r * lnrho), m2 = exp((N - r) * lnrho), mN = exp(N * lnrho);
            // Cf lam^r + Cb lam^(N-r)
            const double nr = cfre[k] * m1 * c1 - cfim[k] * m1 * s1 + cbre[k] * m2 * c2 - cbim[k] * m2 * s2;
            const double ni = cfre[k] * m1 * s1 + cfim[k] * m1 * c1 + cbre[k] * m2 * s2 + cbim[k] * m2 * c2;
            const double tr = nr * bbr - ni * bbi, ti = nr * bbi + ni * bbr;
            const double er = 1.0 - mN * cN, ei = -mN * sN, ee = er * er + ei * ei;
            acc += (tr * er + ti * ei) / ee;                                  // Re(t / (1 - lam^N))
        }
    }
    out[((long long)blk * R + ri) * d + c] = acc;
}

__global__ void k_omega(const double *__restrict__ gf, int N, int d, int periodic, double *__restrict__ omega) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * d) return;
    const int i = idx / d, c = idx % d;
    double acc = 0.0;
    for (int k = 0; k < N; ++k) {
        const int r = k - i;
        const int row = periodic ? (r < 0 ? r + N : r) : r + N - 1;
        acc += gf[(long long)row * d + c];
    }
    omega[idx] = acc / N;
}

cudaError_t launch_taps(const dn_model *m, int N, double *taps64, double *omega64, cudaStream_t st) {
    const int L = m->desc.L, d = m->desc.d, s = m->desc.s, periodic = m->desc.periodic;
    const int R = periodic ? N : 2 * N - 1;
    dim3 grid((R + 127) / 128, d, L + 1);
    {
        ProfScope _ps("k_taps", st);
        k_taps<<<grid, 128, 0, st>>>(m->params_dev, L, d, s, m->layer_size, (long long)L * m->layer_size, N, periodic,
                                     R, taps64);
    }
    {
        ProfScope _ps("k_omega", st);
        k_omega<<<(N * d + 127) / 128, 128, 0, st>>>(taps64 + (long long)L * R * d, N, d, periodic, omega64);
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void k_cast(const double *__restrict__ src, T *__restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
cudaError_t launch_cast(const double *src, T *dst, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    {
        ProfScope _ps("k_cast", st);
        k_cast<T><<<blocks, 256, 0, st>>>(src, dst, n);
    }
    return cudaGetLastError();
}

__global__ void k_check_spins(const int8_t *__restrict__ spins, long long n, int8_t *__restrict__ copy,
                              unsigned *__restrict__ flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int8_t v = spins[i];
        if (copy) copy[i] = v;
        if (v != 1 && v != -1) atomicOr(flag, 1u);
    }
}

cudaError_t launch_check_spins(const int8_t *spins, long long n, int8_t *copy, unsigned *flag, cudaStream_t st) {
    const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    {
        ProfScope _ps("k_check_spins", st);
        k_check_spins<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(spins, n, copy, flag);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------- chi --
// One CTA per (sample, layer, tile of kChiTile sites).  W1 and W2 of the layer are staged
// once (row strides dh + 1 and d + 1, so a warp reading along either index hits distinct
// banks); phi and GELU(z) are kept transposed ([feature][site]) so that a thread (output
// feature, group of 8 sites) reads its 8 sites as two 16-byte broadcasts.
constexpr int kChiTile = 64, kChiRG = 8, kChiTPB = 8;   // sites per tile, per thread group, tiles per CTA
constexpr int kChiTS = kChiTile + 4;   // row stride of the transposed tiles: 16-byte rows that start 4 banks apart

template <typename T>
__global__ void __launch_bounds__(256) k_chi(Geom g, Weights<T> w, const int8_t *__restrict__ spins, int B,
                                             T *__restrict__ chi, int stage) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, dh = g.dh, L = g.L, wd = g.w, W = g.W;
    T *phT = reinterpret_cast<T *>(smraw);      // [dh][kChiTS]
    T *acT = phT + dh * kChiTS;                 // [dh][kChiTS]
    T *sw = acT + dh * kChiTS;                  // [tile + 2w] spins of the tile's windows
    // FP32 with staged weights and dh, d multiples of 4: 4 outputs x 4 sites per thread from
    // 16-byte weight and activation loads (weight rows padded by 4); else 1 output x 8 sites.
    const bool tiled = std::is_same<T, float>::value && stage && dh % 4 == 0 && d % 4 == 0;
    T *W1s = sw + ((kChiTile + 2 * wd + 3) & ~3);   // [f][e] = W1[e][f]
    T *W2s = W1s + dh * (dh + 4);               // [e][c] = W2[c][e]
    const int ntile = (N + kChiTile - 1) / kChiTile;
    const int l = blockIdx.y;
    const T *kap = w.kappa + (long long)l * W * dh;
    const T *beta = w.beta + (long long)l * dh;
    const T *b1 = w.b1 + (long long)l * dh;
    const T *b2 = w.b2 + (long long)l * d;
    // Weights from shared memory (staged once for the CTA's tiles), or from global memory
    // when they do not fit.
    const T *W1p = stage ? W1s : w.W1T + (long long)l * dh * dh;
    const T *W2p = stage ? W2s : w.W2T + (long long)l * dh * d;
    const int s1 = stage ? (tiled ? dh + 4 : dh + 1) : dh, s2 = stage ? (tiled ? d + 4 : d + 1) : d;
    if (stage) {
        for (int q = threadIdx.x; q < dh * dh; q += blockDim.x)
            W1s[(q / dh) * s1 + q % dh] = w.W1T[(long long)l * dh * dh + q];
        for (int q = threadIdx.x; q < dh * d; q += blockDim.x)
            W2s[(q / d) * s2 + q % d] = w.W2T[(long long)l * dh * d + q];
    }
    const long long items = (long long)B * ntile;
    for (int it = 0; it < kChiTPB; ++it) {
        const long long item = (long long)blockIdx.x * kChiTPB + it;
        if (item >= items) break;
        const long long b = item / ntile;
        const int i0 = (int)(item % ntile) * kChiTile;
        const int ns = min(kChiTile, N - i0);
        const int8_t *sp = spins + b * N;
        __syncthreads();   // previous tile's reads of phT / acT / sw (and the weight staging) are done
        for (int q = threadIdx.x; q < kChiTile + 2 * wd; q += blockDim.x) {
            int j = i0 + q - wd;
            T sv;
            if (g.periodic) {
                j = ((j % N) + N) % N;
                sv = (T)sp[j];
            } else {
                sv = (j >= 0 && j < N) ? (T)sp[j] : (T)0;
            }
            sw[q] = sv;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < kChiTile * dh; idx += blockDim.x) {
            const int e = idx / kChiTile, t = idx % kChiTile;   // lanes along sites: conflict-free stores
            T acc = 0;
            if (t < ns) {
                acc = beta[e];
                for (int r = 0; r < W; ++r) acc += kap[r * dh + e] * sw[t + r];
            }
            phT[e * kChiTS + t] = acc;
        }
        __syncthreads();
        if (!tiled) {
            for (int q = threadIdx.x; q < dh * (kChiTile / kChiRG); q += blockDim.x) {
                const int e = q % dh, t0 = (q / dh) * kChiRG;
                T acc[kChiRG];
#pragma unroll
                for (int u = 0; u < kChiRG; ++u) acc[u] = b1[e];
                for (int f = 0; f < dh; ++f) {
                    const T wv = W1p[f * s1 + e];
                    T pv[8];
                    lds8<T>(phT + f * kChiTS + t0, pv);
#pragma unroll
                    for (int u = 0; u < kChiRG; ++u) acc[u] += wv * pv[u];
                }
#pragma unroll
                for (int u = 0; u < kChiRG; ++u) acT[e * kChiTS + t0 + u] = gelu<T>(acc[u]);
            }
            __syncthreads();
            T *dst = chi + ((b * L + l) * N + i0) * d;
            for (int q = threadIdx.x; q < d * (kChiTile / kChiRG); q += blockDim.x) {
                const int c = q % d, t0 = (q / d) * kChiRG;
                T acc[kChiRG];
#pragma unroll
                for (int u = 0; u < kChiRG; ++u) acc[u] = b2[c];
                for (int e = 0; e < dh; ++e) {
                    const T wv = W2p[e * s2 + c];
                    T pv[8];
                    lds8<T>(acT + e * kChiTS + t0, pv);
#pragma unroll
                    for (int u = 0; u < kChiRG; ++u) acc[u] += wv * pv[u];
                }
#pragma unroll
                for (int u = 0; u < kChiRG; ++u)
                    if (t0 + u < ns) dst[(long long)(t0 + u) * d + c] = acc[u];
            }

        } else if constexpr (std::is_same<T, float>::value) {
            for (int q = threadIdx.x; q < (dh / 4) * (kChiTile / 4); q += blockDim.x) {
                const int e0 = (q % (dh / 4)) * 4, t0 = (q / (dh / 4)) * 4;
                float acc[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[j][u] = b1[e0 + j];
#pragma unroll 4
                for (int f = 0; f < dh; ++f) {
                    const float4 wv = *reinterpret_cast<const float4 *>(W1s + f * s1 + e0);
                    const float4 pv = *reinterpret_cast<const float4 *>(phT + f * kChiTS + t0);
                    const float w4[4] = {wv.x, wv.y, wv.z, wv.w}, p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[j][u] = fmaf(w4[j], p4[u], acc[j][u]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<float4 *>(acT + (e0 + j) * kChiTS + t0) =
                        make_float4(gelu<float>(acc[j][0]), gelu<float>(acc[j][1]), gelu<float>(acc[j][2]),
                                    gelu<float>(acc[j][3]));
            }
            __syncthreads();
            float *dst = chi + ((b * L + l) * N + i0) * d;
            for (int q = threadIdx.x; q < (d / 4) * (kChiTile / 4); q += blockDim.x) {
                const int c0 = (q % (d / 4)) * 4, t0 = (q / (d / 4)) * 4;
                float acc[4][4];   // [site][output]
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[u][j] = b2[c0 + j];
#pragma unroll 4
                for (int e = 0; e < dh; ++e) {
                    const float4 wv = *reinterpret_cast<const float4 *>(W2s + e * s2 + c0);
                    const float4 pv = *reinterpret_cast<const float4 *>(acT + e * kChiTS + t0);
                    const float w4[4] = {wv.x, wv.y, wv.z, wv.w}, p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[u][j] = fmaf(w4[j], p4[u], acc[u][j]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t0 + u < ns)
                        *reinterpret_cast<float4 *>(dst + (long long)(t0 + u) * d + c0) =
                            make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
            }
        }
    }
}

template <typename T>
cudaError_t launch_chi(const Geom &g, const Weights<T> &w, const int8_t *spins, int B, T *chi, cudaStream_t st) {
    const int ntile = (g.N + kChiTile - 1) / kChiTile;
    const long long groups = ((long long)B * ntile + kChiTPB - 1) / kChiTPB;
    const size_t act = ((size_t)2 * kChiTS * g.dh + (size_t)((kChiTile + 2 * g.w + 3) & ~3)) * sizeof(T);
    const size_t wts = ((size_t)g.dh * (g.dh + 4) + (size_t)g.dh * (g.d + 4)) * sizeof(T);
    const int stage = act + wts <= 200 * 1024 ? 1 : 0;
    const size_t smem = act + (stage ? wts : 0);
    cudaError_t err = cudaFuncSetAttribute(k_chi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_chi", st);
        k_chi<T><<<dim3((unsigned)groups, (unsigned)g.L), 256, smem, st>>>(g, w, spins, B, chi, stage);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ conv --
// One CTA per (field, channel tile).  Shared memory holds the taps of the
// channel tile extended to offsets r in (-N, N) and the field's channels.
constexpr int kCvOut = 8;   // consecutive outputs per thread
template <typename T>
__global__ void k_conv(Geom g, const T *__restrict__ taps_l, Fields<T> in, const int8_t *__restrict__ spins,
                       const T *__restrict__ e, Fields<T> out, int CT, int transpose, const T *__restrict__ A,
                       const T *__restrict__ omega) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d;
    T *gx = reinterpret_cast<T *>(smraw);     // [2N-1+kCvOut][CT]
    T *x = gx + (2 * N - 1 + kCvOut) * CT;    // [N][CT]
    const int nct = d / CT;
    const long long f = blockIdx.x / nct;
    const int c0 = (int)(blockIdx.x % nct) * CT;
    for (int idx = threadIdx.x; idx < (2 * N - 1) * CT; idx += blockDim.x) {
        const int q = idx / CT, c = idx % CT;
        int r = q - (N - 1);
        if (transpose) r = -r;
        const int row = g.periodic ? (r < 0 ? r + N : r) : r + N - 1;
        gx[idx] = taps_l[(long long)row * d + c0 + c];
    }
    if (spins) {
        const int8_t *sp = spins + f * N;
        for (int idx = threadIdx.x; idx < N * CT; idx += blockDim.x) {
            const int j = idx / CT, c = idx % CT;
            x[idx] = e[c0 + c] * (T)sp[j];
        }
    } else {
        const T *src = in.at(f);
        for (int idx = threadIdx.x; idx < N * CT; idx += blockDim.x) {
            const int j = idx / CT, c = idx % CT;
            x[idx] = src[(long long)j * d + c0 + c];
        }
    }
    // rows 2N-1 .. 2N-1+kCvOut: zero taps read by the last output group past the chain end
    for (int idx = threadIdx.x; idx < kCvOut * CT; idx += blockDim.x) gx[(2 * N - 1) * CT + idx] = 0;
    __syncthreads();
    T *dst = out.at(f);
    const int kk = A ? (int)(f % g.dout) : 0;
    // Thread (group of kCvOut consecutive outputs i0.., channel c): for input site j the taps
    // are g_{i0+u-j}; over a block of 4 sites j..j+3 they form a window of kCvOut + 3 taps,
    // loaded once, so a block costs 4 + kCvOut + 3 loads for 4 kCvOut FMAs.
    const int ngrp = (N + kCvOut - 1) / kCvOut;
    for (int idx = threadIdx.x; idx < ngrp * CT; idx += blockDim.x) {
        const int i0 = (idx / CT) * kCvOut, c = idx % CT;
        const T *gp = gx + (i0 + N - 1) * CT + c;     // g_{i0+u-j} = gp[(u - j) * CT]
        T acc[kCvOut];
#pragma unroll
        for (int u = 0; u < kCvOut; ++u) acc[u] = 0;
        int j = 0;
        for (; j + 4 <= N; j += 4) {
            T xv[4], win[kCvOut + 3];                 // win[m] = g_{i0 + m - 3 - j}
#pragma unroll
            for (int t = 0; t < 4; ++t) xv[t] = x[(j + t) * CT + c];
#pragma unroll
            for (int m = 0; m < kCvOut + 3; ++m) win[m] = gp[(m - 3 - j) * CT];
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int u = 0; u < kCvOut; ++u) acc[u] += win[u - t + 3] * xv[t];
        }
        for (; j < N; ++j) {
            const T xv = x[j * CT + c];
#pragma unroll
            for (int u = 0; u < kCvOut; ++u) acc[u] += gp[(u - j) * CT] * xv;
        }
#pragma unroll
        for (int u = 0; u < kCvOut; ++u) {
            const int i = i0 + u;
            if (i >= N) break;
            T v = acc[u];
            if (A) v += A[(c0 + c) * g.dout + kk] * omega[(long long)i * d + c0 + c];
            dst[(long long)i * d + c0 + c] = v;
        }
    }
}

template <typename T>
static int conv_tile(const Geom &g, size_t *smem) {
    // Largest divisor of d (<= 32) whose taps + field tile fit in 200 KB.
    int best = 1;
    for (int ct = 1; ct <= 32 && ct <= g.d; ++ct) {
        if (g.d % ct) continue;
        size_t bytes = (size_t)(3 * g.N - 1 + kCvOut) * ct * sizeof(T);
        if (bytes <= 200 * 1024) best = ct;
    }
    *smem = (size_t)(3 * g.N - 1 + kCvOut) * best * sizeof(T);
    return best;
}

template <typename T>
cudaError_t launch_conv(const Geom &g, const T *taps_l, Fields<T> in, const int8_t *spins, const T *e, Fields<T> out,
                        long long F, bool transpose, const T *A, const T *omega, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    size_t smem;
    const int CT = conv_tile<T>(g, &smem);
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t err = cudaFuncSetAttribute(k_conv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const long long blocks = F * (g.d / CT);
    {
        ProfScope _ps("k_conv", st);
        k_conv<T><<<(unsigned)blocks, 256, smem, st>>>(g, taps_l, in, spins, e, out, CT, transpose ? 1 : 0, A, omega);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------- mix --
// One CTA per field; the CTA walks the sites in row tiles of TS = blockDim/d.
// Thread (tr, a) owns output channel a of row tr of the tile.
template <typename T>
__global__ void k_mix(Geom g, int l, Weights<T> w, const T *__restrict__ chi, long long chi_stride, long long fps,
                      long long f0, Fields<T> in, Fields<T> out, Fields<T> yout, const T *__restrict__ omega,
                      double *__restrict__ pooled, long long pooled_stride, int adjoint) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d;
    const int TS = blockDim.x / d;
    const int a = threadIdx.x % d, tr = threadIdx.x / d;
    const bool lane_ok = tr < TS;
    T *xs = reinterpret_cast<T *>(smraw);   // [TS][d]
    T *ts = xs + TS * d;                    // [TS][d]
    double *red = reinterpret_cast<double *>(smraw + ((2 * (size_t)TS * d * sizeof(T) + 7) & ~(size_t)7));
    const long long f = blockIdx.x;
    const long long b = (f0 + f) / fps;
    const T *chib = chi + b * chi_stride + (long long)(l - 1) * N * d;
    const long long dd = (long long)d * d, lo = (long long)(l - 1) * dd;
    // m1t[in][out], m2t[in][out]: forward M1 = V, M2 = U; adjoint M1 = U^T, M2 = V^T.
    const T *m1t = adjoint ? w.U + lo : w.VT + lo;
    const T *m2t = adjoint ? w.V + lo : w.UT + lo;
    const T *src = in.at(f);
    T *dst = out.at(f);
    T *ydst = yout.base ? yout.at(f) : nullptr;
    double pacc = 0.0;
    for (int i0 = 0; i0 < N; i0 += TS) {
        const int i = i0 + tr;
        const bool act = lane_ok && i < N;
        if (act) xs[tr * d + a] = src[(long long)i * d + a];
        __syncthreads();
        T yv = 0;
        if (act) {
            for (int bb = 0; bb < d; ++bb) yv += m1t[bb * d + a] * xs[tr * d + bb];
            if (ydst) ydst[(long long)i * d + a] = yv;
            ts[tr * d + a] = chib[(long long)i * d + a] * yv;
        }
        __syncthreads();
        if (act) {
            T hv = 0;
            for (int bb = 0; bb < d; ++bb) hv += m2t[bb * d + a] * ts[tr * d + bb];
            dst[(long long)i * d + a] = hv;
            if (pooled) pacc += (double)omega[(long long)i * d + a] * (double)hv;
        }
        __syncthreads();
    }
    if (pooled) {
        if (lane_ok) red[tr * d + a] = pacc;
        __syncthreads();
        if (tr == 0) {
            double sum = 0.0;
            for (int q = 0; q < TS; ++q) sum += red[q * d + a];
            pooled[f * pooled_stride + a] = sum;
        }
    }
}

// FP32 form of k_mix for d in {16, 32, 64}: the two d x d matrices staged once per
// CTA (rows padded by 4), rows in tiles of RT = 4096 / d, each thread forms 4 outputs x 4 rows
// of both products from 16-byte loads (weights along the outputs, the tile's inputs stored
// transposed along the rows).  Products and summation order per output are those of k_mix.
__global__ void __launch_bounds__(256) k_mix_t(Geom g, int l, Weights<float> w, const float *__restrict__ chi,
                                               long long chi_stride, long long fps, long long f0, Fields<float> in,
                                               Fields<float> out, Fields<float> yout, const float *__restrict__ omega,
                                               double *__restrict__ pooled, long long pooled_stride, int adjoint) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, RT = 4096 / d, ws = d + 4, xs = RT + 4;
    float *M1 = reinterpret_cast<float *>(smraw);   // [bb][a] = m1t[bb d + a], row stride d + 4
    float *M2 = M1 + d * ws;
    float *xT = M2 + d * ws;                        // [bb][r] tile inputs, row stride RT + 4
    float *tT = xT + d * xs;                        // [bb][r] chi . y of the tile
    double *red = reinterpret_cast<double *>(tT + d * xs);   // [RT / 4][d] pooled partials
    const long long f = blockIdx.x;
    const long long b = (f0 + f) / fps;
    const float *chib = chi + b * chi_stride + (long long)(l - 1) * N * d;
    const long long dd = (long long)d * d, lo = (long long)(l - 1) * dd;
    const float *m1t = adjoint ? w.U + lo : w.VT + lo;
    const float *m2t = adjoint ? w.V + lo : w.UT + lo;
    for (int q = threadIdx.x; q < d * d; q += blockDim.x) {
        M1[(q / d) * ws + q % d] = m1t[q];
        M2[(q / d) * ws + q % d] = m2t[q];
    }
    const float *src = in.at(f);
    float *dst = out.at(f);
    float *ydst = yout.base ? yout.at(f) : nullptr;
    const int a0 = 4 * (int)(threadIdx.x % (d / 4)), r0 = 4 * (int)(threadIdx.x / (d / 4));
    double pacc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = 0; i0 < N; i0 += RT) {
        __syncthreads();   // weights staged / the previous tile's xT and tT read
        for (int q = threadIdx.x; q < RT * d; q += blockDim.x) {
            const int r = q / d, bb = q % d;
            xT[bb * xs + r] = i0 + r < N ? src[(long long)(i0 + r) * d + bb] : 0.f;
        }
        __syncthreads();
        float acc[4][4];   // [row][output]
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[u][j] = 0.f;
#pragma unroll 4
        for (int bb = 0; bb < d; ++bb) {
            const float4 mv = *reinterpret_cast<const float4 *>(M1 + bb * ws + a0);
            const float4 xv = *reinterpret_cast<const float4 *>(xT + bb * xs + r0);
            const float m4[4] = {mv.x, mv.y, mv.z, mv.w}, x4[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[u][j] = fmaf(m4[j], x4[u], acc[u][j]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + r0 + u;
            float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < N) {
                if (ydst) *reinterpret_cast<float4 *>(ydst + (long long)i * d + a0) =
                              make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
                cv = *reinterpret_cast<const float4 *>(chib + (long long)i * d + a0);
            }
            tT[(a0 + 0) * xs + r0 + u] = cv.x * acc[u][0];
            tT[(a0 + 1) * xs + r0 + u] = cv.y * acc[u][1];
            tT[(a0 + 2) * xs + r0 + u] = cv.z * acc[u][2];
            tT[(a0 + 3) * xs + r0 + u] = cv.w * acc[u][3];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[u][j] = 0.f;
#pragma unroll 4
        for (int bb = 0; bb < d; ++bb) {
            const float4 mv = *reinterpret_cast<const float4 *>(M2 + bb * ws + a0);
            const float4 tv = *reinterpret_cast<const float4 *>(tT + bb * xs + r0);
            const float m4[4] = {mv.x, mv.y, mv.z, mv.w}, t4[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[u][j] = fmaf(m4[j], t4[u], acc[u][j]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + r0 + u;
            if (i >= N) continue;
            *reinterpret_cast<float4 *>(dst + (long long)i * d + a0) =
                make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
            if (pooled) {
                const float4 om = *reinterpret_cast<const float4 *>(omega + (long long)i * d + a0);
                pacc[0] += (double)om.x * (double)acc[u][0];
                pacc[1] += (double)om.y * (double)acc[u][1];
                pacc[2] += (double)om.z * (double)acc[u][2];
                pacc[3] += (double)om.w * (double)acc[u][3];
            }
        }
    }
    if (pooled) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(r0 / 4) * d + a0 + j] = pacc[j];
        __syncthreads();
        for (int a = threadIdx.x; a < d; a += blockDim.x) {
            double sum = 0.0;
            for (int q = 0; q < RT / 4; ++q) sum += red[q * d + a];
            pooled[f * pooled_stride + a] = sum;
        }
    }
}

template <typename T>
cudaError_t launch_mix(const Geom &g, int l, const Weights<T> &w, const T *chi, long long chi_stride,
                          long long fields_per_sample, long long f0, Fields<T> in, Fields<T> out, Fields<T> yout,
                          const T *omega, double *pooled, long long pooled_stride, long long F, bool adjoint,
                          cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    if constexpr (std::is_same<T, float>::value) {
        if (g.d == 16 || g.d == 32 || g.d == 64) {
            const int RT = 4096 / g.d;
            const size_t smem = (2 * (size_t)g.d * (g.d + 4) + 2 * (size_t)g.d * (RT + 4)) * sizeof(float) +
                                (size_t)(RT / 4) * g.d * sizeof(double);
            cudaError_t err = cudaFuncSetAttribute(k_mix_t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            ProfScope _ps("k_mix", st);
            k_mix_t<<<(unsigned)F, 256, smem, st>>>(g, l, w, chi, chi_stride, fields_per_sample, f0, in, out, yout,
                                                    omega, pooled, pooled_stride, adjoint ? 1 : 0);
            return cudaGetLastError();
        }
    }
    int TS = 256 / g.d;
    if (TS < 1) TS = 1;
    const int threads = TS * g.d;
    const size_t smem = 2 * (size_t)TS * g.d * sizeof(T) + 8 + (size_t)TS * g.d * sizeof(double);
    {
        ProfScope _ps("k_mix", st);
        k_mix<T><<<(unsigned)F, threads, smem, st>>>(g, l, w, chi, chi_stride, fields_per_sample, f0, in, out, yout,
                                                     omega, pooled, pooled_stride, adjoint ? 1 : 0);
    }
    return cudaGetLastError();
}

// --------------------------------------------------------------- readout --
template <typename T>
__global__ void k_pool0(Geom g, const int8_t *__restrict__ spins, const T *__restrict__ e,
                        const T *__restrict__ omega, double *__restrict__ pooled, long long pooled_stride) {
    const long long b = blockIdx.x;
    const int N = g.N, d = g.d;
    const int8_t *sp = spins + b * N;
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < N; ++i) acc += (double)omega[(long long)i * d + c] * (double)sp[i];
        pooled[b * pooled_stride + c] = acc * (double)e[c];
    }
}

template <typename T>
cudaError_t launch_pool0(const Geom &g, const int8_t *spins, const T *e, const T *omega, int B, double *pooled,
                         long long pooled_stride, cudaStream_t st) {
    {
        ProfScope _ps("k_pool0", st);
        k_pool0<T><<<B, 64, 0, st>>>(g, spins, e, omega, pooled, pooled_stride);
    }
    return cudaGetLastError();
}

__device__ __forceinline__ double log_cosh(double x) {
    const double a = fabs(x);
    return a + log1p(exp(-2.0 * a)) - 0.69314718055994530942;
}

__global__ void k_readout(Geom g, int f_kind, const double *__restrict__ A64, const double *__restrict__ pooled,
                          int npool, int B, const int8_t *__restrict__ spins, double *__restrict__ Omega,
                          double *__restrict__ logpsi) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int d = g.d, dout = g.dout;
    bool bad = false;
    if (spins) {
        const int8_t *sp = spins + (long long)b * g.N;
        for (int i = 0; i < g.N; ++i) bad |= (sp[i] != 1 && sp[i] != -1);
    }
    double lp = 0.0;
    for (int k = 0; k < dout; ++k) {
        double acc = 0.0;
        for (int c = 0; c < d; ++c) {
            double pc = 0.0;
            for (int q = 0; q < npool; ++q) pc += pooled[((long long)b * npool + q) * d + c];
            acc += A64[c * dout + k] * pc;
        }
        if (bad) acc = nan("");
        if (Omega) Omega[(long long)b * dout + k] = acc;
        lp += f_kind == 0 ? log_cosh(acc) : acc;
    }
    if (logpsi) logpsi[b] = lp;
}

cudaError_t launch_readout(const Geom &g, int f_kind, const double *A64, const double *pooled, int npool, int B,
                                 const int8_t *spins, double *Omega, double *logpsi, cudaStream_t st) {
    {
        ProfScope _ps("k_readout", st);
        k_readout<<<(B + 127) / 128, 128, 0, st>>>(g, f_kind, A64, pooled, npool, B, spins, Omega, logpsi);
    }
    return cudaGetLastError();
}

// --------------------------------------------------------------- adjoint --
template <typename T>
__global__ void k_rho_init(Geom g, const T *__restrict__ A, const T *__restrict__ omega, Fields<T> out) {
    const long long f = blockIdx.x;
    const int k = (int)(f % g.dout);
    T *dst = out.at(f);
    for (int idx = threadIdx.x; idx < g.N * g.d; idx += blockDim.x) {
        const int c = idx % g.d;
        dst[idx] = A[c * g.dout + k] * omega[idx];
    }
}

template <typename T>
cudaError_t launch_rho_init(const Geom &g, const T *A, const T *omega, Fields<T> out, long long F, cudaStream_t st) {
    {
        ProfScope _ps("k_rho_init", st);
        k_rho_init<T><<<(unsigned)F, 256, 0, st>>>(g, A, omega, out);
    }
    return cudaGetLastError();
}

// t[b][i][k] = e . rho^(0)[b][k][i][:]
template <typename T>
__global__ void k_tlink(Geom g, const T *__restrict__ rho0, const T *__restrict__ e, T *__restrict__ t) {
    const long long b = blockIdx.x;
    const int N = g.N, d = g.d, dout = g.dout;
    for (int idx = threadIdx.x; idx < N * dout; idx += blockDim.x) {
        const int i = idx / dout, k = idx % dout;
        const T *r = rho0 + ((b * dout + k) * N + i) * d;
        T acc = 0;
        for (int c = 0; c < d; ++c) acc += e[c] * r[c];
        t[(b * N + i) * dout + k] = acc;
    }
}

template <typename T>
cudaError_t launch_tlink(const Geom &g, const T *rho0, const T *e, int B, T *t, cudaStream_t st) {
    {
        ProfScope _ps("k_tlink", st);
        k_tlink<T><<<B, 128, 0, st>>>(g, rho0, e, t);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------- instantiations --
#define DN_INST(T)                                                                                                    \
    template cudaError_t launch_cast<T>(const double *, T *, long long, cudaStream_t);                               \
    template cudaError_t launch_chi<T>(const Geom &, const Weights<T> &, const int8_t *, int, T *, cudaStream_t);    \
    template cudaError_t launch_conv<T>(const Geom &, const T *, Fields<T>, const int8_t *, const T *, Fields<T>,     \
                                        long long, bool, const T *, const T *, cudaStream_t);                        \
    template cudaError_t launch_mix<T>(const Geom &, int, const Weights<T> &, const T *, long long, long long,     \
                                          long long, Fields<T>, Fields<T>, Fields<T>, const T *, double *, long long, \
                                          long long, bool, cudaStream_t);                                            \
    template cudaError_t launch_pool0<T>(const Geom &, const int8_t *, const T *, const T *, int, double *,          \
                                         long long, cudaStream_t);                                                   \
    template cudaError_t launch_rho_init<T>(const Geom &, const T *, const T *, Fields<T>, long long, cudaStream_t); \
    template cudaError_t launch_tlink<T>(const Geom &, const T *, const T *, int, T *, cudaStream_t);

DN_INST(double)
DN_INST(float)

}  // namespace dn
