// Interlayer link tensors of the pairs with one intermediate layer (l = m + 2) in the
// frequency domain (App. "Efficient construction of link tensors", the two-layer link by
// matrix-valued FFT; Eq. Lmn).
//
// For such a pair the band entry is a correlation over the intermediate site n:
//   K^(l,m)_{k+dl,k}[c][c'] = sum_n g^(l)_{k+dl-n,c} D0^(m+1)_n[c][c'] g^(m+1)_{n-k,c'}
//                           = sum_n D_n[c][c'] q^dl_{cc'}(n - k),
//   q^dl_{cc'}(t) = g^(l)_{dl-t,c} g^(m+1)_{t,c'},
// so, with hats for DFTs of length M, K^dl_{cc'} = IDFT( D^_{cc'} conj(q^dl_{cc'}^) ).
// On an open chain the sequences are zero-padded to M >= 2N - 1 (t = n - k spans
// (-N, N), so the circular correlation of length M has no wrap-around); on a ring the
// correlation is circular of length N (M = N).  M must be a power of two.
//
// The spectra of q depend only on the weights and N: one kernel computes them for the
// pair, another takes each configuration's vertex matrices D0^(m+1) through the forward
// transform once per (configuration, output channel c, group of source channels c'),
// then for every band offset multiplies, transforms back and writes the band rows.
// Two real sequences travel in one complex transform (x + i y); the transform is a
// radix-2 self-sorting (Stockham) FFT in shared memory with twiddles from sincospi.
// Cost per configuration: d^2 / 2 forward and (2R + 1) d^2 / 2 inverse complex FFTs of
// length M, O((2R + 1) d^2 M log M), against (2R + 1) N^2 d^2 multiply-adds for the
// direct band sum.
#include "dn_internal.cuh"

namespace dn {

namespace {

template <typename T>
struct C2 {
    T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {   // a * conj(b)
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// tw[j] = exp(-2 pi i j / M), j < M / 2.
template <typename T>
__device__ void fill_twiddles(C2<T> *tw, int M) {
    for (int j = threadIdx.x; j < M / 2; j += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)M, &s, &c);
        tw[j] = {(T)c, (T)s};
    }
}

// DFT (sgn = -1) or unscaled inverse DFT (sgn = +1) of nseq complex sequences of length
// M = 2^logM stored one after the other in buf0; buf1 is scratch of the same size.
// Radix-2 Stockham: stage Ns combines pairs (j, j + M/2) with twiddle w^(k M / 2Ns),
// k = j mod Ns, into positions 2(j - k) + k and + Ns; the result comes out in natural
// order.  Returns the buffer that holds it.  Every thread of the block must call it.
template <typename T>
__device__ C2<T> *fft_block(C2<T> *buf0, C2<T> *buf1, const C2<T> *tw, int M, int logM, int nseq, int sgn) {
    const int half = M >> 1;
    C2<T> *in = buf0, *out = buf1;
    for (int s = 0; s < logM; ++s) {
        const int Ns = 1 << s, ts = half >> s;
        for (int q = threadIdx.x; q < nseq * half; q += blockDim.x) {
            const int sq = q >> (logM - 1), j = q & (half - 1);
            const C2<T> *src = in + (long long)sq * M;
            C2<T> *dst = out + (long long)sq * M;
            const int k = j & (Ns - 1);
            C2<T> w = tw[k * ts];
            if (sgn > 0) w.y = -w.y;
            const C2<T> v0 = src[j], v1 = cmul(src[j + half], w);
            const int d0 = 2 * (j - k) + k;
            dst[d0] = {v0.x + v1.x, v0.y + v1.y};
            dst[d0 + Ns] = {v0.x - v1.x, v0.y - v1.y};
        }
        __syncthreads();
        C2<T> *t = in;
        in = out;
        out = t;
    }
    return in;
}

// The two half spectra (nu = 0 .. M/2) of the real sequences x, y from Z = DFT(x + i y):
// X(nu) = (Z(nu) + conj Z(-nu)) / 2, Y(nu) = (Z(nu) - conj Z(-nu)) / (2i).
template <typename T>
__device__ __forceinline__ void split_spectra(const C2<T> *Z, int M, int nu, C2<T> &X, C2<T> &Y) {
    const C2<T> a = Z[nu], b = Z[(M - nu) & (M - 1)];
    X = {(a.x + b.x) / 2, (a.y - b.y) / 2};
    Y = {(a.y + b.y) / 2, (b.x - a.x) / 2};
}

__host__ __device__ inline int ilog2(int M) {
    int l = 0;
    while ((1 << l) < M) ++l;
    return l;
}

}  // namespace

// Spectra of q^dl_{cc'} for one pair: qhat[o][c][c'][nu], o = dl + R, nu = 0 .. M/2.
// One CTA per (offset o, output channel c, group of G source channels).
template <typename T>
__global__ void __launch_bounds__(256) k_link_qhat(int N, int periodic, int d, int R, int M, int G,
                                                   const T *__restrict__ taps_l, const T *__restrict__ taps_m1,
                                                   C2<T> *__restrict__ qhat) {
    extern __shared__ __align__(16) unsigned char smq[];
    const int logM = ilog2(M), half = M / 2, np = G / 2;
    C2<T> *tw = reinterpret_cast<C2<T> *>(smq);
    C2<T> *b0 = tw + half, *b1 = b0 + (size_t)np * M;
    const int o = blockIdx.x, c = blockIdx.y, c0 = blockIdx.z * G, dl = o - R;
    fill_twiddles(tw, M);
    // q^dl_{cc'}(t) at circular index t of length M (signed t in (-N, N) on an open chain).
    auto tap = [&](const T *taps, int r, int ch) -> T {
        if (periodic) return taps[(long long)(((r % N) + N) % N) * d + ch];
        return (r > -N && r < N) ? taps[(long long)(r + N - 1) * d + ch] : (T)0;
    };
    for (int q = threadIdx.x; q < np * M; q += blockDim.x) {
        const int p = q / M, t = q - p * M;
        const int ts = periodic ? t : (t < M / 2 ? t : t - M);
        T v[2] = {0, 0};
        if (periodic || (ts > -N && ts < N)) {
            const T gl = tap(taps_l, dl - ts, c);
            v[0] = gl * tap(taps_m1, ts, c0 + 2 * p);
            v[1] = gl * tap(taps_m1, ts, c0 + 2 * p + 1);
        }
        b0[q] = {v[0], v[1]};
    }
    __syncthreads();
    const C2<T> *Z = fft_block(b0, b1, tw, M, logM, np, -1);
    C2<T> *dst = qhat + (((long long)o * d + c) * d + c0) * (half + 1);
    for (int q = threadIdx.x; q < np * (half + 1); q += blockDim.x) {
        const int p = q / (half + 1), nu = q - p * (half + 1);
        C2<T> X, Y;
        split_spectra(Z + (long long)p * M, M, nu, X, Y);
        dst[(long long)(2 * p) * (half + 1) + nu] = X;
        dst[(long long)(2 * p + 1) * (half + 1) + nu] = Y;
    }
}

// Band rows of one pair for nb configurations.  One CTA per (configuration, output channel
// c, group of G source channels): the G sequences D_n[c][c'] (n < N, zero-padded to M) are
// transformed once and kept as half spectra; for every band offset dl the products
// D^ conj(q^) of two channels form one complex spectrum (Hermitian extension to
// nu > M/2), which is transformed back; row i = k + dl of the band (wrapped on a ring,
// skipped off an open chain) gets K(k) / M for the G channels c', contiguous in memory.
template <typename T>
__global__ void __launch_bounds__(256) k_link_fft(int N, int periodic, int d, int R, int M, int G,
                                                  const T *__restrict__ Dm, long long dm_ss,
                                                  const C2<T> *__restrict__ qhat, T *__restrict__ band, long long bss,
                                                  long long brs, long long bos, long long b0) {
    extern __shared__ __align__(16) unsigned char smf[];
    const int logM = ilog2(M), half = M / 2, np = G / 2, hs = half + 1;
    C2<T> *tw = reinterpret_cast<C2<T> *>(smf);
    C2<T> *spec = tw + half;                         // [G][M/2 + 1]
    C2<T> *b0b = spec + (size_t)G * hs, *b1b = b0b + (size_t)np * M;
    const long long bl = blockIdx.x;
    const int c = blockIdx.y, c0 = blockIdx.z * G;
    fill_twiddles(tw, M);
    const T *D = Dm + bl * dm_ss + (long long)c * d + c0;   // D_n[c][c0 + j] at D[n d^2 + j]
    const long long dd = (long long)d * d;
    for (int q = threadIdx.x; q < np * M; q += blockDim.x) {
        const int p = q / M, n = q - p * M;
        C2<T> v = {0, 0};
        if (n < N) v = {D[n * dd + 2 * p], D[n * dd + 2 * p + 1]};
        b0b[q] = v;
    }
    __syncthreads();
    {
        const C2<T> *Z = fft_block(b0b, b1b, tw, M, logM, np, -1);
        for (int q = threadIdx.x; q < np * hs; q += blockDim.x) {
            const int p = q / hs, nu = q - p * hs;
            C2<T> X, Y;
            split_spectra(Z + (long long)p * M, M, nu, X, Y);
            spec[(2 * p) * hs + nu] = X;
            spec[(2 * p + 1) * hs + nu] = Y;
        }
    }
    __syncthreads();
    const T scale = (T)1 / (T)M;
    for (int o = 0; o < 2 * R + 1; ++o) {
        const int dl = o - R;
        const C2<T> *Q = qhat + (((long long)o * d + c) * d + c0) * hs;
        for (int q = threadIdx.x; q < np * M; q += blockDim.x) {
            const int p = q / M, nu = q - p * M;
            const int nh = nu <= half ? nu : M - nu;
            C2<T> w1 = cmulc(spec[(2 * p) * hs + nh], Q[(long long)(2 * p) * hs + nh]);
            C2<T> w2 = cmulc(spec[(2 * p + 1) * hs + nh], Q[(long long)(2 * p + 1) * hs + nh]);
            if (nu > half) {
                w1.y = -w1.y;
                w2.y = -w2.y;
            }
            b0b[q] = {w1.x - w2.y, w1.y + w2.x};      // w1 + i w2
        }
        __syncthreads();
        const C2<T> *Kt = fft_block(b0b, b1b, tw, M, logM, np, +1);
        T *bb = band + (b0 + bl) * bss + (long long)c * d + c0;
        for (int q = threadIdx.x; q < N * G; q += blockDim.x) {
            const int k = q / G, j = q - k * G;
            int i = k + dl;
            if (periodic) i = ((i % N) + N) % N;
            else if (i < 0 || i >= N) continue;
            const C2<T> v = Kt[(long long)(j >> 1) * M + k];
            bb[(long long)i * brs + (long long)(R - dl) * bos + j] = ((j & 1) ? v.y : v.x) * scale;
        }
        __syncthreads();
    }
}

// Shared memory of the two kernels for group size G, and the group size used: the largest
// even divisor of d whose working set fits (0 if none).
template <typename T>
static size_t link_fft_smem(int M, int G, bool with_spec) {
    return ((size_t)M / 2 + (with_spec ? (size_t)G * (M / 2 + 1) : 0) + (size_t)G * M) * sizeof(C2<T>);
}
template <typename T>
static int link_fft_group(int d, int M) {
    for (int G = d; G >= 2; G /= 2)
        if (d % G == 0 && G % 2 == 0 && link_fft_smem<T>(M, G, true) <= 200 * 1024) return G;
    return 0;
}

template <typename T>
static int link_fft_size(int N, int periodic) {
    if (periodic) return (N >= 2 && (N & (N - 1)) == 0) ? N : 0;
    int M = 2;
    while (M < 2 * N - 1) M *= 2;
    return M;
}

template <typename T>
size_t link_fft_scratch_elems(int N, int periodic, int d, int R) {
    const int M = link_fft_size<T>(N, periodic);
    if (M == 0 || M > 4096 || link_fft_group<T>(d, M) == 0) return 0;
    return (size_t)(2 * R + 1) * d * d * (M / 2 + 1) * 2;   // qhat, in units of T
}

template <typename T>
cudaError_t launch_link_fft(int N, int periodic, int d, int R, const T *taps_l, const T *taps_m1, const T *Dm,
                            long long dm_ss, T *band, long long bss, long long brs, long long bos, long long b0,
                            int nb, T *scratch, size_t scratch_elems, cudaStream_t st) {
    const int M = link_fft_size<T>(N, periodic);
    const size_t need = link_fft_scratch_elems<T>(N, periodic, d, R);
    if (need == 0 || need > scratch_elems || (reinterpret_cast<uintptr_t>(scratch) % sizeof(C2<T>)) != 0)
        return cudaErrorNotSupported;
    const int G = link_fft_group<T>(d, M);
    C2<T> *qhat = reinterpret_cast<C2<T> *>(scratch);
    const size_t sq = link_fft_smem<T>(M, G, false), sf = link_fft_smem<T>(M, G, true);
    cudaError_t err = cudaFuncSetAttribute(k_link_qhat<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sq);
    if (err != cudaSuccess) return err;
    if ((err = cudaFuncSetAttribute(k_link_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf)) != cudaSuccess)
        return err;
    {
        ProfScope _ps("k_link_qhat", st);
        k_link_qhat<T><<<dim3(2 * R + 1, d, d / G), 256, sq, st>>>(N, periodic, d, R, M, G, taps_l, taps_m1, qhat);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    {
        ProfScope _ps("k_link_fft", st);
        k_link_fft<T><<<dim3(nb, d, d / G), 256, sf, st>>>(N, periodic, d, R, M, G, Dm, dm_ss, qhat, band, bss, brs,
                                                           bos, b0);
    }
    return cudaGetLastError();
}

template size_t link_fft_scratch_elems<float>(int, int, int, int);
template size_t link_fft_scratch_elems<double>(int, int, int, int);
template cudaError_t launch_link_fft<float>(int, int, int, int, const float *, const float *, const float *, long long,
                                            float *, long long, long long, long long, long long, int, float *, size_t,
                                            cudaStream_t);
template cudaError_t launch_link_fft<double>(int, int, int, int, const double *, const double *, const double *,
                                             long long, double *, long long, long long, long long, long long, int,
                                             double *, size_t, cudaStream_t);

int g_fft_links = 1;

// ------------------------------------------------------------------------------------------
// The S4 convolution of the forward pass, u = G x per channel (Eq. resolvent: the kernel is
// applied in the frequency domain), as IDFT(G^ X^) of length M: on an open chain M is the
// power of two >= 2N - 1 (the taps g_r, r in (-N, N), sit at circular index r mod M and
// x is zero-padded, so the circular product is the linear convolution); on a ring M = N,
// a power of two (the taps are circulant).  Two channels travel in one complex transform.

// M of the FFT convolution, or 0 where it does not apply.
int conv_fft_size(int N, int periodic) {
    if (periodic) return (N >= 2 && (N & (N - 1)) == 0) ? N : 0;
    int M = 2;
    while (M < 2 * N - 1) M <<= 1;
    return M;
}

namespace {

// Tap spectra of every layer: spec[l][c][nu], nu = 0 .. M/2.  One CTA per (layer, channel pair).
template <typename T>
__global__ void __launch_bounds__(256) k_tap_spec(int N, int periodic, int d, int M, int R, const T *__restrict__ taps,
                                                  C2<T> *__restrict__ spec) {
    extern __shared__ __align__(16) unsigned char smt[];
    const int logM = ilog2(M), half = M / 2, hs = half + 1;
    C2<T> *tw = reinterpret_cast<C2<T> *>(smt);
    C2<T> *b0 = tw + half, *b1 = b0 + M;
    const int l = blockIdx.x, c0 = 2 * blockIdx.y;
    fill_twiddles(tw, M);
    const T *tl = taps + (long long)l * R * d;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        C2<T> v = {0, 0};
        if (periodic) {
            v = {tl[(long long)m * d + c0], tl[(long long)m * d + c0 + 1]};
        } else {
            const int r = m < half ? m : m - M;
            if (r > -N && r < N) v = {tl[(long long)(r + N - 1) * d + c0], tl[(long long)(r + N - 1) * d + c0 + 1]};
        }
        b0[m] = v;
    }
    __syncthreads();
    const C2<T> *Z = fft_block(b0, b1, tw, M, logM, 1, -1);
    C2<T> *dst = spec + ((long long)l * d + c0) * hs;
    for (int nu = threadIdx.x; nu < hs; nu += blockDim.x) {
        C2<T> X, Y;
        split_spectra(Z, M, nu, X, Y);
        dst[nu] = X;
        dst[hs + nu] = Y;
    }
}

// u = G x for F fields, G channels per CTA (G / 2 complex transforms): CTA = (field, group).
// The input is either a field [N][d] or, for the first layer, e_c s_j from the spins.
template <typename T>
__global__ void __launch_bounds__(256) k_conv_fft(int N, int d, int M, int G, const C2<T> *__restrict__ spec_l,
                                                  Fields<T> in, const int8_t *__restrict__ spins,
                                                  const T *__restrict__ e, Fields<T> out) {
    extern __shared__ __align__(16) unsigned char smc[];
    const int logM = ilog2(M), half = M / 2, hs = half + 1, np = G / 2;
    C2<T> *tw = reinterpret_cast<C2<T> *>(smc);
    C2<T> *b0 = tw + half, *b1 = b0 + (size_t)np * M;
    const int ng = d / G;
    const long long f = blockIdx.x / ng;
    const int c0 = (int)(blockIdx.x % ng) * G;
    fill_twiddles(tw, M);
    const T *src = spins ? nullptr : in.at(f);
    const int8_t *sp = spins ? spins + f * N : nullptr;
    for (int q = threadIdx.x; q < np * M; q += blockDim.x) {
        const int p = q / M, n = q - p * M, c = c0 + 2 * p;
        C2<T> v = {0, 0};
        if (n < N) {
            if (sp) {
                const T s = (T)sp[n];
                v = {e[c] * s, e[c + 1] * s};
            } else {
                v = {src[(long long)n * d + c], src[(long long)n * d + c + 1]};
            }
        }
        b0[q] = v;
    }
    __syncthreads();
    const C2<T> *Z = fft_block(b0, b1, tw, M, logM, np, -1);
    C2<T> *W = Z == b0 ? b1 : b0;
    for (int q = threadIdx.x; q < np * M; q += blockDim.x) {
        const int p = q / M, nu = q - p * M, c = c0 + 2 * p;
        const int nh = nu <= half ? nu : M - nu;
        C2<T> X, Y;
        split_spectra(Z + (long long)p * M, M, nh, X, Y);
        C2<T> w1 = cmul(X, spec_l[(long long)c * hs + nh]);
        C2<T> w2 = cmul(Y, spec_l[(long long)(c + 1) * hs + nh]);
        if (nu > half) {   // Hermitian extension of the two real products' spectra
            w1.y = -w1.y;
            w2.y = -w2.y;
        }
        W[q] = {w1.x - w2.y, w1.y + w2.x};      // w1 + i w2
    }
    __syncthreads();
    const C2<T> *U = fft_block(W, W == b0 ? b1 : b0, tw, M, logM, np, +1);
    T *dst = out.at(f);
    const T scale = (T)1 / (T)M;
    for (int q = threadIdx.x; q < np * N; q += blockDim.x) {
        const int n = q / np, p = q - n * np, c = c0 + 2 * p;
        const C2<T> v = U[(long long)p * M + n];
        dst[(long long)n * d + c] = v.x * scale;
        dst[(long long)n * d + c + 1] = v.y * scale;
    }
}

template <typename T>
size_t conv_fft_smem(int M, int G) {
    return ((size_t)M / 2 + 2 * (size_t)(G / 2) * M) * sizeof(C2<T>);
}

// Channels per CTA: the largest of 8, 4, 2 dividing d whose transforms fit in 100 KB.
template <typename T>
int conv_fft_group(int d, int M) {
    for (int G = 8; G >= 2; G >>= 1)
        if (d % G == 0 && conv_fft_smem<T>(M, G) <= 100 * 1024) return G;
    return 0;
}

}  // namespace

template <typename T>
cudaError_t launch_tap_spectra(int N, int periodic, int d, int L, int R, const T *taps, void *spec, cudaStream_t st) {
    const int M = conv_fft_size(N, periodic);
    if (M == 0 || d % 2 != 0) return cudaErrorNotSupported;
    const size_t smem = ((size_t)M / 2 + 2 * (size_t)M) * sizeof(C2<T>);
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    cudaError_t err = cudaFuncSetAttribute(k_tap_spec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_tap_spec<T><<<dim3(L, d / 2), 256, smem, st>>>(N, periodic, d, M, R, taps, static_cast<C2<T> *>(spec));
    return cudaGetLastError();
}

template <typename T>
size_t tap_spectra_bytes(int N, int periodic, int d, int L) {
    const int M = conv_fft_size(N, periodic);
    return M == 0 ? 0 : (size_t)L * d * (M / 2 + 1) * sizeof(C2<T>);
}

template <typename T>
cudaError_t launch_conv_fft(const Geom &g, int l, const void *spec, Fields<T> in, const int8_t *spins, const T *e,
                            Fields<T> out, long long F, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    const int M = conv_fft_size(g.N, g.periodic);
    const int G = M ? conv_fft_group<T>(g.d, M) : 0;
    if (!spec || G == 0) return cudaErrorNotSupported;
    const size_t smem = conv_fft_smem<T>(M, G);
    cudaError_t err = cudaFuncSetAttribute(k_conv_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const C2<T> *spec_l = static_cast<const C2<T> *>(spec) + (long long)(l - 1) * g.d * (M / 2 + 1);
    {
        ProfScope _ps("k_conv_fft", st);
        k_conv_fft<T><<<(unsigned)(F * (g.d / G)), 256, smem, st>>>(g.N, g.d, M, G, spec_l, in, spins, e, out);
    }
    return cudaGetLastError();
}

template cudaError_t launch_tap_spectra<float>(int, int, int, int, int, const float *, void *, cudaStream_t);
template cudaError_t launch_tap_spectra<double>(int, int, int, int, int, const double *, void *, cudaStream_t);
template size_t tap_spectra_bytes<float>(int, int, int, int);
template size_t tap_spectra_bytes<double>(int, int, int, int);
template cudaError_t launch_conv_fft<float>(const Geom &, int, const void *, Fields<float>, const int8_t *,
                                            const float *, Fields<float>, long long, cudaStream_t);
template cudaError_t launch_conv_fft<double>(const Geom &, int, const void *, Fields<double>, const int8_t *,
                                             const double *, Fields<double>, long long, cudaStream_t);

int g_fft_conv = 1;

}  // namespace dn

extern "C" dn_status dn_set_fft_links(int mode) {
    if (mode < 0 || mode > 2) return DN_EINVAL;
    dn::g_fft_links = mode;
    return DN_OK;
}

extern "C" dn_status dn_set_fft_conv(int mode) {
    if (mode < 0 || mode > 2) return DN_EINVAL;
    dn::g_fft_conv = mode;
    return DN_OK;
}
