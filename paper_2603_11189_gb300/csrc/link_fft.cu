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

}  // namespace dn

extern "C" dn_status dn_set_fft_links(int mode) {
    if (mode < 0 || mode > 2) return DN_EINVAL;
    dn::g_fft_links = mode;
    return DN_OK;
}
