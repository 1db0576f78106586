// Interlayer link tensors (Eq. Lmn; App. "Exact algorithm to construct link
// tensors", Eqs. B_def, X_def, L_def) by exact probe propagation.
//
// A probe is a unit source placed at the output of layer m at site k:
//   m = 0:  the embedding e at site k            (N probes per sample);
//   m >= 1: the unit vector e_c' at site k       (N d probes per sample).
// It is propagated through the frozen background B^(n) = D0^(n) G^(n),
// n = m+1, ..., and after G^(l) at every l >= m+2 its rows in the band
// |i - k| <= R are stored:
//   m = 0  -> ell^(l)_{i,k}       = [G^(l) X_{1,l-1} (e delta_k)]_i
//   m >= 1 -> L^(l,m)_{i,k}[:,c'] = [G^(l) X_{m+1,l-1} (e_c' delta_k)]_i
// The first G is the analytic kernel column g^(m+1)_{i-k}.  Only the last
// layer's G is evaluated on the band alone.
#include "dn_internal.cuh"

namespace dn {

__device__ __forceinline__ int tap_row(int r, int N, int periodic) {
    return periodic ? (r < 0 ? r + N : (r >= N ? r - N : r)) : r + N - 1;
}

// u[p][i][c] = g^(m+1)_{i-k, c} * src_c  with src = e (m = 0) or e_c' (m >= 1).
template <typename T>
__global__ void k_probe_src(Geom g, int m, const T *__restrict__ taps, const T *__restrict__ e, long long p0,
                            int nsrc, T *__restrict__ u) {
    const long long pl = blockIdx.x;
    const long long p = p0 + pl;
    const int cp = (int)(p % nsrc);
    const int k = (int)((p / nsrc) % g.N);
    const int N = g.N, d = g.d;
    T *dst = u + pl * N * d;
    for (int idx = threadIdx.x; idx < N * d; idx += blockDim.x) {
        const int i = idx / d, c = idx % d;
        const T gv = taps[(long long)tap_row(i - k, N, g.periodic) * d + c];
        dst[idx] = (m == 0) ? gv * e[c] : (c == cp ? gv : (T)0);
    }
}

struct BandDst {
    long long sample_stride, row_stride, o_stride;
    int R;
};

// Store the band rows of full fields u (probes p0 .. p0+np) into the link array.
template <typename T>
__global__ void k_band_store(Geom g, const T *__restrict__ u, long long p0, int nsrc, T *__restrict__ dst,
                             BandDst bd) {
    const long long pl = blockIdx.x;
    const long long p = p0 + pl;
    const int cp = (int)(p % nsrc);
    const long long q = p / nsrc;
    const int k = (int)(q % g.N);
    const long long b = q / g.N;
    const int N = g.N, d = g.d, nrow = 2 * bd.R + 1;
    const T *src = u + pl * N * d;
    for (int idx = threadIdx.x; idx < nrow * d; idx += blockDim.x) {
        const int dl = idx / d, c = idx % d;
        const int delta = dl - bd.R;
        int i = k + delta;
        if (g.periodic) {
            i = (i + N) % N;
        } else if (i < 0 || i >= N) {
            continue;
        }
        const int o = bd.R - delta;
        dst[b * bd.sample_stride + (long long)i * bd.row_stride + (long long)o * bd.o_stride + (long long)cp * d + c] =
            src[(long long)i * d + c];
    }
}

// Band-only convolution of the last layer: link[i][o] = sum_j g_{i-j} v_j, i = k + delta.
template <typename T>
__global__ void k_conv_band(Geom g, const T *__restrict__ taps, const T *__restrict__ v, long long p0, int nsrc,
                            T *__restrict__ dst, BandDst bd) {
    const long long pl = blockIdx.x;
    const long long p = p0 + pl;
    const int cp = (int)(p % nsrc);
    const long long q = p / nsrc;
    const int k = (int)(q % g.N);
    const long long b = q / g.N;
    const int N = g.N, d = g.d, nrow = 2 * bd.R + 1;
    const T *src = v + pl * N * d;
    for (int idx = threadIdx.x; idx < nrow * d; idx += blockDim.x) {
        const int dl = idx / d, c = idx % d;
        const int delta = dl - bd.R;
        int i = k + delta;
        if (g.periodic) {
            i = (i + N) % N;
        } else if (i < 0 || i >= N) {
            continue;
        }
        T acc = 0;
        for (int j = 0; j < N; ++j) acc += taps[(long long)tap_row(i - j, N, g.periodic) * d + c] * src[(long long)j * d + c];
        const int o = bd.R - delta;
        dst[b * bd.sample_stride + (long long)i * bd.row_stride + (long long)o * bd.o_stride + (long long)cp * d + c] = acc;
    }
}

size_t links_scratch_elems(const dn_model *m, int N, int nb_max) {
    (void)nb_max;
    const long long field = (long long)N * m->desc.d;
    // Two probe batches of up to 2^14 fields, or at least one sample's worth of
    // single-channel probes, whichever is smaller; at least 64 fields.
    long long P = 16384;
    const long long cap = (512ll << 20) / (2 * field * 8);   // ~512 MB at FP64
    if (P > cap) P = cap;
    if (P < 64) P = 64;
    return (size_t)(2 * P * field);
}

template <typename T>
cudaError_t build_links(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, dn_cache *c, T *scratch,
                        size_t scratch_elems, cudaStream_t st) {
    const Geom g = geom_of(m, c->N);
    const int N = g.N, d = g.d, L = g.L;
    if (L < 2) return cudaSuccess;
    const long long field = (long long)N * d;
    const long long Pmax = (long long)(scratch_elems / (2 * field));
    if (Pmax < 1) return cudaErrorInvalidValue;
    T *ubuf = scratch, *vbuf = scratch + Pmax * field;
    const T *chi = static_cast<const T *>(c->chi);
    const long long chi_stride = (long long)L * N * d;
    T *ell = static_cast<T *>(c->ell);
    T *K = static_cast<T *>(c->K);
    const int nRl = 2 * c->Rl + 1, nRk = 2 * c->Rk + 1;
    Fields<T> none{nullptr, 0, 0, 1};
    cudaError_t err;
    for (int msrc = 0; msrc <= L - 2; ++msrc) {
        const int nsrc = msrc == 0 ? 1 : d;
        const long long Q = (long long)c->B * N * nsrc;
        for (long long p0 = 0; p0 < Q; p0 += Pmax) {
            const long long np = (Q - p0 < Pmax) ? Q - p0 : Pmax;
            Fields<T> U{ubuf, field, 0, 1}, V{vbuf, field, 0, 1};
            {
                ProfScope _ps("k_probe_src", st);
                k_probe_src<T><<<(unsigned)np, 256, 0, st>>>(g, msrc, pl.taps + (long long)msrc * g.R * d, w.e, p0, nsrc,
                                                             ubuf);
            }
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            err = launch_mix<T>(g, msrc + 1, w, chi, chi_stride, (long long)N * nsrc, p0, U, V, none, nullptr, nullptr,
                                0, np, false, st);
            if (err != cudaSuccess) return err;
            for (int n = msrc + 2; n <= L; ++n) {
                BandDst bd;
                T *dst;
                if (msrc == 0) {
                    bd.R = c->Rl;
                    bd.sample_stride = (long long)(L - 1) * N * nRl * d;
                    bd.row_stride = (long long)nRl * d;
                    bd.o_stride = d;
                    dst = ell + (long long)(n - 2) * N * nRl * d;
                } else {
                    bd.R = c->Rk;
                    bd.sample_stride = (long long)c->P * N * nRk * d * d;
                    bd.row_stride = (long long)nRk * d * d;
                    bd.o_stride = (long long)d * d;
                    dst = K + (long long)pair_index(n, msrc) * N * nRk * d * d;
                }
                const T *taps_n = pl.taps + (long long)(n - 1) * g.R * d;
                if (n < L) {
                    err = launch_conv<T>(g, taps_n, V, nullptr, nullptr, U, np, false, nullptr, nullptr, st);
                    if (err != cudaSuccess) return err;
                    {
                        ProfScope _ps("k_band_store", st);
                        k_band_store<T><<<(unsigned)np, 256, 0, st>>>(g, ubuf, p0, nsrc, dst, bd);
                    }
                    if ((err = cudaGetLastError()) != cudaSuccess) return err;
                    err = launch_mix<T>(g, n, w, chi, chi_stride, (long long)N * nsrc, p0, U, V, none, nullptr,
                                        nullptr, 0, np, false, st);
                    if (err != cudaSuccess) return err;
                } else {
                    {
                        ProfScope _ps("k_conv_band", st);
                        k_conv_band<T><<<(unsigned)np, 256, 0, st>>>(g, taps_n, vbuf, p0, nsrc, dst, bd);
                    }
                    if ((err = cudaGetLastError()) != cudaSuccess) return err;
                }
            }
        }
    }
    return cudaSuccess;
}

template cudaError_t build_links<double>(const dn_model *, const Plan<double> &, const Weights<double> &, dn_cache *,
                                         double *, size_t, cudaStream_t);
template cudaError_t build_links<float>(const dn_model *, const Plan<float> &, const Weights<float> &, dn_cache *,
                                        float *, size_t, cudaStream_t);

}  // namespace dn
