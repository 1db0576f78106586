// Internal declarations of the DysonNet / ABACUS CUDA library (sm_103a).
//
// Data layout in HBM (per cache, B samples, T = double or float):
//   spins  int8 [B][N]
//   chi    T    [B][L][N][d]        local vertex spectrum chi^(l)_i (Eq. Dpractical)
//   y      T    [B][L][N][d]        pre-gate channel mix y = V u0, u0 = G h0 (slice
//                                   activations h~_0 of Eq. recur_step)
//   rho    T    [B][L][dout][N][d]  output links T^(l) with A folded in (Eq. Tl)
//   t      T    [B][N][dout]        embedding output link e . rho^(0)
//   ell    T    [B][L-1][N][2Rl+1][d]      ell^(l)_{i, i+o-Rl}: background response
//                                          at layer l to the embedding of site i+o-Rl
//   K      T    [B][P][N][2Rk+1][d][d]     links L^(l,m) (Eq. Lmn) on the band
//                                          |i-k| <= Rk, k = i+o-Rk, each d x d block
//                                          row-major [c_out][c_in]
//   Omega  f64  [B][dout], logpsi f64 [B], flag u32
// with W_F = 2w + max_cluster, Rk = W_F - 1, Rl = W_F - 1 - w and
// P = (L-1)(L-2)/2 layer pairs (l, m), 1 <= m <= l-2, indexed (l-3)(l-2)/2 + m-1.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "dysonnet.h"

namespace dn {

constexpr int kMaxD = 128;
constexpr int kMaxDh = 128;
constexpr int kMaxDout = 8;
constexpr int kMaxL = 12;

// Device copies of the layer weights.  Matrices come in both orientations:
// M[out][in] and MT[in][out] (MT puts the output index fastest, so a warp whose
// lanes own consecutive outputs reads consecutive addresses).
template <typename T>
struct Weights {
    T *kappa = nullptr;  // [L][W][dh]
    T *beta = nullptr;   // [L][dh]
    T *W1T = nullptr;    // [L][dh_in][dh_out]
    T *b1 = nullptr;     // [L][dh]
    T *W2T = nullptr;    // [L][dh][d]
    T *b2 = nullptr;     // [L][d]
    T *U = nullptr, *UT = nullptr, *V = nullptr, *VT = nullptr;  // [L][d][d]
    T *A = nullptr;      // [d][dout]
    T *e = nullptr;      // [d]
    void *block = nullptr;
    size_t bytes = 0;
};

// Weights-only tables for one chain length N (S4 kernel taps in FP64, cast).
template <typename T>
struct Plan {
    int N = 0, R = 0;
    T *taps = nullptr;        // [L][R][d], row r + N - 1 (open) or r (periodic)
    T *omega = nullptr;       // [N][d] pooling weights (1/N) sum_k g^f_{k-i}
    double *taps64 = nullptr; // [L+1][R][d]
    double *omega64 = nullptr;
    void *spec = nullptr;     // [L][d][M/2 + 1] complex tap spectra for the FFT convolution, or null
    void *block = nullptr;
    size_t bytes = 0;
};

}  // namespace dn

struct dn_model {
    dn_model_desc desc;
    int W = 0;
    size_t nparams = 0;
    std::vector<double> params;
    double *params_dev = nullptr;
    double *A64 = nullptr;  // [d][dout]
    long long s4_size = 0, layer_size = 0;
    dn::Weights<double> w64;
    dn::Weights<float> w32;
    std::map<int, dn::Plan<double>> plan64;
    std::map<int, dn::Plan<float>> plan32;
    bool weights_ready[2] = {false, false};
};

struct dn_cache {
    dn_model *model = nullptr;
    int N = 0, B = 0, prec = 0, max_cluster = 1;
    int WF = 0, Rk = 0, Rl = 0, P = 0;
    cudaStream_t stream = nullptr;
    void *block = nullptr;
    size_t bytes = 0;
    int8_t *spins = nullptr;
    void *chi = nullptr, *y = nullptr, *rho = nullptr, *t = nullptr, *ell = nullptr, *K = nullptr;
    double *Omega = nullptr, *logpsi = nullptr;
    unsigned *flag = nullptr;
};

namespace dn {

// Eight consecutive values from shared memory at a 16-byte-aligned address.
template <typename T>
__device__ __forceinline__ void lds8(const T *p, T (&v)[8]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            const double2 a = *reinterpret_cast<const double2 *>(p + u);
            v[u] = a.x;
            v[u + 1] = a.y;
        }
    }
}

// ------------------------------------------------------------------ memory --
void *dev_alloc(size_t bytes, cudaStream_t stream);
void dev_free(void *p, size_t bytes, cudaStream_t stream);

// Bump allocator inside one device block, 256-byte aligned sub-arrays.
struct Carve {
    size_t off = 0;
    template <typename X>
    size_t take(size_t count) {
        size_t o = (off + 255) & ~size_t(255);
        off = o + count * sizeof(X);
        return o;
    }
};

// ---------------------------------------------------------------- tracing --
// RAII scope around one kernel launch: counts it and, while tracing is on,
// records CUDA events before and after it on the launch stream.
class ProfScope {
   public:
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

   private:
    cudaStream_t st_;
    int tag_ = -1;
    cudaEvent_t start_ = nullptr;
};

// Names the enclosing stage of a call ("forward", "links", ...); launches
// inside are traced as "stage/kernel" (stages nest).
class ProfPhase {
   public:
    explicit ProfPhase(const char *name);
    ~ProfPhase();
    ProfPhase(const ProfPhase &) = delete;
    ProfPhase &operator=(const ProfPhase &) = delete;
};

// --------------------------------------------------------------- geometry --
struct Geom {
    int N, L, d, dh, dout, w, W, periodic, R;
};

inline Geom geom_of(const dn_model *m, int N) {
    Geom g;
    g.N = N; g.L = m->desc.L; g.d = m->desc.d; g.dh = m->desc.d_h; g.dout = m->desc.d_out;
    g.w = m->desc.w; g.W = 2 * m->desc.w + 1; g.periodic = m->desc.periodic;
    g.R = g.periodic ? N : 2 * N - 1;
    return g;
}

__host__ __device__ inline int pair_index(int l, int m) { return (l - 3) * (l - 2) / 2 + (m - 1); }

// Generic addressing of a batch of [N][d] fields: field f lives at
// base + (f / inner) * outer + (f % inner) * stride_inner.
template <typename T>
struct Fields {
    T *base;
    long long outer, stride_inner;
    int inner;
    __host__ __device__ T *at(long long f) const {
        return base + (f / inner) * outer + (f % inner) * stride_inner;
    }
};

// ---------------------------------------------------------------- kernels --
// Launchers (forward.cu).
cudaError_t launch_taps(const dn_model *m, int N, double *taps64, double *omega64, cudaStream_t st);
template <typename T>
cudaError_t launch_cast(const double *src, T *dst, long long n, cudaStream_t st);
cudaError_t launch_check_spins(const int8_t *spins, long long n, int8_t *copy, unsigned *flag, cudaStream_t st);

template <typename T>
cudaError_t launch_chi(const Geom &g, const Weights<T> &w, const int8_t *spins, int B, T *chi,
                       cudaStream_t st);

// u = G x (transpose: G^T x) per channel.  x from `in` fields, or, when
// spins != nullptr, x_j = e * sigma_j of sample f.  With add_Aw the output is
// A[:, k] * omega + G^T x for field f = (b, k) (adjoint recursion).
template <typename T>
cudaError_t launch_conv(const Geom &g, const T *taps_l, Fields<T> in, const int8_t *spins, const T *e,
                        Fields<T> out, long long F, bool transpose, const T *A, const T *omega, cudaStream_t st);

// Site-wise vertex: forward  h = U (chi * (V u)), optionally storing y = V u and
// the pooled sum_i omega_i h_i (FP64) per field; adjoint z = V^T (chi * (U^T x)).
// Field f (global index f0 + f) uses the vertex of sample (f0 + f) / fields_per_sample.
template <typename T>
cudaError_t launch_mix(const Geom &g, int l, const Weights<T> &w, const T *chi, long long chi_stride,
                       long long fields_per_sample, long long f0, Fields<T> in, Fields<T> out, Fields<T> yout,
                       const T *omega, double *pooled, long long pooled_stride, long long F, bool adjoint,
                       cudaStream_t st);

template <typename T>
cudaError_t launch_pool0(const Geom &g, const int8_t *spins, const T *e, const T *omega, int B, double *pooled,
                         long long pooled_stride, cudaStream_t st);
cudaError_t launch_readout(const Geom &g, int f_kind, const double *A64, const double *pooled, int npool, int B,
                           const int8_t *spins, double *Omega, double *logpsi, cudaStream_t st);
template <typename T>
cudaError_t launch_rho_init(const Geom &g, const T *A, const T *omega, Fields<T> out, long long F, cudaStream_t st);
template <typename T>
cudaError_t launch_tlink(const Geom &g, const T *rho0, const T *e, int B, T *t, cudaStream_t st);

// Links (links.cu): build ell and K for every sample of a cache, in batches of
// probes that fit the scratch buffer.
template <typename T>
cudaError_t build_links(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, dn_cache *c, T *scratch,
                        size_t scratch_elems, cudaStream_t st);
size_t links_scratch_elems(const dn_model *m, int N, int B);

// Toeplitz hop of the FP32 link build on the tcgen05 tensor cores (tc_gemm.cu):
// Y[b][a] = T_a X[b][a] (X generated from gtaps/gDm when gtaps != nullptr), band
// rows to band (may be null).  cudaErrorNotSupported when the shape does not fit.
// planes = BF16 terms per operand value: 1 (plain BF16), 2 (three products, about
// 2^-18 relative), 3 (six products, FP32-grade).
cudaError_t launch_tgemm_tc(const Geom &g, const float *taps, int P, const float *X, const float *gtaps,
                            const float *gDm, long long dm_ss, float *Y, float *band, long long bss, long long brs,
                            long long bos, int bR, int bns, long long b0, int nb, unsigned *flag, cudaStream_t st,
                            int planes = 2);

// Vertex hop X[b][c][n][p] = sum_a D0_n[c][a] Y[b][a][n][p] on the tensor cores (tc_gemm.cu),
// planes BF16 terms per value (3: FP32-grade, 1: BF16); cudaErrorNotSupported for other d.
cudaError_t launch_dhop_tc(int d, int N, int P, const float *Dm, long long dm_ss, const float *Y, float *Xo, int nb,
                           int planes, unsigned *flag, cudaStream_t st);

// Last vertex hop of a chain fused with the last layer's band convolution (dband_tc.cu):
// band of G^(L) D0^(L-1) Y for interlayer sources (nsrc = d), FP32 with 3 BF16 planes.
// dband_tc_ok() tells whether launch_dband_tc() takes the shape (else cudaErrorNotSupported).
bool dband_tc_ok(int d, int N, int periodic, int P, int nsrc, int R);
cudaError_t launch_dband_tc(int d, int N, int periodic, int P, int nsrc, int R, const float *taps, const float *Dm,
                            long long dm_ss, const float *Y, float *band, long long bss, long long brs, long long bos,
                            long long b0, int nb, unsigned *flag, cudaStream_t st);
// Process-wide choice between the fused and the two-kernel chain ends (both exact; on by default).
extern int g_fused_links;

// Band links of a pair with one intermediate layer by FFT (link_fft.cu): scratch (units of T)
// for the spectra of the pair (0: shape not supported), and the launch (cudaErrorNotSupported
// when the shape or the scratch does not fit).  g_fft_links: on by default.
template <typename T>
size_t link_fft_scratch_elems(int N, int periodic, int d, int R);
template <typename T>
cudaError_t launch_link_fft(int N, int periodic, int d, int R, const T *taps_l, const T *taps_m1, const T *Dm,
                            long long dm_ss, T *band, long long bss, long long brs, long long bos, long long b0,
                            int nb, T *scratch, size_t scratch_elems, cudaStream_t st);
extern int g_fft_links;
// The forward pass's S4 convolution by FFT (link_fft.cu): conv_fft_size is the transform
// length (0 where it does not apply: a ring whose N is not a power of two); the tap spectra
// of all layers are built with the plan.  g_fft_conv: 0 direct, 1 FP32 with N >= 512
// (default), 2 wherever the spectra exist.
int conv_fft_size(int N, int periodic);
template <typename T>
size_t tap_spectra_bytes(int N, int periodic, int d, int L);
template <typename T>
cudaError_t launch_tap_spectra(int N, int periodic, int d, int L, int R, const T *taps, void *spec, cudaStream_t st);
template <typename T>
cudaError_t launch_conv_fft(const Geom &g, int l, const void *spec, Fields<T> in, const int8_t *spins, const T *e,
                            Fields<T> out, long long F, cudaStream_t st);
extern int g_fft_conv;
template <typename T>
inline bool use_fft_conv(const Geom &g, const Plan<T> &pl) {
    if (!pl.spec || g_fft_conv == 0) return false;
    return g_fft_conv == 2 || (sizeof(T) == 4 && g.N >= 512);
}

// Reverse pass for the parameter log-derivatives (grad.cu).  Operands of the per-sample
// outer-product sums of one layer, [B][N][.] each.
template <typename T>
struct GradScratch {
    T *tY, *dy, *dchi;          // chi . y, chi . dt, y . dt      [B][N][d]
    T *a1, *phi, *dz, *dphi;    // GELU(z), phi, dz, W1^T dz      [B][N][dh]
    T *win;                     // sigma_{i+r}, r = -w..w         [B][N][W]
};
template <typename T>
cudaError_t launch_h0(int N, int d, int B, const int8_t *spins, const T *e, T *h, cudaStream_t st);
template <typename T>
cudaError_t launch_grad_readout(const Geom &g, int f_kind, int npool, int B, const double *A64, const double *pooled,
                                const double *Omega, double *acoef, T *O, long long P, long long offA, cudaStream_t st);
template <typename T>
cudaError_t launch_add_omega(const Geom &g, int B, const T *omega, const double *acoef, T *dst, bool add,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_mlp_back(const Geom &g, int l, const Weights<T> &w, const int8_t *spins, int B, const T *chi,
                            const T *y, const T *dtv, const GradScratch<T> &s, cudaStream_t st);
template <typename T>
cudaError_t launch_outer(int N, int B, int dx, int dyc, const T *X, const T *Y, T *O, long long P, long long off,
                         int ldo, cudaStream_t st);
template <typename T>
cudaError_t launch_dtaps(const Geom &g, int B, const T *du, const T *h, T *dg, cudaStream_t st);
template <typename T>
cudaError_t launch_grad_e(const Geom &g, int B, const T *dh0, const int8_t *spins, T *O, long long P, long long off,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_grad_gf(const Geom &g, int B, const T *h, long long lstride, const double *acoef, T *dgf,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_s4_pow(const dn_model *m, int N, T *pw, cudaStream_t st);
template <typename T>
cudaError_t launch_vjp(const T *O, const double *wts, int B, long long P, double *vjp, cudaStream_t st);
// Column means of O [B][P] into mean [P]; gram [B][B] = Oc Oc^T / B and Ssub [nk][nk] =
// Oc[:, k0:k0+nk]^T Oc[:, k0:k0+nk] / B with Oc the centred O (either may be null).
// part (may be null: CUDA-core kernel) holds the tensor-core Gram's K-split partials.
template <typename T>
cudaError_t launch_sr_matrices(const T *O, int B, long long P, double *gram, long long k0, int nk, double *Ssub,
                               T *mean, float *part, int nsplit, cudaStream_t st);
template <typename T>
cudaError_t launch_s4_grad(const dn_model *m, int blk, int N, int B, const T *dg, const T *pw, T *O, long long P,
                           cudaStream_t st);

// Sample-space Gram on the tensor cores (tc_gemm.cu): S [n][n] = scale Xc Xc^T, Xc = X - m,
// X [n][K] float row-major; partial buffer of gram_tc_partial_elems() floats.
size_t gram_tc_partial_elems(int n, long long K, int *nsplit);
bool link_rows_map(CUtensorMap *tm, const float *base, unsigned long long rows, int d, int box_rows);
// Tensor map of a hop output Y [zs][N][P] (float) in boxes of 128 columns x 1 site x 32 z (tc_gemm.cu).
bool dband_input_map(CUtensorMap *tm, const float *Y, int N, int P, long long zs);
cudaError_t launch_gram_tc(const float *X, int n, long long K, const float *m, double scale, double *S, float *part,
                           int nsplit, unsigned *flag, cudaStream_t st);

// Screened typewriter sampler (sampler.cu).
cudaError_t launch_flip_list(int C, int K, const int32_t *sites, const int32_t *row, const int32_t *kfrom,
                             int32_t *sample, int32_t *fsites, cudaStream_t st);
cudaError_t launch_screened_sweep(int N, int C, int K, int dout, int f_kind, double eps, const int32_t *sites,
                                  const double *u, const double *dOm, double *Om, int32_t *kpos, int8_t *spins,
                                  int8_t *acc, int32_t *amb, unsigned long long *counters, cudaStream_t st);
cudaError_t launch_pair_configs(int N, int K, int n, const int32_t *list, const int32_t *amb, const int32_t *sites,
                                const int8_t *spins, int8_t *cfg, cudaStream_t st);
cudaError_t launch_exact_decide(int N, int K, int n, const int32_t *list, const int32_t *amb, const int32_t *sites,
                                const double *u, const double *lp, int8_t *spins, int8_t *acc, int32_t *kpos,
                                unsigned long long *counters, cudaStream_t st);
cudaError_t launch_gather_rows(int N, int n, const int32_t *list, const int8_t *spins, int8_t *dst, cudaStream_t st);
cudaError_t launch_scatter_refresh(int K, int dout, int n, const int32_t *list, const int32_t *kpos,
                                   const double *Om_new, const double *dOm_new, double *Om, double *dOm,
                                   cudaStream_t st);

// Tensor-core forward pass (forward_tc.cu); activations channel-major h[c][n B + b].
bool forward_tc_ok(const Geom &g);
cudaError_t launch_h0_cm(const Geom &g, const int8_t *spins, const float *e, int B, float *h, cudaStream_t st);
cudaError_t launch_pool_cm(const Geom &g, int l, const float *h, const float *omega, int B, double *pooled,
                           long long pstride, cudaStream_t st);
// chi and y (may be null) are the caches' base pointers [B][L][N][d]; layer l is selected inside.
cudaError_t launch_mix_tc(const Geom &g, int l, const Weights<float> &w, const float *ucm, const float *chi, float *y,
                          float *hcm, int B, int planes, unsigned *flag, cudaStream_t st);

// ABACUS (abacus.cu).
// out [F] (may be null) log-amplitude ratios; dOmega [F][dout] (may be null) update vectors.
template <typename T>
cudaError_t launch_abacus(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c,
                          const int32_t *sample, const int32_t *sites, int F, double *out, cudaStream_t st,
                          double *dOmega = nullptr);
// Flip sets of several caches of one model in one launch (serving): descs is a device
// array of abacus_desc_bytes<T>() records filled by abacus_desc<T>(); flip f uses
// cache cache_of[f]; all caches share max_cluster (slice width WF).
template <typename T>
size_t abacus_desc_bytes();
template <typename T>
void abacus_desc(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c, void *dst);
template <typename T>
cudaError_t launch_abacus_multi(const dn_model *m, int WF, const void *descs, const int32_t *cache_of,
                                const int32_t *sample, const int32_t *sites, int F, double *out, cudaStream_t st);

// Persistent serving kernel (abacus.cu): work items in host-mapped memory, taken by
// ticket (item base + ctl[0]++) and served once the host has published them (item i is
// available when i < q->tail).  Item slot s = i mod cap holds cache[s] (descriptor
// index), sites[2 s .. 2 s + 1] and the state word done[s] (2i + 1 after publication);
// the kernel writes out[s] and then done[s] = 2i + 2.  When the tail has not moved for
// idle_ns nanoseconds a CTA sets q->status = DN_ETIMEOUT and ctl[1] = 1; on ctl[1] or
// q->stop every CTA leaves once its ticket is not published.  ctl (device memory, two
// words) is zeroed before each launch.
struct ServeQueue {
    unsigned long long tail;   // items published (host)
    unsigned int stop;         // host: leave as soon as no item is available
    int status;                // kernel: DN_OK, or DN_ETIMEOUT after the idle limit
};
struct ServeItems {
    int32_t *cache;            // [cap]
    int32_t *sites;            // [cap][2]
    double *out;               // [cap]
    unsigned long long *done;  // [cap] state of slot i % cap: 2i + 1 published, 2i + 2 served
    int cap;
};
template <typename T>
cudaError_t launch_abacus_serve(const dn_model *m, int WF, const void *descs, ServeQueue *q, ServeItems it,
                                unsigned long long *ctl, unsigned long long base, long long idle_ns, int ctas,
                                cudaStream_t st);
// All N single flips of every cached configuration, out[b N + j], layer by
// layer; scratch of singles_scratch_bytes() bytes (cudaErrorNotSupported when
// the shape does not fit the kernels).
size_t singles_scratch_bytes(const dn_model *m, const dn_cache *c);
template <typename T>
cudaError_t launch_abacus_singles(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c,
                                  void *scratch, double *out, cudaStream_t st);
// The pair flips {j, j + bonds[bo]} (1 <= nb <= 2 bonds, 1 <= bonds[bo] <= max_cluster - 1)
// of every site j of every cached configuration, out[(b nb + bo) N + j] (0 where the pair
// runs past an open end, and with anti set where its two spins are aligned), layer by
// layer; scratch of pairs_scratch_bytes() bytes (cudaErrorNotSupported when the shape does
// not fit the kernels).
// Whether the grouped kernels take the pattern (else the flip-list kernel serves it).
bool pairs_grouped_fits(const dn_model *m, const dn_cache *c, int nb, const int *bonds);
size_t pairs_scratch_bytes(const dn_model *m, const dn_cache *c, int nb, const int *bonds);
template <typename T>
cudaError_t launch_abacus_pairs(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c, int nb,
                                const int *bonds, bool anti, void *scratch, double *out, cudaStream_t st);
// The same pairs as a flip list for the flip-list kernel: entry (b nb + bo) N + j (empty
// entries where the pair runs past an open end or, with anti set, its spins are aligned).
cudaError_t launch_make_pair_flips(int N, int B, int periodic, int nb, const int *bonds, bool anti,
                                   const int8_t *spins, int32_t *sample, int32_t *sites, cudaStream_t st);
cudaError_t launch_make_flips(int kind, int N, int B, int periodic, const int8_t *spins, int32_t *sample,
                              int32_t *sites, cudaStream_t st);
cudaError_t launch_eloc_reduce(const dn_hamiltonian &H, int N, int B, const int8_t *spins, const double *coupling,
                               const double *dlogpsi, double *eloc, cudaStream_t st);
cudaError_t launch_expand_flips(int N, const int8_t *spins, const int32_t *sample, const int32_t *sites, int F,
                                int B, int8_t *out, unsigned *flag, cudaStream_t st);
cudaError_t launch_sub_base(const double *lp_flip, const double *lp_base, const int32_t *sample, const int32_t *sites,
                            int F, int B, int N, double *out, cudaStream_t st);

}  // namespace dn
