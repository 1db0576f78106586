// Full-forward evaluation that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a host whose
// device memory is fully reserved up front by another runtime or arena, a
// serving process that forbids allocation after warm-up so that its memory
// footprint stays fixed, or code that runs where a cudaMalloc (or a caching
// allocator that may fall back to one) could block or fail.  For them this
// file provides dn_full_forward_noalloc(): the same log-amplitude as
// dn_full_forward(), computed with every temporary in one fixed, file-scope
// device array instead of freshly allocated buffers.
//
// The array is kNoAllocScratchBytes large and lives on every device that
// loads the library until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress, on the first call made with that
// device current); that first call should therefore happen before any stream
// capture.  The looked-up address is kept for the life of the process: a
// cudaDeviceReset() (or any reset of the primary context by the host program)
// reloads the module and invalidates it, so this entry point must not be used
// on a device after such a reset.  All calls share the array and it keeps the contents of the last
// call: every value a call reads is written earlier in the same call, so
// nothing needs clearing, but two calls that overlap on the GPU (different
// streams, or different host threads) race on it.

#include "dn_internal.cuh"

namespace dn {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of the scratch array in the current context.  Looked up on every call
// (a host-side query that allocates nothing), so that a device or primary-context reset,
// which reloads the module at a new address, never leaves a stale pointer behind.
cudaError_t noalloc_scratch(void **out) { return cudaGetSymbolAddress(out, g_noalloc_scratch); }

// Pack the layer weights of the FP64 parameter vector into the kernels' layout
// (both orientations of every matrix) in precision T.
template <typename T>
__global__ void k_pack_weights(const double *__restrict__ P, int L, int d, int dh, int W, int dout,
                               long long layer_size, long long s4_size, Weights<T> w) {
    const long long dd = (long long)d * d;
    const long long per_layer = (long long)W * dh + 2 * dh + (long long)dh * dh + (long long)d * dh + d + 2 * dd;
    const long long total = L * per_layer + (long long)d * dout + d;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx >= L * per_layer) {
            const long long q = idx - L * per_layer;
            const double *fin = P + L * layer_size + s4_size;
            if (q < (long long)d * dout) w.A[q] = (T)fin[q];
            else w.e[q - (long long)d * dout] = (T)fin[q];
            continue;
        }
        const int l = (int)(idx / per_layer);
        long long q = idx % per_layer;
        const double *kap = P + l * layer_size + s4_size;
        const double *beta = kap + (long long)W * dh, *W1 = beta + dh, *b1 = W1 + (long long)dh * dh, *W2 = b1 + dh,
                     *b2 = W2 + (long long)d * dh, *U = b2 + d, *V = U + dd;
        if (q < (long long)W * dh) { w.kappa[(long long)l * W * dh + q] = (T)kap[q]; continue; }
        q -= (long long)W * dh;
        if (q < dh) { w.beta[(long long)l * dh + q] = (T)beta[q]; continue; }
        q -= dh;
        if (q < (long long)dh * dh) {      // W1[e][f] -> W1T[f][e]
            const long long e = q / dh, f = q % dh;
            w.W1T[((long long)l * dh + f) * dh + e] = (T)W1[q];
            continue;
        }
        q -= (long long)dh * dh;
        if (q < dh) { w.b1[(long long)l * dh + q] = (T)b1[q]; continue; }
        q -= dh;
        if (q < (long long)d * dh) {       // W2[c][e] -> W2T[e][c]
            const long long c = q / dh, e = q % dh;
            w.W2T[((long long)l * dh + e) * d + c] = (T)W2[q];
            continue;
        }
        q -= (long long)d * dh;
        if (q < d) { w.b2[(long long)l * d + q] = (T)b2[q]; continue; }
        q -= d;
        if (q < dd) {                      // U[a][b]
            const long long a = q / d, b = q % d;
            w.U[l * dd + q] = (T)U[q];
            w.UT[l * dd + b * d + a] = (T)U[q];
            continue;
        }
        q -= dd;
        {                                  // V[a][b]
            const long long a = q / d, b = q % d;
            w.V[l * dd + q] = (T)V[q];
            w.VT[l * dd + b * d + a] = (T)V[q];
        }
    }
}

struct NoAllocLayout {
    size_t kappa, beta, W1T, b1, W2T, b2, U, UT, V, VT, A, e, taps64, omega64, taps, omega, chi, h, u, pooled, total;
};

template <typename T>
NoAllocLayout noalloc_layout(const dn_model_desc &D, int N, int B) {
    const int L = D.L, d = D.d, dh = D.d_h, W = 2 * D.w + 1, dout = D.d_out;
    const size_t R = D.periodic ? (size_t)N : 2 * (size_t)N - 1;
    Carve cv;
    NoAllocLayout s;
    s.kappa = cv.take<T>((size_t)L * W * dh);
    s.beta = cv.take<T>((size_t)L * dh);
    s.W1T = cv.take<T>((size_t)L * dh * dh);
    s.b1 = cv.take<T>((size_t)L * dh);
    s.W2T = cv.take<T>((size_t)L * dh * d);
    s.b2 = cv.take<T>((size_t)L * d);
    s.U = cv.take<T>((size_t)L * d * d);
    s.UT = cv.take<T>((size_t)L * d * d);
    s.V = cv.take<T>((size_t)L * d * d);
    s.VT = cv.take<T>((size_t)L * d * d);
    s.A = cv.take<T>((size_t)d * dout);
    s.e = cv.take<T>((size_t)d);
    s.taps64 = cv.take<double>((size_t)(L + 1) * R * d);
    s.omega64 = cv.take<double>((size_t)N * d);
    s.taps = cv.take<T>((size_t)L * R * d);
    s.omega = cv.take<T>((size_t)N * d);
    s.chi = cv.take<T>((size_t)B * L * N * d);
    s.h = cv.take<T>((size_t)B * N * d);
    s.u = cv.take<T>((size_t)B * N * d);
    s.pooled = cv.take<double>((size_t)B * (L + 1) * d);
    s.total = cv.off;
    return s;
}

template <typename T>
cudaError_t noalloc_forward(const dn_model *m, int N, const int8_t *spins, int B, char *base, const NoAllocLayout &s,
                            cudaStream_t st, double *logpsi, double *Omega) {
    const dn_model_desc &D = m->desc;
    const Geom g = geom_of(m, N);
    const int L = g.L, d = g.d;
    auto P = [&](size_t off) { return reinterpret_cast<T *>(base + off); };
    Weights<T> w;
    w.kappa = P(s.kappa); w.beta = P(s.beta); w.W1T = P(s.W1T); w.b1 = P(s.b1); w.W2T = P(s.W2T); w.b2 = P(s.b2);
    w.U = P(s.U); w.UT = P(s.UT); w.V = P(s.V); w.VT = P(s.VT); w.A = P(s.A); w.e = P(s.e);
    double *taps64 = reinterpret_cast<double *>(base + s.taps64);
    double *omega64 = reinterpret_cast<double *>(base + s.omega64);
    T *taps = P(s.taps), *omega = P(s.omega), *chi = P(s.chi), *h = P(s.h), *u = P(s.u);
    double *pooled = reinterpret_cast<double *>(base + s.pooled);
    cudaError_t err;
    {
        ProfScope _ps("k_pack_weights", st);
        k_pack_weights<T><<<64, 256, 0, st>>>(m->params_dev, L, d, D.d_h, 2 * D.w + 1, D.d_out, m->layer_size,
                                              m->s4_size, w);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = launch_taps(m, N, taps64, omega64, st)) != cudaSuccess) return err;
    if ((err = launch_cast<T>(taps64, taps, (long long)L * g.R * d, st)) != cudaSuccess) return err;
    if ((err = launch_cast<T>(omega64, omega, (long long)N * d, st)) != cudaSuccess) return err;
    const long long field = (long long)N * d;
    if ((err = launch_chi<T>(g, w, spins, B, chi, st)) != cudaSuccess) return err;
    if ((err = launch_pool0<T>(g, spins, w.e, omega, B, pooled, (long long)(L + 1) * d, st)) != cudaSuccess) return err;
    Fields<T> H{h, field, 0, 1}, U{u, field, 0, 1}, none{nullptr, 0, 0, 1};
    for (int l = 1; l <= L; ++l) {
        err = launch_conv<T>(g, taps + (long long)(l - 1) * g.R * d, H, l == 1 ? spins : nullptr, w.e, U, B, false,
                             nullptr, nullptr, st);
        if (err != cudaSuccess) return err;
        err = launch_mix<T>(g, l, w, chi, (long long)L * field, 1, 0, U, H, none, omega, pooled + (long long)l * d,
                            (long long)(L + 1) * d, B, false, st);
        if (err != cudaSuccess) return err;
    }
    return launch_readout(g, D.f_kind, m->A64, pooled, L + 1, B, spins, Omega, logpsi, st);
}

}  // namespace
}  // namespace dn

extern "C" dn_status dn_full_forward_noalloc(const dn_model *m, int N, const int8_t *spins_dev, int B,
                                             dn_precision prec, void *stream, double *logpsi_dev, double *Omega_dev) {
    if (!m || !spins_dev || !logpsi_dev || N < 1 || B < 1) return DN_EINVAL;
    if (prec == DN_BF16) return DN_EUNSUPPORTED;
    if (prec != DN_FP64 && prec != DN_FP32) return DN_EINVAL;
    const size_t need = prec == DN_FP64 ? dn::noalloc_layout<double>(m->desc, N, B).total
                                        : dn::noalloc_layout<float>(m->desc, N, B).total;
    if (need > dn::kNoAllocScratchBytes) return DN_EINVAL;   // request larger than the fixed scratch
    void *scratch = nullptr;
    cudaError_t err = dn::noalloc_scratch(&scratch);
    if (err != cudaSuccess) return DN_ECUDA;
    dn::ProfPhase phase("noalloc");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(scratch);
    err = prec == DN_FP64 ? dn::noalloc_forward<double>(m, N, spins_dev, B, base,
                                                         dn::noalloc_layout<double>(m->desc, N, B), st, logpsi_dev,
                                                         Omega_dev)
                          : dn::noalloc_forward<float>(m, N, spins_dev, B, base, dn::noalloc_layout<float>(m->desc, N, B),
                                                       st, logpsi_dev, Omega_dev);
    return err == cudaSuccess ? DN_OK : DN_ECUDA;
}
