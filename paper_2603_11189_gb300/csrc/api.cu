// C ABI of the DysonNet / ABACUS library: argument checks, memory and the
// order of the kernels.  See include/dysonnet.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "dn_internal.cuh"

namespace {

dn_alloc_fn g_alloc = nullptr;
dn_free_fn g_free = nullptr;
void *g_ctx = nullptr;

// Upper bound on the bytes of caches that local_energy() keeps at once.
constexpr size_t kLocalEnergyBudget = size_t(8) << 30;
// Upper bound on the scratch of the recompute baseline per chunk of flips.
constexpr size_t kRecomputeBudget = size_t(2) << 30;

struct Fail {
    dn_status s;
};

inline void ck(cudaError_t e) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) throw Fail{DN_ENOMEM};
    throw Fail{DN_ECUDA};
}

// RAII device buffer from the installed allocator.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t s) : bytes(n), st(s) {
        p = dn::dev_alloc(n, s);
        if (!p) throw Fail{DN_ENOMEM};
    }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) dn::dev_free(p, bytes, st);
    }
    template <typename X>
    X *as(size_t off = 0) const {
        return reinterpret_cast<X *>(static_cast<char *>(p) + off);
    }
};

template <typename F>
dn_status guard(F &&fn) {
    try {
        return fn();
    } catch (const Fail &f) {
        return f.s;
    } catch (const std::bad_alloc &) {
        return DN_ENOMEM;
    } catch (...) {
        return DN_ECUDA;
    }
}

long long s4_size_of(const dn_model_desc &d) { return 8ll * d.d * d.s + d.d; }
long long layer_size_of(const dn_model_desc &d) {
    const long long W = 2 * d.w + 1;
    return s4_size_of(d) + W * d.d_h + d.d_h + (long long)d.d_h * d.d_h + d.d_h + (long long)d.d * d.d_h + d.d +
           2ll * d.d * d.d;
}
long long nparams_of(const dn_model_desc &d) {
    return d.L * layer_size_of(d) + s4_size_of(d) + (long long)d.d * d.d_out + d.d;
}

bool desc_ok(const dn_model_desc *d) {
    return d && d->L >= 1 && d->L <= dn::kMaxL && d->d >= 1 && d->d <= dn::kMaxD && d->s >= 1 && d->s <= 256 &&
           d->w >= 0 && d->w <= 6 && d->d_h >= 1 && d->d_h <= dn::kMaxDh && d->d_out >= 1 &&
           d->d_out <= dn::kMaxDout && (d->periodic == 0 || d->periodic == 1) && (d->f_kind == 0 || d->f_kind == 1);
}

template <typename T>
dn::Weights<T> &weights_of(dn_model *m);
template <>
dn::Weights<double> &weights_of<double>(dn_model *m) { return m->w64; }
template <>
dn::Weights<float> &weights_of<float>(dn_model *m) { return m->w32; }
template <typename T>
std::map<int, dn::Plan<T>> &plans_of(dn_model *m);
template <>
std::map<int, dn::Plan<double>> &plans_of<double>(dn_model *m) { return m->plan64; }
template <>
std::map<int, dn::Plan<float>> &plans_of<float>(dn_model *m) { return m->plan32; }

// Device weights in precision T (built once per model and precision).
template <typename T>
const dn::Weights<T> &ensure_weights(dn_model *m, cudaStream_t st) {
    const int slot = sizeof(T) == 8 ? 0 : 1;
    dn::Weights<T> &w = weights_of<T>(m);
    if (m->weights_ready[slot]) return w;
    const dn_model_desc &D = m->desc;
    const int L = D.L, d = D.d, dh = D.d_h, W = 2 * D.w + 1, dout = D.d_out;
    const long long n_kappa = (long long)L * W * dh, n_beta = (long long)L * dh, n_W1 = (long long)L * dh * dh,
                    n_b1 = (long long)L * dh, n_W2 = (long long)L * dh * d, n_b2 = (long long)L * d,
                    n_mat = (long long)L * d * d, n_A = (long long)d * dout, n_e = d;
    dn::Carve cv;
    const size_t o_kappa = cv.take<T>(n_kappa), o_beta = cv.take<T>(n_beta), o_W1 = cv.take<T>(n_W1),
                 o_b1 = cv.take<T>(n_b1), o_W2 = cv.take<T>(n_W2), o_b2 = cv.take<T>(n_b2), o_U = cv.take<T>(n_mat),
                 o_UT = cv.take<T>(n_mat), o_V = cv.take<T>(n_mat), o_VT = cv.take<T>(n_mat), o_A = cv.take<T>(n_A),
                 o_e = cv.take<T>(n_e);
    std::vector<unsigned char> host(cv.off, 0);
    auto H = [&](size_t off) { return reinterpret_cast<T *>(host.data() + off); };
    const double *P = m->params.data();
    for (int l = 0; l < L; ++l) {
        const double *q = P + (long long)l * m->layer_size + m->s4_size;
        const double *kap = q, *beta = kap + W * dh, *W1 = beta + dh, *b1 = W1 + dh * dh, *W2 = b1 + dh,
                     *b2 = W2 + (long long)d * dh, *U = b2 + d, *V = U + (long long)d * d;
        for (int i = 0; i < W * dh; ++i) H(o_kappa)[(long long)l * W * dh + i] = (T)kap[i];
        for (int i = 0; i < dh; ++i) H(o_beta)[(long long)l * dh + i] = (T)beta[i];
        for (int i = 0; i < dh; ++i) H(o_b1)[(long long)l * dh + i] = (T)b1[i];
        for (int e = 0; e < dh; ++e)
            for (int f = 0; f < dh; ++f) H(o_W1)[((long long)l * dh + f) * dh + e] = (T)W1[e * dh + f];
        for (int c = 0; c < d; ++c)
            for (int e = 0; e < dh; ++e) H(o_W2)[((long long)l * dh + e) * d + c] = (T)W2[c * dh + e];
        for (int c = 0; c < d; ++c) H(o_b2)[(long long)l * d + c] = (T)b2[c];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                const long long base = (long long)l * d * d;
                H(o_U)[base + a * d + b] = (T)U[a * d + b];
                H(o_UT)[base + b * d + a] = (T)U[a * d + b];
                H(o_V)[base + a * d + b] = (T)V[a * d + b];
                H(o_VT)[base + b * d + a] = (T)V[a * d + b];
            }
    }
    const double *fin = P + (long long)L * m->layer_size + m->s4_size;
    for (int i = 0; i < d * dout; ++i) H(o_A)[i] = (T)fin[i];
    for (int i = 0; i < d; ++i) H(o_e)[i] = (T)fin[d * dout + i];
    void *blk = dn::dev_alloc(cv.off, st);
    if (!blk) throw Fail{DN_ENOMEM};
    cudaError_t err = cudaMemcpyAsync(blk, host.data(), cv.off, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
        dn::dev_free(blk, cv.off, st);
        ck(err);
    }
    auto D_ = [&](size_t off) { return reinterpret_cast<T *>(static_cast<char *>(blk) + off); };
    w.kappa = D_(o_kappa); w.beta = D_(o_beta); w.W1T = D_(o_W1); w.b1 = D_(o_b1); w.W2T = D_(o_W2);
    w.b2 = D_(o_b2); w.U = D_(o_U); w.UT = D_(o_UT); w.V = D_(o_V); w.VT = D_(o_VT); w.A = D_(o_A); w.e = D_(o_e);
    w.block = blk;
    w.bytes = cv.off;
    m->weights_ready[slot] = true;
    return w;
}

// Kernel taps and pooling weights for chain length N (once per model, N and precision).
template <typename T>
const dn::Plan<T> &ensure_plan(dn_model *m, int N, cudaStream_t st) {
    auto &plans = plans_of<T>(m);
    auto it = plans.find(N);
    if (it != plans.end()) return it->second;
    dn::ProfPhase phase("plan");
    const dn_model_desc &D = m->desc;
    const int R = D.periodic ? N : 2 * N - 1;
    dn::Carve cv;
    const size_t o_t64 = cv.take<double>((size_t)(D.L + 1) * R * D.d), o_w64 = cv.take<double>((size_t)N * D.d),
                 o_t = cv.take<T>((size_t)D.L * R * D.d), o_w = cv.take<T>((size_t)N * D.d);
    const size_t spec_bytes = dn::tap_spectra_bytes<T>(N, D.periodic, D.d, D.L);
    const size_t o_s = spec_bytes ? cv.take<double>((spec_bytes + 7) / 8) : 0;
    void *blk = dn::dev_alloc(cv.off, st);
    if (!blk) throw Fail{DN_ENOMEM};
    dn::Plan<T> pl;
    pl.N = N;
    pl.R = R;
    pl.block = blk;
    pl.bytes = cv.off;
    char *base = static_cast<char *>(blk);
    pl.taps64 = reinterpret_cast<double *>(base + o_t64);
    pl.omega64 = reinterpret_cast<double *>(base + o_w64);
    pl.taps = reinterpret_cast<T *>(base + o_t);
    pl.omega = reinterpret_cast<T *>(base + o_w);
    cudaError_t err = dn::launch_taps(m, N, pl.taps64, pl.omega64, st);
    if (err == cudaSuccess) err = dn::launch_cast<T>(pl.taps64, pl.taps, (long long)D.L * R * D.d, st);
    if (err == cudaSuccess) err = dn::launch_cast<T>(pl.omega64, pl.omega, (long long)N * D.d, st);
    if (err == cudaSuccess && spec_bytes) {
        // tap spectra of the FFT convolution (weights only); where the transform does not fit,
        // the forward keeps the direct convolution
        pl.spec = base + o_s;
        err = dn::launch_tap_spectra<T>(N, D.periodic, D.d, D.L, R, pl.taps, pl.spec, st);
        if (err == cudaErrorNotSupported) {
            cudaGetLastError();
            pl.spec = nullptr;
            err = cudaSuccess;
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) {
        dn::dev_free(blk, cv.off, st);
        ck(err);
    }
    return plans.emplace(N, pl).first->second;
}

// Forward pass over B validated configurations.  chi [B][L][N][d] is written;
// y (may be null) receives V u0 per layer; Omega/logpsi in FP64.
template <typename T>
void run_forward(dn_model *m, const dn::Plan<T> &pl, const dn::Weights<T> &w, int N, const int8_t *spins, int B,
                 T *chi, T *y, double *Omega, double *logpsi, int prec, unsigned *flag, cudaStream_t st) {
    dn::ProfPhase phase("forward");
    const dn::Geom g = dn::geom_of(m, N);
    const int L = g.L, d = g.d;
    const long long field = (long long)N * d;
    DevBuf hb((size_t)B * field * sizeof(T), st), ub((size_t)B * field * sizeof(T), st),
        pb((size_t)B * (L + 1) * d * sizeof(double), st);
    T *h = hb.as<T>(), *u = ub.as<T>();
    double *pooled = pb.as<double>();
    ck(dn::launch_chi<T>(g, w, spins, B, chi, st));
    ck(dn::launch_pool0<T>(g, spins, w.e, pl.omega, B, pooled, (long long)(L + 1) * d, st));
    if constexpr (sizeof(T) == 4) {
        if (prec == DN_BF16 && dn::forward_tc_ok(g)) {
            // BF16: tensor cores, channel-major activations h[c][n B + b] (forward_tc.cu),
            // every operand carried as two BF16 terms (hi + lo; products hi*hi + hi*lo + lo*hi,
            // FP32 accumulation).  One BF16 term per operand gave log-amplitude-ratio errors of
            // 1e-3 absolute (0.11 in the ratio metric) on the J1-J2 N = 256, 6 x 64 x 64 model.
            // The FP32 forward stays on the FMA kernels: tensor-core FP32 accumulation over
            // the K = N sites of the convolution, even with operands split into three BF16
            // planes, measured 1.1e-4 on log-ratios of the N = 128 workload model, above the
            // FP32 bound.
            const int planes = 2;
            ck(dn::launch_h0_cm(g, spins, w.e, B, h, st));
            for (int l = 1; l <= L; ++l) {
                const T *taps_l = pl.taps + (long long)(l - 1) * g.R * d;
                ck(dn::launch_tgemm_tc(g, taps_l, B, h, nullptr, nullptr, 0, u, nullptr, 0, 0, 0, 0, 1, 0, 1, flag, st,
                                       planes));
                ck(dn::launch_mix_tc(g, l, w, u, chi, y, h, B, planes, flag, st));
                ck(dn::launch_pool_cm(g, l, h, pl.omega, B, pooled, (long long)(L + 1) * d, st));
            }
            ck(dn::launch_readout(g, m->desc.f_kind, m->A64, pooled, L + 1, B, spins, Omega, logpsi, st));
            return;
        }
    }
    if (prec == DN_BF16) throw Fail{DN_EUNSUPPORTED};
    dn::Fields<T> H{h, field, 0, 1}, Uf{u, field, 0, 1}, none{nullptr, 0, 0, 1};
    const bool fft_conv = dn::use_fft_conv<T>(g, pl);
    for (int l = 1; l <= L; ++l) {
        const T *taps_l = pl.taps + (long long)(l - 1) * g.R * d;
        if (fft_conv)
            ck(dn::launch_conv_fft<T>(g, l, pl.spec, H, l == 1 ? spins : nullptr, w.e, Uf, B, st));
        else
            ck(dn::launch_conv<T>(g, taps_l, H, l == 1 ? spins : nullptr, w.e, Uf, B, false, nullptr, nullptr, st));
        dn::Fields<T> Y = y ? dn::Fields<T>{y + (long long)(l - 1) * field, (long long)L * field, 0, 1} : none;
        ck(dn::launch_mix<T>(g, l, w, chi, (long long)L * field, 1, 0, Uf, H, Y, pl.omega, pooled + (long long)l * d,
                             (long long)(L + 1) * d, B, false, st));
    }
    ck(dn::launch_readout(g, m->desc.f_kind, m->A64, pooled, L + 1, B, spins, Omega, logpsi, st));
}

// Adjoint of the frozen network (output links rho, t).
template <typename T>
void run_adjoint(dn_model *m, const dn::Plan<T> &pl, const dn::Weights<T> &w, dn_cache *c, cudaStream_t st) {
    dn::ProfPhase phase("adjoint");
    const dn::Geom g = dn::geom_of(m, c->N);
    const int L = g.L, d = g.d, dout = g.dout, N = c->N, B = c->B;
    const long long field = (long long)N * d;
    const long long F = (long long)B * dout;
    DevBuf zb((size_t)F * field * sizeof(T), st), r0((size_t)F * field * sizeof(T), st);
    T *rho = static_cast<T *>(c->rho);
    auto rho_layer = [&](int l) { return dn::Fields<T>{rho + (long long)(l - 1) * dout * field, (long long)L * dout * field, field, dout}; };
    dn::Fields<T> Z{zb.as<T>(), field, 0, 1}, R0{r0.as<T>(), field, 0, 1}, none{nullptr, 0, 0, 1};
    ck(dn::launch_rho_init<T>(g, w.A, pl.omega, rho_layer(L), F, st));
    for (int l = L; l >= 1; --l) {
        ck(dn::launch_mix<T>(g, l, w, static_cast<const T *>(c->chi), (long long)L * field, dout, 0, rho_layer(l), Z,
                             none, nullptr, nullptr, 0, F, true, st));
        dn::Fields<T> out = l >= 2 ? rho_layer(l - 1) : R0;
        ck(dn::launch_conv<T>(g, pl.taps + (long long)(l - 1) * g.R * d, Z, nullptr, nullptr, out, F, true, w.A,
                              pl.omega, st));
    }
    ck(dn::launch_tlink<T>(g, r0.as<T>(), w.e, B, static_cast<T *>(c->t), st));
}

struct CacheLayout {
    size_t spins, chi, y, rho, t, ell, K, Omega, logpsi, flag, total;
};

template <typename T>
CacheLayout cache_layout(const dn_model_desc &D, int N, int B, int max_cluster) {
    const int W = 2 * D.w + 1, WF = W + max_cluster - 1, Rk = WF - 1, Rl = WF - 1 - D.w;
    const long long P = D.L >= 3 ? (long long)(D.L - 1) * (D.L - 2) / 2 : 0;
    const long long field = (long long)N * D.d;
    dn::Carve cv;
    CacheLayout cl;
    cl.spins = cv.take<int8_t>((size_t)B * N);
    cl.chi = cv.take<T>((size_t)B * D.L * field);
    cl.y = cv.take<T>((size_t)B * D.L * field);
    cl.rho = cv.take<T>((size_t)B * D.L * D.d_out * field);
    cl.t = cv.take<T>((size_t)B * N * D.d_out);
    cl.ell = cv.take<T>((size_t)B * (D.L - 1) * N * (2 * Rl + 1) * D.d);
    cl.K = cv.take<T>((size_t)B * P * N * (2 * Rk + 1) * D.d * D.d);
    cl.Omega = cv.take<double>((size_t)B * D.d_out);
    cl.logpsi = cv.take<double>((size_t)B);
    cl.flag = cv.take<unsigned>(1);
    cl.total = (cv.off + 255) & ~size_t(255);
    return cl;
}

size_t cache_bytes(const dn_model_desc &D, int N, int B, int prec, int mc) {
    return prec == DN_FP64 ? cache_layout<double>(D, N, B, mc).total : cache_layout<float>(D, N, B, mc).total;
}

bool prec_valid(int prec) { return prec == DN_FP64 || prec == DN_FP32 || prec == DN_BF16; }

// BF16 runs only where the tensor-core forward applies.
bool prec_supported(const dn_model *m, int prec) {
    if (prec != DN_BF16) return true;
    const int d = m->desc.d;
    return d % 16 == 0 && d >= 16 && d <= 128;
}

bool cache_args_ok(const dn_model *m, int N, int B, int mc) {
    if (!m || N < 1 || B < 1 || mc < 1 || mc > 3) return false;
    const int W = 2 * m->desc.w + 1, WF = W + mc - 1;
    if (WF > 16) return false;
    if (m->desc.periodic && N < 2 * WF - 1) return false;
    return true;
}

template <typename T>
dn_cache *build_cache(dn_model *m, int N, const int8_t *spins_dev, int B, int prec, int mc, cudaStream_t st) {
    const dn::Plan<T> &pl = ensure_plan<T>(m, N, st);
    const dn::Weights<T> &w = ensure_weights<T>(m, st);
    const dn_model_desc &D = m->desc;
    const CacheLayout cl = cache_layout<T>(D, N, B, mc);
    dn_cache *c = new dn_cache();
    c->model = m;
    c->N = N;
    c->B = B;
    c->prec = prec;
    c->max_cluster = mc;
    c->WF = 2 * D.w + mc;
    c->Rk = c->WF - 1;
    c->Rl = c->WF - 1 - D.w;
    c->P = D.L >= 3 ? (D.L - 1) * (D.L - 2) / 2 : 0;
    c->stream = st;
    c->block = dn::dev_alloc(cl.total, st);
    if (!c->block) {
        delete c;
        throw Fail{DN_ENOMEM};
    }
    c->bytes = cl.total;
    char *base = static_cast<char *>(c->block);
    c->spins = reinterpret_cast<int8_t *>(base + cl.spins);
    c->chi = base + cl.chi;
    c->y = base + cl.y;
    c->rho = base + cl.rho;
    c->t = base + cl.t;
    c->ell = base + cl.ell;
    c->K = base + cl.K;
    c->Omega = reinterpret_cast<double *>(base + cl.Omega);
    c->logpsi = reinterpret_cast<double *>(base + cl.logpsi);
    c->flag = reinterpret_cast<unsigned *>(base + cl.flag);
    try {
        ck(cudaMemsetAsync(c->flag, 0, sizeof(unsigned), st));
        ck(dn::launch_check_spins(spins_dev, (long long)B * N, c->spins, c->flag, st));
        run_forward<T>(m, pl, w, N, c->spins, B, static_cast<T *>(c->chi), static_cast<T *>(c->y), c->Omega,
                       c->logpsi, prec, c->flag, st);
        run_adjoint<T>(m, pl, w, c, st);
        if (D.L >= 2) {
            dn::ProfPhase phase("links");
            const size_t elems = dn::links_scratch_elems(m, N, B);
            DevBuf sb(elems * sizeof(T), st);
            ck(dn::build_links<T>(m, pl, w, c, sb.as<T>(), elems, st));
        }
    } catch (...) {
        dn::dev_free(c->block, c->bytes, st);
        delete c;
        throw;
    }
    return c;
}

template <typename T>
void full_forward(dn_model *m, int N, const int8_t *spins_dev, int B, int prec, cudaStream_t st, double *logpsi,
                  double *Omega) {
    const dn::Plan<T> &pl = ensure_plan<T>(m, N, st);
    const dn::Weights<T> &w = ensure_weights<T>(m, st);
    DevBuf chi((size_t)B * m->desc.L * N * m->desc.d * sizeof(T), st);
    // No cache flag here: a timed-out tensor-core tile writes NaN, which reaches logpsi.
    run_forward<T>(m, pl, w, N, spins_dev, B, chi.as<T>(), nullptr, Omega, logpsi, prec, nullptr, st);
}

// Upper bound on the activations kept by dn_logpsi_grad() per chunk of samples.
constexpr size_t kGradBudget = size_t(6) << 30;

// Per-configuration log-derivatives (grad.cu): forward keeping every activation, then the
// reverse pass layer by layer.  O [B][P] in T (may be null when only vjp is wanted);
// vjp [P] (may be null) += sum_b wts_b O_b.
template <typename T>
void run_grad(dn_model *m, int N, const int8_t *spins_dev, int B, cudaStream_t st, double *logpsi, T *O,
              const double *wts, double *vjp) {
    dn::ProfPhase phase("grad");
    const dn::Plan<T> &pl = ensure_plan<T>(m, N, st);
    const dn::Weights<T> &w = ensure_weights<T>(m, st);
    const dn::Geom g = dn::geom_of(m, N);
    const dn_model_desc &D = m->desc;
    const int L = g.L, d = g.d, dh = g.dh, W = g.W, dout = g.dout, R = g.R;
    const long long P = (long long)m->nparams, field = (long long)N * d, fh = (long long)N * dh;
    const size_t per = sizeof(T) * ((size_t)(4 * L + 1) * field + 6 * field + 4 * fh + (size_t)N * W +
                                    (size_t)R * d + (O ? 0 : (size_t)P)) +
                       sizeof(double) * ((size_t)(L + 1) * d + d + dout + 1) + (size_t)N + 4096;
    const int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)B, kGradBudget / per));
    DevBuf flag(sizeof(unsigned), st);
    DevBuf pw((size_t)(L + 1) * d * D.s * (N + 1) * 2 * sizeof(T), st);
    ck(cudaMemsetAsync(flag.p, 0, sizeof(unsigned), st));
    ck(dn::launch_s4_pow<T>(m, N, pw.as<T>(), st));
    if (vjp) ck(cudaMemsetAsync(vjp, 0, (size_t)P * sizeof(double), st));
    dn::Carve cv;
    const size_t o_sp = cv.take<int8_t>((size_t)nb * N), o_chi = cv.take<T>((size_t)nb * L * field),
                 o_h = cv.take<T>((size_t)(L + 1) * nb * field), o_u = cv.take<T>((size_t)L * nb * field),
                 o_y = cv.take<T>((size_t)L * nb * field), o_dH = cv.take<T>((size_t)nb * field),
                 o_dU = cv.take<T>((size_t)nb * field), o_dT = cv.take<T>((size_t)nb * field),
                 o_tY = cv.take<T>((size_t)nb * field), o_dy = cv.take<T>((size_t)nb * field),
                 o_dchi = cv.take<T>((size_t)nb * field), o_a1 = cv.take<T>((size_t)nb * fh),
                 o_phi = cv.take<T>((size_t)nb * fh), o_dz = cv.take<T>((size_t)nb * fh),
                 o_dphi = cv.take<T>((size_t)nb * fh), o_win = cv.take<T>((size_t)nb * N * W),
                 o_dg = cv.take<T>((size_t)nb * R * d), o_pool = cv.take<double>((size_t)nb * (L + 1) * d),
                 o_om = cv.take<double>((size_t)nb * dout), o_lp = cv.take<double>((size_t)nb),
                 o_ac = cv.take<double>((size_t)nb * d), o_O = cv.take<T>(O ? 0 : (size_t)nb * P);
    DevBuf work(cv.off, st);
    int8_t *sp = work.as<int8_t>(o_sp);
    T *chi = work.as<T>(o_chi), *h = work.as<T>(o_h), *u = work.as<T>(o_u), *y = work.as<T>(o_y);
    T *dH = work.as<T>(o_dH), *dU = work.as<T>(o_dU), *dT = work.as<T>(o_dT), *dg = work.as<T>(o_dg);
    dn::GradScratch<T> scr{work.as<T>(o_tY), work.as<T>(o_dy), work.as<T>(o_dchi), work.as<T>(o_a1),
                           work.as<T>(o_phi), work.as<T>(o_dz), work.as<T>(o_dphi), work.as<T>(o_win)};
    double *pooled = work.as<double>(o_pool), *Omega = work.as<double>(o_om), *acoef = work.as<double>(o_ac);
    const long long pstride = (long long)(L + 1) * d;
    const long long s4 = m->s4_size, ls = m->layer_size;
    const long long offA = (long long)L * ls + s4, offE = offA + (long long)d * dout;
    for (int b0 = 0; b0 < B; b0 += nb) {
        const int n = std::min(nb, B - b0);
        const long long nf = (long long)n * field;
        T *Ob = O ? O + (long long)b0 * P : work.as<T>(o_O);
        double *lp = logpsi ? logpsi + b0 : work.as<double>(o_lp);
        auto F1 = [&](T *base) { return dn::Fields<T>{base, field, 0, 1}; };
        // forward, every activation kept (layer-major h^(0..L), u, y)
        ck(dn::launch_check_spins(spins_dev + (long long)b0 * N, (long long)n * N, sp, flag.as<unsigned>(), st));
        ck(dn::launch_chi<T>(g, w, sp, n, chi, st));
        ck(dn::launch_h0<T>(N, d, n, sp, w.e, h, st));
        ck(dn::launch_pool0<T>(g, sp, w.e, pl.omega, n, pooled, pstride, st));
        for (int l = 1; l <= L; ++l) {
            const T *taps_l = pl.taps + (long long)(l - 1) * R * d;
            ck(dn::launch_conv<T>(g, taps_l, F1(h + (l - 1) * nf), nullptr, w.e, F1(u + (l - 1) * nf), n, false,
                                  nullptr, nullptr, st));
            ck(dn::launch_mix<T>(g, l, w, chi, (long long)L * field, 1, 0, F1(u + (l - 1) * nf), F1(h + l * nf),
                                 F1(y + (l - 1) * nf), pl.omega, pooled + (long long)l * d, pstride, n, false, st));
        }
        ck(dn::launch_readout(g, D.f_kind, m->A64, pooled, L + 1, n, sp, Omega, lp, st));
        if (!O && !vjp) continue;
        // reverse pass
        ck(dn::launch_grad_readout<T>(g, D.f_kind, L + 1, n, m->A64, pooled, Omega, acoef, Ob, P, offA, st));
        ck(dn::launch_add_omega<T>(g, n, pl.omega, acoef, dH, false, st));
        for (int l = L; l >= 1; --l) {
            const long long base = (long long)(l - 1) * ls;
            const long long oK = base + s4, oBeta = oK + (long long)W * dh, oW1 = oBeta + dh, oB1 = oW1 + (long long)dh * dh,
                            oW2 = oB1 + dh, oB2 = oW2 + (long long)d * dh, oU = oB2 + d, oV = oU + (long long)d * d;
            ck(dn::launch_mix<T>(g, l, w, chi, (long long)L * field, 1, 0, F1(dH), F1(dU), F1(dT), nullptr, nullptr, 0,
                                 n, true, st));
            ck(dn::launch_mlp_back<T>(g, l, w, sp, n, chi, y + (l - 1) * nf, dT, scr, st));
            ck(dn::launch_outer<T>(N, n, d, d, dH, scr.tY, Ob, P, oU, d, st));
            ck(dn::launch_outer<T>(N, n, d, d, scr.dy, u + (l - 1) * nf, Ob, P, oV, d, st));
            ck(dn::launch_outer<T>(N, n, d, dh, scr.dchi, scr.a1, Ob, P, oW2, dh, st));
            ck(dn::launch_outer<T>(N, n, d, 1, scr.dchi, nullptr, Ob, P, oB2, 1, st));
            ck(dn::launch_outer<T>(N, n, dh, dh, scr.dz, scr.phi, Ob, P, oW1, dh, st));
            ck(dn::launch_outer<T>(N, n, dh, 1, scr.dz, nullptr, Ob, P, oB1, 1, st));
            ck(dn::launch_outer<T>(N, n, W, dh, scr.win, scr.dphi, Ob, P, oK, dh, st));
            ck(dn::launch_outer<T>(N, n, dh, 1, scr.dphi, nullptr, Ob, P, oBeta, 1, st));
            ck(dn::launch_dtaps<T>(g, n, dU, h + (l - 1) * nf, dg, st));
            ck(dn::launch_s4_grad<T>(m, l - 1, N, n, dg, pw.as<T>(), Ob, P, st));
            ck(dn::launch_conv<T>(g, pl.taps + (long long)(l - 1) * R * d, F1(dU), nullptr, nullptr, F1(dH), n, true,
                                  nullptr, nullptr, st));
            ck(dn::launch_add_omega<T>(g, n, pl.omega, acoef, dH, true, st));
        }
        ck(dn::launch_grad_e<T>(g, n, dH, sp, Ob, P, offE, st));
        ck(dn::launch_grad_gf<T>(g, n, h, nf, acoef, dg, st));
        ck(dn::launch_s4_grad<T>(m, L, N, n, dg, pw.as<T>(), Ob, P, st));
        if (vjp) ck(dn::launch_vjp<T>(Ob, wts + b0, n, P, vjp, st));
    }
    unsigned bad = 0;
    ck(cudaMemcpyAsync(&bad, flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (bad) throw Fail{DN_EINVAL};
}

}  // namespace

namespace dn {

// Every block is released by the allocator that produced it, even if another
// allocator has been installed in between.
struct Owner {
    dn_free_fn free_fn;
    void *ctx;
};
static std::mutex g_owner_mu;
static std::unordered_map<void *, Owner> g_owner;

void *dev_alloc(size_t bytes, cudaStream_t stream) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    dn_alloc_fn a;
    dn_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_owner_mu);
        a = g_alloc;
        f = g_free;
        ctx = g_ctx;
    }
    if (a) {
        p = a(bytes, (void *)stream, ctx);
    } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        std::lock_guard<std::mutex> lk(g_owner_mu);
        g_owner[p] = Owner{a ? f : nullptr, ctx};
    }
    return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t stream) {
    if (!p) return;
    Owner o{nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lk(g_owner_mu);
        auto it = g_owner.find(p);
        if (it != g_owner.end()) {
            o = it->second;
            g_owner.erase(it);
        }
    }
    if (o.free_fn) o.free_fn(p, bytes, (void *)stream, o.ctx);
    else cudaFreeAsync(p, stream);
}

}  // namespace dn

extern "C" {

dn_status dn_set_allocator(dn_alloc_fn alloc, dn_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return DN_EINVAL;
    std::lock_guard<std::mutex> lk(dn::g_owner_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = ctx;
    return DN_OK;
}

const char *dn_status_string(dn_status s) {
    switch (s) {
        case DN_OK: return "DN_OK";
        case DN_EINVAL: return "DN_EINVAL: invalid argument or invalid device data";
        case DN_ENOMEM: return "DN_ENOMEM: device allocation refused";
        case DN_ECUDA: return "DN_ECUDA: CUDA runtime or launch error";
        case DN_ETIMEOUT: return "DN_ETIMEOUT: bounded device wait gave up";
        case DN_EUNSUPPORTED: return "DN_EUNSUPPORTED: not implemented by this library";
    }
    return "unknown dn_status";
}

dn_status dn_model_create(const dn_model_desc *desc, const double *params_host, size_t n_params,
                          dn_model **model_out) {
    if (!model_out) return DN_EINVAL;
    *model_out = nullptr;
    if (!desc_ok(desc) || !params_host) return DN_EINVAL;
    if ((long long)n_params != nparams_of(*desc)) return DN_EINVAL;
    return guard([&]() -> dn_status {
        dn_model *m = new dn_model();
        m->desc = *desc;
        m->W = 2 * desc->w + 1;
        m->nparams = n_params;
        m->s4_size = s4_size_of(*desc);
        m->layer_size = layer_size_of(*desc);
        m->params.assign(params_host, params_host + n_params);
        const size_t nA = (size_t)desc->d * desc->d_out;
        void *blk = dn::dev_alloc((n_params + nA) * sizeof(double), nullptr);
        if (!blk) {
            delete m;
            return DN_ENOMEM;
        }
        m->params_dev = static_cast<double *>(blk);
        m->A64 = m->params_dev + n_params;
        const double *A = params_host + desc->L * m->layer_size + m->s4_size;
        cudaError_t err = cudaMemcpyAsync(m->params_dev, params_host, n_params * sizeof(double),
                                          cudaMemcpyHostToDevice, nullptr);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(m->A64, A, nA * sizeof(double), cudaMemcpyHostToDevice, nullptr);
        if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
        if (err != cudaSuccess) {
            dn::dev_free(blk, (n_params + nA) * sizeof(double), nullptr);
            delete m;
            return err == cudaErrorMemoryAllocation ? DN_ENOMEM : DN_ECUDA;
        }
        *model_out = m;
        return DN_OK;
    });
}

void dn_model_destroy(dn_model *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    for (auto &kv : m->plan64) dn::dev_free(kv.second.block, kv.second.bytes, nullptr);
    for (auto &kv : m->plan32) dn::dev_free(kv.second.block, kv.second.bytes, nullptr);
    if (m->w64.block) dn::dev_free(m->w64.block, m->w64.bytes, nullptr);
    if (m->w32.block) dn::dev_free(m->w32.block, m->w32.bytes, nullptr);
    dn::dev_free(m->params_dev, (m->nparams + (size_t)m->desc.d * m->desc.d_out) * sizeof(double), nullptr);
    cudaStreamSynchronize(nullptr);
    delete m;
}

size_t dn_cache_bytes(const dn_model *m, int N, int batch, dn_precision prec, int max_cluster) {
    if (!cache_args_ok(m, N, batch, max_cluster) || !prec_valid(prec)) return 0;
    return cache_bytes(m->desc, N, batch, prec, max_cluster);
}

dn_status dysonnet_forward_cache(dn_model *m, int N, const int8_t *spins_dev, int B, dn_precision prec,
                                 int max_cluster, void *stream, dn_cache **cache_out, double *logpsi_dev) {
    if (!cache_out) return DN_EINVAL;
    *cache_out = nullptr;
    if (!cache_args_ok(m, N, B, max_cluster) || !spins_dev || !prec_valid(prec)) return DN_EINVAL;
    if (!prec_supported(m, prec)) return DN_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn_cache *c = prec == DN_FP64 ? build_cache<double>(m, N, spins_dev, B, prec, max_cluster, st)
                                      : build_cache<float>(m, N, spins_dev, B, prec, max_cluster, st);
        if (logpsi_dev) {
            cudaError_t err = cudaMemcpyAsync(logpsi_dev, c->logpsi, (size_t)B * sizeof(double),
                                              cudaMemcpyDeviceToDevice, st);
            if (err != cudaSuccess) {
                dn::dev_free(c->block, c->bytes, st);
                delete c;
                ck(err);
            }
        }
        *cache_out = c;
        return DN_OK;
    });
}

dn_status abacus_flip_ratios(const dn_cache *c, const int32_t *sample_dev, const int32_t *sites_dev, int F,
                             double *dlogpsi_dev, void *stream) {
    if (!c || F < 0) return DN_EINVAL;
    if (F == 0) return DN_OK;
    if (!sample_dev || !sites_dev || !dlogpsi_dev) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("abacus");
        dn_model *m = c->model;
        if (c->prec == DN_FP64)
            ck(dn::launch_abacus<double>(m, m->plan64.at(c->N), m->w64, c, sample_dev, sites_dev, F, dlogpsi_dev, st));
        else
            ck(dn::launch_abacus<float>(m, m->plan32.at(c->N), m->w32, c, sample_dev, sites_dev, F, dlogpsi_dev, st));
        return DN_OK;
    });
}

dn_status abacus_single_flip_ratios(const dn_cache *c, double *dlogpsi_dev, void *stream) {
    if (!c || !dlogpsi_dev) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("abacus");
        dn_model *m = c->model;
        DevBuf scratch(dn::singles_scratch_bytes(m, c), st);
        cudaError_t err = c->prec == DN_FP64 ? dn::launch_abacus_singles<double>(m, m->plan64.at(c->N), m->w64, c,
                                                                                  scratch.p, dlogpsi_dev, st)
                                             : dn::launch_abacus_singles<float>(m, m->plan32.at(c->N), m->w32, c,
                                                                                 scratch.p, dlogpsi_dev, st);
        if (err == cudaErrorNotSupported) {
            // Shapes outside the grouped kernel: the general kernel on the explicit list.
            cudaGetLastError();
            const long long F = (long long)c->B * c->N;
            DevBuf smp((size_t)F * sizeof(int32_t), st), sts((size_t)F * 2 * sizeof(int32_t), st);
            ck(dn::launch_make_flips(0, c->N, c->B, 0, c->spins, smp.as<int32_t>(), sts.as<int32_t>(), st));
            if (c->prec == DN_FP64)
                err = dn::launch_abacus<double>(m, m->plan64.at(c->N), m->w64, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                                (int)F, dlogpsi_dev, st);
            else
                err = dn::launch_abacus<float>(m, m->plan32.at(c->N), m->w32, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                               (int)F, dlogpsi_dev, st);
        }
        ck(err);
        return DN_OK;
    });
}

// Pair flips grouped by site (anti: antialigned pairs only, the others 0); arguments checked.
static dn_status pair_ratios(const dn_cache *c, int n_bonds, const int32_t *bonds, bool anti, double *dlogpsi_dev,
                            void *stream) {
    if (!c || !bonds || !dlogpsi_dev || n_bonds < 1 || n_bonds > 2) return DN_EINVAL;
    for (int q = 0; q < n_bonds; ++q)
        if (bonds[q] < 1 || bonds[q] > c->max_cluster - 1) return DN_EINVAL;
    if (n_bonds == 2 && bonds[0] == bonds[1]) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("abacus");
        dn_model *m = c->model;
        const int bd[2] = {bonds[0], n_bonds > 1 ? bonds[1] : 0};
        cudaError_t err = cudaErrorNotSupported;
        if (dn::pairs_grouped_fits(m, c, n_bonds, bd)) {
            DevBuf scratch(dn::pairs_scratch_bytes(m, c, n_bonds, bd), st);
            err = c->prec == DN_FP64 ? dn::launch_abacus_pairs<double>(m, m->plan64.at(c->N), m->w64, c, n_bonds, bd,
                                                                      anti, scratch.p, dlogpsi_dev, st)
                                     : dn::launch_abacus_pairs<float>(m, m->plan32.at(c->N), m->w32, c, n_bonds, bd,
                                                                     anti, scratch.p, dlogpsi_dev, st);
        }
        if (err == cudaErrorNotSupported) {
            // Shapes outside the grouped kernel: the flip-list kernel on the same pairs.
            cudaGetLastError();
            const long long F = (long long)c->B * n_bonds * c->N;
            DevBuf smp((size_t)F * sizeof(int32_t), st), sts((size_t)F * 2 * sizeof(int32_t), st);
            ck(dn::launch_make_pair_flips(c->N, c->B, m->desc.periodic, n_bonds, bd, anti, c->spins,
                                          smp.as<int32_t>(), sts.as<int32_t>(), st));
            if (c->prec == DN_FP64)
                err = dn::launch_abacus<double>(m, m->plan64.at(c->N), m->w64, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                                (int)F, dlogpsi_dev, st);
            else
                err = dn::launch_abacus<float>(m, m->plan32.at(c->N), m->w32, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                               (int)F, dlogpsi_dev, st);
        }
        ck(err);
        return DN_OK;
    });
}

dn_status abacus_pair_flip_ratios(const dn_cache *c, int n_bonds, const int32_t *bonds, double *dlogpsi_dev,
                                  void *stream) {
    return pair_ratios(c, n_bonds, bonds, false, dlogpsi_dev, stream);
}

dn_status local_energy(dn_model *m, const dn_hamiltonian *H, int N, const int8_t *spins_dev, int B,
                       dn_precision prec, void *stream, double *eloc_dev) {
    if (!m || !H || !spins_dev || !eloc_dev || B < 1 || N < 1) return DN_EINVAL;
    if (!prec_valid(prec)) return DN_EINVAL;
    if (!prec_supported(m, prec)) return DN_EUNSUPPORTED;
    if (H->kind != 0 && H->kind != 1) return DN_EINVAL;
    if (H->kind == 1 && N < 3) return DN_EINVAL;
    if (H->kind == 0 && !(H->alpha >= 0.0)) return DN_EINVAL;
    const int mc = H->kind == 0 ? 1 : 3;
    if (!cache_args_ok(m, N, 1, mc)) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("eloc");
        const size_t per_sample = cache_bytes(m->desc, N, 1, prec, mc);
        int nb = (int)std::max<size_t>(1, kLocalEnergyBudget / std::max<size_t>(per_sample, 1));
        nb = std::min(nb, B);
        const int per = H->kind == 0 ? N : 2 * N;
        // Couplings J r^-alpha / N_a for r = 0..N-1 (TFIM).
        std::vector<double> coup(N, 0.0);
        if (H->kind == 0) {
            double norm = 1.0;
            if (H->kac) {
                norm = 0.0;
                for (int r = 1; r <= N / 2; ++r) norm += 2.0 * std::pow((double)r, -H->alpha);
            }
            for (int r = 1; r < N; ++r) coup[r] = H->J * std::pow((double)r, -H->alpha) / norm;
        }
        DevBuf cb((size_t)N * sizeof(double), st), smp((size_t)nb * per * sizeof(int32_t), st),
            sts((size_t)nb * per * 2 * sizeof(int32_t), st), dl((size_t)nb * per * sizeof(double), st);
        ck(cudaMemcpyAsync(cb.p, coup.data(), (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st));
        for (int b0 = 0; b0 < B; b0 += nb) {
            const int n = std::min(nb, B - b0);
            dn_cache *c = nullptr;
            dn_status s = dysonnet_forward_cache(m, N, spins_dev + (long long)b0 * N, n, prec, mc, stream, &c, nullptr);
            if (s != DN_OK) return s;
            cudaError_t err = cudaSuccess;
            if (H->kind == 0) {
                s = abacus_single_flip_ratios(c, dl.as<double>(), stream);
            } else if (H->periodic == m->desc.periodic) {
                // the antialigned pairs (j, j+1), (j, j+2) grouped by site: entry b 2N + (bond-1) N + j,
                // the layout k_eloc_reduce reads
                const int32_t bonds[2] = {1, 2};
                s = pair_ratios(c, 2, bonds, true, dl.as<double>(), stream);
            } else {
                err = dn::launch_make_flips(H->kind, N, n, H->periodic, c->spins, smp.as<int32_t>(), sts.as<int32_t>(),
                                            st);
                if (err == cudaSuccess)
                    s = abacus_flip_ratios(c, smp.as<int32_t>(), sts.as<int32_t>(), n * per, dl.as<double>(), stream);
            }
            if (err == cudaSuccess && s == DN_OK)
                err = dn::launch_eloc_reduce(*H, N, n, c->spins, cb.as<double>(), dl.as<double>(), eloc_dev + b0, st);
            dn_cache_destroy(c);
            if (s != DN_OK) return s;
            ck(err);
        }
        // Keep the host coupling table alive until its copy has run.
        ck(cudaStreamSynchronize(st));
        return DN_OK;
    });
}

dn_status dn_full_forward(dn_model *m, int N, const int8_t *spins_dev, int B, dn_precision prec, void *stream,
                          double *logpsi_dev, double *Omega_dev) {
    if (!m || !spins_dev || !logpsi_dev || N < 1 || B < 1) return DN_EINVAL;
    if (!prec_valid(prec)) return DN_EINVAL;
    if (!prec_supported(m, prec)) return DN_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        if (prec == DN_FP64) full_forward<double>(m, N, spins_dev, B, prec, st, logpsi_dev, Omega_dev);
        else full_forward<float>(m, N, spins_dev, B, prec, st, logpsi_dev, Omega_dev);
        return DN_OK;
    });
}

size_t dn_model_nparams(const dn_model *m) { return m ? m->nparams : 0; }

dn_status dn_logpsi_grad(dn_model *m, int N, const int8_t *spins_dev, int B, dn_precision prec, void *stream,
                         double *logpsi_dev, void *O_dev, const double *w_dev, double *vjp_dev) {
    if (!m || !spins_dev || N < 1 || B < 1) return DN_EINVAL;
    if ((w_dev == nullptr) != (vjp_dev == nullptr)) return DN_EINVAL;
    if (!O_dev && !vjp_dev && !logpsi_dev) return DN_EINVAL;
    if (!prec_valid(prec)) return DN_EINVAL;
    if (prec == DN_BF16) return DN_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        if (prec == DN_FP64) run_grad<double>(m, N, spins_dev, B, st, logpsi_dev, static_cast<double *>(O_dev), w_dev, vjp_dev);
        else run_grad<float>(m, N, spins_dev, B, st, logpsi_dev, static_cast<float *>(O_dev), w_dev, vjp_dev);
        return DN_OK;
    });
}

dn_status dn_sr_matrices(const void *O_dev, int B, size_t n_params, dn_precision prec, void *stream, double *gram_dev,
                         size_t k0, int nk, double *s_dev) {
    if (!O_dev || B < 1 || n_params < 1) return DN_EINVAL;
    if (prec != DN_FP64 && prec != DN_FP32) return DN_EINVAL;
    if (!gram_dev && !s_dev) return DN_EINVAL;
    if (s_dev && (nk < 1 || k0 + (size_t)nk > n_params)) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("sr");
        DevBuf mean(n_params * sizeof(double), st);
        if (prec == DN_FP64) {
            ck(dn::launch_sr_matrices<double>(static_cast<const double *>(O_dev), B, (long long)n_params, gram_dev,
                                              (long long)k0, s_dev ? nk : 0, s_dev, mean.as<double>(), nullptr, 0,
                                              st));
        } else {
            int nsplit = 1;
            const size_t pe = gram_dev ? dn::gram_tc_partial_elems(B, (long long)n_params, &nsplit) : 0;
            DevBuf part(std::max<size_t>(pe, 1) * sizeof(float), st);
            ck(dn::launch_sr_matrices<float>(static_cast<const float *>(O_dev), B, (long long)n_params, gram_dev,
                                             (long long)k0, s_dev ? nk : 0, s_dev, mean.as<float>(),
                                             gram_dev ? part.as<float>() : nullptr, nsplit, st));
        }
        return DN_OK;
    });
}

dn_status dn_sampler_batch(dn_model *m, int N, int8_t *spins_dev, int C, const int32_t *sites_dev, const double *u_dev,
                           int K, double eps, dn_precision prec, void *stream, int8_t *accepted_dev,
                           dn_sampler_stats *stats) {
    if (!m || !spins_dev || !sites_dev || !u_dev || N < 1 || C < 1 || K < 1 || !(eps >= 0.0)) return DN_EINVAL;
    if (!prec_valid(prec)) return DN_EINVAL;
    if (prec == DN_BF16) return DN_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("sampler");
        const int dout = m->desc.d_out;
        const long long F = (long long)C * K;
        DevBuf dom((size_t)F * dout * sizeof(double), st), om((size_t)C * dout * sizeof(double), st),
            kpos((size_t)C * sizeof(int32_t), st), amb((size_t)C * sizeof(int32_t), st),
            list((size_t)C * sizeof(int32_t), st), smp((size_t)F * sizeof(int32_t), st),
            sts((size_t)F * 2 * sizeof(int32_t), st), cnt(3 * sizeof(unsigned long long), st);
        ck(cudaMemsetAsync(cnt.p, 0, 3 * sizeof(unsigned long long), st));
        ck(cudaMemsetAsync(kpos.p, 0, (size_t)C * sizeof(int32_t), st));
        if (accepted_dev) ck(cudaMemsetAsync(accepted_dev, 0, (size_t)F, st));
        auto abacus_updates = [&](dn_cache *c, long long nf, double *dst) {
            if (c->prec == DN_FP64)
                ck(dn::launch_abacus<double>(m, m->plan64.at(N), m->w64, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                             (int)nf, nullptr, st, dst));
            else
                ck(dn::launch_abacus<float>(m, m->plan32.at(N), m->w32, c, smp.as<int32_t>(), sts.as<int32_t>(),
                                            (int)nf, nullptr, st, dst));
        };
        auto check_cache = [&](dn_cache *c) {
            const dn_status s = dn_cache_check(c, stream);
            if (s != DN_OK) {
                dn_cache_destroy(c);
                throw Fail{s};
            }
        };
        // caches of the starting configurations and the update vector of every proposal
        {
            dn_cache *c = nullptr;
            dn_status s = dysonnet_forward_cache(m, N, spins_dev, C, prec, 1, stream, &c, nullptr);
            if (s != DN_OK) return s;
            check_cache(c);
            try {
                ck(dn::launch_flip_list(C, K, sites_dev, nullptr, nullptr, smp.as<int32_t>(), sts.as<int32_t>(), st));
                abacus_updates(c, F, dom.as<double>());
                ck(cudaMemcpyAsync(om.p, c->Omega, (size_t)C * dout * sizeof(double), cudaMemcpyDeviceToDevice, st));
                check_cache(c);
            } catch (...) {
                dn_cache_destroy(c);
                throw;
            }
            dn_cache_destroy(c);
        }
        std::vector<int32_t> ambh((size_t)C);
        for (;;) {
            ck(dn::launch_screened_sweep(N, C, K, dout, m->desc.f_kind, eps, sites_dev, u_dev, dom.as<double>(),
                                         om.as<double>(), kpos.as<int32_t>(), spins_dev, accepted_dev,
                                         amb.as<int32_t>(), cnt.as<unsigned long long>(), st));
            ck(cudaMemcpyAsync(ambh.data(), amb.p, (size_t)C * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            ck(cudaStreamSynchronize(st));
            std::vector<int32_t> lst;
            for (int c = 0; c < C; ++c)
                if (ambh[c] >= 0) lst.push_back(c);
            if (lst.empty()) break;
            const int n = (int)lst.size();
            ck(cudaMemcpyAsync(list.p, lst.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            // exact decisions: log psi of the current configuration and of the proposal
            DevBuf cfg((size_t)2 * n * N, st), lp((size_t)2 * n * sizeof(double), st), rows((size_t)n * N, st);
            ck(dn::launch_pair_configs(N, K, n, list.as<int32_t>(), amb.as<int32_t>(), sites_dev, spins_dev,
                                       cfg.as<int8_t>(), st));
            dn_status s = dn_full_forward(m, N, cfg.as<int8_t>(), 2 * n, prec, stream, lp.as<double>(), nullptr);
            if (s != DN_OK) return s;
            ck(dn::launch_exact_decide(N, K, n, list.as<int32_t>(), amb.as<int32_t>(), sites_dev, u_dev,
                                       lp.as<double>(), spins_dev, accepted_dev, kpos.as<int32_t>(),
                                       cnt.as<unsigned long long>(), st));
            // refresh: caches of the new configurations, update vectors of the remaining proposals
            ck(dn::launch_gather_rows(N, n, list.as<int32_t>(), spins_dev, rows.as<int8_t>(), st));
            dn_cache *c = nullptr;
            s = dysonnet_forward_cache(m, N, rows.as<int8_t>(), n, prec, 1, stream, &c, nullptr);
            if (s != DN_OK) return s;
            try {
                DevBuf domn((size_t)n * K * dout * sizeof(double), st);
                ck(dn::launch_flip_list(n, K, sites_dev, list.as<int32_t>(), kpos.as<int32_t>(), smp.as<int32_t>(),
                                        sts.as<int32_t>(), st));
                abacus_updates(c, (long long)n * K, domn.as<double>());
                ck(dn::launch_scatter_refresh(K, dout, n, list.as<int32_t>(), kpos.as<int32_t>(), c->Omega,
                                              domn.as<double>(), om.as<double>(), dom.as<double>(), st));
                check_cache(c);
            } catch (...) {
                dn_cache_destroy(c);
                throw;
            }
            dn_cache_destroy(c);
        }
        if (stats) {
            unsigned long long h[3];
            ck(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, st));
            ck(cudaStreamSynchronize(st));
            stats->proposals = h[0];
            stats->accepted = h[1];
            stats->refreshes = h[2];
        }
        return DN_OK;
    });
}

dn_status dn_recompute_flip_ratios(dn_model *m, int N, const int8_t *spins_dev, int B, const int32_t *sample_dev,
                                   const int32_t *sites_dev, int F, dn_precision prec, void *stream,
                                   double *dlogpsi_dev) {
    if (!m || !spins_dev || N < 1 || B < 1 || F < 0) return DN_EINVAL;
    if (!prec_valid(prec)) return DN_EINVAL;
    if (!prec_supported(m, prec)) return DN_EUNSUPPORTED;
    if (F == 0) return DN_OK;
    if (!sample_dev || !sites_dev || !dlogpsi_dev) return DN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return guard([&]() -> dn_status {
        dn::ProfPhase phase("recompute");
        const size_t tb = prec == DN_FP64 ? 8 : 4;
        const size_t per_cfg = (size_t)N * m->desc.d * tb * (2 + m->desc.L) + (size_t)N + 64;
        int chunk = (int)std::max<size_t>(1, kRecomputeBudget / per_cfg);
        chunk = std::min(chunk, F);
        DevBuf base((size_t)B * sizeof(double), st), flag(sizeof(unsigned), st), cfg((size_t)chunk * N, st),
            lp((size_t)chunk * sizeof(double), st);
        ck(cudaMemsetAsync(flag.p, 0, sizeof(unsigned), st));
        dn_status s = dn_full_forward(m, N, spins_dev, B, prec, stream, base.as<double>(), nullptr);
        if (s != DN_OK) return s;
        for (int f0 = 0; f0 < F; f0 += chunk) {
            const int n = std::min(chunk, F - f0);
            ck(dn::launch_expand_flips(N, spins_dev, sample_dev + f0, sites_dev + 2ll * f0, n, B, cfg.as<int8_t>(),
                                       flag.as<unsigned>(), st));
            s = dn_full_forward(m, N, cfg.as<int8_t>(), n, prec, stream, lp.as<double>(), nullptr);
            if (s != DN_OK) return s;
            ck(dn::launch_sub_base(lp.as<double>(), base.as<double>(), sample_dev + f0, sites_dev + 2ll * f0, n, B, N,
                                   dlogpsi_dev + f0, st));
        }
        return DN_OK;
    });
}

dn_status dn_cache_check(const dn_cache *c, void *stream) {
    if (!c) return DN_EINVAL;
    unsigned flag = 0;
    cudaError_t err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (err == cudaSuccess) err = cudaMemcpy(&flag, c->flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return DN_ECUDA;
    return flag ? DN_EINVAL : DN_OK;
}

dn_status dn_cache_info(const dn_cache *c, int *N, int *B, int *prec, int *max_cluster) {
    if (!c) return DN_EINVAL;
    if (N) *N = c->N;
    if (B) *B = c->B;
    if (prec) *prec = c->prec;
    if (max_cluster) *max_cluster = c->max_cluster;
    return DN_OK;
}

dn_status dn_cache_tensor(const dn_cache *c, const char *name, void **dev_ptr, size_t *count, int *elem_bytes) {
    if (!c || !name || !dev_ptr) return DN_EINVAL;
    const dn_model_desc &D = c->model->desc;
    const long long B = c->B, N = c->N, L = D.L, d = D.d, dout = D.d_out;
    const int tb = c->prec == DN_FP64 ? 8 : 4;
    const long long P = c->P;
    struct Entry {
        const char *n;
        void *p;
        long long cnt;
        int eb;
    } tab[] = {
        {"spins", c->spins, B * N, 1},
        {"chi", c->chi, B * L * N * d, tb},
        {"y", c->y, B * L * N * d, tb},
        {"rho", c->rho, B * L * dout * N * d, tb},
        {"t", c->t, B * N * dout, tb},
        {"ell", c->ell, B * (L - 1) * N * (2 * c->Rl + 1) * d, tb},
        {"K", c->K, B * P * N * (2 * c->Rk + 1) * d * d, tb},
        {"Omega", c->Omega, B * dout, 8},
        {"logpsi", c->logpsi, B, 8},
    };
    for (const Entry &e : tab) {
        if (std::strcmp(e.n, name) == 0) {
            *dev_ptr = e.p;
            if (count) *count = (size_t)e.cnt;
            if (elem_bytes) *elem_bytes = e.eb;
            return DN_OK;
        }
    }
    return DN_EINVAL;
}

void dn_cache_destroy(dn_cache *c) {
    if (!c) return;
    dn::dev_free(c->block, c->bytes, c->stream);
    delete c;
}

}  // extern "C"
