// ABACUS local update (Alg. 1; Eqs. recur_step and recur_out; Theorem 1) and
// the local estimator (Eq. local-estimator) on sm_103a.
//
// One CTA per flip set F (one site, or two sites at separation <= max_cluster-1)
// on the slice S = [first - w, last + w] (width wf <= W_F).  For l = 1..L:
//   p_i   = sum_{k in S} g^(l)_{i-k} s^(l-1)_k                 (M~ s, slice Toeplitz)
//         + sum_{j in F} dsigma_j ell^(l)_{i,j}                (background-propagated
//                                                                embedding change, l >= 2)
//         + sum_{m=1}^{l-2} sum_{k in S} L^(l,m)_{i,k} s^(m)_k  (Eq. Lmn links)
//   s^(l)_i = U (dchi^(l)_i * (y^(l)_i + V p_i))     [= dD (h~_0 + ...) of Eq. recur_step]
//   dOmega += rho^(l)_i . s^(l)_i                     [T^(l) of Eq. recur_out]
// with s^(0)_j = e dsigma_j; dOmega also collects the flip's unscattered
// contribution sum_j t_j dsigma_j.  Output: sum_k f(Omega_k + dOmega_k) - f(Omega_k).
#include <math.h>

#include <cstring>
#include <type_traits>

#include "dn_internal.cuh"

namespace dn {

template <typename T>
__device__ __forceinline__ T gelu_ab(T x);
template <>
__device__ __forceinline__ double gelu_ab<double>(double x) {
    return 0.5 * x * (1.0 + erf(x * 0.70710678118654752440));
}
template <>
__device__ __forceinline__ float gelu_ab<float>(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678f));
}

__device__ __forceinline__ double log_cosh_ab(double x) {
    const double a = fabs(x);
    return a + log1p(exp(-2.0 * a)) - 0.69314718055994530942;
}

// 16-byte aligned, so that an array of these (the serving kernel's descriptor table, filled
// by the host with abacus_desc_bytes() per record) has the same stride on both sides.
template <typename T>
struct alignas(16) AbArgs {
    Geom g;
    int B, WF, Rk, Rl, P, max_cluster, f_kind;
    const int8_t *spins;
    const T *chi, *y, *rho, *t, *ell, *K, *taps;
    const double *Omega;
    unsigned *flag;
    Weights<T> w;
    double *dOmega;             // optional [F][dout]: the update vector of each flip set (Alg. 2), or null
};

constexpr int kAbThreads = 256;

// Body of the flip-list kernel: flip set f of the cache described by a, one CTA.
template <typename T>
__device__ __forceinline__ void abacus_flip_set(const AbArgs<T> &a, long long f, const int32_t *__restrict__ sample,
                                                const int32_t *__restrict__ sites, double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const Geom &g = a.g;
    const int N = g.N, d = g.d, dh = g.dh, L = g.L, WF = a.WF, dout = g.dout, wd = g.w;
    T *S = reinterpret_cast<T *>(smraw);          // [L+1][WF][d]
    T *p = S + (size_t)(L + 1) * WF * d;          // [WF][d]
    T *gz = p + (size_t)WF * d;                   // [WF][d]
    T *phi = gz + (size_t)WF * d;                 // [WF][dh]
    T *act = phi + (size_t)WF * dh;               // [WF][dh]
    double *red = reinterpret_cast<double *>(smraw + ((((size_t)(L + 3) * WF * d + 2 * (size_t)WF * dh) * sizeof(T) + 7) & ~(size_t)7));
    __shared__ int info[8];
    __shared__ int pos[16];
    const int tid = threadIdx.x;
    if (tid == 0) {
        int status = 0, b = sample[f], j0 = sites[2 * f], j1 = sites[2 * f + 1];
        int first = j0, sep = 0;
        if (j0 == -1) {
            status = 1;
        } else if (b < 0 || b >= a.B || j0 < 0 || j0 >= N) {
            status = 2;
        } else if (j1 != -1) {
            if (j1 < 0 || j1 >= N || j1 == j0) {
                status = 2;
            } else if (g.periodic) {
                const int dd = ((j1 - j0) % N + N) % N;
                sep = dd < N - dd ? dd : N - dd;
                first = (dd == sep) ? j0 : j1;
            } else {
                sep = j1 > j0 ? j1 - j0 : j0 - j1;
                first = j0 < j1 ? j0 : j1;
            }
            if (status == 0 && sep > a.max_cluster - 1) status = 2;
        }
        info[0] = status;
        info[1] = b;
        info[2] = j0;
        info[3] = j1;
        info[4] = first - wd;   // slice start
        info[5] = g.W + sep;    // slice width
    }
    __syncthreads();
    const int status = info[0];
    if (status == 1 || status == 2) {
        // empty entry: zero; invalid entry: NaN and the sticky flag (each output is optional)
        if (tid == 0) {
            const double v = status == 1 ? 0.0 : nan("");
            if (out) out[f] = v;
            if (a.dOmega)
                for (int k = 0; k < dout; ++k) a.dOmega[f * dout + k] = v;
            if (status == 2) atomicOr(a.flag, 2u);
        }
        return;
    }
    const long long b = info[1];
    const int j0 = info[2], j1 = info[3], start = info[4], wf = info[5];
    const int8_t *sp = a.spins + b * N;
    if (tid < wf) {
        int i = start + tid;
        if (g.periodic) i = ((i % N) + N) % N;
        else if (i < 0 || i >= N) i = -1;
        pos[tid] = i;
    }
    const int nflip = j1 >= 0 ? 2 : 1;
    const int jf[2] = {j0, j1};
    const T ds[2] = {(T)(-2 * sp[j0]), j1 >= 0 ? (T)(-2 * sp[j1]) : (T)0};
    __syncthreads();

    // Band offset k - i mapped to (-(WF-1), WF-1].
    auto offs = [&](int k, int i) -> int {
        int dl = k - i;
        if (g.periodic) {
            dl = ((dl % N) + N) % N;
            if (dl > WF - 1) dl -= N;
        }
        return dl;
    };
    auto tap = [&](int l, int r, int c) -> T {
        int row;
        if (g.periodic) {
            r = ((r % N) + N) % N;
            row = r;
        } else {
            row = r + N - 1;
        }
        return a.taps[((long long)(l - 1) * g.R + row) * d + c];
    };
    auto spin_new = [&](int j) -> T {
        if (g.periodic) j = ((j % N) + N) % N;
        else if (j < 0 || j >= N) return (T)0;
        T v = (T)sp[j];
        if (j == j0 || (j1 >= 0 && j == j1)) v = -v;
        return v;
    };

    double dom[kMaxDout];
#pragma unroll
    for (int k = 0; k < kMaxDout; ++k) dom[k] = 0.0;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    const long long dd = (long long)d * d;

    for (int l = 1; l <= L; ++l) {
        // (1) p = propagated change reaching the slice at layer l
        for (int idx = tid; idx < wf * d; idx += blockDim.x) {
            const int t = idx / d, c = idx % d;
            const int i = pos[t];
            T acc = 0;
            if (i >= 0) {
                if (l == 1) {
                    for (int q = 0; q < nflip; ++q) acc += tap(1, i - jf[q], c) * a.w.e[c] * ds[q];
                } else {
                    const T *Sp = S + (size_t)(l - 1) * WF * d;
                    for (int t2 = 0; t2 < wf; ++t2) {
                        const int k = pos[t2];
                        if (k >= 0) acc += tap(l, i - k, c) * Sp[t2 * d + c];
                    }
                    const T *el = a.ell + (((b * (L - 1) + (l - 2)) * N + i) * nRl) * d;
                    for (int q = 0; q < nflip; ++q) acc += ds[q] * el[(offs(jf[q], i) + a.Rl) * d + c];
                    for (int m = 1; m <= l - 2; ++m) {
                        const T *Kr = a.K + ((b * a.P + pair_index(l, m)) * N + i) * nRk * dd + (long long)c * d;
                        const T *Sm = S + (size_t)m * WF * d;
                        for (int t2 = 0; t2 < wf; ++t2) {
                            const int k = pos[t2];
                            if (k < 0) continue;
                            const T *Kb = Kr + (long long)(offs(k, i) + a.Rk) * dd;
                            const T *sv = Sm + t2 * d;
#pragma unroll 8
                            for (int c2 = 0; c2 < d; ++c2) acc += Kb[c2] * sv[c2];
                        }
                    }
                }
            }
            p[idx] = acc;
        }
        // (2) phi' on the slice with the flipped spins
        const T *kap = a.w.kappa + (long long)(l - 1) * g.W * dh;
        const T *beta = a.w.beta + (long long)(l - 1) * dh;
        for (int idx = tid; idx < wf * dh; idx += blockDim.x) {
            const int t = idx / dh, e = idx % dh;
            T acc = 0;
            if (pos[t] >= 0) {
                acc = beta[e];
                const int i = start + t;
                for (int r = -wd; r <= wd; ++r) acc += kap[(r + wd) * dh + e] * spin_new(i + r);
            }
            phi[idx] = acc;
        }
        __syncthreads();
        const T *W1T = a.w.W1T + (long long)(l - 1) * dh * dh;
        const T *b1 = a.w.b1 + (long long)(l - 1) * dh;
        for (int idx = tid; idx < wf * dh; idx += blockDim.x) {
            const int t = idx / dh, e = idx % dh;
            T acc = b1[e];
            for (int f2 = 0; f2 < dh; ++f2) acc += W1T[f2 * dh + e] * phi[t * dh + f2];
            act[idx] = gelu_ab<T>(acc);
        }
        __syncthreads();
        // (3) gz = dchi * (y + V p)
        const T *W2T = a.w.W2T + (long long)(l - 1) * dh * d;
        const T *b2 = a.w.b2 + (long long)(l - 1) * d;
        const T *VT = a.w.VT + (long long)(l - 1) * dd;
        for (int idx = tid; idx < wf * d; idx += blockDim.x) {
            const int t = idx / d, c = idx % d;
            const int i = pos[t];
            T val = 0;
            if (i >= 0) {
                T chin = b2[c];
                for (int e = 0; e < dh; ++e) chin += W2T[e * d + c] * act[t * dh + e];
                const long long ci = ((b * L + (l - 1)) * N + i) * d + c;
                const T dchi = chin - a.chi[ci];
                T z = a.y[ci];
                for (int c2 = 0; c2 < d; ++c2) z += VT[c2 * d + c] * p[t * d + c2];
                val = dchi * z;
            }
            gz[idx] = val;
        }
        __syncthreads();
        // (4) s^(l) = U gz ; dOmega += rho^(l) . s^(l)
        const T *UT = a.w.UT + (long long)(l - 1) * dd;
        T *Sl = S + (size_t)l * WF * d;
        for (int idx = tid; idx < wf * d; idx += blockDim.x) {
            const int t = idx / d, c = idx % d;
            const int i = pos[t];
            T sv = 0;
            if (i >= 0) {
                for (int c2 = 0; c2 < d; ++c2) sv += UT[c2 * d + c] * gz[t * d + c2];
#pragma unroll
                for (int k = 0; k < kMaxDout; ++k)
                    if (k < dout) dom[k] += (double)a.rho[(((b * L + (l - 1)) * dout + k) * N + i) * d + c] * (double)sv;
            }
            Sl[idx] = sv;
        }
        __syncthreads();
    }
    // Block reduction of dOmega.
#pragma unroll
    for (int k = 0; k < kMaxDout; ++k)
        if (k < dout) red[k * blockDim.x + tid] = dom[k];
    __syncthreads();
    if (tid < dout) {
        const int k = tid;
        double sum = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) sum += red[k * blockDim.x + q];
        for (int q = 0; q < nflip; ++q) sum += (double)a.t[(b * N + jf[q]) * dout + k] * (double)ds[q];
        red[k * blockDim.x] = sum;
    }
    __syncthreads();
    if (tid == 0) {
        double res = 0.0;
        for (int k = 0; k < dout; ++k) {
            const double om = a.Omega[b * dout + k];
            const double dk = red[k * blockDim.x];
            res += a.f_kind == 0 ? (log_cosh_ab(om + dk) - log_cosh_ab(om)) : dk;
            if (a.dOmega) a.dOmega[f * dout + k] = dk;
        }
        if (out) out[f] = res;
    }
}

template <typename T>
__global__ void __launch_bounds__(kAbThreads) k_abacus(AbArgs<T> a, const int32_t *__restrict__ sample,
                                                       const int32_t *__restrict__ sites, int F,
                                                       double *__restrict__ out) {
    abacus_flip_set<T>(a, blockIdx.x, sample, sites, out);
}

// Flip sets of several caches (of one model, same max_cluster) in one launch:
// flip set f belongs to cache cache_of[f], described by descs[cache_of[f]].
template <typename T>
__global__ void __launch_bounds__(kAbThreads) k_abacus_multi(const AbArgs<T> *__restrict__ descs,
                                                             const int32_t *__restrict__ cache_of,
                                                             const int32_t *__restrict__ sample,
                                                             const int32_t *__restrict__ sites, int F,
                                                             double *__restrict__ out) {
    __shared__ AbArgs<T> sa;
    const long long f = blockIdx.x;
    if (threadIdx.x == 0) sa = descs[cache_of[f]];
    __syncthreads();
    abacus_flip_set<T>(sa, f, sample, sites, out);
}

// Persistent serving loop.  A CTA takes a ticket (the next item number, from a counter
// that starts at `base`), waits until the host's tail passes it, runs the flip-list body
// on the item and hands the ratio back through host-mapped memory.  One atomic per item
// and no retry loop: claiming items by compare-and-swap against the tail served at most
// one claim per round trip.  The state word of ring slot i % cap is 2i + 1 once the host
// has published item i and 2i + 2 once a CTA has served it; a ticket whose slot says
// anything but 2i + 1 was served by an earlier launch and is dropped.
//
// Leaving: when the host asks to stop, or when the tail has not moved for idle_ns of
// %globaltimer time (the CTA then records DN_ETIMEOUT and raises the closing word), a CTA
// leaves as soon as its ticket is not published.  Tickets held by leaving CTAs are
// served by the next launch, which the host makes, from the first item not yet served,
// once every CTA is gone.
__device__ __forceinline__ unsigned long long load_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__global__ void __launch_bounds__(kAbThreads) k_abacus_serve(const AbArgs<T> *__restrict__ descs, ServeQueue *q,
                                                             ServeItems it, unsigned long long *ctl,
                                                             unsigned long long base, long long idle_ns) {
    __shared__ AbArgs<T> sa;
    __shared__ int32_t s_sample[1], s_sites[2];
    __shared__ double s_out[1];
    __shared__ long long s_item;
    unsigned long long tail_seen = 0ull, t_change = global_ns();   // thread 0's view of the tail
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            long long item = -1;
            unsigned long long h = base + atomicAdd(ctl, 1ull);
            unsigned int nap = 256;
            for (;;) {
                const unsigned long long tail = load_acquire_sys(&q->tail);
                const unsigned long long now = global_ns();
                if (tail != tail_seen) {
                    tail_seen = tail;
                    t_change = now;
                }
                if (h < tail) {
                    const int slot = (int)(h % (unsigned long long)it.cap);
                    if (load_acquire_sys(it.done + slot) == 2 * h + 1) {
                        item = (long long)h;
                        break;
                    }
                    h = base + atomicAdd(ctl, 1ull);   // served by an earlier launch
                    nap = 256;
                    continue;
                }
                if (*((volatile unsigned int *)&q->stop) || *((volatile unsigned long long *)(ctl + 1))) break;
                if ((long long)(now - t_change) > idle_ns) {
                    *((volatile unsigned long long *)(ctl + 1)) = 1ull;
                    *((volatile int *)&q->status) = (int)DN_ETIMEOUT;   // every leaving CTA writes the same value
                    __threadfence_system();
                    break;
                }
                __nanosleep(nap);
                if (nap < 8192) nap *= 2;
            }
            s_item = item;
            if (item >= 0) {
                const int slot = (int)(item % it.cap);
                sa = descs[((volatile int32_t *)it.cache)[slot]];
                s_sample[0] = 0;
                s_sites[0] = ((volatile int32_t *)it.sites)[2 * slot];
                s_sites[1] = ((volatile int32_t *)it.sites)[2 * slot + 1];
            }
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0) break;
        abacus_flip_set<T>(sa, 0, s_sample, s_sites, s_out);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int slot = (int)(item % it.cap);
            ((volatile double *)it.out)[slot] = s_out[0];
            __threadfence_system();
            ((volatile unsigned long long *)it.done)[slot] = 2 * (unsigned long long)item + 2;
        }
    }
}

template <typename T>
cudaError_t launch_abacus(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c,
                          const int32_t *sample, const int32_t *sites, int F, double *out, cudaStream_t st,
                          double *dOmega) {
    if (F <= 0) return cudaSuccess;
    AbArgs<T> a;
    a.dOmega = dOmega;
    a.g = geom_of(m, c->N);
    a.B = c->B;
    a.WF = c->WF;
    a.Rk = c->Rk;
    a.Rl = c->Rl;
    a.P = c->P;
    a.max_cluster = c->max_cluster;
    a.f_kind = m->desc.f_kind;
    a.spins = c->spins;
    a.chi = static_cast<const T *>(c->chi);
    a.y = static_cast<const T *>(c->y);
    a.rho = static_cast<const T *>(c->rho);
    a.t = static_cast<const T *>(c->t);
    a.ell = static_cast<const T *>(c->ell);
    a.K = static_cast<const T *>(c->K);
    a.taps = pl.taps;
    a.Omega = c->Omega;
    a.flag = c->flag;
    a.w = w;
    const Geom &g = a.g;
    const size_t tsz = ((size_t)(g.L + 3) * c->WF * g.d + 2 * (size_t)c->WF * g.dh) * sizeof(T);
    const size_t smem = ((tsz + 7) & ~(size_t)7) + (size_t)kMaxDout * kAbThreads * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_abacus<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_abacus", st);
        k_abacus<T><<<F, kAbThreads, smem, st>>>(a, sample, sites, F, out);
    }
    return cudaGetLastError();
}

// ------------------------------------------- all single flips, by layer ----
// The local estimator of a transverse field needs every single flip j of every
// configuration.  The recurrence is evaluated for all of them one layer at a
// time, each flip's slice state s^(l) kept in a scratch array between layers:
//  k_dchi_table  dchi^(l) on every slot (flip j, slot t -> site j - w + t) for all
//                layers: a batched per-site MLP with the flipped spin;
//  k_ab_layer    layer l: one warp per (configuration, site i).  Site i is slot
//                t = q of the W flips j = i + w - q.  The warp reads the link
//                blocks L^(l,m)_{i,k} (|i-k| <= 2w) of its site once (lane = output
//                channel, the lane's row of each block) and applies each to every
//                flip whose slice holds both i and k; then it forms
//                s^(l) = U (dchi * (y + V p)) for its W (flip, slot) pairs and adds
//                rho^(l) . s^(l) to their partial dOmega;
//  k_ab_final    dOmega_j = sum_t partial + t_j dsigma_j, and the log cosh difference.
// Every link byte of a configuration is read once per call.
constexpr int kLayMaxW = 9;
constexpr int kDxTPB = 8;   // most row tiles per CTA of k_dchi_table (fewer when the grid would not fill the GPU)

// The flips that the grouped kernels evaluate for every site j of every configuration:
// for each of nb bonds the set {j, j + delta} (delta = 0: the single flip of j).  A
// flip's slice is the W + delta sites j - w ... j + delta + w (Sec. "ABACUS", cluster
// flips: the window grows by the extent of the cluster); its rows are padded to Wm =
// W + the largest delta slots.  Row r = ((b N + j) nb + bond) Wm + t holds slot t (site
// j - w + t) of the flip; slots t >= W + delta are unused.  Single flips are
// {nb = 1, Wm = W, delta = 0}.  With anti set, only the pairs of antialigned spins are
// evaluated (the connected configurations of an exchange coupling); the others give 0.
struct FlipPattern {
    int nb, Wm;
    int bond[2];
    int anti;
};
// fp.bond[k] without a dynamic index into the parameter (which would copy it to local memory)
__device__ __forceinline__ int bond_of(const FlipPattern &fp, int k) { return k == 0 ? fp.bond[0] : fp.bond[1]; }

// A CTA takes up to tpb consecutive tiles of 64 (flip, slot) rows of one layer and stages
// that layer's MLP weights once for all of them.  The activations are kept transposed
// ([feature][row]), so a thread reads its rows as 16-byte broadcasts.  Each tile first
// resolves its rows once: the flipped spin window of the row (W values) and the offset of
// the row's chi entry (-1 where slot site j - w + t lies off an open chain).
template <typename T, bool PR>
__global__ void __launch_bounds__(256) k_dchi_table(AbArgs<T> a, FlipPattern fp, T *__restrict__ DX, int tpb) {
    if constexpr (!PR) fp = FlipPattern{1, 2 * a.g.w + 1, {0, 0}, 0};   // single flips: compile-time row layout
    extern __shared__ __align__(16) unsigned char smraw[];
    const Geom &g = a.g;
    const int N = g.N, d = g.d, dh = g.dh, L = g.L, wd = g.w, W = g.W;
    constexpr int RT = 64, RG = 8, TS = RT + 4;             // rows per tile, rows per thread, row stride
    long long *roff = reinterpret_cast<long long *>(smraw);   // [RT] chi offset of the row's site, or -1
    T *phT = reinterpret_cast<T *>(roff + RT);              // [dh][TS]  phi
    T *acT = phT + dh * TS;                                 // [dh][TS]  GELU(z)
    // FP32 with dh and d multiples of 4: each thread forms 4 outputs x 4 rows (16-byte weight
    // and activation loads); otherwise 1 output x 8 rows.  Weight rows are padded to keep
    // the 16-byte loads aligned (stride + 4) or the scalar ones off one bank (stride + 1).
    const bool tiled = std::is_same<T, float>::value && dh % 4 == 0 && d % 4 == 0;
    const int ws1 = tiled ? dh + 4 : dh + 1, ws2 = tiled ? d + 4 : d + 1;
    T *W1s = acT + dh * TS;                                 // [f][e] = W1[e][f], row stride ws1
    T *W2s = W1s + dh * ws1;                                // [e][c] = W2[c][e], row stride ws2
    T *win = W2s + dh * ws2;                                // [RT][W] flipped spin window of the row
    const int l = blockIdx.y;
    const int Wm = PR ? fp.Wm : W, nb = PR ? fp.nb : 1;
    const long long rows = (long long)a.B * N * nb * Wm;
    const T *W1T = a.w.W1T + (long long)l * dh * dh, *W2T = a.w.W2T + (long long)l * dh * d;
    const T *b1 = a.w.b1 + (long long)l * dh, *b2 = a.w.b2 + (long long)l * d;
    const T *kap = a.w.kappa + (long long)l * W * dh, *beta = a.w.beta + (long long)l * dh;
    for (int q = threadIdx.x; q < dh * dh; q += blockDim.x) W1s[(q / dh) * ws1 + q % dh] = W1T[q];
    for (int q = threadIdx.x; q < dh * d; q += blockDim.x) W2s[(q / d) * ws2 + q % d] = W2T[q];
    for (int it = 0; it < tpb; ++it) {
        const long long r0 = ((long long)blockIdx.x * tpb + it) * RT;
        if (r0 >= rows) break;
        __syncthreads();   // the previous tile's reads of phT / acT / roff (and the weight staging) are done
        for (int rr = threadIdx.x; rr < RT; rr += blockDim.x) {
            const long long r = r0 + rr;
            long long off = -1;
            if (r < rows) {
                const int t = (int)(r % Wm);
                const long long fb = r / Wm;   // (b N + j) nb + bond
                const int dl = PR ? bond_of(fp, (int)(fb % nb)) : 0, j = (int)((fb / nb) % N);
                const long long b = fb / ((long long)nb * N);
                const int8_t *sp = a.spins + b * N;
                const int iu = j - wd + t;
                // partner of a pair (-1: none); a pair past an open end is not a flip
                int jp = -1;
                if (dl > 0) jp = g.periodic ? (j + dl) % N : (j + dl < N ? j + dl : -2);
                if (PR && fp.anti && jp >= 0 && sp[j] == sp[jp]) jp = -2;
                if (t < W + dl && jp != -2 && (g.periodic || (iu >= 0 && iu < N))) {
                    off = ((b * L + l) * N + (g.periodic ? ((iu % N) + N) % N : iu)) * d;
                    for (int o = -wd; o <= wd; ++o) {
                        int jn = iu + o;
                        T v;
                        if (g.periodic) {
                            jn = ((jn % N) + N) % N;
                            v = (T)sp[jn];
                        } else {
                            v = (jn >= 0 && jn < N) ? (T)sp[jn] : (T)0;
                        }
                        if (jn == j || jn == jp) v = -v;
                        win[rr * W + o + wd] = v;
                    }
                }
            }
            roff[rr] = off;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < RT * dh; q += blockDim.x) {
            const int e = q / RT, rr = q % RT;   // lanes along rows: conflict-free stores
            T acc = 0;
            if (roff[rr] >= 0) {
                acc = beta[e];
                for (int o = 0; o < W; ++o) acc += kap[o * dh + e] * win[rr * W + o];
            }
            phT[e * TS + rr] = acc;
        }
        __syncthreads();
        if (!tiled) {
            for (int q = threadIdx.x; q < dh * (RT / RG); q += blockDim.x) {
                const int e = q % dh, t0 = (q / dh) * RG;
                T acc[RG];
        #pragma unroll
                for (int u = 0; u < RG; ++u) acc[u] = b1[e];
                for (int f = 0; f < dh; ++f) {
                    const T wv = W1s[f * ws1 + e];
                    T pv[RG];
                    lds8<T>(phT + f * TS + t0, pv);
        #pragma unroll
                    for (int u = 0; u < RG; ++u) acc[u] += wv * pv[u];
                }
        #pragma unroll
                for (int u = 0; u < RG; ++u) acT[e * TS + t0 + u] = gelu_ab<T>(acc[u]);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < d * (RT / RG); q += blockDim.x) {
                const int c = q % d, t0 = (q / d) * RG;
                T acc[RG];
        #pragma unroll
                for (int u = 0; u < RG; ++u) acc[u] = b2[c];
                for (int e = 0; e < dh; ++e) {
                    const T wv = W2s[e * ws2 + c];
                    T pv[RG];
                    lds8<T>(acT + e * TS + t0, pv);
        #pragma unroll
                    for (int u = 0; u < RG; ++u) acc[u] += wv * pv[u];
                }
        #pragma unroll
                for (int u = 0; u < RG; ++u) {
                    const long long r = r0 + t0 + u;
                    if (r >= rows) continue;
                    const long long off = roff[t0 + u];
                    DX[((long long)l * rows + r) * d + c] = off >= 0 ? acc[u] - a.chi[off + c] : (T)0;
                }
            }

        } else if constexpr (std::is_same<T, float>::value) {
            // 4 outputs x 4 rows per thread
            for (int q = threadIdx.x; q < (dh / 4) * (RT / 4); q += blockDim.x) {
                const int e0 = (q % (dh / 4)) * 4, t0 = (q / (dh / 4)) * 4;
                float acc[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[j][u] = b1[e0 + j];
#pragma unroll 4
                for (int f = 0; f < dh; ++f) {
                    const float4 wv = *reinterpret_cast<const float4 *>(W1s + f * ws1 + e0);
                    const float4 pv = *reinterpret_cast<const float4 *>(phT + f * TS + t0);
                    const float w4[4] = {wv.x, wv.y, wv.z, wv.w}, p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[j][u] = fmaf(w4[j], p4[u], acc[j][u]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<float4 *>(acT + (e0 + j) * TS + t0) =
                        make_float4(gelu_ab<float>(acc[j][0]), gelu_ab<float>(acc[j][1]), gelu_ab<float>(acc[j][2]),
                                    gelu_ab<float>(acc[j][3]));
            }
            __syncthreads();
            for (int q = threadIdx.x; q < (d / 4) * (RT / 4); q += blockDim.x) {
                const int c0 = (q % (d / 4)) * 4, t0 = (q / (d / 4)) * 4;
                float acc[4][4];   // [row][output]
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[u][j] = b2[c0 + j];
#pragma unroll 4
                for (int e = 0; e < dh; ++e) {
                    const float4 wv = *reinterpret_cast<const float4 *>(W2s + e * ws2 + c0);
                    const float4 pv = *reinterpret_cast<const float4 *>(acT + e * TS + t0);
                    const float w4[4] = {wv.x, wv.y, wv.z, wv.w}, p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[u][j] = fmaf(w4[j], p4[u], acc[u][j]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long r = r0 + t0 + u;
                    if (r >= rows) continue;
                    const long long off = roff[t0 + u];
                    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (off >= 0) {
                        const float4 ch = *reinterpret_cast<const float4 *>(a.chi + off + c0);
                        o = make_float4(acc[u][0] - ch.x, acc[u][1] - ch.y, acc[u][2] - ch.z, acc[u][3] - ch.w);
                    }
                    *reinterpret_cast<float4 *>(DX + ((long long)l * rows + r) * d + c0) = o;
                }
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int HD>
__global__ void __launch_bounds__(256) k_ab_layer(AbArgs<T> a, int l, T *__restrict__ S, const T *__restrict__ DX,
                                                  double *__restrict__ PART) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const Geom &g = a.g;
    const int N = g.N, d = g.d, L = g.L, wd = g.w, W = g.W, dout = g.dout;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long dd = (long long)d * d;
    T *VTs = reinterpret_cast<T *>(smraw);                  // [d][d] = V^T
    T *UTs = VTs + dd;                                      // [d][d] = U^T
    T *wb = UTs + dd + (size_t)warp * (W * W * d + 2 * W * d);
    T *Ss = wb;                                             // [W][W][d]  s^(m) of the warp's flips
    T *pq = Ss + W * W * d;                                 // [W][d]
    T *gq = pq + W * d;                                     // [W][d]
    const long long lo = l - 1;
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        VTs[q] = a.w.VT[lo * dd + q];
        UTs[q] = a.w.UT[lo * dd + q];
    }
    __syncthreads();
    const long long b = blockIdx.y;
    const int i = blockIdx.x * 8 + warp;
    if (i >= N) return;
    const int8_t *sp = a.spins + b * N;
    const long long rows = (long long)a.B * N * W;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    // Flips served by this site: q -> j = i + w - q, slot t = q.
    int jq[kLayMaxW];
    T dsq[kLayMaxW];
    unsigned valid = 0;
#pragma unroll
    for (int q = 0; q < kLayMaxW; ++q) {
        int j = i + wd - q;
        bool ok = q < W;
        if (g.periodic) j = ((j % N) + N) % N;
        else ok = ok && j >= 0 && j < N;
        jq[q] = ok ? j : 0;
        dsq[q] = ok ? (T)(-2 * sp[j]) : (T)0;
        if (ok) valid |= 1u << q;
    }
    auto tap = [&](int ll, int r, int c) -> T {
        const int row = g.periodic ? ((r % N) + N) % N : r + N - 1;
        return a.taps[((long long)(ll - 1) * g.R + row) * d + c];
    };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    T acc[HD][kLayMaxW];
#pragma unroll
    for (int h = 0; h < HD; ++h)
#pragma unroll
        for (int q = 0; q < kLayMaxW; ++q) acc[h][q] = 0;
    // Slice Toeplitz and embedding terms.
#pragma unroll
    for (int q = 0; q < kLayMaxW; ++q) {
        if (!((valid >> q) & 1u)) continue;
        const int j = jq[q];
#pragma unroll
        for (int h = 0; h < HD; ++h) {
            const int c = lane + 32 * h;
            if (c >= d) continue;
            T v;
            if (l == 1) {
                v = tap(1, q - wd, c) * a.w.e[c] * dsq[q];
            } else {
                v = 0;
                const T *Sp = S + (lo - 1) * rows * d + (((long long)b * N + j) * W) * d + c;
                for (int t2 = 0; t2 < W; ++t2)
                    if (site_ok(j - wd + t2)) v += tap(l, q - t2, c) * Sp[(long long)t2 * d];
                v += dsq[q] * a.ell[(((b * (L - 1) + (l - 2)) * N + i) * nRl + (wd - q + a.Rl)) * d + c];
            }
            acc[h][q] = v;
        }
    }
    // Interlayer links.
    for (int m = 1; m <= l - 2; ++m) {
        for (int x = lane; x < W * W * d; x += 32) {
            const int q = x / (W * d);
            const int t2 = (x / d) % W, c2 = x % d;
            Ss[x] = ((valid >> q) & 1u) ? S[(long long)(m - 1) * rows * d + (((long long)b * N + jq[q]) * W + t2) * d + c2]
                                        : (T)0;
        }
        __syncwarp();
        const T *Kr = a.K + ((b * a.P + pair_index(l, m)) * N + i) * nRk * dd;
        for (int dl = -2 * wd; dl <= 2 * wd; ++dl) {
            const int k = i + dl;
            if (!site_ok(k)) continue;
            const int qlo = dl < 0 ? -dl : 0, qhi = dl > 0 ? 2 * wd - dl : 2 * wd;
            const T *Kb = Kr + (long long)(dl + a.Rk) * dd;
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c >= d) continue;
                const T *kr = Kb + (long long)c * d;
                for (int c2 = 0; c2 < d; c2 += 4) {
                    T kv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) kv[u] = (c2 + u < d) ? kr[c2 + u] : (T)0;
#pragma unroll
                    for (int q = 0; q < kLayMaxW; ++q) {
                        if (q < qlo || q > qhi) continue;
                        const T *sv = Ss + ((q * W) + (dl + q)) * d + c2;
                        T sacc = 0;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (c2 + u < d) sacc += kv[u] * sv[u];
                        acc[h][q] += sacc;
                    }
                }
            }
        }
        __syncwarp();
    }
    // s^(l) = U (dchi * (y + V p)) and its contribution to dOmega.
#pragma unroll
    for (int q = 0; q < kLayMaxW; ++q) {
        if (q >= W) break;
#pragma unroll
        for (int h = 0; h < HD; ++h) {
            const int c = lane + 32 * h;
            if (c < d) pq[q * d + c] = acc[h][q];
        }
    }
    __syncwarp();
    const T *yrow = a.y + ((b * L + lo) * N + i) * d;
#pragma unroll
    for (int q = 0; q < kLayMaxW; ++q) {
        if (q >= W) break;
        const bool ok = (valid >> q) & 1u;
#pragma unroll
        for (int h = 0; h < HD; ++h) {
            const int c = lane + 32 * h;
            if (c >= d) continue;
            T z = yrow[c];
            for (int c2 = 0; c2 < d; ++c2) z += VTs[c2 * d + c] * pq[q * d + c2];
            const T dx = ok ? DX[(lo * rows + ((long long)b * N + jq[q]) * W + q) * d + c] : (T)0;
            gq[q * d + c] = dx * z;
        }
    }
    __syncwarp();
    const T *rho = a.rho + ((b * L + lo) * dout) * (long long)N * d + (long long)i * d;
#pragma unroll
    for (int q = 0; q < kLayMaxW; ++q) {
        if (q >= W) break;
        if (!((valid >> q) & 1u)) continue;
        T sv[HD];
#pragma unroll
        for (int h = 0; h < HD; ++h) {
            const int c = lane + 32 * h;
            T s = 0;
            if (c < d) {
                for (int c2 = 0; c2 < d; ++c2) s += UTs[c2 * d + c] * gq[q * d + c2];
                if (l < L) S[(lo * rows + ((long long)b * N + jq[q]) * W + q) * d + c] = s;
            }
            sv[h] = s;
        }
        for (int k = 0; k < dout; ++k) {
            double v = 0.0;
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c < d) v += (double)rho[(long long)k * N * d + c] * (double)sv[h];
            }
            v = warp_sum<double>(v);
            if (lane == 0) PART[(((long long)b * N + jq[q]) * W + q) * dout + k] += v;
        }
    }
}

// Layer l of the grouped pair flips of a FlipPattern.  A CTA of nw warps takes a run of nw
// consecutive sites i0 .. i0 + nw - 1 of one configuration, warp r the site i = i0 + r.
// For bond delta the site is slot q of the W + delta flips j = i + w - q (pairs
// {j, j + delta}); consecutive sites share all but one of them, so the run needs only the
// nw + W + delta - 1 flips of a window, whose states s^(m) are staged once per CTA.  Every
// link block K^(l,m)_{i, i+dk} (|dk| <= Wm - 1) is read once per site and applied to the
// flips of all bonds whose slice holds site i + dk.  The terms are those of the flip-list
// kernel with the slice [j - w, j + delta + w]: the slice Toeplitz term of the previous
// layer's states, the embedding links of both flipped sites (Eq. Lmn with m = 0), the
// interlayer links (Eq. recur_step), then s^(l) = U (dchi * (y + V p)) and its
// contribution rho^(l) . s^(l) to the flip's partial dOmega.
constexpr int kPrMaxWs = 8;   // slots per flip (W + delta)
constexpr int kPrMaxFl = 48;  // flips per bond in a CTA's window (nw + W + delta - 1)

template <typename T, int HD, bool VEC>
__global__ void __launch_bounds__(256) k_ab_pairs(AbArgs<T> a, FlipPattern fp, int l, T *__restrict__ S,
                                                  const T *__restrict__ DX, double *__restrict__ PART) {
    static_assert(!VEC || std::is_same<T, float>::value, "16-byte loads of FP32 link rows (d a multiple of 16)");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int jwin[2][kPrMaxFl];   // wrapped flip site of window entry fl, or -1 (no flip)
    const Geom &g = a.g;
    const int N = g.N, d = g.d, L = g.L, wd = g.w, W = g.W, dout = g.dout, nb = fp.nb, Wm = fp.Wm;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long dd = (long long)d * d;
    const int ws0 = W + fp.bond[0], ws1 = nb > 1 ? W + fp.bond[1] : 0;
    T *VTs = reinterpret_cast<T *>(smraw);                       // [d][d] = V^T
    T *UTs = VTs + dd;                                           // [d][d] = U^T
    T *Sw0 = UTs + dd;                                           // bond 0: [nw + ws0 - 1][ws0][d]
    T *Sw1 = Sw0 + (size_t)(nw + ws0 - 1) * ws0 * d;             // bond 1: [nw + ws1 - 1][ws1][d]
    T *pq = Sw1 + (size_t)(nw + ws1 - 1) * ws1 * d + (size_t)warp * (nb * Wm + 1) * d;   // [nb][Wm][d] of the warp
    T *gb = pq + (size_t)nb * Wm * d;                            // [d]
    const long long lo = l - 1;
    const long long b = blockIdx.y;
    const int i0 = blockIdx.x * nw, i = i0 + warp;
    const bool active = i < N;
    const int8_t *sp = a.spins + b * N;
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        VTs[q] = a.w.VT[lo * dd + q];
        UTs[q] = a.w.UT[lo * dd + q];
    }
    for (int x = threadIdx.x; x < 2 * kPrMaxFl; x += blockDim.x) {
        const int bo = x / kPrMaxFl, fl = x % kPrMaxFl;
        int jw = -1;
        if (bo < nb) {
            const int dl = bond_of(fp, bo), ws = W + dl;
            if (fl < nw + ws - 1) {
                const int ju = i0 + wd - ws + 1 + fl;
                if (g.periodic) {
                    const int j = ((ju % N) + N) % N;
                    if (!fp.anti || sp[j] != sp[(j + dl) % N]) jw = j;
                } else if (ju >= 0 && ju + dl < N && (!fp.anti || sp[ju] != sp[ju + dl])) {
                    jw = ju;
                }
            }
        }
        jwin[bo][fl] = jw;
    }
    __syncthreads();
    const long long rows = (long long)a.B * N * nb * Wm;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    auto row_of = [&](int j, int bo) -> long long { return (((long long)b * N + j) * nb + bo) * Wm; };
    auto tap = [&](int ll, int r, int c) -> T {
        const int row = g.periodic ? ((r % N) + N) % N : r + N - 1;
        return a.taps[((long long)(ll - 1) * g.R + row) * d + c];
    };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    // flip (bond bo, slot q) of this warp's site: window entry warp + ws - 1 - q
    auto flip_of = [&](int bo, int q) -> int {
        const int ws = bo == 0 ? ws0 : ws1;
        return jwin[bo][warp + ws - 1 - q];
    };
    unsigned valid = 0;   // bit bo * kPrMaxWs + q
    if (active)
        for (int bo = 0; bo < nb; ++bo)
            for (int q = 0; q < (bo == 0 ? ws0 : ws1); ++q)
                if (flip_of(bo, q) >= 0) valid |= 1u << (bo * kPrMaxWs + q);
    T acc[HD][2][kPrMaxWs];
#pragma unroll
    for (int h = 0; h < HD; ++h)
#pragma unroll
        for (int bo = 0; bo < 2; ++bo)
#pragma unroll
            for (int q = 0; q < kPrMaxWs; ++q) acc[h][bo][q] = 0;
    // Slice Toeplitz and embedding terms.
#pragma unroll
    for (int bo = 0; bo < 2; ++bo) {
        if (bo >= nb) break;
        const int dl = fp.bond[bo];
#pragma unroll
        for (int q = 0; q < kPrMaxWs; ++q) {
            if (!((valid >> (bo * kPrMaxWs + q)) & 1u)) continue;
            const int j = flip_of(bo, q), jp = g.periodic ? (j + dl) % N : j + dl;
            const T ds = (T)(-2 * sp[j]), dsp = (T)(-2 * sp[jp]);
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c >= d) continue;
                T v;
                if (l == 1) {
                    v = tap(1, q - wd, c) * a.w.e[c] * ds + tap(1, q - wd - dl, c) * a.w.e[c] * dsp;
                } else {
                    v = 0;
                    const T *Sp = S + (lo - 1) * rows * d + row_of(j, bo) * d + c;
                    for (int t2 = 0; t2 < W + dl; ++t2)
                        if (site_ok(i - q + t2)) v += tap(l, q - t2, c) * Sp[(long long)t2 * d];
                    const T *el = a.ell + (((b * (L - 1) + (l - 2)) * N + i) * nRl) * d + c;
                    v += ds * el[(long long)(wd - q + a.Rl) * d] + dsp * el[(long long)(wd - q + dl + a.Rl) * d];
                }
                acc[h][bo][q] = v;
            }
        }
    }
    // Interlayer links.  Each flip's 16-term dot product runs as four partial sums, so its
    // dependent chain is 4 + 2 deep rather than 16.
    for (int m = 1; m <= l - 2; ++m) {
        __syncthreads();   // the previous m's window is no longer read
        for (int bo = 0; bo < nb; ++bo) {
            const int ws = bo == 0 ? ws0 : ws1, per = ws * d;
            T *dst = bo == 0 ? Sw0 : Sw1;
            const T *src = S + (long long)(m - 1) * rows * d;
            for (int x = threadIdx.x; x < (nw + ws - 1) * per; x += blockDim.x) {
                const int fl = x / per, rem = x % per;
                const int j = jwin[bo][fl];
                dst[x] = j >= 0 ? src[row_of(j, bo) * d + rem] : (T)0;
            }
        }
        __syncthreads();
        if (!active) continue;
        const T *Kr = a.K + ((b * a.P + pair_index(l, m)) * N + i) * nRk * dd;
        for (int dk = -(Wm - 1); dk <= Wm - 1; ++dk) {
            if (!site_ok(i + dk)) continue;
            const T *Kb = Kr + (long long)(dk + a.Rk) * dd;
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c >= d) continue;
                const T *kr = Kb + (long long)c * d;
                for (int c2 = 0; c2 < d; c2 += 16) {
                    T kv[16];
                    if constexpr (VEC) {
#pragma unroll
                        for (int u = 0; u < 16; u += 4) {
                            const float4 k4 = __ldg(reinterpret_cast<const float4 *>(kr + c2 + u));
                            kv[u] = k4.x;
                            kv[u + 1] = k4.y;
                            kv[u + 2] = k4.z;
                            kv[u + 3] = k4.w;
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u) kv[u] = (c2 + u < d) ? kr[c2 + u] : (T)0;
                    }
#pragma unroll
                    for (int bo = 0; bo < 2; ++bo) {
                        if (bo >= nb) break;
                        const int ws = bo == 0 ? ws0 : ws1;
                        const T *Swb = bo == 0 ? Sw0 : Sw1;
#pragma unroll
                        for (int q = 0; q < kPrMaxWs; ++q) {
                            const int t2 = dk + q;
                            if (q >= ws || t2 < 0 || t2 >= ws || !((valid >> (bo * kPrMaxWs + q)) & 1u)) continue;
                            const T *sv = Swb + ((size_t)(warp + ws - 1 - q) * ws + t2) * d + c2;
                            T ps[4] = {0, 0, 0, 0};
                            if constexpr (VEC) {
#pragma unroll
                                for (int u = 0; u < 16; u += 4) {
                                    const float4 s4 = *reinterpret_cast<const float4 *>(sv + u);
                                    ps[0] = fmaf(kv[u], s4.x, ps[0]);
                                    ps[1] = fmaf(kv[u + 1], s4.y, ps[1]);
                                    ps[2] = fmaf(kv[u + 2], s4.z, ps[2]);
                                    ps[3] = fmaf(kv[u + 3], s4.w, ps[3]);
                                }
                            } else {
#pragma unroll
                                for (int u = 0; u < 16; ++u)
                                    if (c2 + u < d) ps[u & 3] += kv[u] * sv[u];
                            }
                            acc[h][bo][q] += (ps[0] + ps[1]) + (ps[2] + ps[3]);
                        }
                    }
                }
            }
        }
    }
    if (!active) return;
    // s^(l) = U (dchi * (y + V p)) and its contribution to dOmega, one flip at a time.
#pragma unroll
    for (int bo = 0; bo < 2; ++bo) {
        if (bo >= nb) break;
#pragma unroll
        for (int q = 0; q < kPrMaxWs; ++q) {
            if (q >= Wm) break;
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c < d) pq[(bo * Wm + q) * d + c] = acc[h][bo][q];
            }
        }
    }
    __syncwarp();
    const T *yrow = a.y + ((b * L + lo) * N + i) * d;
    const T *rho = a.rho + ((b * L + lo) * dout) * (long long)N * d + (long long)i * d;
    for (int bo = 0; bo < nb; ++bo) {
        for (int q = 0; q < (bo == 0 ? ws0 : ws1); ++q) {
            if (!((valid >> (bo * kPrMaxWs + q)) & 1u)) continue;
            const long long row = row_of(flip_of(bo, q), bo) + q;
            const T *pv = pq + (bo * Wm + q) * d;
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                if (c >= d) continue;
                T z = yrow[c];
                for (int c2 = 0; c2 < d; ++c2) z += VTs[c2 * d + c] * pv[c2];
                gb[c] = DX[(lo * rows + row) * d + c] * z;
            }
            __syncwarp();
            T sv[HD];
#pragma unroll
            for (int h = 0; h < HD; ++h) {
                const int c = lane + 32 * h;
                T s = 0;
                if (c < d) {
                    for (int c2 = 0; c2 < d; ++c2) s += UTs[c2 * d + c] * gb[c2];
                    if (l < L) S[(lo * rows + row) * d + c] = s;
                }
                sv[h] = s;
            }
            __syncwarp();   // gb is rewritten by the next flip
            for (int k = 0; k < dout; ++k) {
                double v = 0.0;
#pragma unroll
                for (int h = 0; h < HD; ++h) {
                    const int c = lane + 32 * h;
                    if (c < d) v += (double)rho[(long long)k * N * d + c] * (double)sv[h];
                }
                v = warp_sum<double>(v);
                if (lane == 0) PART[row * dout + k] += v;
            }
        }
    }
}

constexpr long kSpinLimit = 1L << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < kSpinLimit; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_addr(mbar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Streaming fast path of k_ab_layer for FP32 with d = 32.  Warp w of a CTA owns a
// run of R consecutive sites of one sample and walks them in order; for every
// site it needs
//  * the link blocks K^(l,m)_{i, i+dl} (m = 1..l-2, |dl| <= 2w), 4 KB each, which
//    lie back to back in memory along the run; they are streamed through a ring
//    of NS shared-memory slots by TMA tensor copies, and the ring is kept full
//    across site boundaries, so the copies of the next site are in flight while
//    the current site's slice terms, matvecs and outputs are computed;
//  * the states s^(m) (m = 1..l-1) of the W flips whose slice holds the site.
//    Consecutive sites share W-1 of these flips, so they live in a window of
//    W+1 flip slots per m (slot = flip mod (W+1)): moving one site on loads one
//    new flip (W d contiguous values per m, one bulk copy), issued a site early
//    into the slot that the previous site has released;
//  * y, dchi, rho and the embedding links of the site, loaded into registers one
//    site ahead.
// Lane c owns output channel c.  Link blocks are copied by TMA with the 128-byte
// swizzle (chunk j of row r lands at chunk j ^ (r mod 8)), so when every lane reads
// chunk s of its own row the 8 lanes of a shared-memory phase hit 8 different bank
// groups, and the matching chunk s of a slice state is one broadcast to all lanes.  Every wait is bounded; a
// timeout raises bit 4 of the cache flag, lets the copies in flight land and
// ends the warp.
constexpr int kStWarps = 8;
constexpr int kStMaxNS = 4;
constexpr int kStMaxDout = 2;

__device__ __forceinline__ void mbar_expect(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}

// Bulk copy whose completion counts against a byte total announced by mbar_expect.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// One 4 KB link block (32 rows of 32 floats starting at row `row` of the tensor map) into a
// 1024-byte-aligned slot, 128B-swizzled: chunk j of row r lands at chunk j ^ (r mod 8).
__device__ __forceinline__ void tma_block(void *dst, const CUtensorMap *tm, int row, uint64_t *mbar) {
    mbar_expect(mbar, 4096u);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(row), "r"(smem_addr(mbar))
        : "memory");
}

// One 4 KB chunk of 16 rows of 64 floats (starting at row `row` of the tensor map) as two
// 32-column boxes: columns 0-31 to dst, columns 32-63 to dst + 2 KB, both 128B-swizzled.
__device__ __forceinline__ void tma_chunk64(float *dst, const CUtensorMap *tm, int row, uint64_t *mbar) {
    mbar_expect(mbar, 4096u);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                smem_addr(dst + sg * 512)),
            "l"(reinterpret_cast<uint64_t>(tm)), "r"(32 * sg), "r"(row), "r"(smem_addr(mbar))
            : "memory");
}

__device__ __forceinline__ int floor_mod(int x, int m) {
    const int r = x % m;
    return r < 0 ? r + m : r;
}

// Sums NV <= 16 values over the warp; lane t with even t ends up holding the total
// of value (t >> 1) & 15 (recursive halving: 16 + 15 shuffles instead of 5 NV).
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane) {
#pragma unroll
    for (int h = 8, off = 16; h >= 1; h >>= 1, off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int u = 0; u < h; ++u) {
            const float send = up ? v[u] : v[u + h];
            const float keep = up ? v[u + h] : v[u];
            v[u] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int WW, int NS>
__global__ void __launch_bounds__(32 * kStWarps, NS == 0 ? 2 : 1) k_ab_stream(AbArgs<float> a, int l, int R,
                                                                              float *__restrict__ S,
                                                                              const float *__restrict__ DX,
                                                                              double *__restrict__ PART,
                                                                              const __grid_constant__ CUtensorMap tmK) {
    extern __shared__ __align__(1024) unsigned char smst[];
    unsigned char *smraw = smst;
    constexpr int d = 32, dd = d * d;
    const Geom &g = a.g;
    if ((smem_addr(smraw) & 1023u) != 0u) {   // the swizzled ring needs 1024-byte-aligned slots
        if (threadIdx.x == 0) atomicOr(a.flag, 8u);
        return;
    }
    constexpr int W = WW, wd = (WW - 1) / 2, W1 = W + 1;
    const int N = g.N, L = g.L, dout = g.dout;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = lane;
    const int nwin = l - 1, nlink = l > 2 ? l - 2 : 0, nper = 4 * wd + 1;
    float *Kring = reinterpret_cast<float *>(smraw) + (size_t)warp * NS * dd;   // [NS][d][d], 4 KB-aligned slots
    float *VTs = reinterpret_cast<float *>(smraw) + (size_t)kStWarps * NS * dd;  // [d][d]
    float *UTs = VTs + dd;                                          // [d][d]
    float *Gs = UTs + dd;                                           // [4w+1][d] taps g^(l)_{-2w..2w}
    float *Zs = Gs + nper * d;                                      // [d] zeros
    const int per_warp = nwin * W1 * W * d + 2 * W * d;
    float *Win = Zs + d + (size_t)warp * per_warp;                  // [nwin][W+1][W][d]
    float *pq = Win + nwin * W1 * W * d;                            // [W][d]
    float *gq = pq + W * d;                                         // [W][d]
    uint64_t *mb = reinterpret_cast<uint64_t *>(Zs + d + (size_t)kStWarps * per_warp) +
                   (size_t)warp * (kStMaxNS + 2);                   // NS ring barriers, 2 window barriers
    int8_t *sps = reinterpret_cast<int8_t *>(reinterpret_cast<uint64_t *>(Zs + d + (size_t)kStWarps * per_warp) +
                                             (size_t)kStWarps * (kStMaxNS + 2));
    const long long lo = l - 1;
    const long long b = blockIdx.y;
    // VT and UT interleaved as [k/4][c][k%4]: one 16-byte load gives rows k..k+3 of column c.
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        const int k = q / d, cc = q % d, x = ((k >> 2) * d + cc) * 4 + (k & 3);
        VTs[x] = a.w.VT[lo * dd + q];
        UTs[x] = a.w.UT[lo * dd + q];
    }
    for (int q = threadIdx.x; q < nper * d; q += blockDim.x) {
        const int r = q / d - 2 * wd, cc = q % d;
        const int row = g.periodic ? ((r % N) + N) % N : (r > -N && r < N ? r + N - 1 : -1);
        Gs[q] = row >= 0 ? a.taps[(lo * g.R + row) * d + cc] : 0.f;
    }
    for (int q = threadIdx.x; q < N; q += blockDim.x) sps[q] = a.spins[b * N + q];
    for (int q = threadIdx.x; q < d; q += blockDim.x) Zs[q] = 0.f;
    if (lane == 0) {
        for (int s = 0; s < kStMaxNS + 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb + s)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    const int i0 = (blockIdx.x * kStWarps + warp) * R;
    const int nsite = N - i0 < R ? N - i0 : R;
    if (nsite <= 0) return;
    uint64_t *wmb = mb + kStMaxNS;
    const long long rows = (long long)a.B * N * W;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    auto wrap = [&](int x) -> int { return g.periodic ? floor_mod(x, N) : x; };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    // Window copies: flip jj (unwrapped) of every m into slot jj mod (W+1).
    // One arrival per phase carries the byte count of all the phase's copies.
    auto issue_flip = [&](int jj, uint64_t *bar) {
        if (!site_ok(jj)) return;
        const int j = wrap(jj), slot = floor_mod(jj, W1);
        for (int m = 1; m <= nwin; ++m)
            bulk_copy(Win + ((m - 1) * W1 + slot) * W * d, S + ((m - 1) * rows + (b * N + j) * W) * d,
                      (uint32_t)(W * d * sizeof(float)), bar);
    };
    auto flip_bytes = [&](int jj) -> uint32_t { return site_ok(jj) ? (uint32_t)(nwin * W * d * sizeof(float)) : 0u; };
    // Link blocks, in stream order (site r, pair m, offset dl): the nper blocks of one (r, m)
    // are contiguous.  Issue and consume positions advance incrementally (no divisions).
    const int nblk = nsite * nlink * nper;
    int iss_r = 0, iss_m = 1, iss_dl = 0;          // next block to issue
    const float *iss_src = nullptr;
    auto iss_base = [&]() {
        iss_src = a.K + (((b * a.P + pair_index(l, iss_m)) * N + (i0 + iss_r)) * nRk + (a.Rk - 2 * wd)) * (long long)dd;
    };
    auto iss_advance = [&]() {
        if (++iss_dl == nper) {
            iss_dl = 0;
            if (++iss_m > nlink) {
                iss_m = 1;
                ++iss_r;
            }
            if (iss_r < nsite) iss_base();
        } else {
            iss_src += dd;
        }
    };
    int issued = 0, consumed = 0, iss_slot = 0, con_slot = 0;
    uint32_t con_phase = 0;
    uint32_t wpend[2] = {0u, 0u}, wuse[2] = {0u, 0u};
    if (NS > 0 && nblk > 0) {
        iss_base();
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (; issued < nblk && issued < NS; ++issued) {
            if (lane == 0) tma_block(Kring + iss_slot * dd, &tmK, (int)((iss_src - a.K) >> 5), mb + iss_slot);
            iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
            iss_advance();
        }
    }
    if (nwin > 0) {
        uint32_t bytes = 0;
        for (int jj = i0 - wd; jj <= i0 + wd; ++jj) bytes += flip_bytes(jj);
        if (lane == 0 && bytes) {
            mbar_expect(wmb, bytes);
            for (int jj = i0 - wd; jj <= i0 + wd; ++jj) issue_flip(jj, wmb);
        }
        wpend[0] = bytes ? 1u : 0u;
    }
    bool timed_out = false;
    // Per-site vectors of site r (cur) and r + 1 (nxt).
    float y_c, dx_c[W], rh_c[kStMaxDout], el_c[W];
    auto load_site = [&](int i, float &yv, float (&dx)[W], float (&rh)[kStMaxDout], float (&el)[W]) {
        yv = a.y[((b * L + lo) * N + i) * d + c];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            dx[q] = 0.f;
            el[q] = 0.f;
            if (q >= W) continue;
            const int jj = i + wd - q;
            if (!site_ok(jj)) continue;
            dx[q] = DX[(lo * rows + (b * N + wrap(jj)) * W + q) * d + c];
            if (l >= 2) el[q] = a.ell[((b * (L - 1) + (l - 2)) * N + i) * nRl * d + (wd - q + a.Rl) * d + c];
        }
#pragma unroll
        for (int k = 0; k < kStMaxDout; ++k) rh[k] = k < dout ? a.rho[((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d + c] : 0.f;
    };
    load_site(i0, y_c, dx_c, rh_c, el_c);
    for (int r = 0; r < nsite && !timed_out; ++r) {
        const int i = i0 + r;
        int jq[W], wsl[W];
        float dsq[W];
        unsigned valid = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int jj = i + wd - q;
            const bool ok = q < W && site_ok(jj);
            jq[q] = ok ? wrap(jj) : 0;
            wsl[q] = floor_mod(jj, W1);
            dsq[q] = ok ? (float)(-2 * sps[jq[q]]) : 0.f;
            if (ok) valid |= 1u << q;
        }
        // This site's window copies, then the next site's new flip into the released slot.
        if (nwin > 0) {
            const int pb = r & 1;
            if (wpend[pb]) {
                if (!mbar_wait(wmb + pb, wuse[pb] & 1u)) {
                    timed_out = true;
                    break;
                }
                wuse[pb]++;
                wpend[pb] = 0;
            }
            if (r + 1 < nsite) {
                const int jn = i + 1 + wd;
                const uint32_t bytes = flip_bytes(jn);
                if (lane == 0 && bytes) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect(wmb + (pb ^ 1), bytes);
                    issue_flip(jn, wmb + (pb ^ 1));
                }
                wpend[pb ^ 1] = bytes ? 1u : 0u;
            }
        }
        float y_n = 0.f, dx_n[W], rh_n[kStMaxDout], el_n[W];
        if (r + 1 < nsite) load_site(i + 1, y_n, dx_n, rh_n, el_n);
        float acc[W];
#pragma unroll
        for (int q = 0; q < W; ++q) acc[q] = 0.f;
        if (l == 1) {
#pragma unroll
            for (int q = 0; q < W; ++q)
                if ((valid >> q) & 1u) acc[q] = Gs[(q - wd + 2 * wd) * d + c] * a.w.e[c] * dsq[q];
        } else {
            const float *wl = Win + (size_t)(l - 2) * W1 * W * d;
#pragma unroll
            for (int q = 0; q < W; ++q) {
                if (!((valid >> q) & 1u)) continue;
                float v = dsq[q] * el_c[q];
                const float *ws = wl + wsl[q] * W * d;
                for (int t2 = 0; t2 < W; ++t2)
                    if (site_ok(jq[q] - wd + t2)) v += Gs[(q - t2 + 2 * wd) * d + c] * ws[t2 * d + c];
                acc[q] = v;
            }
        }
        // Link blocks of this site.  Slot q of block dl multiplies the state of flip q at
        // slice position q + dl; where that position is off the slice or the flip does not
        // exist, the slot reads the zero row instead, so the inner loop has no branches.
        // Even and odd 16-byte chunks go to separate accumulators (two FMA chains per slot).
        float acc2[W];
#pragma unroll
        for (int q = 0; q < W; ++q) acc2[q] = 0.f;
        for (int mi = 0; mi < nlink && !timed_out; ++mi) {
            const float *wm = Win + (size_t)mi * W1 * W * d;
            for (int bi = 0; bi < nper; ++bi) {
                const int slot = con_slot;
                if (!mbar_wait(mb + slot, con_phase)) {
                    timed_out = true;
                    break;
                }
                ++consumed;
                if (++con_slot == NS) {
                    con_slot = 0;
                    con_phase ^= 1u;
                }
                const int dl = bi - 2 * wd;
                if (site_ok(i + dl)) {
                    const float *Kb = Kring + slot * dd + c * d;   // row c, 16-byte chunks swizzled by c mod 8
                    const int sw = c & 7;
                    const float *sp[W];
#pragma unroll
                    for (int q = 0; q < W; ++q) {
                        const int t2 = q + dl;
                        sp[q] = (t2 >= 0 && t2 < W && ((valid >> q) & 1u)) ? wm + (wsl[q] * W + t2) * d : Zs;
                    }
#pragma unroll
                    for (int s2 = 0; s2 < d / 4; s2 += 2) {
                        const int ch0 = s2, ch1 = s2 + 1;
                        const float4 k0 = *reinterpret_cast<const float4 *>(Kb + 4 * (ch0 ^ sw));
                        const float4 k1 = *reinterpret_cast<const float4 *>(Kb + 4 * (ch1 ^ sw));
#pragma unroll
                        for (int q = 0; q < W; ++q) {
                            const float4 s0 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch0);
                            const float4 s1 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch1);
                            acc[q] = fmaf(k0.x, s0.x, acc[q]);
                            acc2[q] = fmaf(k1.x, s1.x, acc2[q]);
                            acc[q] = fmaf(k0.y, s0.y, acc[q]);
                            acc2[q] = fmaf(k1.y, s1.y, acc2[q]);
                            acc[q] = fmaf(k0.z, s0.z, acc[q]);
                            acc2[q] = fmaf(k1.z, s1.z, acc2[q]);
                            acc[q] = fmaf(k0.w, s0.w, acc[q]);
                            acc2[q] = fmaf(k1.w, s1.w, acc2[q]);
                        }
                    }
                }
                __syncwarp();
                if (issued < nblk) {
                    if (lane == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        tma_block(Kring + iss_slot * dd, &tmK, (int)((iss_src - a.K) >> 5), mb + iss_slot);
                    }
                    ++issued;
                    iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
                    iss_advance();
                }
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q) acc[q] += acc2[q];
        if (timed_out) break;
        // s^(l) = U (dchi * (y + V p)) and its contribution to dOmega.
#pragma unroll
        for (int q = 0; q < W; ++q)
            if (q < W) pq[q * d + c] = acc[q];
        __syncwarp();
        float z[W];
#pragma unroll
        for (int q = 0; q < W; ++q) z[q] = y_c;
#pragma unroll 2
        for (int c2 = 0; c2 < d; c2 += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(VTs + ((c2 >> 2) * d + c) * 4);
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const float4 pv = *reinterpret_cast<const float4 *>(pq + q * d + c2);
                z[q] += v.x * pv.x + v.y * pv.y + v.z * pv.z + v.w * pv.w;
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q)
            if (q < W) gq[q * d + c] = dx_c[q] * z[q];
        __syncwarp();
        float sv[W];
#pragma unroll
        for (int q = 0; q < W; ++q) sv[q] = 0.f;
#pragma unroll 2
        for (int c2 = 0; c2 < d; c2 += 4) {
            const float4 u = *reinterpret_cast<const float4 *>(UTs + ((c2 >> 2) * d + c) * 4);
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const float4 gv = *reinterpret_cast<const float4 *>(gq + q * d + c2);
                sv[q] += u.x * gv.x + u.y * gv.y + u.z * gv.z + u.w * gv.w;
            }
        }
        float part[16];   // FP32 dot over the 32 channels; summed over layers in FP64
#pragma unroll
        for (int u = 0; u < 16; ++u) part[u] = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (q >= W || !((valid >> q) & 1u)) continue;
            if (l < L) S[(lo * rows + (b * N + jq[q]) * W + q) * d + c] = sv[q];
#pragma unroll
            for (int k = 0; k < kStMaxDout; ++k)
                if (q * kStMaxDout + k < 16) part[q * kStMaxDout + k] = rh_c[k] * sv[q];
        }
        const float tot = warp_sum16(part, lane);
        const int idx = (lane >> 1) & 15, qi = idx / kStMaxDout, ki = idx % kStMaxDout;
        if (!(lane & 1) && qi < W && ki < dout && ((valid >> qi) & 1u)) {
            double *dst = PART + ((b * N + wrap(i + wd - qi)) * W + qi) * dout + ki;
            *dst += (double)tot;
        }
        __syncwarp();
        y_c = y_n;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            dx_c[q] = dx_n[q];
            el_c[q] = el_n[q];
        }
#pragma unroll
        for (int k = 0; k < kStMaxDout; ++k) rh_c[k] = rh_n[k];
    }
    if (timed_out) {
        if (lane == 0) atomicOr(a.flag, 4u);
        // Let the copies in flight land before the shared memory is released.
        while (consumed < issued) {
            mbar_wait(mb + con_slot, con_phase);
            ++consumed;
            if (++con_slot == NS) {
                con_slot = 0;
                con_phase ^= 1u;
            }
        }
        for (int pb = 0; pb < 2; ++pb)
            if (wpend[pb]) mbar_wait(wmb + pb, wuse[pb] & 1u);
    }
}

// Cooperative streaming fast path of k_ab_layer for FP32 with d = 64 (the kernel is
// written for d in {32, 64}): the 8 warps of a CTA work on the same site of a run of
// consecutive sites.
//  * Link blocks K^(l,m)_{i,i+dl} are cut into 4 KB chunks of 1024 / d rows; warp w
//    owns row chunk j = w mod (d^2/1024) of every block whose index is congruent to
//    w div (d^2/1024) modulo 8 / (d^2/1024), and streams its chunks through its own
//    ring of NS shared-memory slots (cp.async.bulk, mbarrier completion).  The ring
//    runs ahead across sites, so the copies of the next sites are in flight while the
//    CTA finishes the current one.
//  * A lane owns one row of a chunk and 32 of its d columns; slot q of block dl
//    multiplies the state of flip q at slice position q + dl (the zero row where that
//    position or flip does not exist).  Partial sums go through shared memory and are
//    reduced per (slot, channel).
//  * The states s^(m) of the W flips around the site live in a window of W+1 flip
//    slots per m shared by the CTA (one bulk copy per m and site, issued a site early).
//  * The per-site epilogue (slice Toeplitz and embedding terms, V and U matvecs,
//    outputs, dOmega partials) is spread over the 256 threads.
// Every wait is bounded; a timeout raises bit 4 of the cache flag and the CTA lets its
// copies land before it ends.
constexpr int kCoWarps = 8;
constexpr int kCoPk = 2;   // (flip, output) pairs per warp whose inputs are loaded a contraction early

template <int D, int WW, int NS>
__global__ void __launch_bounds__(32 * kCoWarps, NS == 0 ? 2 : 1) k_ab_coop(AbArgs<float> a, int l, int R,
                                                                            float *__restrict__ S,
                                                                            const float *__restrict__ DX,
                                                                            double *__restrict__ PART,
                                                                            const __grid_constant__ CUtensorMap tmK) {
    extern __shared__ __align__(1024) unsigned char smco[];
    unsigned char *smraw = smco;
    constexpr int d = D, dd = D * D, W = WW, wd = (WW - 1) / 2, W1 = W + 1;
    constexpr int RC = 1024 / D;          // rows per 4 KB chunk
    constexpr int CPB = dd / 1024;        // chunks per block
    constexpr int WPJ = kCoWarps / CPB;   // warps per chunk row class
    constexpr int nper = 4 * wd + 1;
    constexpr int kCoIt = (W * D + 32 * kCoWarps - 1) / (32 * kCoWarps);   // (flip, channel) items per thread
    const Geom &g = a.g;
    const int N = g.N, L = g.L, dout = g.dout;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwin = l - 1, nlink = l > 2 ? l - 2 : 0;
    if ((smem_addr(smraw) & 1023u) != 0u) {   // the swizzled ring needs 1024-byte-aligned slots
        if (tid == 0) atomicOr(a.flag, 8u);
        return;
    }
    // Ring slots hold a chunk as [32-column segment][row][32], 128B-swizzled: chunk j of
    // line r (= segment * RC + row) sits at chunk j ^ (r mod 8).
    float *Kring = reinterpret_cast<float *>(smraw);   // [8][NS][1024], 4 KB-aligned slots
    float *VTs = Kring + kCoWarps * NS * 1024;         // [c'][c] = V[c][c']
    float *UTs = VTs + dd;
    float *Gs = UTs + dd;                            // [4w+1][d] taps g^(l)_{-2w..2w}
    float *Zs = Gs + nper * d;                       // [d] zeros
    float *Win = Zs + d;                             // [nwin][W+1][W][d]
    float *Pb = Win + nwin * W1 * W * d;             // [8][W][32] partial sums
    float *pq = Pb + kCoWarps * W * 32;              // [W][d]
    float *gq = pq + W * d;                          // [W][d]
    uint64_t *mbw = reinterpret_cast<uint64_t *>(gq + W * d);   // [8][NS] ring, then 2 window
    uint64_t *wmb = mbw + kCoWarps * NS;
    int *s_fail_p = reinterpret_cast<int *>(wmb + 2);
    int8_t *sps = reinterpret_cast<int8_t *>(s_fail_p + 2);
    const long long lo = l - 1;
    const long long b = blockIdx.y;
    for (int q = tid; q < dd; q += blockDim.x) {
        VTs[q] = a.w.VT[lo * dd + q];
        UTs[q] = a.w.UT[lo * dd + q];
    }
    for (int q = tid; q < nper * d; q += blockDim.x) {
        const int r = q / d - 2 * wd, cc = q % d;
        const int row = g.periodic ? ((r % N) + N) % N : (r > -N && r < N ? r + N - 1 : -1);
        Gs[q] = row >= 0 ? a.taps[(lo * g.R + row) * d + cc] : 0.f;
    }
    for (int q = tid; q < d; q += blockDim.x) Zs[q] = 0.f;
    for (int q = tid; q < N; q += blockDim.x) sps[q] = a.spins[b * N + q];
    if (tid == 0) {
        for (int s = 0; s < kCoWarps * NS + 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbw + s)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    const int i0 = blockIdx.x * R;
    const int nsite = N - i0 < R ? N - i0 : R;
    if (nsite <= 0) return;
    const long long rows = (long long)a.B * N * W;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    auto wrap = [&](int x) -> int { return g.periodic ? floor_mod(x, N) : x; };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    // ---- window of flip states (thread 0 issues) ----
    auto flip_bytes = [&](int jj) -> uint32_t { return site_ok(jj) ? (uint32_t)(nwin * W * d * sizeof(float)) : 0u; };
    auto issue_flip = [&](int jj, uint64_t *bar) {
        if (!site_ok(jj)) return;
        const int j = wrap(jj), slot = floor_mod(jj, W1);
        for (int m = 1; m <= nwin; ++m)
            bulk_copy(Win + ((m - 1) * W1 + slot) * W * d, S + ((m - 1) * rows + (b * N + j) * W) * d,
                      (uint32_t)(W * d * sizeof(float)), bar);
    };
    uint32_t wpend[2] = {0u, 0u}, wuse[2] = {0u, 0u};
    if (nwin > 0) {
        uint32_t bytes = 0;
        for (int jj = i0 - wd; jj <= i0 + wd; ++jj) bytes += flip_bytes(jj);
        if (tid == 0 && bytes) {
            mbar_expect(wmb, bytes);
            for (int jj = i0 - wd; jj <= i0 + wd; ++jj) issue_flip(jj, wmb);
        }
        wpend[0] = bytes ? 1u : 0u;
    }
    // ---- this warp's chunk stream ----
    const int jrow = warp % CPB, bcls = warp / CPB;
    const int nb_site = nlink * nper;
    int my_per_site = 0;
    for (int bb = bcls; bb < nb_site; bb += WPJ) ++my_per_site;
    const int nchunk = nsite * my_per_site;
    uint64_t *mb = mbw + warp * NS;
    float *ring = Kring + warp * NS * 1024;
    int iss_r = 0, iss_b = bcls, issued = 0, consumed = 0, iss_slot = 0, con_slot = 0;
    uint32_t con_phase = 0;
    auto iss_src = [&]() -> const float * {
        const int m = iss_b / nper + 1, dl = iss_b % nper - 2 * wd;
        return a.K + (((b * a.P + pair_index(l, m)) * N + (i0 + iss_r)) * nRk + (dl + a.Rk)) * (long long)dd +
               jrow * 1024;
    };
    auto iss_advance = [&]() {
        iss_b += WPJ;
        if (iss_b >= nb_site) {
            iss_b = bcls;
            ++iss_r;
        }
    };
    if (NS > 0 && nchunk > 0) {
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (; issued < nchunk && issued < NS; ++issued) {
            if (lane == 0) tma_chunk64(ring + iss_slot * 1024, &tmK, (int)((iss_src() - a.K) / d), mb + iss_slot);
            iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
            iss_advance();
        }
    }
    int &s_fail = *s_fail_p;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const int lrow = lane % RC, seg = lane / RC;      // chunk row, 32-column segment
    bool failed = false;
    for (int r = 0; r < nsite; ++r) {
        const int i = i0 + r;
        int jq[W], wsl[W];
        unsigned valid = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int jj = i + wd - q;
            const bool ok = site_ok(jj);
            jq[q] = ok ? wrap(jj) : 0;
            wsl[q] = floor_mod(jj, W1);
            if (ok) valid |= 1u << q;
        }
        // The epilogue's inputs from global memory (y, dchi, the embedding links, rho and
        // the dOmega partials of the earlier layers), loaded now so that their latency
        // hides behind the link contraction: thread tid owns items tid + 256 u of the
        // (flip, channel) loops, warp w the (flip, output) pairs w + 8 u.
        float pre_y[kCoIt], pre_dx[kCoIt], pre_el[kCoIt], pre_rho[kCoPk][D / 32];
        double pre_part[kCoPk];
#pragma unroll
        for (int u = 0; u < kCoIt; ++u) {
            const int it = tid + u * 32 * kCoWarps;
            pre_y[u] = pre_dx[u] = pre_el[u] = 0.f;
            if (it < W * d) {
                const int q = it / d, c = it % d;
                pre_y[u] = a.y[((b * L + lo) * N + i) * d + c];
                if ((valid >> q) & 1u) {
                    pre_dx[u] = DX[(lo * rows + (b * N + jq[q]) * W + q) * d + c];
                    if (l > 1) pre_el[u] = a.ell[((b * (L - 1) + (l - 2)) * N + i) * nRl * d + (wd - q + a.Rl) * d + c];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kCoPk; ++u) {
            const int pk = warp + u * kCoWarps, q = pk / dout, k = pk % dout;
            pre_part[u] = 0.0;
#pragma unroll
            for (int h = 0; h < D / 32; ++h) pre_rho[u][h] = 0.f;
            if (pk < W * dout && ((valid >> q) & 1u)) {
                const float *rho = a.rho + ((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d;
#pragma unroll
                for (int h = 0; h < D / 32; ++h) pre_rho[u][h] = rho[lane + 32 * h];
                if (lane == 0) pre_part[u] = PART[((b * N + jq[q]) * W + q) * dout + k];
            }
        }
        // Window of this site; then the next site's new flip into the slot released by the last one.
        if (nwin > 0) {
            const int pb = r & 1;
            if (wpend[pb]) {
                if (tid == 0 && !mbar_wait(wmb + pb, wuse[pb] & 1u)) s_fail = 1;
                wuse[pb]++;
                wpend[pb] = 0;
            }
            __syncthreads();
            if (s_fail) {
                failed = true;
                break;
            }
            if (r + 1 < nsite) {
                const int jn = i + 1 + wd;
                const uint32_t bytes = flip_bytes(jn);
                if (tid == 0 && bytes) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect(wmb + (pb ^ 1), bytes);
                    issue_flip(jn, wmb + (pb ^ 1));
                }
                wpend[pb ^ 1] = bytes ? 1u : 0u;
            }
        }
        // Link chunks of this warp for site r.
        float acc[W], acc2[W];
#pragma unroll
        for (int q = 0; q < W; ++q) acc[q] = acc2[q] = 0.f;
        for (int bb = bcls; bb < nb_site && !failed; bb += WPJ) {
            if (!mbar_wait(mb + con_slot, con_phase)) {
                failed = true;
                break;
            }
            const int slot = con_slot;
            ++consumed;
            if (++con_slot == NS) {
                con_slot = 0;
                con_phase ^= 1u;
            }
            const int mi = bb / nper, dl = bb % nper - 2 * wd;
            if (site_ok(i + dl)) {
                const float *wm = Win + (size_t)mi * W1 * W * d + seg * 32;
                const float *Kc = ring + slot * 1024 + (seg * RC + lrow) * 32;   // line seg * RC + lrow
                const int sw = lrow & 7;
                const float *sp[W];
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    const int t2 = q + dl;
                    sp[q] = (t2 >= 0 && t2 < W && ((valid >> q) & 1u)) ? wm + (wsl[q] * W + t2) * d : Zs;
                }
#pragma unroll
                for (int s2 = 0; s2 < 8; s2 += 2) {
                    const int ch0 = s2, ch1 = s2 + 1;
                    const float4 k0 = *reinterpret_cast<const float4 *>(Kc + 4 * (ch0 ^ sw));
                    const float4 k1 = *reinterpret_cast<const float4 *>(Kc + 4 * (ch1 ^ sw));
#pragma unroll
                    for (int q = 0; q < W; ++q) {
                        const float4 s0 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch0);
                        const float4 s1 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch1);
                        acc[q] = fmaf(k0.x, s0.x, acc[q]);
                        acc2[q] = fmaf(k1.x, s1.x, acc2[q]);
                        acc[q] = fmaf(k0.y, s0.y, acc[q]);
                        acc2[q] = fmaf(k1.y, s1.y, acc2[q]);
                        acc[q] = fmaf(k0.z, s0.z, acc[q]);
                        acc2[q] = fmaf(k1.z, s1.z, acc2[q]);
                        acc[q] = fmaf(k0.w, s0.w, acc[q]);
                        acc2[q] = fmaf(k1.w, s1.w, acc2[q]);
                    }
                }
            }
            __syncwarp();
            if (issued < nchunk) {
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_chunk64(ring + iss_slot * 1024, &tmK, (int)((iss_src() - a.K) / d), mb + iss_slot);
                }
                ++issued;
                iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
                iss_advance();
            }
        }
        if (failed) s_fail = 1;
#pragma unroll
        for (int q = 0; q < W; ++q) Pb[(warp * W + q) * 32 + lane] = acc[q] + acc2[q];
        __syncthreads();
        if (s_fail) {
            failed = true;
            break;
        }
        // Reduce the partials per (q, c), add the slice Toeplitz and embedding terms.
#pragma unroll
        for (int u = 0; u < kCoIt; ++u) {
            const int it = tid + u * 32 * kCoWarps;
            if (it >= W * d) break;
            const int q = it / d, c = it % d;
            float v = 0.f;
            if (nlink > 0) {
                const int jj = c / RC, rr = c % RC;
#pragma unroll
                for (int bc = 0; bc < WPJ; ++bc)
#pragma unroll
                    for (int sg = 0; sg < 32 / RC; ++sg) v += Pb[((jj + bc * CPB) * W + q) * 32 + sg * RC + rr];
            }
            if ((valid >> q) & 1u) {
                const float dsq = (float)(-2 * sps[jq[q]]);
                if (l == 1) {
                    v += Gs[(q - wd + 2 * wd) * d + c] * a.w.e[c] * dsq;
                } else {
                    v += dsq * pre_el[u];
                    const float *ws = Win + ((size_t)(l - 2) * W1 + wsl[q]) * W * d;
                    for (int t2 = 0; t2 < W; ++t2)
                        if (site_ok(jq[q] - wd + t2)) v += Gs[(q - t2 + 2 * wd) * d + c] * ws[t2 * d + c];
                }
            }
            pq[it] = v;
        }
        __syncthreads();
        // z = y + V p, then the gate with dchi.
#pragma unroll
        for (int u = 0; u < kCoIt; ++u) {
            const int it = tid + u * 32 * kCoWarps;
            if (it >= W * d) break;
            const int q = it / d, c = it % d;
            // four partial sums: the chain of dependent FMAs is a quarter as long
            float z0 = pre_y[u], z1 = 0.f, z2 = 0.f, z3 = 0.f;
            const float *pr = pq + q * d;
#pragma unroll 4
            for (int c2 = 0; c2 < d; c2 += 4) {
                const float4 pv = *reinterpret_cast<const float4 *>(pr + c2);
                z0 = fmaf(VTs[c2 * d + c], pv.x, z0);
                z1 = fmaf(VTs[(c2 + 1) * d + c], pv.y, z1);
                z2 = fmaf(VTs[(c2 + 2) * d + c], pv.z, z2);
                z3 = fmaf(VTs[(c2 + 3) * d + c], pv.w, z3);
            }
            gq[it] = pre_dx[u] * ((z0 + z1) + (z2 + z3));
        }
        __syncthreads();
        // s^(l) = U g; written to S (next layers) and kept in pq for the dOmega partials.
        for (int it = tid; it < W * d; it += blockDim.x) {
            const int q = it / d, c = it % d;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            const float *gr = gq + q * d;
#pragma unroll 4
            for (int c2 = 0; c2 < d; c2 += 4) {
                const float4 gv = *reinterpret_cast<const float4 *>(gr + c2);
                s0 = fmaf(UTs[c2 * d + c], gv.x, s0);
                s1 = fmaf(UTs[(c2 + 1) * d + c], gv.y, s1);
                s2 = fmaf(UTs[(c2 + 2) * d + c], gv.z, s2);
                s3 = fmaf(UTs[(c2 + 3) * d + c], gv.w, s3);
            }
            const float s = (s0 + s1) + (s2 + s3);
            pq[it] = s;
            if (l < L && ((valid >> q) & 1u)) S[(lo * rows + (b * N + jq[q]) * W + q) * d + c] = s;
        }
        __syncthreads();
        // dOmega_k partial of (flip q, layer l): rho^(l)_k(i) . s, in FP64; one warp per (q, k).
#pragma unroll
        for (int u = 0; u < kCoPk; ++u) {
            const int pk = warp + u * kCoWarps, q = pk / dout, k = pk % dout;
            if (pk >= W * dout || !((valid >> q) & 1u)) continue;
            // FP32 dot over the channels (FP64 arithmetic is scarce on this part); the
            // partials of the layers are summed in FP64
            float v = 0.f;
#pragma unroll
            for (int h = 0; h < D / 32; ++h) v = fmaf(pre_rho[u][h], pq[q * d + lane + 32 * h], v);
            v = warp_sum<float>(v);
            if (lane == 0) PART[((b * N + jq[q]) * W + q) * dout + k] = pre_part[u] + (double)v;
        }
        for (int pk = warp + kCoPk * kCoWarps; pk < W * dout; pk += kCoWarps) {
            const int q = pk / dout, k = pk % dout;
            if (!((valid >> q) & 1u)) continue;
            const float *rho = a.rho + ((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d;
            float v = 0.f;
            for (int c = lane; c < d; c += 32) v = fmaf(rho[c], pq[q * d + c], v);
            v = warp_sum<float>(v);
            if (lane == 0) PART[((b * N + jq[q]) * W + q) * dout + k] += (double)v;
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicOr(a.flag, 4u);
        // Let the copies in flight land before the shared memory is released.
        while (consumed < issued) {
            mbar_wait(mb + con_slot, con_phase);
            ++consumed;
            if (++con_slot == NS) {
                con_slot = 0;
                con_phase ^= 1u;
            }
        }
        if (tid == 0)
            for (int pb = 0; pb < 2; ++pb)
                if (wpend[pb]) mbar_wait(wmb + pb, wuse[pb] & 1u);
        __syncthreads();
    }
}

// Warp-specialised form of k_ab_coop for the layers with link blocks (l > 2), FP32,
// d = 64.  The link contraction of a site and its epilogue no longer alternate on the
// same warps: the contraction of site r + 1 streams link chunks while the epilogue of
// site r runs, so the CTA-wide steps of the epilogue no longer stall the HBM stream.
//  * warps 0-7 (contraction): as in k_ab_coop, warp w streams row chunk w mod 4 of the
//    link blocks of class w div 4 through its own ring of NS slots, and multiplies them
//    with the slice states of the window; its per-flip partials go to one of two
//    partial buffers.  Warp 0 also copies the next site's new flip into the window.
//  * warps 8-15 (epilogue): reduce the partials, add the slice Toeplitz and embedding
//    terms, the V and U matvecs with the gate, the states s^(l) (to S) and the dOmega
//    partials; their global inputs are loaded before they wait for the partials.
// Hand-offs are mbarriers: full[b] (all contraction threads arrive after writing partial
// buffer b), empty[b] (the epilogue arrives once it has read buffer b and the window
// slots of that site), and four window barriers by site (r mod 4).  The window has
// W + 2 flip slots, so that the copy for site r + 1 only overwrites a flip that site r - 2
// used last.  Every wait is bounded; a wait that gives up raises bit 4 of the cache flag
// and sets the CTA's stop word, every role leaves its loop, and the copies in flight are
// waited for (bounded) before the CTA ends.
constexpr int kCoEpiWarps = 8;

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}
// Barrier 1 over the epilogue warps, returning whether `ok` holds on every thread.
__device__ __forceinline__ bool epi_all(bool ok) {
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)ok), "n"(32 * kCoEpiWarps)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kCoEpiWarps) : "memory"); }

template <int D, int WW, int NS>
__global__ void __launch_bounds__(32 * (kCoWarps + kCoEpiWarps), 1)
    k_ab_coop_ws(AbArgs<float> a, int l, int R, float *__restrict__ S, const float *__restrict__ DX,
                 double *__restrict__ PART, const __grid_constant__ CUtensorMap tmK) {
    extern __shared__ __align__(1024) unsigned char smws[];
    unsigned char *smraw = smws;
    constexpr int d = D, dd = D * D, W = WW, wd = (WW - 1) / 2, W2 = W + 2;
    constexpr int RC = 1024 / D;          // rows per 4 KB chunk
    constexpr int CPB = dd / 1024;        // chunks per block
    constexpr int WPJ = kCoWarps / CPB;   // warps per chunk row class
    constexpr int nper = 4 * wd + 1;
    constexpr int kET = 32 * kCoEpiWarps;                 // epilogue threads
    constexpr int kEIt = (W * D + kET - 1) / kET;         // (flip, channel) items per epilogue thread
    constexpr int kEPk = 3;                              // (flip, output) pairs per warp loaded early
    const Geom &g = a.g;
    const int N = g.N, L = g.L, dout = g.dout;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwin = l - 1, nlink = l - 2;
    if ((smem_addr(smraw) & 1023u) != 0u) {   // the swizzled ring needs 1024-byte-aligned slots
        if (tid == 0) atomicOr(a.flag, 8u);
        return;
    }
    float *Kring = reinterpret_cast<float *>(smraw);   // [8][NS][1024], 4 KB-aligned slots
    float *VTs = Kring + kCoWarps * NS * 1024;         // [c'][c] = V[c][c']
    float *UTs = VTs + dd;
    float *Gs = UTs + dd;                              // [4w+1][d] taps g^(l)_{-2w..2w}
    float *Zs = Gs + nper * d;                         // [d] zeros
    float *Win = Zs + d;                               // [nwin][W + 2][W][d]
    float *Pb = Win + nwin * W2 * W * d;               // [2][8][W][32] partial sums
    float *pq = Pb + 2 * kCoWarps * W * 32;            // [W][d]
    float *gq = pq + W * d;                            // [W][d]
    uint64_t *mbw = reinterpret_cast<uint64_t *>(gq + W * d);   // [8][NS] ring
    uint64_t *wmb = mbw + kCoWarps * NS;                         // [4] window, by site mod 4
    uint64_t *full = wmb + 4;                                    // [2]
    uint64_t *empty = full + 2;                                  // [2]
    int *s_stop = reinterpret_cast<int *>(empty + 2);
    int8_t *sps = reinterpret_cast<int8_t *>(s_stop + 2);
    const long long lo = l - 1;
    const long long b = blockIdx.y;
    for (int q = tid; q < dd; q += blockDim.x) {
        VTs[q] = a.w.VT[lo * dd + q];
        UTs[q] = a.w.UT[lo * dd + q];
    }
    for (int q = tid; q < nper * d; q += blockDim.x) {
        const int r = q / d - 2 * wd, cc = q % d;
        const int row = g.periodic ? ((r % N) + N) % N : (r > -N && r < N ? r + N - 1 : -1);
        Gs[q] = row >= 0 ? a.taps[(lo * g.R + row) * d + cc] : 0.f;
    }
    for (int q = tid; q < d; q += blockDim.x) Zs[q] = 0.f;
    for (int q = tid; q < N; q += blockDim.x) sps[q] = a.spins[b * N + q];
    if (tid == 0) {
        for (int s = 0; s < kCoWarps * NS + 4; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbw + s)), "r"(1));
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + s)), "r"(32 * kCoWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(empty + s)), "r"(1));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_stop = 0;
    }
    __syncthreads();
    const int i0 = blockIdx.x * R;
    const int nsite = N - i0 < R ? N - i0 : R;
    if (nsite <= 0) return;
    const long long rows = (long long)a.B * N * W;
    const long long nRk = 2 * a.Rk + 1, nRl = 2 * a.Rl + 1;
    auto wrap = [&](int x) -> int { return g.periodic ? floor_mod(x, N) : x; };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    auto stopped = [&]() -> bool { return *((volatile int *)s_stop) != 0; };
    // flips of site i: slot q holds flip i + wd - q
    auto flips_of = [&](int i, int (&jq)[W], int (&wsl)[W]) -> unsigned {
        unsigned valid = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int jj = i + wd - q;
            const bool ok = site_ok(jj);
            jq[q] = ok ? wrap(jj) : 0;
            wsl[q] = floor_mod(jj, W2);
            if (ok) valid |= 1u << q;
        }
        return valid;
    };
    if (warp < kCoWarps) {
        // ------------------------------------------------------------ contraction --
        auto flip_bytes = [&](int jj) -> uint32_t {
            return site_ok(jj) ? (uint32_t)(nwin * W * d * sizeof(float)) : 0u;
        };
        auto issue_flip = [&](int jj, uint64_t *bar) {
            if (!site_ok(jj)) return;
            const int j = wrap(jj), slot = floor_mod(jj, W2);
            for (int m = 1; m <= nwin; ++m)
                bulk_copy(Win + ((m - 1) * W2 + slot) * W * d, S + ((m - 1) * rows + (b * N + j) * W) * d,
                          (uint32_t)(W * d * sizeof(float)), bar);
        };
        const bool leader = warp == 0 && lane == 0;
        int wissued = 0, wdone = 0;   // window phases armed / observed by this warp (leader's bookkeeping)
        if (leader) {
            uint32_t bytes = 0;
            for (int jj = i0 - wd; jj <= i0 + wd; ++jj) bytes += flip_bytes(jj);
            mbar_expect(wmb, bytes);
            for (int jj = i0 - wd; jj <= i0 + wd; ++jj) issue_flip(jj, wmb);
        }
        wissued = 1;
        // this warp's chunk stream
        const int jrow = warp % CPB, bcls = warp / CPB;
        const int nb_site = nlink * nper;
        int my_per_site = 0;
        for (int bb = bcls; bb < nb_site; bb += WPJ) ++my_per_site;
        const int nchunk = nsite * my_per_site;
        uint64_t *mb = mbw + warp * NS;
        float *ring = Kring + warp * NS * 1024;
        int iss_r = 0, iss_b = bcls, issued = 0, consumed = 0, iss_slot = 0, con_slot = 0;
        uint32_t con_phase = 0;
        auto iss_row = [&]() -> int {
            const int m = iss_b / nper + 1, dl = iss_b % nper - 2 * wd;
            const float *src = a.K + (((b * a.P + pair_index(l, m)) * N + (i0 + iss_r)) * nRk + (dl + a.Rk)) *
                                         (long long)dd + jrow * 1024;
            return (int)((src - a.K) / d);
        };
        auto iss_advance = [&]() {
            iss_b += WPJ;
            if (iss_b >= nb_site) {
                iss_b = bcls;
                ++iss_r;
            }
        };
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (; issued < nchunk && issued < NS; ++issued) {
            if (lane == 0) tma_chunk64(ring + iss_slot * 1024, &tmK, iss_row(), mb + iss_slot);
            iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
            iss_advance();
        }
        const int lrow = lane % RC, seg = lane / RC;      // chunk row, 32-column segment
        bool failed = false;
        for (int r = 0; r < nsite && !failed; ++r) {
            const int i = i0 + r, buf = r & 1;
            int jq[W], wsl[W];
            const unsigned valid = flips_of(i, jq, wsl);
            // partial buffer `buf` and the window slot of flip i - wd - 2 were released by the
            // epilogue of site r - 2
            bool ok = !stopped();
            if (ok && r >= 2) ok = mbar_wait(empty + buf, ((r - 2) >> 1) & 1);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            if (leader && r + 1 < nsite) {
                const int jn = i + 1 + wd;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect(wmb + ((r + 1) & 3), flip_bytes(jn));   // 0 bytes: a plain arrive
                issue_flip(jn, wmb + ((r + 1) & 3));
            }
            if (r + 1 < nsite) wissued = r + 2;
            ok = mbar_wait(wmb + (r & 3), (r >> 2) & 1);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            wdone = r + 1;
            float acc[W], acc2[W];
#pragma unroll
            for (int q = 0; q < W; ++q) acc[q] = acc2[q] = 0.f;
            for (int bb = bcls; bb < nb_site; bb += WPJ) {
                ok = mbar_wait(mb + con_slot, con_phase);
                if (!__all_sync(0xffffffffu, ok)) {
                    failed = true;
                    break;
                }
                const int slot = con_slot;
                ++consumed;
                if (++con_slot == NS) {
                    con_slot = 0;
                    con_phase ^= 1u;
                }
                const int mi = bb / nper, dl = bb % nper - 2 * wd;
                if (site_ok(i + dl)) {
                    const float *wm = Win + (size_t)mi * W2 * W * d + seg * 32;
                    const float *Kc = ring + slot * 1024 + (seg * RC + lrow) * 32;   // line seg * RC + lrow
                    const int sw = lrow & 7;
                    const float *sp[W];
#pragma unroll
                    for (int q = 0; q < W; ++q) {
                        const int t2 = q + dl;
                        sp[q] = (t2 >= 0 && t2 < W && ((valid >> q) & 1u)) ? wm + (wsl[q] * W + t2) * d : Zs;
                    }
#pragma unroll
                    for (int s2 = 0; s2 < 8; s2 += 2) {
                        const int ch0 = s2, ch1 = s2 + 1;
                        const float4 k0 = *reinterpret_cast<const float4 *>(Kc + 4 * (ch0 ^ sw));
                        const float4 k1 = *reinterpret_cast<const float4 *>(Kc + 4 * (ch1 ^ sw));
#pragma unroll
                        for (int q = 0; q < W; ++q) {
                            const float4 s0 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch0);
                            const float4 s1 = *reinterpret_cast<const float4 *>(sp[q] + 4 * ch1);
                            acc[q] = fmaf(k0.x, s0.x, acc[q]);
                            acc2[q] = fmaf(k1.x, s1.x, acc2[q]);
                            acc[q] = fmaf(k0.y, s0.y, acc[q]);
                            acc2[q] = fmaf(k1.y, s1.y, acc2[q]);
                            acc[q] = fmaf(k0.z, s0.z, acc[q]);
                            acc2[q] = fmaf(k1.z, s1.z, acc2[q]);
                            acc[q] = fmaf(k0.w, s0.w, acc[q]);
                            acc2[q] = fmaf(k1.w, s1.w, acc2[q]);
                        }
                    }
                }
                __syncwarp();
                if (issued < nchunk) {
                    if (lane == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        tma_chunk64(ring + iss_slot * 1024, &tmK, iss_row(), mb + iss_slot);
                    }
                    ++issued;
                    iss_slot = iss_slot + 1 == NS ? 0 : iss_slot + 1;
                    iss_advance();
                }
            }
            if (failed) break;
            float *pb = Pb + ((size_t)buf * kCoWarps + warp) * W * 32;
#pragma unroll
            for (int q = 0; q < W; ++q) pb[q * 32 + lane] = acc[q] + acc2[q];
            mbar_arrive_cta(full + buf);
        }
        if (failed) {
            if (lane == 0) {
                *((volatile int *)s_stop) = 1;
                atomicOr(a.flag, 4u);
            }
            // Let the copies in flight land before the shared memory is released.
            while (consumed < issued) {
                mbar_wait(mb + con_slot, con_phase);
                ++consumed;
                if (++con_slot == NS) {
                    con_slot = 0;
                    con_phase ^= 1u;
                }
            }
            if (leader)
                for (int s = wdone; s < wissued; ++s) mbar_wait(wmb + (s & 3), (s >> 2) & 1);
        }
    } else {
        // --------------------------------------------------------------- epilogue --
        const int et = tid - 32 * kCoWarps, ew = warp - kCoWarps;
        bool good = true;
        for (int r = 0; r < nsite; ++r) {
            const int i = i0 + r, buf = r & 1;
            int jq[W], wsl[W];
            const unsigned valid = flips_of(i, jq, wsl);
            // Global inputs of this site, loaded before the wait for its partials: thread et
            // owns items et + 256 u of the (flip, channel) loops, warp ew the (flip, output)
            // pairs ew + 8 u.
            float pre_y[kEIt], pre_dx[kEIt], pre_el[kEIt], pre_rho[kEPk][D / 32];
            double pre_part[kEPk];
#pragma unroll
            for (int u = 0; u < kEIt; ++u) {
                const int it = et + u * kET;
                pre_y[u] = pre_dx[u] = pre_el[u] = 0.f;
                if (it < W * d) {
                    const int q = it / d, c = it % d;
                    pre_y[u] = a.y[((b * L + lo) * N + i) * d + c];
                    if ((valid >> q) & 1u) {
                        pre_dx[u] = DX[(lo * rows + (b * N + jq[q]) * W + q) * d + c];
                        pre_el[u] = a.ell[((b * (L - 1) + (l - 2)) * N + i) * nRl * d + (wd - q + a.Rl) * d + c];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kEPk; ++u) {
                const int pk = ew + u * kCoEpiWarps, q = pk / dout, k = pk % dout;
                pre_part[u] = 0.0;
#pragma unroll
                for (int h = 0; h < D / 32; ++h) pre_rho[u][h] = 0.f;
                if (pk < W * dout && ((valid >> q) & 1u)) {
                    const float *rho = a.rho + ((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d;
#pragma unroll
                    for (int h = 0; h < D / 32; ++h) pre_rho[u][h] = rho[lane + 32 * h];
                    if (lane == 0) pre_part[u] = PART[((b * N + jq[q]) * W + q) * dout + k];
                }
            }
            const bool ok = !stopped() && mbar_wait(full + buf, (r >> 1) & 1);
            if (!epi_all(ok)) {
                good = false;
                break;
            }
            // Reduce the partials per (q, c), add the slice Toeplitz and embedding terms.
            const float *pbuf = Pb + (size_t)buf * kCoWarps * W * 32;
#pragma unroll
            for (int u = 0; u < kEIt; ++u) {
                const int it = et + u * kET;
                if (it >= W * d) break;
                const int q = it / d, c = it % d;
                float v = 0.f;
                const int jj = c / RC, rr = c % RC;
#pragma unroll
                for (int bc = 0; bc < WPJ; ++bc)
#pragma unroll
                    for (int sg = 0; sg < 32 / RC; ++sg) v += pbuf[((jj + bc * CPB) * W + q) * 32 + sg * RC + rr];
                if ((valid >> q) & 1u) {
                    const float dsq = (float)(-2 * sps[jq[q]]);
                    v += dsq * pre_el[u];
                    const float *ws = Win + ((size_t)(l - 2) * W2 + wsl[q]) * W * d;
                    for (int t2 = 0; t2 < W; ++t2)
                        if (site_ok(jq[q] - wd + t2)) v += Gs[(q - t2 + 2 * wd) * d + c] * ws[t2 * d + c];
                }
                pq[it] = v;
            }
            epi_sync();
            if (et == 0) mbar_arrive_cta(empty + buf);   // partials and window slots of site r read
            // z = y + V p, then the gate with dchi.
#pragma unroll
            for (int u = 0; u < kEIt; ++u) {
                const int it = et + u * kET;
                if (it >= W * d) break;
                const int q = it / d, c = it % d;
                float z0 = pre_y[u], z1 = 0.f, z2 = 0.f, z3 = 0.f;
                const float *pr = pq + q * d;
#pragma unroll 4
                for (int c2 = 0; c2 < d; c2 += 4) {
                    const float4 pv = *reinterpret_cast<const float4 *>(pr + c2);
                    z0 = fmaf(VTs[c2 * d + c], pv.x, z0);
                    z1 = fmaf(VTs[(c2 + 1) * d + c], pv.y, z1);
                    z2 = fmaf(VTs[(c2 + 2) * d + c], pv.z, z2);
                    z3 = fmaf(VTs[(c2 + 3) * d + c], pv.w, z3);
                }
                gq[it] = pre_dx[u] * ((z0 + z1) + (z2 + z3));
            }
            epi_sync();
            // s^(l) = U g; written to S (next layers) and kept in pq for the dOmega partials.
#pragma unroll
            for (int u = 0; u < kEIt; ++u) {
                const int it = et + u * kET;
                if (it >= W * d) break;
                const int q = it / d, c = it % d;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                const float *gr = gq + q * d;
#pragma unroll 4
                for (int c2 = 0; c2 < d; c2 += 4) {
                    const float4 gv = *reinterpret_cast<const float4 *>(gr + c2);
                    s0 = fmaf(UTs[c2 * d + c], gv.x, s0);
                    s1 = fmaf(UTs[(c2 + 1) * d + c], gv.y, s1);
                    s2 = fmaf(UTs[(c2 + 2) * d + c], gv.z, s2);
                    s3 = fmaf(UTs[(c2 + 3) * d + c], gv.w, s3);
                }
                const float s = (s0 + s1) + (s2 + s3);
                pq[it] = s;
                if (l < L && ((valid >> q) & 1u)) S[(lo * rows + (b * N + jq[q]) * W + q) * d + c] = s;
            }
            epi_sync();
            // dOmega_k partial of (flip q, layer l): rho^(l)_k(i) . s (FP32 dot, FP64 sum over layers).
#pragma unroll
            for (int u = 0; u < kEPk; ++u) {
                const int pk = ew + u * kCoEpiWarps, q = pk / dout, k = pk % dout;
                if (pk >= W * dout || !((valid >> q) & 1u)) continue;
                float v = 0.f;
#pragma unroll
                for (int h = 0; h < D / 32; ++h) v = fmaf(pre_rho[u][h], pq[q * d + lane + 32 * h], v);
                v = warp_sum<float>(v);
                if (lane == 0) PART[((b * N + jq[q]) * W + q) * dout + k] = pre_part[u] + (double)v;
            }
            for (int pk = ew + kEPk * kCoEpiWarps; pk < W * dout; pk += kCoEpiWarps) {
                const int q = pk / dout, k = pk % dout;
                if (!((valid >> q) & 1u)) continue;
                const float *rho = a.rho + ((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d;
                float v = 0.f;
                for (int c = lane; c < d; c += 32) v = fmaf(rho[c], pq[q * d + c], v);
                v = warp_sum<float>(v);
                if (lane == 0) PART[((b * N + jq[q]) * W + q) * dout + k] += (double)v;
            }
            epi_sync();   // pq and gq are rewritten by the next site
        }
        if (!good && et == 0) {
            *((volatile int *)s_stop) = 1;
            atomicOr(a.flag, 4u);
        }
    }
}

// The link-free layers (l <= 2: no interlayer link block, at most one window of slice
// states) of an FP32 cache with d = 64 and d_out <= 2.  Their work per site is small
// (two 64 x 64 matvecs on W flips) and bounded by latency, so every warp walks its own
// run of R sites with no CTA-wide step, 16 warps per CTA: lane t owns channels t and
// t + 32.  The per-warp window of layer-1 slice states (l = 2) is kept as in
// k_ab_stream: W + 1 flip slots, one bulk copy per new flip, issued a site early.  Every
// wait is bounded; a timeout raises bit 4 of the cache flag and the warp lets its copies
// land before it ends.
constexpr int kLfWarps = 16;

template <int WW>
__global__ void __launch_bounds__(32 * kLfWarps, 1) k_ab_lf64(AbArgs<float> a, int l, int R, float *__restrict__ S,
                                                              const float *__restrict__ DX,
                                                              double *__restrict__ PART) {
    extern __shared__ __align__(16) unsigned char smlf[];
    constexpr int d = 64, dd = d * d, W = WW, wd = (WW - 1) / 2, W1 = W + 1, nper = 4 * wd + 1;
    const Geom &g = a.g;
    const int N = g.N, L = g.L, dout = g.dout;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwin = l - 1;
    float *VTs = reinterpret_cast<float *>(smlf);   // [k/4][c][k%4]: one 16-byte load = rows k..k+3 of column c
    float *UTs = VTs + dd;
    float *Gs = UTs + dd;                           // [4w+1][d] taps g^(l)_{-2w..2w}
    const int per_warp = nwin * W1 * W * d + 2 * W * d;
    float *Win = Gs + nper * d + (size_t)warp * per_warp;   // [nwin][W+1][W][d]
    float *pq = Win + nwin * W1 * W * d;                    // [W][d]
    float *gq = pq + W * d;                                 // [W][d]
    uint64_t *wmb = reinterpret_cast<uint64_t *>(Gs + nper * d + (size_t)kLfWarps * per_warp) + 2 * warp;
    int8_t *sps = reinterpret_cast<int8_t *>(reinterpret_cast<uint64_t *>(Gs + nper * d + (size_t)kLfWarps * per_warp) +
                                             2 * kLfWarps);
    const long long lo = l - 1;
    const long long b = blockIdx.y;
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        const int k = q / d, cc = q % d, x = ((k >> 2) * d + cc) * 4 + (k & 3);
        VTs[x] = a.w.VT[lo * dd + q];
        UTs[x] = a.w.UT[lo * dd + q];
    }
    for (int q = threadIdx.x; q < nper * d; q += blockDim.x) {
        const int r = q / d - 2 * wd, cc = q % d;
        const int row = g.periodic ? ((r % N) + N) % N : (r > -N && r < N ? r + N - 1 : -1);
        Gs[q] = row >= 0 ? a.taps[(lo * g.R + row) * d + cc] : 0.f;
    }
    for (int q = threadIdx.x; q < N; q += blockDim.x) sps[q] = a.spins[b * N + q];
    if (lane == 0) {
        for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(wmb + s)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    const int i0 = (blockIdx.x * kLfWarps + warp) * R;
    const int nsite = N - i0 < R ? N - i0 : R;
    if (nsite <= 0) return;
    const long long rows = (long long)a.B * N * W;
    const long long nRl = 2 * a.Rl + 1;
    auto wrap = [&](int x) -> int { return g.periodic ? floor_mod(x, N) : x; };
    auto site_ok = [&](int k) -> bool { return g.periodic || (k >= 0 && k < N); };
    // Window copies (l = 2): flip jj (unwrapped) of layer 1 into slot jj mod (W+1).
    auto issue_flip = [&](int jj, uint64_t *bar) {
        if (!site_ok(jj)) return;
        bulk_copy(Win + floor_mod(jj, W1) * W * d, S + (b * N + wrap(jj)) * W * d, (uint32_t)(W * d * sizeof(float)),
                  bar);
    };
    auto flip_bytes = [&](int jj) -> uint32_t { return site_ok(jj) ? (uint32_t)(W * d * sizeof(float)) : 0u; };
    uint32_t wpend[2] = {0u, 0u}, wuse[2] = {0u, 0u};
    if (nwin > 0) {
        uint32_t bytes = 0;
        for (int jj = i0 - wd; jj <= i0 + wd; ++jj) bytes += flip_bytes(jj);
        if (lane == 0 && bytes) {
            mbar_expect(wmb, bytes);
            for (int jj = i0 - wd; jj <= i0 + wd; ++jj) issue_flip(jj, wmb);
        }
        wpend[0] = bytes ? 1u : 0u;
    }
    float e_h[2] = {0.f, 0.f};
    if (l == 1) {
        e_h[0] = a.w.e[lane];
        e_h[1] = a.w.e[lane + 32];
    }
    // Per-site inputs of site r (cur) and r + 1 (nxt), channels lane and lane + 32.
    struct In {
        float y[2], dx[W][2], el[W][2], rh[kStMaxDout][2];
    };
    auto load_site = [&](int i, In &v) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            v.y[h] = a.y[((b * L + lo) * N + i) * d + c];
#pragma unroll
            for (int q = 0; q < W; ++q) {
                v.dx[q][h] = 0.f;
                v.el[q][h] = 0.f;
                const int jj = i + wd - q;
                if (!site_ok(jj)) continue;
                v.dx[q][h] = DX[(lo * rows + (b * N + wrap(jj)) * W + q) * d + c];
                if (l >= 2) v.el[q][h] = a.ell[((b * (L - 1) + (l - 2)) * N + i) * nRl * d + (wd - q + a.Rl) * d + c];
            }
#pragma unroll
            for (int k = 0; k < kStMaxDout; ++k)
                v.rh[k][h] = k < dout ? a.rho[((b * L + lo) * dout + k) * (long long)N * d + (long long)i * d + c] : 0.f;
        }
    };
    In cur, nxt;
    load_site(i0, cur);
    nxt = cur;
    bool timed_out = false;
    for (int r = 0; r < nsite; ++r) {
        const int i = i0 + r;
        int jq[W], wsl[W];
        float dsq[W];
        unsigned valid = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int jj = i + wd - q;
            const bool ok = site_ok(jj);
            jq[q] = ok ? wrap(jj) : 0;
            wsl[q] = floor_mod(jj, W1);
            dsq[q] = ok ? (float)(-2 * sps[jq[q]]) : 0.f;
            if (ok) valid |= 1u << q;
        }
        if (nwin > 0) {
            const int pb = r & 1;
            if (wpend[pb]) {
                if (!mbar_wait(wmb + pb, wuse[pb] & 1u)) {
                    timed_out = true;
                    break;
                }
                wuse[pb]++;
                wpend[pb] = 0;
            }
            if (r + 1 < nsite) {
                const int jn = i + 1 + wd;
                const uint32_t bytes = flip_bytes(jn);
                if (lane == 0 && bytes) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect(wmb + (pb ^ 1), bytes);
                    issue_flip(jn, wmb + (pb ^ 1));
                }
                wpend[pb ^ 1] = bytes ? 1u : 0u;
            }
        }
        if (r + 1 < nsite) load_site(i + 1, nxt);
        // p: slice Toeplitz and embedding terms (l = 2) or the embedding column (l = 1).
#pragma unroll
        for (int q = 0; q < W; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                float v = 0.f;
                if ((valid >> q) & 1u) {
                    if (l == 1) {
                        v = Gs[(q - wd + 2 * wd) * d + c] * e_h[h] * dsq[q];
                    } else {
                        v = dsq[q] * cur.el[q][h];
                        const float *ws = Win + wsl[q] * W * d;
                        for (int t2 = 0; t2 < W; ++t2)
                            if (site_ok(jq[q] - wd + t2)) v += Gs[(q - t2 + 2 * wd) * d + c] * ws[t2 * d + c];
                    }
                }
                pq[q * d + c] = v;
            }
        }
        __syncwarp();
        // z = y + V p, gate with dchi
        float z[W][2];
#pragma unroll
        for (int q = 0; q < W; ++q) z[q][0] = z[q][1] = 0.f;
#pragma unroll 2
        for (int c2 = 0; c2 < d; c2 += 4) {
            const float4 v0 = *reinterpret_cast<const float4 *>(VTs + ((c2 >> 2) * d + lane) * 4);
            const float4 v1 = *reinterpret_cast<const float4 *>(VTs + ((c2 >> 2) * d + lane + 32) * 4);
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const float4 pv = *reinterpret_cast<const float4 *>(pq + q * d + c2);
                z[q][0] += v0.x * pv.x + v0.y * pv.y + v0.z * pv.z + v0.w * pv.w;
                z[q][1] += v1.x * pv.x + v1.y * pv.y + v1.z * pv.z + v1.w * pv.w;
            }
        }
#pragma unroll
        for (int q = 0; q < W; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) gq[q * d + lane + 32 * h] = cur.dx[q][h] * (cur.y[h] + z[q][h]);
        __syncwarp();
        // s = U g
#pragma unroll
        for (int q = 0; q < W; ++q) z[q][0] = z[q][1] = 0.f;
#pragma unroll 2
        for (int c2 = 0; c2 < d; c2 += 4) {
            const float4 u0 = *reinterpret_cast<const float4 *>(UTs + ((c2 >> 2) * d + lane) * 4);
            const float4 u1 = *reinterpret_cast<const float4 *>(UTs + ((c2 >> 2) * d + lane + 32) * 4);
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const float4 gv = *reinterpret_cast<const float4 *>(gq + q * d + c2);
                z[q][0] += u0.x * gv.x + u0.y * gv.y + u0.z * gv.z + u0.w * gv.w;
                z[q][1] += u1.x * gv.x + u1.y * gv.y + u1.z * gv.z + u1.w * gv.w;
            }
        }
        float part[16];   // FP32 dot over the channels; summed over layers in FP64
#pragma unroll
        for (int u = 0; u < 16; ++u) part[u] = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            if (!((valid >> q) & 1u)) continue;
            if (l < L)
#pragma unroll
                for (int h = 0; h < 2; ++h) S[(lo * rows + (b * N + jq[q]) * W + q) * d + lane + 32 * h] = z[q][h];
#pragma unroll
            for (int k = 0; k < kStMaxDout; ++k)
                if (q * kStMaxDout + k < 16) part[q * kStMaxDout + k] = cur.rh[k][0] * z[q][0] + cur.rh[k][1] * z[q][1];
        }
        const float tot = warp_sum16(part, lane);
        const int idx = (lane >> 1) & 15, qi = idx / kStMaxDout, ki = idx % kStMaxDout;
        if (!(lane & 1) && qi < W && ki < dout && ((valid >> qi) & 1u))
            PART[((b * N + wrap(i + wd - qi)) * W + qi) * dout + ki] += (double)tot;
        __syncwarp();   // pq and gq are rewritten by the next site
        cur = nxt;
    }
    if (timed_out) {
        if (lane == 0) atomicOr(a.flag, 4u);
        for (int pb = 0; pb < 2; ++pb)
            if (wpend[pb]) mbar_wait(wmb + pb, wuse[pb] & 1u);
    }
}

// out[(b nb + bond) N + j]: the sum of a flip's slot partials and its embedding terms
// t_j ds_j (Eq. recur_out), through the readout.  A pair past an open end gives 0.
__global__ void k_ab_final(Geom g, FlipPattern fp, int B, int f_kind, const int8_t *__restrict__ spins,
                           const double *__restrict__ Omega, const double *__restrict__ PART,
                           const void *__restrict__ tlink, int tsize, double *__restrict__ out) {
    const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int N = g.N, W = g.W, dout = g.dout, nb = fp.nb, Wm = fp.Wm;
    if (f >= (long long)B * nb * N) return;
    const long long b = f / ((long long)nb * N);
    const int bond = (int)((f / N) % nb), j = (int)(f % N);
    const int dl = bond_of(fp, bond);
    int jp = -1;
    if (dl > 0) {
        jp = g.periodic ? (j + dl) % N : j + dl;
        if (jp >= N || (fp.anti && spins[b * N + j] == spins[b * N + jp])) {
            out[f] = 0.0;
            return;
        }
    }
    const double ds = -2.0 * spins[b * N + j], dsp = jp >= 0 ? -2.0 * spins[b * N + jp] : 0.0;
    const long long row0 = ((b * N + j) * nb + bond) * Wm;
    auto tval = [&](long long ti) -> double {
        return tsize == 8 ? static_cast<const double *>(tlink)[ti] : (double)static_cast<const float *>(tlink)[ti];
    };
    double res = 0.0;
    for (int k = 0; k < dout; ++k) {
        double s = tval((b * N + j) * dout + k) * ds;
        if (jp >= 0) s += tval((b * N + jp) * dout + k) * dsp;
        for (int t = 0; t < W + dl; ++t) s += PART[(row0 + t) * dout + k];
        const double om = Omega[b * dout + k];
        res += f_kind == 0 ? (log_cosh_ab(om + s) - log_cosh_ab(om)) : s;
    }
    out[f] = res;
}

template <typename T>
static AbArgs<T> ab_args(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c) {
    AbArgs<T> a;
    a.g = geom_of(m, c->N);
    a.B = c->B;
    a.WF = c->WF;
    a.Rk = c->Rk;
    a.Rl = c->Rl;
    a.P = c->P;
    a.max_cluster = c->max_cluster;
    a.f_kind = m->desc.f_kind;
    a.spins = c->spins;
    a.chi = static_cast<const T *>(c->chi);
    a.y = static_cast<const T *>(c->y);
    a.rho = static_cast<const T *>(c->rho);
    a.t = static_cast<const T *>(c->t);
    a.ell = static_cast<const T *>(c->ell);
    a.K = static_cast<const T *>(c->K);
    a.taps = pl.taps;
    a.Omega = c->Omega;
    a.flag = c->flag;
    a.w = w;
    a.dOmega = nullptr;
    return a;
}

// Descriptor of a cache for k_abacus_multi (a plain struct, copied to the device by the caller).
template <typename T>
size_t abacus_desc_bytes() {
    static_assert(sizeof(AbArgs<T>) % 16 == 0, "descriptor records are read as an array on the device");
    return sizeof(AbArgs<T>);
}

template <typename T>
void abacus_desc(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c, void *dst) {
    const AbArgs<T> a = ab_args<T>(m, pl, w, c);
    memcpy(dst, &a, sizeof(a));
}

template <typename T>
cudaError_t launch_abacus_multi(const dn_model *m, int WF, const void *descs, const int32_t *cache_of,
                                const int32_t *sample, const int32_t *sites, int F, double *out, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    const dn_model_desc &D = m->desc;
    const size_t tsz = ((size_t)(D.L + 3) * WF * D.d + 2 * (size_t)WF * D.d_h) * sizeof(T);
    const size_t smem = ((tsz + 7) & ~(size_t)7) + (size_t)kMaxDout * kAbThreads * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_abacus_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_abacus_multi", st);
        k_abacus_multi<T><<<F, kAbThreads, smem, st>>>(static_cast<const AbArgs<T> *>(descs), cache_of, sample, sites,
                                                       F, out);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_abacus_serve(const dn_model *m, int WF, const void *descs, ServeQueue *q, ServeItems it,
                                unsigned long long *ctl, unsigned long long base, long long idle_ns, int ctas,
                                cudaStream_t st) {
    const dn_model_desc &D = m->desc;
    const size_t tsz = ((size_t)(D.L + 3) * WF * D.d + 2 * (size_t)WF * D.d_h) * sizeof(T);
    const size_t smem = ((tsz + 7) & ~(size_t)7) + (size_t)kMaxDout * kAbThreads * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_abacus_serve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_abacus_serve", st);
        k_abacus_serve<T><<<ctas, kAbThreads, smem, st>>>(static_cast<const AbArgs<T> *>(descs), q, it, ctl, base,
                                                          idle_ns);
    }
    return cudaGetLastError();
}

template size_t abacus_desc_bytes<double>();
template size_t abacus_desc_bytes<float>();
template void abacus_desc<double>(const dn_model *, const Plan<double> &, const Weights<double> &, const dn_cache *,
                                  void *);
template void abacus_desc<float>(const dn_model *, const Plan<float> &, const Weights<float> &, const dn_cache *,
                                 void *);
template cudaError_t launch_abacus_serve<double>(const dn_model *, int, const void *, ServeQueue *, ServeItems,
                                                 unsigned long long *, unsigned long long, long long, int, cudaStream_t);
template cudaError_t launch_abacus_serve<float>(const dn_model *, int, const void *, ServeQueue *, ServeItems,
                                                unsigned long long *, unsigned long long, long long, int, cudaStream_t);
template cudaError_t launch_abacus_multi<double>(const dn_model *, int, const void *, const int32_t *, const int32_t *,
                                                 const int32_t *, int, double *, cudaStream_t);
template cudaError_t launch_abacus_multi<float>(const dn_model *, int, const void *, const int32_t *, const int32_t *,
                                                const int32_t *, int, double *, cudaStream_t);

size_t singles_scratch_bytes(const dn_model *m, const dn_cache *c) {
    const size_t W = 2 * m->desc.w + 1, rows = (size_t)c->B * c->N * W;
    const size_t tb = c->prec == DN_FP64 ? 8 : 4;
    return 2 * (size_t)m->desc.L * rows * m->desc.d * tb + rows * m->desc.d_out * 8 + 1024;
}

template <typename T, int HD>
static cudaError_t launch_ab_layer(const AbArgs<T> &a, int l, T *S, const T *DX, double *PART, cudaStream_t st) {
    const Geom &g = a.g;
    const size_t smem = (2 * (size_t)g.d * g.d + 8 * ((size_t)g.W * g.W * g.d + 2 * (size_t)g.W * g.d)) * sizeof(T);
    cudaError_t err = cudaFuncSetAttribute(k_ab_layer<T, HD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid((g.N + 7) / 8, a.B);
    {
        ProfScope _ps("k_ab_layer", st);
        k_ab_layer<T, HD><<<grid, 256, smem, st>>>(a, l, S, DX, PART);
    }
    return cudaGetLastError();
}

// Shared memory of k_ab_stream with NS ring slots; 0 if it does not fit.
static size_t ab_stream_smem(const Geom &g, int l, int NS) {
    const size_t d = 32, W = g.W, nwin = l - 1;
    const size_t per_warp = NS * d * d + nwin * (W + 1) * W * d + 2 * W * d;   // ring slots first, then the rest
    const size_t floats = 2 * d * d + (size_t)(4 * g.w + 2) * d + kStWarps * per_warp;
    const size_t bytes = floats * sizeof(float) + (size_t)kStWarps * (kStMaxNS + 2) * sizeof(uint64_t) +
                         (((size_t)g.N + 15) & ~(size_t)15);
    return bytes <= 227 * 1024 ? bytes : 0;
}

template <int WW, int NS>
static cudaError_t launch_ab_stream_one(const AbArgs<float> &a, int l, int R, dim3 grid, size_t smem, float *S,
                                       const float *DX, double *PART, const CUtensorMap &tmK, cudaStream_t st) {
    cudaError_t err = cudaFuncSetAttribute(k_ab_stream<WW, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_ab_layer", st);
        k_ab_stream<WW, NS><<<grid, 32 * kStWarps, smem, st>>>(a, l, R, S, DX, PART, tmK);
    }
    return cudaGetLastError();
}

template <int WW>
static cudaError_t launch_ab_stream_ns(const AbArgs<float> &a, int l, int R, int NS, dim3 grid, size_t smem, float *S,
                                      const float *DX, double *PART, const CUtensorMap &tmK, cudaStream_t st) {
    switch (NS) {
    case 0: return launch_ab_stream_one<WW, 0>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 2: return launch_ab_stream_one<WW, 2>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 3: return launch_ab_stream_one<WW, 3>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 4: return launch_ab_stream_one<WW, 4>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    default: return cudaErrorNotSupported;
    }
}

static cudaError_t launch_ab_stream(const AbArgs<float> &a, int l, float *S, const float *DX, double *PART,
                                    cudaStream_t st) {
    const Geom &g = a.g;
    int NS = 0;
    size_t smem = ab_stream_smem(g, l, 0);
    if (l > 2) {
        for (NS = kStMaxNS; NS >= 2; --NS)
            if ((smem = ab_stream_smem(g, l, NS)) != 0) break;
        if (NS < 2) return cudaErrorNotSupported;
    }
    if (smem == 0) return cudaErrorNotSupported;
    // Runs of R sites per warp (8 warps per CTA, one CTA per SM): 8 keeps the copy ring
    // full across sites; shorter runs where 8 leaves the last wave of CTAs mostly empty.
    int R = 8;
    {
        auto tail = [&](int r) {
            const long long ctas = (long long)((g.N + kStWarps * r - 1) / (kStWarps * r)) * a.B;
            const long long w = (ctas + 151) / 152;
            return (double)(w * 152 - ctas) / (double)(w * 152);
        };
        if (tail(8) > 0.25 && tail(4) < tail(8)) R = 4;
    }
    dim3 grid((unsigned)((g.N + kStWarps * R - 1) / (kStWarps * R)), (unsigned)a.B);
    // Link blocks through a tensor map over the cache's K array viewed as rows of 32 floats
    // (unused by the link-free layers l <= 2).
    alignas(64) CUtensorMap tmK;
    std::memset(&tmK, 0, sizeof(tmK));
    if (l > 2) {
        const unsigned long long rows =
            (unsigned long long)a.B * a.P * g.N * (2ull * a.Rk + 1) * 32ull;
        if (!a.K || !link_rows_map(&tmK, a.K, rows, 32, 32)) return cudaErrorNotSupported;
    }
    if (g.W == 5) return launch_ab_stream_ns<5>(a, l, R, NS, grid, smem, S, DX, PART, tmK, st);
    if (g.W == 3) return launch_ab_stream_ns<3>(a, l, R, NS, grid, smem, S, DX, PART, tmK, st);
    return cudaErrorNotSupported;
}

// Shared memory of k_ab_coop with NS ring slots per warp; 0 if it does not fit.
static size_t ab_coop_smem(const Geom &g, int l, int NS) {
    const size_t d = g.d, W = g.W, nwin = l - 1, nper = 4 * g.w + 1;
    const size_t floats = 2 * d * d + nper * d + d + nwin * (W + 1) * W * d + (size_t)kCoWarps * W * 32 + 2 * W * d +
                          (size_t)kCoWarps * NS * 1024;
    const size_t bytes = floats * sizeof(float) + ((size_t)kCoWarps * NS + 2) * sizeof(uint64_t) + 2 * sizeof(int) +
                         (((size_t)g.N + 15) & ~(size_t)15);
    return bytes <= 227 * 1024 ? bytes : 0;
}

template <int D, int WW, int NS>
static cudaError_t launch_ab_coop_one(const AbArgs<float> &a, int l, int R, dim3 grid, size_t smem, float *S,
                                      const float *DX, double *PART, const CUtensorMap &tmK, cudaStream_t st) {
    cudaError_t err = cudaFuncSetAttribute(k_ab_coop<D, WW, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_ab_layer", st);
        k_ab_coop<D, WW, NS><<<grid, 32 * kCoWarps, smem, st>>>(a, l, R, S, DX, PART, tmK);
    }
    return cudaGetLastError();
}

template <int D, int WW>
static cudaError_t launch_ab_coop_ns(const AbArgs<float> &a, int l, int R, int NS, dim3 grid, size_t smem, float *S,
                                     const float *DX, double *PART, const CUtensorMap &tmK, cudaStream_t st) {
    switch (NS) {
    case 0: return launch_ab_coop_one<D, WW, 0>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 2: return launch_ab_coop_one<D, WW, 2>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 4: return launch_ab_coop_one<D, WW, 4>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 6: return launch_ab_coop_one<D, WW, 6>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    default: return cudaErrorNotSupported;
    }
}

// Shared memory of k_ab_coop_ws with NS ring slots per contraction warp; 0 if it does not fit.
static size_t ab_coop_ws_smem(const Geom &g, int l, int NS) {
    const size_t d = g.d, W = g.W, nwin = l - 1, nper = 4 * g.w + 1;
    const size_t floats = 2 * d * d + nper * d + d + nwin * (W + 2) * W * d + 2 * (size_t)kCoWarps * W * 32 +
                          2 * W * d + (size_t)kCoWarps * NS * 1024;
    const size_t bytes = floats * sizeof(float) + ((size_t)kCoWarps * NS + 8) * sizeof(uint64_t) + 2 * sizeof(int) +
                         (((size_t)g.N + 15) & ~(size_t)15);
    return bytes <= 227 * 1024 ? bytes : 0;
}

template <int D, int WW, int NS>
static cudaError_t launch_ab_coop_ws_one(const AbArgs<float> &a, int l, int R, dim3 grid, size_t smem, float *S,
                                         const float *DX, double *PART, const CUtensorMap &tmK, cudaStream_t st) {
    cudaError_t err =
        cudaFuncSetAttribute(k_ab_coop_ws<D, WW, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_ab_layer", st);
        k_ab_coop_ws<D, WW, NS><<<grid, 32 * (kCoWarps + kCoEpiWarps), smem, st>>>(a, l, R, S, DX, PART, tmK);
    }
    return cudaGetLastError();
}

template <int D, int WW>
static cudaError_t launch_ab_coop_ws_ns(const AbArgs<float> &a, int l, int R, int NS, dim3 grid, size_t smem,
                                        float *S, const float *DX, double *PART, const CUtensorMap &tmK,
                                        cudaStream_t st) {
    switch (NS) {
    case 2: return launch_ab_coop_ws_one<D, WW, 2>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 4: return launch_ab_coop_ws_one<D, WW, 4>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    case 6: return launch_ab_coop_ws_one<D, WW, 6>(a, l, R, grid, smem, S, DX, PART, tmK, st);
    default: return cudaErrorNotSupported;
    }
}

// Shared memory of k_ab_lf64; 0 if it does not fit.
static size_t ab_lf64_smem(const Geom &g, int l) {
    const size_t d = 64, W = g.W, nwin = l - 1, nper = 4 * g.w + 1;
    const size_t per_warp = nwin * (W + 1) * W * d + 2 * W * d;
    const size_t floats = 2 * d * d + nper * d + (size_t)kLfWarps * per_warp;
    const size_t bytes = floats * sizeof(float) + 2 * (size_t)kLfWarps * sizeof(uint64_t) + (((size_t)g.N + 15) & ~(size_t)15);
    return bytes <= 227 * 1024 ? bytes : 0;
}

template <int WW>
static cudaError_t launch_ab_lf64(const AbArgs<float> &a, int l, float *S, const float *DX, double *PART,
                                  size_t smem, cudaStream_t st) {
    const Geom &g = a.g;
    cudaError_t err = cudaFuncSetAttribute(k_ab_lf64<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    // Runs of R sites per warp, R chosen so that the warps of one CTA per SM cover the sites.
    const long long sites = (long long)g.N * a.B, slots = 152LL * kLfWarps;
    long long R = (sites + slots - 1) / slots;
    R = R < 1 ? 1 : (R > 32 ? 32 : R);
    dim3 grid((unsigned)((g.N + kLfWarps * R - 1) / (kLfWarps * R)), (unsigned)a.B);
    {
        ProfScope _ps("k_ab_layer", st);
        k_ab_lf64<WW><<<grid, 32 * kLfWarps, smem, st>>>(a, l, (int)R, S, DX, PART);
    }
    return cudaGetLastError();
}

static cudaError_t launch_ab_coop(const AbArgs<float> &a, int l, float *S, const float *DX, double *PART,
                                  cudaStream_t st) {
    const Geom &g = a.g;
    if (l <= 2 && g.d == 64 && g.dout <= kStMaxDout) {
        const size_t sml = ab_lf64_smem(g, l);
        if (sml && g.W == 5) return launch_ab_lf64<5>(a, l, S, DX, PART, sml, st);
        if (sml && g.W == 3) return launch_ab_lf64<3>(a, l, S, DX, PART, sml, st);
    }
    int NS = 0;
    size_t smem = ab_coop_smem(g, l, 0);
    if (l > 2) {
        for (NS = 6; NS >= 2; NS -= 2)
            if ((smem = ab_coop_smem(g, l, NS)) != 0) break;
        if (NS < 2) return cudaErrorNotSupported;
    }
    if (smem == 0) return cudaErrorNotSupported;
    // Runs of R sites per CTA (one CTA per SM fits with a link ring, two without): R is chosen
    // so that the runs make whole waves of 152 (304) CTAs, with runs of at most 32 sites - a
    // grid of 2.07 waves spent a third round on its last 11 CTAs.
    const long long sites = (long long)g.N * a.B;
    const long long slots = NS == 0 ? 2 * 152 : 152;   // link-free layers: two CTAs per SM fit
    const long long waves = (sites + slots * 32 - 1) / (slots * 32);
    long long R = (sites + slots * waves - 1) / (slots * waves);
    R = R < 2 ? 2 : (R > 32 ? 32 : R);
    dim3 grid((unsigned)((g.N + R - 1) / R), (unsigned)a.B);
    const int Ri = (int)R;
    // Link chunks through a tensor map over the cache's K array viewed as rows of 64 floats
    // (unused by the link-free layers l <= 2).
    alignas(64) CUtensorMap tmK;
    std::memset(&tmK, 0, sizeof(tmK));
    if (l > 2) {
        const unsigned long long rows = (unsigned long long)a.B * a.P * g.N * (2ull * a.Rk + 1) * 64ull;
        if (g.d != 64 || !a.K || !link_rows_map(&tmK, a.K, rows, 64, 16)) return cudaErrorNotSupported;
    }
    if (l > 2) {
        // Layers with link blocks: the warp-specialised kernel (contraction and epilogue
        // overlapped), with the deepest ring that fits.
        int NSw = 6;
        size_t smw = 0;
        for (; NSw >= 2; NSw -= 2)
            if ((smw = ab_coop_ws_smem(g, l, NSw)) != 0) break;
        if (NSw >= 2) {
            if (g.W == 5) return launch_ab_coop_ws_ns<64, 5>(a, l, Ri, NSw, grid, smw, S, DX, PART, tmK, st);
            if (g.W == 3) return launch_ab_coop_ws_ns<64, 3>(a, l, Ri, NSw, grid, smw, S, DX, PART, tmK, st);
        }
    }
    if (g.d == 64 && g.W == 5) return launch_ab_coop_ns<64, 5>(a, l, Ri, NS, grid, smem, S, DX, PART, tmK, st);
    if (g.d == 64 && g.W == 3) return launch_ab_coop_ns<64, 3>(a, l, Ri, NS, grid, smem, S, DX, PART, tmK, st);
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_abacus_singles(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c,
                                  void *scratch, double *out, cudaStream_t st) {
    const Geom g = geom_of(m, c->N);
    if (g.W > kLayMaxW || g.d > 128) return cudaErrorNotSupported;
    const size_t lsm = (2 * (size_t)g.d * g.d + 8 * ((size_t)g.W * g.W * g.d + 2 * (size_t)g.W * g.d)) * sizeof(T);
    const size_t tsm = 64 * sizeof(long long) +
                       ((size_t)g.dh * (g.dh + 4) + (size_t)g.dh * (g.d + 4) + 2 * 68 * (size_t)g.dh + 64 * (size_t)g.W) *
                           sizeof(T);
    if (lsm > 220 * 1024 || tsm > 220 * 1024) return cudaErrorNotSupported;
    const AbArgs<T> a = ab_args<T>(m, pl, w, c);
    const FlipPattern singles{1, g.W, {0, 0}, 0};
    const long long rows = (long long)c->B * c->N * g.W;
    T *DX = static_cast<T *>(scratch);
    T *S = DX + (size_t)g.L * rows * g.d;
    double *PART = reinterpret_cast<double *>(S + (size_t)g.L * rows * g.d);
    cudaError_t err = cudaMemsetAsync(PART, 0, (size_t)rows * g.dout * sizeof(double), st);
    if (err != cudaSuccess) return err;
    if ((err = cudaFuncSetAttribute(k_dchi_table<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) !=
        cudaSuccess)
        return err;
    {
        ProfScope _ps("k_dchi_table", st);
        // Tiles of 64 rows, up to kDxTPB per CTA (the weights are staged once per CTA), but
        // enough CTAs for four per SM.
        const long long tiles = (rows + 63) / 64;
        long long tpb = (tiles * g.L + 4 * 152 - 1) / (4 * 152);
        tpb = tpb < 1 ? 1 : (tpb > kDxTPB ? kDxTPB : tpb);
        k_dchi_table<T, false><<<dim3((unsigned)((tiles + tpb - 1) / tpb), g.L), 256, tsm, st>>>(a, singles, DX, (int)tpb);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int hd = (g.d + 31) / 32;
    // The streaming kernel takes FP32 caches with d = 32, W in {3, 5} and d_out <= 2; a
    // layer whose shared memory would not fit falls back to k_ab_layer.
    const bool stream_ok = sizeof(T) == 4 && g.d == 32 && (g.W == 3 || g.W == 5) && g.dout <= kStMaxDout;
    // d = 64 takes the cooperative kernel; at d = 32 a site's link rows (72 KB at L = 4) are too
    // little work to amortise its CTA-wide steps and the per-warp kernel is faster (measured).
    const bool coop_ok = sizeof(T) == 4 && g.d == 64 && (g.W == 3 || g.W == 5);
    for (int l = 1; l <= g.L; ++l) {
        err = cudaErrorNotSupported;
        if constexpr (std::is_same_v<T, float>) {
            if (coop_ok) err = launch_ab_coop(a, l, S, DX, PART, st);
            if (err == cudaErrorNotSupported && stream_ok) {
                cudaGetLastError();
                err = launch_ab_stream(a, l, S, DX, PART, st);
            }
        }
        if (err == cudaSuccess) continue;
        if (err != cudaErrorNotSupported) return err;
        cudaGetLastError();
        if (hd == 1) err = launch_ab_layer<T, 1>(a, l, S, DX, PART, st);
        else if (hd == 2) err = launch_ab_layer<T, 2>(a, l, S, DX, PART, st);
        else err = launch_ab_layer<T, 4>(a, l, S, DX, PART, st);
        if (err != cudaSuccess) return err;
    }
    {
        ProfScope _ps("k_ab_final", st);
        k_ab_final<<<(unsigned)(((long long)c->B * c->N + 255) / 256), 256, 0, st>>>(
            g, singles, c->B, m->desc.f_kind, c->spins, c->Omega, PART, c->t, (int)sizeof(T), out);
    }
    return cudaGetLastError();
}

template cudaError_t launch_abacus_singles<double>(const dn_model *, const Plan<double> &, const Weights<double> &,
                                                   const dn_cache *, void *, double *, cudaStream_t);
template cudaError_t launch_abacus_singles<float>(const dn_model *, const Plan<float> &, const Weights<float> &,
                                                  const dn_cache *, void *, double *, cudaStream_t);

static int pattern_wm(const dn_model *m, int nb, const int *bonds) {
    int mx = 0;
    for (int q = 0; q < nb; ++q) mx = bonds[q] > mx ? bonds[q] : mx;
    return 2 * m->desc.w + 1 + mx;
}

bool pairs_grouped_fits(const dn_model *m, const dn_cache *c, int nb, const int *bonds) {
    const int Wm = pattern_wm(m, nb, bonds);
    return nb >= 1 && nb <= 2 && Wm <= kPrMaxWs && Wm <= c->WF && m->desc.d <= 64 && c->B <= 65535;
}

size_t pairs_scratch_bytes(const dn_model *m, const dn_cache *c, int nb, const int *bonds) {
    const size_t rows = (size_t)c->B * c->N * nb * pattern_wm(m, nb, bonds);
    const size_t tb = c->prec == DN_FP64 ? 8 : 4;
    return 2 * (size_t)m->desc.L * rows * m->desc.d * tb + rows * m->desc.d_out * 8 + 1024;
}

template <typename T>
cudaError_t launch_abacus_pairs(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, const dn_cache *c, int nb,
                                const int *bonds, bool anti, void *scratch, double *out, cudaStream_t st) {
    const Geom g = geom_of(m, c->N);
    if (nb < 1 || nb > 2) return cudaErrorInvalidValue;
    FlipPattern fp{nb, pattern_wm(m, nb, bonds), {bonds[0], nb > 1 ? bonds[1] : 0}, anti ? 1 : 0};
    for (int q = 0; q < nb; ++q)
        if (bonds[q] < 1 || bonds[q] > c->max_cluster - 1) return cudaErrorInvalidValue;
    if (!pairs_grouped_fits(m, c, nb, bonds)) return cudaErrorNotSupported;
    const size_t tsm = 64 * sizeof(long long) +
                       ((size_t)g.dh * (g.dh + 4) + (size_t)g.dh * (g.d + 4) + 2 * 68 * (size_t)g.dh + 64 * (size_t)g.W) *
                           sizeof(T);
    // Sites per CTA (one warp each): the most resident warps per SM for the shared flip
    // windows and the per-warp buffers.
    const int ws0 = g.W + fp.bond[0], ws1 = nb > 1 ? g.W + fp.bond[1] : 0;
    auto lsm_of = [&](int nw) -> size_t {
        return (2 * (size_t)g.d * g.d + (size_t)(nw + ws0 - 1) * ws0 * g.d + (size_t)(nw + ws1 - 1) * ws1 * g.d +
                (size_t)nw * (nb * fp.Wm + 1) * g.d) *
               sizeof(T);
    };
    const bool two = g.d > 32;
    constexpr bool F32 = std::is_same<T, float>::value;
    const bool vec = F32 && g.d % 16 == 0;
    auto kfn = two ? (vec ? k_ab_pairs<T, 2, F32> : k_ab_pairs<T, 2, false>)
                   : (vec ? k_ab_pairs<T, 1, F32> : k_ab_pairs<T, 1, false>);
    cudaError_t err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (err != cudaSuccess) return err;
    int wpc = 0, best = 0;
    for (int nw = 1; nw <= 8; ++nw) {
        if (lsm_of(nw) > 220 * 1024) break;
        int blocks = 0;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kfn, 32 * nw, lsm_of(nw))) != cudaSuccess)
            return err;
        if (blocks * nw >= best && blocks > 0) {
            best = blocks * nw;
            wpc = nw;
        }
    }
    if (wpc == 0 || tsm > 220 * 1024) return cudaErrorNotSupported;
    const size_t lsm = lsm_of(wpc);
    const AbArgs<T> a = ab_args<T>(m, pl, w, c);
    const long long rows = (long long)c->B * c->N * nb * fp.Wm;
    T *DX = static_cast<T *>(scratch);
    T *S = DX + (size_t)g.L * rows * g.d;
    double *PART = reinterpret_cast<double *>(S + (size_t)g.L * rows * g.d);
    err = cudaMemsetAsync(PART, 0, (size_t)rows * g.dout * sizeof(double), st);
    if (err != cudaSuccess) return err;
    if ((err = cudaFuncSetAttribute(k_dchi_table<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) !=
        cudaSuccess)
        return err;
    {
        ProfScope _ps("k_dchi_table", st);
        const long long tiles = (rows + 63) / 64;
        long long tpb = (tiles * g.L + 4 * 152 - 1) / (4 * 152);
        tpb = tpb < 1 ? 1 : (tpb > kDxTPB ? kDxTPB : tpb);
        k_dchi_table<T, true><<<dim3((unsigned)((tiles + tpb - 1) / tpb), g.L), 256, tsm, st>>>(a, fp, DX, (int)tpb);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const dim3 grid((unsigned)((g.N + wpc - 1) / wpc), (unsigned)c->B);
    for (int l = 1; l <= g.L; ++l) {
        ProfScope _ps("k_ab_pairs", st);
        kfn<<<grid, 32 * wpc, lsm, st>>>(a, fp, l, S, DX, PART);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    {
        ProfScope _ps("k_ab_final", st);
        k_ab_final<<<(unsigned)(((long long)c->B * nb * c->N + 255) / 256), 256, 0, st>>>(
            g, fp, c->B, m->desc.f_kind, c->spins, c->Omega, PART, c->t, (int)sizeof(T), out);
    }
    return cudaGetLastError();
}

template cudaError_t launch_abacus_pairs<double>(const dn_model *, const Plan<double> &, const Weights<double> &,
                                                 const dn_cache *, int, const int *, bool, void *, double *,
                                                 cudaStream_t);
template cudaError_t launch_abacus_pairs<float>(const dn_model *, const Plan<float> &, const Weights<float> &,
                                                const dn_cache *, int, const int *, bool, void *, double *,
                                                cudaStream_t);

template cudaError_t launch_abacus<double>(const dn_model *, const Plan<double> &, const Weights<double> &,
                                           const dn_cache *, const int32_t *, const int32_t *, int, double *,
                                           cudaStream_t, double *);
template cudaError_t launch_abacus<float>(const dn_model *, const Plan<float> &, const Weights<float> &,
                                          const dn_cache *, const int32_t *, const int32_t *, int, double *,
                                          cudaStream_t, double *);

// ------------------------------------------------------ local estimator ----
// Connected flip sets.  kind 0 (TFIM): every single site, f = b N + i.
// kind 1 (J1-J2): pairs (i, i+1) then (i, i+2), f = b 2N + (bond-1) N + i;
// aligned pairs and pairs past an open end are empty entries.
__global__ void k_make_flips(int kind, int N, int B, int periodic, const int8_t *__restrict__ spins,
                             int32_t *__restrict__ sample, int32_t *__restrict__ sites) {
    const long long per = kind == 0 ? N : 2 * N;
    const long long F = per * B;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < F; f += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(f / per);
        const int r = (int)(f % per);
        sample[f] = b;
        if (kind == 0) {
            sites[2 * f] = r;
            sites[2 * f + 1] = -1;
        } else {
            const int bond = r / N + 1, i = r % N;
            int j = i + bond;
            bool ok = true;
            if (periodic) j %= N;
            else if (j >= N) ok = false;
            if (ok && spins[(long long)b * N + i] == spins[(long long)b * N + j]) ok = false;
            sites[2 * f] = ok ? i : -1;
            sites[2 * f + 1] = ok ? j : -1;
        }
    }
}

__global__ void k_make_pair_flips(int N, int B, int periodic, FlipPattern fp, const int8_t *__restrict__ spins,
                                  int32_t *__restrict__ sample, int32_t *__restrict__ sites) {
    const long long F = (long long)B * fp.nb * N;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < F; f += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(f % N), bo = (int)((f / N) % fp.nb);
        int jp = j + bond_of(fp, bo);
        bool ok = true;
        if (periodic) jp %= N;
        else if (jp >= N) ok = false;
        const long long b = f / ((long long)fp.nb * N);
        if (ok && fp.anti && spins[b * N + j] == spins[b * N + jp]) ok = false;
        sample[f] = (int32_t)b;
        sites[2 * f] = ok ? j : -1;
        sites[2 * f + 1] = ok ? jp : -1;
    }
}

cudaError_t launch_make_pair_flips(int N, int B, int periodic, int nb, const int *bonds, bool anti,
                                   const int8_t *spins, int32_t *sample, int32_t *sites, cudaStream_t st) {
    const FlipPattern fp{nb, 0, {bonds[0], nb > 1 ? bonds[1] : 0}, anti ? 1 : 0};
    {
        ProfScope _ps("k_make_flips", st);
        k_make_pair_flips<<<1024, 256, 0, st>>>(N, B, periodic, fp, spins, sample, sites);
    }
    return cudaGetLastError();
}

cudaError_t launch_make_flips(int kind, int N, int B, int periodic, const int8_t *spins, int32_t *sample,
                              int32_t *sites, cudaStream_t st) {
    {
        ProfScope _ps("k_make_flips", st);
        k_make_flips<<<1024, 256, 0, st>>>(kind, N, B, periodic, spins, sample, sites);
    }
    return cudaGetLastError();
}

// E_loc(b) = <sigma|H|sigma> + sum over connected sigma' of H_{sigma sigma'} exp(dlogpsi).
// coupling[r] = J r^-alpha / N_a (TFIM, r = 1..N-1).
__global__ void k_eloc_reduce(dn_hamiltonian H, int N, int B, const int8_t *__restrict__ spins,
                              const double *__restrict__ coupling, const double *__restrict__ dlogpsi,
                              double *__restrict__ eloc) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    const int8_t *sp = spins + (long long)b * N;
    double acc = 0.0;
    if (H.kind == 0) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            double row = 0.0;
            for (int j = i + 1; j < N; ++j) {
                int r = j - i;
                if (H.periodic && N - r < r) r = N - r;
                row += coupling[r] * sp[j];
            }
            acc += row * sp[i];
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) acc += H.h * exp(dlogpsi[(long long)b * N + i]);
    } else {
        for (int q = threadIdx.x; q < 2 * N; q += blockDim.x) {
            const int bond = q / N + 1, i = q % N;
            const double Jb = bond == 1 ? H.J1 : H.J2;
            int j = i + bond;
            if (H.periodic) j %= N;
            else if (j >= N) continue;
            acc += 0.25 * Jb * sp[i] * sp[j];
            if (sp[i] != sp[j]) acc += 0.5 * Jb * exp(dlogpsi[(long long)b * 2 * N + q]);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) s += red[q];
        eloc[b] = s;
    }
}

cudaError_t launch_eloc_reduce(const dn_hamiltonian &H, int N, int B, const int8_t *spins, const double *coupling,
                               const double *dlogpsi, double *eloc, cudaStream_t st) {
    {
        ProfScope _ps("k_eloc_reduce", st);
        k_eloc_reduce<<<B, 256, 0, st>>>(H, N, B, spins, coupling, dlogpsi, eloc);
    }
    return cudaGetLastError();
}

// ------------------------------------------------- full-recompute baseline --
__global__ void k_expand_flips(int N, const int8_t *__restrict__ spins, const int32_t *__restrict__ sample,
                               const int32_t *__restrict__ sites, int F, int B, int8_t *__restrict__ out,
                               unsigned *__restrict__ flag) {
    const long long f = blockIdx.x;
    if (f >= F) return;
    const int b = sample[f], j0 = sites[2 * f], j1 = sites[2 * f + 1];
    const bool bad = (b < 0 || b >= B) || (j0 < -1 || j0 >= N) || (j1 < -1 || j1 >= N) || (j0 == -1 && j1 != -1) ||
                     (j0 >= 0 && j0 == j1);
    if (bad && threadIdx.x == 0) atomicOr(flag, 2u);
    const int8_t *src = spins + (long long)(bad ? 0 : b) * N;
    int8_t *dst = out + f * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int8_t v = src[i];
        if (!bad && (i == j0 || i == j1)) v = (int8_t)(-v);
        dst[i] = v;
    }
}

cudaError_t launch_expand_flips(int N, const int8_t *spins, const int32_t *sample, const int32_t *sites, int F,
                                int B, int8_t *out, unsigned *flag, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    {
        ProfScope _ps("k_expand_flips", st);
        k_expand_flips<<<F, 128, 0, st>>>(N, spins, sample, sites, F, B, out, flag);
    }
    return cudaGetLastError();
}

__global__ void k_sub_base(const double *__restrict__ lp_flip, const double *__restrict__ lp_base,
                           const int32_t *__restrict__ sample, const int32_t *__restrict__ sites, int F, int B, int N,
                           double *__restrict__ out) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int b = sample[f], j0 = sites[2 * f], j1 = sites[2 * f + 1];
    const bool bad = (b < 0 || b >= B) || (j0 < -1 || j0 >= N) || (j1 < -1 || j1 >= N) || (j0 == -1 && j1 != -1) ||
                     (j0 >= 0 && j0 == j1);
    if (bad) {
        out[f] = nan("");
        return;
    }
    out[f] = j0 == -1 ? 0.0 : lp_flip[f] - lp_base[b];
}

cudaError_t launch_sub_base(const double *lp_flip, const double *lp_base, const int32_t *sample, const int32_t *sites,
                            int F, int B, int N, double *out, cudaStream_t st) {
    if (F <= 0) return cudaSuccess;
    {
        ProfScope _ps("k_sub_base", st);
        k_sub_base<<<(F + 255) / 256, 256, 0, st>>>(lp_flip, lp_base, sample, sites, F, B, N, out);
    }
    return cudaGetLastError();
}

}  // namespace dn
