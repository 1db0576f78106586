/*
 * dysonnet.h -- C ABI of the GB300 DysonNet / ABACUS local-estimator library.
 *
 * The library evaluates, for a batch of spin configurations sigma in {+1,-1}^N,
 * the DysonNet log-amplitude (Sec. "DysonNet", Eq. wavefunc), fills the per-
 * sample caches that ABACUS needs (link tensors T and L, Eqs. Tl and Lmn),
 * and computes log psi(sigma') - log psi(sigma) for local updates sigma' by
 * the slice-local recurrence of Alg. 1 (Eqs. recur_step and recur_out), whose
 * exactness is Theorem 1.  The local energy of Eq. local-estimator is built on
 * top of it for the long-range transverse-field Ising chain (Sec.
 * "Benchmarking") and the J1-J2 Heisenberg chain (Eq. j1j2_hamiltonian).
 *
 * Conventions shared by every call:
 *  - Pointers named *_dev are caller-owned CUDA device memory on the current
 *    device; *_host pointers are host memory.  Arrays are C-contiguous.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous: results are valid once the stream has
 *    reached them.  Host-side argument checks happen before anything is
 *    enqueued; a failing check returns DN_EINVAL and enqueues nothing.
 *  - Invalid data that only the device can see (a spin that is not +-1, a site
 *    out of range, a flip set wider than the cache allows) never causes an
 *    out-of-bounds access: the affected output is set to NaN and a sticky flag
 *    is raised, reported by dn_cache_check() (or by the next call on the cache).
 *  - dn_model and dn_cache are opaque and library-owned.  Device memory they
 *    hold comes from the allocator installed with dn_set_allocator() (default:
 *    cudaMallocAsync/cudaFreeAsync on the call's stream).  A failed allocation
 *    returns DN_ENOMEM and leaves no partial object behind.
 *  - A model may be used by one host thread at a time.
 *  - No C++ exception, abort() or exit() crosses this interface.
 */
#ifndef DYSONNET_H
#define DYSONNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DN_OK = 0,
    DN_EINVAL = 1,        /* bad argument (checked on the host) or bad device data (sticky flag) */
    DN_ENOMEM = 2,        /* the allocator refused a request */
    DN_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    DN_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    DN_EUNSUPPORTED = 5   /* valid request the library does not implement */
} dn_status;

/* Arithmetic of the network and of the caches.  Every precision generates the
 * S4 kernel taps in FP64 and accumulates the pooled readout and the final
 * log cosh difference in FP64.
 *   DN_FP64: everything in double.
 *   DN_FP32: activations, caches and link contractions in float.  The forward
 *     pass runs on FP32 FMA kernels; the Toeplitz hops of the link construction
 *     run on the tcgen05 tensor cores as three BF16 products
 *     (hi*hi + hi*lo + lo*hi) with FP32 accumulation.
 *   DN_BF16: the S4 convolutions and the channel-mixing GEMMs of the forward pass
 *     on the tensor cores in BF16 arithmetic, each operand carried as two BF16
 *     terms (hi*hi + hi*lo + lo*hi, FP32 accumulation); the link tensors are built
 *     as for DN_FP32; caches, the adjoint and the ABACUS contractions stay in
 *     float.  Requires d a multiple of 16, d <= 128 (else DN_EUNSUPPORTED).  Its
 *     error against the FP64 definition is larger than DN_FP32's; the tests state
 *     the bound. */
typedef enum {
    DN_FP64 = 0,
    DN_FP32 = 1,
    DN_BF16 = 2
} dn_precision;

/* N-agnostic hyper-parameters (Sec. "Implementation of DysonNet", App.
 * "Details on the implementation of the DysonNet block"):
 *   L layers of h' = D(sigma) G h with d channels; diagonal S4 kernels with s
 *   complex modes per channel; window half-width w (W = 2w+1) of the local
 *   vertex; d_h hidden units of the per-site MLP; d_out readout units.
 *   periodic = 1: ring (circulant kernels, wrapped windows); 0: open chain.
 *   f_kind = 0: log psi = sum_k log cosh Omega_k (Eq. wavefunc);
 *   f_kind = 1: log psi = sum_k Omega_k (the Jastrow limit of App. power-law). */
typedef struct {
    int L, d, s, w, d_h, d_out;
    int periodic;
    int f_kind;
} dn_model_desc;

/* Hamiltonian for local_energy().
 *   kind 0, long-range TFIM:  H = (J/N_a) sum_{i<j} r_ij^-alpha sz_i sz_j + h sum_i sx_i
 *           r_ij = |i-j| (open) or min(|i-j|, N-|i-j|) (periodic);
 *           N_a = 1, or the Kac factor 2 sum_{r=1}^{N/2} r^-alpha when kac = 1.
 *           (The paper's form -J'/N_a sum_{i!=j} ... - h' sum sx is J = -2J', h = -h'.)
 *   kind 1, J1-J2 chain: H = J1 sum_i S_i.S_{i+1} + J2 sum_i S_i.S_{i+2}, S = sigma/2,
 *           sums over i = 0..N-1 with wrap-around when periodic = 1, else up to N-1-b.
 *           Requires N >= 3. */
typedef struct {
    int kind;
    double J, alpha, h;
    double J1, J2;
    int periodic, kac;
} dn_hamiltonian;

typedef struct dn_model dn_model;
typedef struct dn_cache dn_cache;

/* Allocator hook.  alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, bytes, stream, ctx) releases it.  Passing NULL for both restores
 * the default.  Applies to allocations made after the call. */
typedef void *(*dn_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*dn_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
dn_status dn_set_allocator(dn_alloc_fn alloc, dn_free_fn free_fn, void *ctx);

/* Human-readable name of a status. */
const char *dn_status_string(dn_status s);

/* Create a model from the flat FP64 parameter vector params_host[n_params].
 * Layout (W = 2w+1; matrices row-major, output index first):
 *   S4 block (8 d s + d values): lam_re[d][s] lam_im[d][s] (continuous-time
 *     diagonal state matrix, Re < 0), log_dt[d], b_re[d][s] b_im[d][s],
 *     cf_re[d][s] cf_im[d][s] (forward output), cb_re[d][s] cb_im[d][s]
 *     (backward output);
 *   for l = 1..L: S4 block | kappa[W][d_h] (window weight at offset r is row
 *     r+w) | beta[d_h] | W1[d_h][d_h] | b1[d_h] | W2[d][d_h] | b2[d] | U[d][d] | V[d][d];
 *   then: readout S4 block (G^f) | A[d][d_out] | e[d].
 * The parameters are copied; the caller keeps ownership of params_host.
 * DN_EINVAL if a size is non-positive, w < 0, n_params does not match the
 * layout, or d > 128, d_h > 128, d_out > 8, s > 256, L > 12. */
dn_status dn_model_create(const dn_model_desc *desc, const double *params_host, size_t n_params,
                          dn_model **model_out);
void dn_model_destroy(dn_model *model);

/* Device bytes a cache for (N, batch, precision, max_cluster) will hold; 0 on
 * bad arguments.  Used to admit work against a memory budget. */
size_t dn_cache_bytes(const dn_model *model, int N, int batch, dn_precision prec, int max_cluster);

/* One full DysonNet forward pass over B configurations and the construction
 * of the ABACUS caches (Eqs. wavefunc, Tl, Lmn; App. "Efficient construction
 * of link tensors"):
 *   spins_dev [B][N] int8, each +1 or -1;
 *   max_cluster in {1, 2, 3}: the flip sets the cache must serve -- single
 *     sites (1), pairs at separation 1 (2) or separations 1 and 2 (3); the
 *     slice width is W_F = 2w + max_cluster;
 *   logpsi_dev [B] float64 (may be NULL): log psi(sigma).
 * On DN_OK *cache_out owns the caches; destroy with dn_cache_destroy().
 * Errors: DN_EINVAL (N < 1, B < 1, null pointers, max_cluster out of range,
 * periodic with N < 2 W_F - 1), DN_ENOMEM, DN_ECUDA. */
dn_status dysonnet_forward_cache(dn_model *model, int N, const int8_t *spins_dev, int B,
                                 dn_precision prec, int max_cluster, void *stream,
                                 dn_cache **cache_out, double *logpsi_dev);

/* ABACUS (Alg. 1; Eqs. recur_step, recur_out; Theorem 1): for F flip sets
 *   sample_dev [F] int32: index of the cached configuration (0 <= b < B);
 *   sites_dev [F][2] int32: flipped sites; sites[f][1] = -1 for a single flip;
 *     a pair must be distinct and at ring/chain separation <= max_cluster - 1;
 *     sites[f][0] = -1 marks an empty entry (output 0);
 *   dlogpsi_dev [F] float64: log psi(sigma') - log psi(sigma).
 * Cost per flip is independent of N.  Entries with invalid sites get NaN and
 * raise the cache's sticky flag.  Errors: DN_EINVAL, DN_ECUDA. */
dn_status abacus_flip_ratios(const dn_cache *cache, const int32_t *sample_dev, const int32_t *sites_dev,
                             int F, double *dlogpsi_dev, void *stream);

/* ABACUS for every single flip of every cached configuration (the connected
 * configurations of a transverse field, Sec. "Benchmarking"):
 *   dlogpsi_dev [B][N] float64: entry (b, j) = log psi(sigma_b with site j
 *   flipped) - log psi(sigma_b).
 * Same results as abacus_flip_ratios() on the list of all single flips; the
 * flips of a configuration are processed in groups of consecutive sites so that
 * each link block is read from memory once per group.
 * Errors: DN_EINVAL, DN_ECUDA. */
dn_status abacus_single_flip_ratios(const dn_cache *cache, double *dlogpsi_dev, void *stream);

/* ABACUS for the pair flips {j, j + delta} of every site j of every cached
 * configuration, for n_bonds (1 or 2) distinct separations (the connected
 * configurations of a J1-J2 chain are the antialigned pairs at delta = 1, 2;
 * Sec. "ABACUS", cluster flips):
 *   bonds [n_bonds] int32, HOST memory: the separations delta,
 *     1 <= delta <= max_cluster - 1 of the cache;
 *   dlogpsi_dev [B][n_bonds][N] float64: entry (b, k, j) = log psi(sigma_b with
 *     sites j and j + bonds[k] flipped) - log psi(sigma_b); on a ring j + delta
 *     wraps, on an open chain a pair past the end gives 0.
 * Same results as abacus_flip_ratios() on the list of these pairs; the pairs of a
 * configuration are processed by site, both separations together, so that each
 * link block is read from memory once per site and layer pair.
 * Errors: DN_EINVAL (null pointers, n_bonds not 1 or 2, a separation out of
 * range, equal separations), DN_ECUDA. */
dn_status abacus_pair_flip_ratios(const dn_cache *cache, int n_bonds, const int32_t *bonds, double *dlogpsi_dev,
                                  void *stream);

/* Local energy E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma')/psi(sigma)
 * (Eq. local-estimator) for B configurations, every ratio by ABACUS:
 *   eloc_dev [B] float64.  Builds and frees its own caches (in chunks of
 *   samples bounded by an internal memory budget).
 * Errors: DN_EINVAL, DN_ENOMEM, DN_ECUDA. */
dn_status local_energy(dn_model *model, const dn_hamiltonian *ham, int N, const int8_t *spins_dev, int B,
                       dn_precision prec, void *stream, double *eloc_dev);

/* Full-forward baseline: log psi for B configurations, recomputing the whole
 * network (Eq. wavefunc).  logpsi_dev [B] float64; Omega_dev [B][d_out]
 * float64 (may be NULL). */
dn_status dn_full_forward(dn_model *model, int N, const int8_t *spins_dev, int B, dn_precision prec,
                          void *stream, double *logpsi_dev, double *Omega_dev);

/* The computation ABACUS replaces (Sec. "ABACUS", discussion of runtime):
 * log psi(sigma') - log psi(sigma) for each flip set by building every
 * flipped configuration on the device and recomputing the whole network.
 * Same flip-set format as abacus_flip_ratios(); spins_dev [B][N]. */
dn_status dn_recompute_flip_ratios(dn_model *model, int N, const int8_t *spins_dev, int B,
                                   const int32_t *sample_dev, const int32_t *sites_dev, int F,
                                   dn_precision prec, void *stream, double *dlogpsi_dev);

/* dn_full_forward() for callers that cannot allocate device memory during
 * the call -- for example a host whose device memory is reserved up front by
 * another runtime, or a server that forbids allocation after warm-up to keep
 * its footprint fixed.  The paper has no counterpart; it is a deployment
 * variant of the full forward pass.
 * Same arguments and results as dn_full_forward().  Every temporary (packed
 * weights, kernel taps, activations, pooled sums) lives in one fixed 16 MiB
 * device array that each device loading the library holds until the process
 * exits; no cudaMalloc, cudaFree or allocator call is made.  A call needs
 * about B*N*d*(L+2)*t + B*(L+1)*d*8 bytes plus the weights and kernel taps
 * (t = 8 for DN_FP64, 4 for DN_FP32); a request that does not fit returns
 * DN_EINVAL and does nothing.  Every call looks up the array's device address
 * in the current context (cudaGetSymbolAddress, a host-side query; the first one
 * on a device loads the library's device code, so make it before any stream
 * capture).  All calls share the array and nothing in it needs clearing, but
 * calls that overlap on the GPU (other streams or threads) race on it. */
dn_status dn_full_forward_noalloc(const dn_model *model, int N, const int8_t *spins_dev, int B, dn_precision prec,
                                  void *stream, double *logpsi_dev, double *Omega_dev);

/* Length of the parameter vector of a model (n_params of dn_model_create); 0 for NULL. */
size_t dn_model_nparams(const dn_model *model);

/* Per-configuration log-derivatives of the wave function with respect to every
 * parameter, O[b][k] = d log psi(sigma_b) / d theta_k (the variational
 * derivatives of the energy gradient and of stochastic reconfiguration, Sec.
 * "Variational Monte Carlo"; Eq. wavefunc differentiated through every layer,
 * the S4 kernels through their discretisation, App. "Details on the
 * implementation of the DysonNet block"):
 *   spins_dev [B][N] int8, each +1 or -1;
 *   prec DN_FP64 or DN_FP32 (DN_BF16: DN_EUNSUPPORTED);
 *   logpsi_dev [B] float64 (may be NULL);
 *   O_dev [B][n_params] (may be NULL): float64 for DN_FP64, float32 for DN_FP32,
 *     k in the layout of the parameter vector given to dn_model_create();
 *   w_dev [B] float64 and vjp_dev [n_params] float64, both NULL or both set:
 *     vjp = sum_b w_b O[b] (the vector-Jacobian product of a backward pass;
 *     computed without O_dev when O_dev is NULL).
 * At least one output must be given.  Samples are processed in chunks bounded
 * by an internal memory budget.  The call synchronises `stream` at its end.
 * Errors: DN_EINVAL (bad arguments, spins not +-1), DN_EUNSUPPORTED, DN_ENOMEM, DN_ECUDA. */
dn_status dn_logpsi_grad(dn_model *model, int N, const int8_t *spins_dev, int B, dn_precision prec, void *stream,
                         double *logpsi_dev, void *O_dev, const double *w_dev, double *vjp_dev);

/* Stochastic-reconfiguration matrices (Sec. "Variational Monte Carlo") from the
 * log-derivatives O_dev [B][n_params] of dn_logpsi_grad() (float64 for DN_FP64,
 * float32 for DN_FP32), centred over the samples, Oc = O - mean_b O:
 *   gram_dev [B][B] float64 (may be NULL): Oc Oc^T / B, the sample-space form whose
 *     size does not grow with the parameter count;
 *   s_dev [nk][nk] float64 (may be NULL): Oc[:, k0:k0+nk]^T Oc[:, k0:k0+nk] / B, the
 *     parameter-space matrix of a contiguous block of parameters.
 * float64 O: FMA products accumulated in float64.  float32 O: the Gram matrix runs on
 * the tensor cores with every value split into three BF16 terms (6 products, about
 * float32 accuracy), accumulated in float32 over K splits of at most 16384 parameters,
 * the splits summed in float64; the parameter block s_dev accumulates FMA products in
 * float32 in partial sums of 512 terms added into a second float32 sum.
 * Errors: DN_EINVAL, DN_ENOMEM, DN_ECUDA. */
dn_status dn_sr_matrices(const void *O_dev, int B, size_t n_params, dn_precision prec, void *stream, double *gram_dev,
                         size_t k0, int nk, double *s_dev);

/* Counters of dn_sampler_batch(): proposals decided, proposals accepted, and proposals
 * that fell into the ambiguous window (each decided exactly and followed by a cache
 * refresh of its chain). */
typedef struct {
    unsigned long long proposals, accepted, refreshes;
} dn_sampler_stats;

/* One batch of the screened typewriter sampler (Alg. 2, Sec. "Screened typewriter
 * sampler"; screened acceptance, App. "Screened Metropolis sampler is exact") on C
 * Markov chains:
 *   spins_dev [C][N] int8 (+-1), updated in place;
 *   sites_dev [C][K] int32: single-site proposals of each chain, decided in order
 *     (-1 = no proposal).  The proposals of a batch are evaluated against the caches of
 *     the configuration the batch starts from (independent scattering approximation), so
 *     they should be spaced by at least the window (the typewriter schedule: one site in
 *     every other block of width s >= w);
 *   u_dev [C][K] float64: the uniforms of the Metropolis tests;
 *   eps >= 0: half-width of the ambiguous window.  A proposal with |u - min(1, R~)| <= eps
 *     (R~ the ratio from the scattering approximation) is decided with the exact ratio
 *     from two full forward passes, and its chain's caches are rebuilt from the new
 *     configuration before the chain continues.  Decisions equal exact Metropolis
 *     decisions whenever |min(1, R~) - min(1, R)| <= eps for every proposal;
 *   accepted_dev [C][K] int8 (may be NULL): 1 where the proposal was accepted;
 *   stats (may be NULL): counters of the call.
 * prec DN_FP64 or DN_FP32.  The call synchronises `stream`.
 * Errors: DN_EINVAL (bad arguments, spins not +-1), DN_EUNSUPPORTED (DN_BF16), DN_ENOMEM,
 * DN_ECUDA. */
dn_status dn_sampler_batch(dn_model *model, int N, int8_t *spins_dev, int C, const int32_t *sites_dev,
                           const double *u_dev, int K, double eps, dn_precision prec, void *stream,
                           int8_t *accepted_dev, dn_sampler_stats *stats);

/* Wait for `stream`, then report the cache's sticky device flag:
 * DN_OK, DN_EINVAL (invalid spins or flip sites were seen), DN_ECUDA. */
dn_status dn_cache_check(const dn_cache *cache, void *stream);

/* Read-only view of one cache array (device pointer owned by the cache):
 * name is one of "spins" (int8 [B][N]), "chi" and "y" ([B][L][N][d]),
 * "rho" ([B][L][d_out][N][d]: output links, Eq. Tl with A folded in),
 * "t" ([B][N][d_out]), "ell" ([B][L-1][N][2Rl+1][d]: response at layer l of
 * the embedding at site i+o-Rl, Rl = W_F-1-w), "K" ([B][P][N][2Rk+1][d][d]:
 * links L^(l,m) of Eq. Lmn on the band |i-k| <= Rk = W_F-1, stored
 * [i][o][c_out][c_in] with k = i+o-Rk, pairs ordered (l,m) = (3,1), (4,1),
 * (4,2), ...), "Omega" (f64 [B][d_out]) or "logpsi" (f64 [B]).  Elements are
 * float64 for DN_FP64 caches and float32 for DN_FP32 caches.  Band entries
 * whose partner site lies off an open chain are unspecified.
 * DN_EINVAL for an unknown name. */
dn_status dn_cache_tensor(const dn_cache *cache, const char *name, void **dev_ptr, size_t *count, int *elem_bytes);

/* Shape of a cache: N, B, precision, max_cluster (any pointer may be NULL). */
dn_status dn_cache_info(const dn_cache *cache, int *N, int *B, int *prec, int *max_cluster);

/* Tracing.  dn_launch_count(): kernels launched by the library since load.
 * dn_profile_enable(1) starts recording a pair of CUDA events around every
 * kernel launch (on its stream), grouped by kernel name; dn_profile_enable(0)
 * stops.  dn_profile_count() is the number of kernel names seen;
 * dn_profile_get(i, ...) synchronises the device and returns name i, its
 * launches and total device milliseconds since tracing was last enabled. */
long long dn_launch_count(void);
dn_status dn_profile_enable(int on);
int dn_profile_count(void);
dn_status dn_profile_get(int i, char *name, size_t name_len, long long *launches, double *total_ms);

/* Choice between two exact implementations of the end of a link-propagation chain
 * (App. "Exact algorithm to construct link tensors", Eqs. X_def, L_def): on (1, the
 * default) the last vertex hop D0^(L-1) and the band of G^(L) run as one fused kernel
 * where it supports the shape (FP32 caches, d = 32, band half-width Rk <= 4); off (0)
 * they run as two kernels with the hop output in device memory.  Both give the same
 * link tensors.  Process-wide; affects caches built after the call.  Always DN_OK. */
dn_status dn_set_fused_links(int on);

/* Choice between two exact constructions of the band links of a pair with one
 * intermediate layer, L^(m+2,m) (App. "Efficient construction of link tensors": the
 * two-layer link by FFT): as circular correlations by FFT of length M = the power of
 * two >= 2N - 1 (open chain) or N (ring, N a power of two), O((2R+1) d^2 M log M) per
 * configuration, or as the direct band sum, (2R+1) N^2 d^2 multiply-adds.  mode 1 (the
 * default): FFT where the direct sum has no fast kernel or N >= 512; 2: FFT wherever
 * the shape allows; 0: never.  The two agree to rounding.  Process-wide; affects caches
 * built after the call.  DN_EINVAL for another mode. */
dn_status dn_set_fft_links(int mode);

/* The S4 convolution of the forward pass (Eq. resolvent, Sec. "Implementation of
 * DysonNet"): directly as a Toeplitz / circulant sum, O(N^2 d) per layer, or through
 * DFTs of length M (the power of two >= 2N - 1 on an open chain; M = N on a ring whose N
 * is a power of two), O(N log N d), with the tap spectra built once per (model, N).
 * mode 1 (default): FFT for FP32 with N >= 512; 2: FFT wherever it applies (FP64 too);
 * 0: never.  The two agree to rounding.  Process-wide; applies to forward passes (caches,
 * full forward, recompute) launched after the call.  DN_EINVAL for another mode. */
dn_status dn_set_fft_conv(int mode);

/* Release a cache (stream-ordered on the stream of the call that built it). */
void dn_cache_destroy(dn_cache *cache);

/* ------------------------------------------------------------- serving --
 * Continuous-batching request loop over resident caches: the way ABACUS is
 * used inside Markov-chain Monte Carlo, where each chain proposes flips and
 * needs their log-amplitude ratios (Sec. "ABACUS"; the batching and masking of
 * App. "Implementation" for many chains).  A server owns a library worker
 * thread and two CUDA streams.  Chains (one configuration of N sites each, any
 * N) are registered with dn_server_set_chain; a request carries F single-site
 * proposals for one chain and receives F ratios log psi(s') - log psi(s) in
 * FP64.  Requests that arrive while earlier batches run join the next batch;
 * one kernel serves all requests of a batch, whatever their chains.  A chain
 * without a resident cache gets one built when it is first admitted (or at
 * dn_server_set_chain with build_now); when the caches would exceed the
 * device-memory budget, the least recently used idle ones are dropped.
 * DN_SERVE_RECOMPUTE serves the same requests by a full forward pass of every
 * proposal (the baseline).  DN_SERVE_PERSISTENT serves them with one resident
 * kernel (one or two CTAs per SM) instead of a launch per batch: admitted
 * proposals are appended to a work queue in host-mapped memory and published by
 * a counter; the items are dealt to the kernel's CTAs in turn, each serves its
 * items as they appear and returns each ratio through mapped memory, so requests
 * that arrive while others run are served with no launch in between.  When the
 * counter has not moved for an idle limit (dn_server_set_idle_limit, default
 * 0.2 s) the kernel leaves with DN_ETIMEOUT (dn_server_kernel_status); the worker
 * launches it again when work arrives and stops it while a new chain's cache is
 * built.  While a server exists, its model
 * must not be used by other calls.  Results of a request do not depend on which
 * other requests share its batch. */
typedef struct dn_server dn_server;
typedef enum { DN_SERVE_ABACUS = 0, DN_SERVE_RECOMPUTE = 1, DN_SERVE_PERSISTENT = 2 } dn_serve_mode;
typedef struct {
    unsigned long long requests, flips, batches, cache_builds, evictions;
    size_t resident_bytes; /* device bytes of the resident caches */
} dn_server_stats;

/* hbm_budget_bytes bounds the resident caches; a batch holds at most
 * max_batch_flips proposals and max_batch_chains chains (a request larger than
 * max_batch_flips is rejected by dn_server_submit).  DN_EINVAL, DN_ENOMEM. */
dn_status dn_server_create(dn_model *model, dn_precision prec, int mode, size_t hbm_budget_bytes, int max_batch_flips,
                           int max_batch_chains, dn_server **server_out);

/* Register chain `chain` (>= 0) with configuration spins_host[N] (+1/-1, copied),
 * replacing an earlier one (and its cache).  build_now != 0 builds its cache in
 * this call (ABACUS and persistent modes).  DN_EINVAL while requests of the chain are pending or
 * in flight, or for spins other than +1/-1. */
dn_status dn_server_set_chain(dn_server *server, int chain, int N, const int8_t *spins_host, int build_now);

/* Queue F proposals for `chain`: sites_host[F][2] (site, -1) is copied; the F
 * ratios are written to out_host[F], which must stay valid until the request
 * completes.  *ticket identifies the request.  Returns at once. */
dn_status dn_server_submit(dn_server *server, int chain, const int32_t *sites_host, int F, double *out_host,
                           unsigned long long *ticket);

/* Wait until request `ticket` completes (timeout_s < 0: no limit) and release
 * it; *latency_s (may be NULL) is the host time from submission to the result in
 * out_host.  Returns the request's status (DN_ETIMEOUT leaves it pending). */
dn_status dn_server_wait(dn_server *server, unsigned long long ticket, double timeout_s, double *latency_s);

dn_status dn_server_get_stats(dn_server *server, dn_server_stats *out);

/* DN_SERVE_PERSISTENT: how long (seconds, > 0) the kernel waits for work before it
 * leaves; applies to launches after the call.  DN_EINVAL for other modes. */
dn_status dn_server_set_idle_limit(dn_server *server, double seconds);

/* DN_SERVE_PERSISTENT: wait up to wait_s seconds for the resident kernel to have
 * left; *running (may be NULL) = 1 if it is still running.  Returns DN_OK while it
 * runs or after the worker stopped it, DN_ETIMEOUT when its last exit was the idle
 * limit running out with the queue unfed.  DN_EINVAL for other modes. */
dn_status dn_server_kernel_status(dn_server *server, double wait_s, int *running);

/* Finish every queued request, stop the worker and release the caches. */
void dn_server_destroy(dn_server *server);

#ifdef __cplusplus
}
#endif
#endif /* DYSONNET_H */
