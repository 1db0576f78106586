// Screened typewriter sampler (Sec. "Screened typewriter sampler", Alg. 2): device kernels.
//
// A batch of K single-site proposals per chain is evaluated against the caches of a
// reference configuration sigma0: ABACUS gives each proposal's update vector dOmega_k
// (the latent change of the flip alone, independent scattering approximation).  The
// proposals are then decided in order per chain (k_screened_sweep): with the current
// latents Omega (Omega(sigma0) plus the update vectors of the accepted proposals),
//   R~ = |f(Omega + dOmega_k) / f(Omega)|^2,  P~ = min(1, R~),
// accept if u_k < P~ - unless |u_k - P~| <= eps, the ambiguous window, where the chain
// stops and the host decides the proposal exactly (full forward passes of the current
// configuration and of the proposal, k_exact_decide) and refreshes the chain's caches.
// With log psi = sum_k log cosh Omega_k, |f(Omega')/f(Omega)|^2 = exp(2 sum_k [log cosh
// Omega'_k - log cosh Omega_k]).
#include <math.h>

#include "dn_internal.cuh"

namespace dn {

namespace {

__device__ __forceinline__ double log_cosh_s(double x) {
    const double a = fabs(x);
    return a + log1p(exp(-2.0 * a)) - 0.69314718055994530942;
}

}  // namespace

// Flip list for ABACUS: entry (c, k) = flip of sites[c][k] on configuration row[c], or an
// empty entry when the site is -1 or k < kfrom[row[c]] (kfrom may be null: every k).
__global__ void k_flip_list(int C, int K, const int32_t *__restrict__ sites, const int32_t *__restrict__ row,
                            const int32_t *__restrict__ kfrom, int32_t *__restrict__ sample,
                            int32_t *__restrict__ fsites) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)C * K) return;
    const int c = (int)(x / K), k = (int)(x % K);
    const int src = row ? row[c] : c;
    const bool on = !kfrom || k >= kfrom[src];
    sample[x] = c;
    fsites[2 * x] = on ? sites[(long long)src * K + k] : -1;
    fsites[2 * x + 1] = -1;
}

// One thread per chain: decide proposals kpos[c] .. K-1 in order (see the file comment).
// amb[c] = index of the proposal that fell into the ambiguous window, or -1 when the batch
// is done.  Counters: [0] proposals decided here, [1] accepted here, [2] ambiguous.
__global__ void k_screened_sweep(int N, int C, int K, int dout, int f_kind, double eps,
                                 const int32_t *__restrict__ sites, const double *__restrict__ u,
                                 const double *__restrict__ dOm, double *__restrict__ Om, int32_t *__restrict__ kpos,
                                 int8_t *__restrict__ spins, int8_t *__restrict__ acc, int32_t *__restrict__ amb,
                                 unsigned long long *__restrict__ counters) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int k = kpos[c];
    amb[c] = -1;
    if (k >= K) return;
    double om[kMaxDout];
    for (int j = 0; j < dout; ++j) om[j] = Om[(long long)c * dout + j];
    unsigned long long nprop = 0, nacc = 0;
    for (; k < K; ++k) {
        const int site = sites[(long long)c * K + k];
        if (site < 0 || site >= N) {
            if (acc) acc[(long long)c * K + k] = 0;
            continue;
        }
        const double *dk = dOm + ((long long)c * K + k) * dout;
        double dl = 0.0;
        for (int j = 0; j < dout; ++j) dl += f_kind == 0 ? log_cosh_s(om[j] + dk[j]) - log_cosh_s(om[j]) : dk[j];
        const double p = fmin(1.0, exp(2.0 * dl));
        const double uk = u[(long long)c * K + k];
        if (fabs(uk - p) <= eps) {
            amb[c] = k;
            atomicAdd(counters + 2, 1ull);
            break;
        }
        ++nprop;
        const bool a = uk < p;
        if (acc) acc[(long long)c * K + k] = a ? 1 : 0;
        if (a) {
            ++nacc;
            spins[(long long)c * N + site] = (int8_t)(-spins[(long long)c * N + site]);
            for (int j = 0; j < dout; ++j) om[j] += dk[j];
        }
    }
    for (int j = 0; j < dout; ++j) Om[(long long)c * dout + j] = om[j];
    kpos[c] = k;
    if (nprop) atomicAdd(counters, nprop);
    if (nacc) atomicAdd(counters + 1, nacc);
}

// For the n ambiguous chains list[a] (proposal amb[list[a]]): cfg[2a] = current
// configuration, cfg[2a+1] = the same with the proposal's site flipped.
__global__ void k_pair_configs(int N, int K, int n, const int32_t *__restrict__ list, const int32_t *__restrict__ amb,
                               const int32_t *__restrict__ sites, const int8_t *__restrict__ spins,
                               int8_t *__restrict__ cfg) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)n * N) return;
    const int a = (int)(x / N), i = (int)(x % N);
    const int c = list[a];
    const int site = sites[(long long)c * K + amb[c]];
    const int8_t s = spins[(long long)c * N + i];
    cfg[(2LL * a) * N + i] = s;
    cfg[(2LL * a + 1) * N + i] = i == site ? (int8_t)(-s) : s;
}

// Exact Metropolis decision of each ambiguous proposal: accept iff u < min(1, |psi'/psi|^2).
// Then the chain resumes after the proposal (kpos) once its caches are refreshed.
__global__ void k_exact_decide(int N, int K, int n, const int32_t *__restrict__ list, const int32_t *__restrict__ amb,
                               const int32_t *__restrict__ sites, const double *__restrict__ u,
                               const double *__restrict__ lp, int8_t *__restrict__ spins, int8_t *__restrict__ acc,
                               int32_t *__restrict__ kpos, unsigned long long *__restrict__ counters) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int c = list[a], k = amb[c];
    const int site = sites[(long long)c * K + k];
    const double p = fmin(1.0, exp(2.0 * (lp[2 * a + 1] - lp[2 * a])));
    const bool take = u[(long long)c * K + k] < p;
    if (take) spins[(long long)c * N + site] = (int8_t)(-spins[(long long)c * N + site]);
    if (acc) acc[(long long)c * K + k] = take ? 1 : 0;
    kpos[c] = k + 1;
    atomicAdd(counters, 1ull);
    if (take) atomicAdd(counters + 1, 1ull);
}

// Refreshed chains: spins of list[a] gathered into rows a; after the caches are rebuilt,
// their latents and the update vectors of the remaining proposals are scattered back.
__global__ void k_gather_rows(int N, int n, const int32_t *__restrict__ list, const int8_t *__restrict__ spins,
                              int8_t *__restrict__ dst) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)n * N) return;
    const int a = (int)(x / N), i = (int)(x % N);
    dst[x] = spins[(long long)list[a] * N + i];
}

__global__ void k_scatter_refresh(int K, int dout, int n, const int32_t *__restrict__ list,
                                  const int32_t *__restrict__ kpos, const double *__restrict__ Om_new,
                                  const double *__restrict__ dOm_new, double *__restrict__ Om,
                                  double *__restrict__ dOm) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)n * K) return;
    const int a = (int)(x / K), k = (int)(x % K);
    const int c = list[a];
    if (k >= kpos[c])
        for (int j = 0; j < dout; ++j) dOm[((long long)c * K + k) * dout + j] = dOm_new[x * dout + j];
    if (k == 0)
        for (int j = 0; j < dout; ++j) Om[(long long)c * dout + j] = Om_new[(long long)a * dout + j];
}

// ------------------------------------------------------------------ host --
static unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_flip_list(int C, int K, const int32_t *sites, const int32_t *row, const int32_t *kfrom,
                             int32_t *sample, int32_t *fsites, cudaStream_t st) {
    ProfScope _ps("k_flip_list", st);
    k_flip_list<<<blocks_for((long long)C * K, 256), 256, 0, st>>>(C, K, sites, row, kfrom, sample, fsites);
    return cudaGetLastError();
}

cudaError_t launch_screened_sweep(int N, int C, int K, int dout, int f_kind, double eps, const int32_t *sites,
                                  const double *u, const double *dOm, double *Om, int32_t *kpos, int8_t *spins,
                                  int8_t *acc, int32_t *amb, unsigned long long *counters, cudaStream_t st) {
    ProfScope _ps("k_screened_sweep", st);
    k_screened_sweep<<<blocks_for(C, 128), 128, 0, st>>>(N, C, K, dout, f_kind, eps, sites, u, dOm, Om, kpos, spins,
                                                         acc, amb, counters);
    return cudaGetLastError();
}

cudaError_t launch_pair_configs(int N, int K, int n, const int32_t *list, const int32_t *amb, const int32_t *sites,
                                const int8_t *spins, int8_t *cfg, cudaStream_t st) {
    ProfScope _ps("k_pair_configs", st);
    k_pair_configs<<<blocks_for((long long)n * N, 256), 256, 0, st>>>(N, K, n, list, amb, sites, spins, cfg);
    return cudaGetLastError();
}

cudaError_t launch_exact_decide(int N, int K, int n, const int32_t *list, const int32_t *amb, const int32_t *sites,
                                const double *u, const double *lp, int8_t *spins, int8_t *acc, int32_t *kpos,
                                unsigned long long *counters, cudaStream_t st) {
    ProfScope _ps("k_exact_decide", st);
    k_exact_decide<<<blocks_for(n, 128), 128, 0, st>>>(N, K, n, list, amb, sites, u, lp, spins, acc, kpos, counters);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(int N, int n, const int32_t *list, const int8_t *spins, int8_t *dst, cudaStream_t st) {
    ProfScope _ps("k_gather_rows", st);
    k_gather_rows<<<blocks_for((long long)n * N, 256), 256, 0, st>>>(N, n, list, spins, dst);
    return cudaGetLastError();
}

cudaError_t launch_scatter_refresh(int K, int dout, int n, const int32_t *list, const int32_t *kpos,
                                   const double *Om_new, const double *dOm_new, double *Om, double *dOm,
                                   cudaStream_t st) {
    ProfScope _ps("k_scatter_refresh", st);
    k_scatter_refresh<<<blocks_for((long long)n * K, 256), 256, 0, st>>>(K, dout, n, list, kpos, Om_new, dOm_new, Om,
                                                                         dOm);
    return cudaGetLastError();
}

}  // namespace dn
