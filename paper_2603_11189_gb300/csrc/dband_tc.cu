// Last vertex hop of a link-propagation chain fused with the last layer's band
// convolution, on the tcgen05 tensor cores (FP32 path, d = 32 channels, source
// columns p = k d + c' of interlayer sources).
//
// A chain from source layer m ends, for the pair (L, m) of Eq. Lmn, with
//   Z[c][n][p]                  = sum_a D0^(L-1)_n[c][a] Y[a][n][p]       (vertex hop)
//   band[k+dl][R-dl][c][c']     = sum_n g^(L)_{k+dl-n,c} Z[c][n][k d + c']   (G^(L) on the band)
// where Y = G^(L-1) X_{m+1,L-2} (e_c' delta_k) is the previous Toeplitz hop (App. "Exact
// algorithm to construct link tensors", Eqs. X_def, L_def).  Run as two kernels, Z is
// written to HBM and read back; here it never leaves the chip.
//
// One CTA per (configuration, tile of 128 source columns = 4 source sites), looping
// over all N sites n:
//   - Y[:, n, tile] (32 x 128 floats) and D0_n (32 x 32) arrive by cp.async in a
//     four-stage ring, so that the HBM reads of later sites are in flight;
//   - both are split into three BF16 planes (v = p0 + p1 + p2 + rest) and one elected
//     thread issues the six plane products with pa + pb <= 2 (M = 128 columns,
//     N = 32 output channels, K = 32 input channels, FP32 accumulation in tensor
//     memory), the same products and order as the separate vertex-hop kernel;
//   - each warp announces its staged planes on an mbarrier; only the MMA-issuing thread
//     waits for all sixteen, the others go on to the band sums;
//   - while the MMAs of site n run, every thread adds site n-1 into its band sums:
//     warp w owns TMEM lanes 32 (w & 3) .. + 31 (one source site, lane = source channel
//     c') and output channels 8 (w >> 2) .. + 7, with the 2R+1 band offsets held in
//     registers (taps from a shared table, already wrapped for rings).  The band sums
//     are formed in the same order (site n ascending, fmaf(tap, z, acc)) as the separate
//     band kernel, so the fused result equals the two-kernel one.
// Every mbarrier wait is bounded; a wait that gives up raises bit 8 of the cache flag,
// the CTA drains its own copies, frees its tensor memory and writes nothing.
#include "dn_internal.cuh"
#include "tc_common.cuh"

namespace dn {

namespace {

constexpr int kDbD = 32;                             // channels
constexpr int kDbCols = 128;                         // source columns per CTA
constexpr int kDbStages = 4;                         // depth of the input ring
constexpr int kDbThreads = 512;
constexpr uint32_t kDbUBytes = kDbD * kDbCols * 4;   // Y[:, n, tile]: 16 KB
constexpr uint32_t kDbDBytes = kDbD * kDbD * 4;      // D0_n: 4 KB
constexpr uint32_t kDbStage = kDbUBytes + kDbDBytes;
constexpr uint32_t kDbASlab = kDbCols * 32;          // one 16-wide K slab of 128 BF16 rows
constexpr uint32_t kDbAPlane = 2 * kDbASlab;         // K = 32
constexpr uint32_t kDbBSlab = kDbD * 32;
constexpr uint32_t kDbBPlane = 2 * kDbBSlab;
constexpr uint32_t kDbABuf = 3 * kDbAPlane;          // three planes
constexpr uint32_t kDbBBuf = 3 * kDbBPlane;
constexpr uint32_t kDbFixed = 2 * kDbABuf + 2 * kDbBBuf + kDbStages * kDbStage;

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

}  // namespace

template <int NB>
__global__ void __launch_bounds__(kDbThreads, 1)
    k_dband_tc(int N, int periodic, int P, const float *__restrict__ taps, const float *__restrict__ Dm,
               long long dm_ss, const float *__restrict__ Y, float *__restrict__ band, long long bss, long long brs,
               long long bos, long long b0, unsigned *__restrict__ flag) {
    constexpr int R = (NB - 1) / 2;
    extern __shared__ __align__(1024) unsigned char smb[];
    unsigned char *Abuf = smb;                                   // [2][3 planes][2 slabs]
    unsigned char *Bbuf = Abuf + 2 * kDbABuf;                    // [2][3 planes][2 slabs]
    unsigned char *ring = Bbuf + 2 * kDbBBuf;                    // [stages][Y slice | D0_n]
    float *tap_s = reinterpret_cast<float *>(ring + kDbStages * kDbStage);   // [N + 3 + 2R][32]
    const int ntap = N + 3 + 2 * R;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tap_s + (size_t)ntap * kDbD);   // [2] MMAs of site n done
    uint64_t *staged = mbar + 2;                                                   // [2] operands of site n staged
    uint32_t *tslot = reinterpret_cast<uint32_t *>(staged + 2);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = (P + kDbCols - 1) / kDbCols;
    const long long blk = blockIdx.x;
    const int p0 = (int)(blk % tiles) * kDbCols;
    const long long bl = blk / tiles;
    const int k0 = p0 / kDbD;
    const float *Yb = Y + bl * (long long)kDbD * N * P;          // [a][n][p] of this configuration
    const float *Db = Dm + bl * dm_ss;                           // [n][c][a]

    // tap_s[j][c] = g_{r,c}, r = k0 - R - (N - 1) + j (circulant index on a ring, zero outside (-N, N)
    // on an open chain): site n's tap for band offset dl of source site k0 + q is row q + dl + N - 1 - n.
    for (int q = tid; q < ntap * kDbD; q += kDbThreads) {
        const int j = q / kDbD, c = q % kDbD;
        int r = k0 - R - (N - 1) + j;
        float v = 0.f;
        if (periodic) {
            r = ((r % N) + N) % N;
            v = taps[(long long)r * kDbD + c];
        } else if (r > -N && r < N) {
            v = taps[(long long)(r + N - 1) * kDbD + c];
        }
        tap_s[q] = v;
    }
    // Site n's inputs into ring stage st: 1024 + 256 chunks of 16 bytes.
    auto issue = [&](int n, int st) {
        unsigned char *dst = ring + st * kDbStage;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = tid + u * kDbThreads;
            const int a = j >> 5, c16 = j & 31;
            const int p = p0 + c16 * 4;
            const bool ok = p < P;
            cp_async16(dst + a * (kDbCols * 4) + c16 * 16, ok ? Yb + ((long long)a * N + n) * P + p : Yb, ok ? 16u : 0u);
        }
        if (tid < 256) cp_async16(dst + kDbUBytes + tid * 16, Db + (long long)n * (kDbD * kDbD) + tid * 4, 16u);
    };
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(&staged[0], kDbThreads / 32);
        tc::mbar_init(&staged[1], kDbThreads / 32);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 64);
#pragma unroll
    for (int s = 0; s < kDbStages - 1; ++s) {
        if (s < N) issue(s, s);
        cp_async_commit();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, kDbD);
    const int q4 = warp & 3, cg = warp >> 2;                      // lane quadrant, group of 8 output channels
    const uint32_t tlane = (uint32_t)(32 * q4) << 16;

    float acc[NB][8];
#pragma unroll
    for (int dl = 0; dl < NB; ++dl)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[dl][c] = 0.f;

    bool good = true;
    for (int n = 0; n <= N; ++n) {
        if (n < N) {
            cp_async_wait<kDbStages - 2>();
            __syncthreads();
            if (!*s_ok) {
                good = false;
                break;
            }
            {
                const int nn = n + kDbStages - 1;
                if (nn < N) issue(nn, nn % kDbStages);
                cp_async_commit();
            }
            const unsigned char *st = ring + (n % kDbStages) * kDbStage;
            unsigned char *A = Abuf + (n & 1) * kDbABuf;
            unsigned char *Bp = Bbuf + (n & 1) * kDbBBuf;
            {
                // A operand: rows = the tile's columns p, K = input channel a (this thread: 8 of them).
                const int pl = tid & 127, a8 = (tid >> 7) * 8;
                const float *us = reinterpret_cast<const float *>(st) + a8 * kDbCols + pl;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = us[u * kDbCols];
                tc::stage8_planes<3>(A, kDbAPlane, (uint32_t)(a8 >> 4) * kDbASlab + tc::canon(pl, a8 & 15), v);
            }
            if (tid < 128) {
                // B operand: rows = output channel c, K = input channel a.
                const int c = tid >> 2, k8 = (tid & 3) * 8;
                const float *ds = reinterpret_cast<const float *>(st + kDbUBytes) + c * kDbD + k8;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ds[u];
                tc::stage8_planes<3>(Bp, kDbBPlane, (uint32_t)(k8 >> 4) * kDbBSlab + tc::canon(c, k8 & 15), v);
            }
            // Every thread's plane stores become visible to the tensor cores, then one arrival per warp.
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&staged[n & 1])) : "memory");
            if (tid == 0) {
                if (!tc::wait(&staged[n & 1], (uint32_t)((n >> 1) & 1))) {
                    *s_ok = 0;
                } else {
                    tc::fence_after();
#pragma unroll 1
                    for (int s = 0; s < 2; ++s)
#pragma unroll
                        for (int pa = 0; pa < 3; ++pa)
#pragma unroll
                            for (int pb = 0; pa + pb < 3; ++pb)
                                tc::mma_bf16(tmem + (uint32_t)((n & 1) * kDbD),
                                             tc::desc(tc::smem_u32(A + pa * kDbAPlane + s * kDbASlab)),
                                             tc::desc(tc::smem_u32(Bp + pb * kDbBPlane + s * kDbBSlab)), idesc,
                                             (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
                    tc::commit(&mbar[n & 1]);
                }
            }
        }
        if (n >= 1) {
            // Band sums of site m = n - 1 (its MMAs were issued one iteration ago).
            const int m = n - 1;
            // One waiter per warp; the shuffle keeps the warp converged for the
            // warp-wide tensor-memory load that follows.
            uint32_t done = 1u;
            if (lane == 0) done = tc::wait(&mbar[m & 1], (uint32_t)((m >> 1) & 1)) ? 1u : 0u;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) {
                if (lane == 0) *s_ok = 0;
                good = false;
                if (n == N) break;
                continue;
            }
            tc::fence_after();
            float z[8];
            tc::tmem_ld8(tmem + tlane + (uint32_t)((m & 1) * kDbD + 8 * cg), z);
            const float *trow = tap_s + (size_t)(q4 + N - 1 - m) * kDbD + 8 * cg;
#pragma unroll
            for (int dl = 0; dl < NB; ++dl) {
                const float4 *t4 = reinterpret_cast<const float4 *>(trow + dl * kDbD);
#pragma unroll
                for (int c4 = 0; c4 < 2; ++c4) {
                    const float4 t = t4[c4];
                    acc[dl][4 * c4 + 0] = fmaf(t.x, z[4 * c4 + 0], acc[dl][4 * c4 + 0]);
                    acc[dl][4 * c4 + 1] = fmaf(t.y, z[4 * c4 + 1], acc[dl][4 * c4 + 1]);
                    acc[dl][4 * c4 + 2] = fmaf(t.z, z[4 * c4 + 2], acc[dl][4 * c4 + 2]);
                    acc[dl][4 * c4 + 3] = fmaf(t.w, z[4 * c4 + 3], acc[dl][4 * c4 + 3]);
                }
            }
            tc::fence_before();
        }
    }
    cp_async_wait<0>();
    tc::fence_before();
    __syncthreads();
    if (!*s_ok) good = false;
    if (good) {
        const int k = k0 + q4;
        if (k < N && p0 + 32 * q4 < P) {
            float *colb = band + (b0 + bl) * bss + (long long)(8 * cg) * kDbD + lane;
#pragma unroll
            for (int dl = 0; dl < NB; ++dl) {
                int i = k + dl - R;
                if (periodic) i = ((i % N) + N) % N;
                else if (i < 0 || i >= N) continue;
                float *dst = colb + (long long)i * brs + (long long)(2 * R - dl) * bos;
#pragma unroll
                for (int c = 0; c < 8; ++c) dst[c * kDbD] = acc[dl][c];
            }
        }
    } else if (tid == 0 && flag) {
        atomicOr(flag, 8u);
    }
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, 64);
}

template <int NB>
static cudaError_t launch_dband_nb(int N, int periodic, int P, const float *taps, const float *Dm, long long dm_ss,
                                   const float *Y, float *band, long long bss, long long brs, long long bos,
                                   long long b0, int nb, unsigned *flag, cudaStream_t st) {
    constexpr int R = (NB - 1) / 2;
    const size_t smem = kDbFixed + (size_t)(N + 3 + 2 * R) * kDbD * 4 + 64;
    if (smem > 225 * 1024) return cudaErrorNotSupported;
    cudaError_t err = cudaFuncSetAttribute(k_dband_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const long long blocks = (long long)nb * ((P + kDbCols - 1) / kDbCols);
    ProfScope _ps("k_dband", st);
    k_dband_tc<NB><<<(unsigned)blocks, kDbThreads, smem, st>>>(N, periodic, P, taps, Dm, dm_ss, Y, band, bss, brs,
                                                                bos, b0, flag);
    return cudaGetLastError();
}

int g_fused_links = 1;

bool dband_tc_ok(int d, int N, int periodic, int P, int nsrc, int R) {
    if (d != kDbD || nsrc != kDbD || P != N * kDbD || N < 1) return false;
    if (periodic && N < 2 * R + 1) return false;
    if (R != 2 && R != 3 && R != 4) return false;
    return kDbFixed + (size_t)(N + 3 + 2 * R) * kDbD * 4 + 64 <= 225 * 1024;   // mbarriers and slots: 40 B
}

cudaError_t launch_dband_tc(int d, int N, int periodic, int P, int nsrc, int R, const float *taps, const float *Dm,
                            long long dm_ss, const float *Y, float *band, long long bss, long long brs, long long bos,
                            long long b0, int nb, unsigned *flag, cudaStream_t st) {
    if (!dband_tc_ok(d, N, periodic, P, nsrc, R)) return cudaErrorNotSupported;
    switch (2 * R + 1) {
        case 5: return launch_dband_nb<5>(N, periodic, P, taps, Dm, dm_ss, Y, band, bss, brs, bos, b0, nb, flag, st);
        case 7: return launch_dband_nb<7>(N, periodic, P, taps, Dm, dm_ss, Y, band, bss, brs, bos, b0, nb, flag, st);
        case 9: return launch_dband_nb<9>(N, periodic, P, taps, Dm, dm_ss, Y, band, bss, brs, bos, b0, nb, flag, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace dn

extern "C" dn_status dn_set_fused_links(int on) {
    dn::g_fused_links = on ? 1 : 0;
    return DN_OK;
}
