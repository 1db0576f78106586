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
// over all N sites n, with specialised warps connected by mbarriers:
//   - warpgroup 3: one thread brings Y[:, n, tile] (32 x 128 floats, one TMA tensor copy)
//     and D0_n (32 x 32, one bulk copy) into a four-stage ring as stages free up; another
//     issues, per site, the five BF16 plane products with pa < 2, pa + pb <= 2 (M = 128 columns,
//     N = 32 output channels, K = 32 input channels, FP32 accumulation into one of three
//     tensor-memory buffers): the same products and order as the separate vertex-hop
//     kernel;
//   - warpgroup 0 splits every value into BF16 planes (v = p0 + p1 + rest): the A operand
//     (the hop output slice, row = column p, two planes: it carries the previous Toeplitz
//     hop's two-plane error already) into one of three tensor-memory buffers, the B
//     operand (D0_n, three planes) into one of three shared-memory buffers; the MMAs read
//     A from tensor memory, which keeps the plane products' operand reads off the
//     shared-memory port;
//   - warpgroups 1-2 (warps 4-11) only add each site into the band sums: warp w owns
//     TMEM lanes 32 (w & 3) .. + 31 (one source site, lane = source channel c') and
//     output channels 16 ((w - 4) >> 2) .. + 15, with the 2R+1 band offsets in registers
//     (taps from a shared table, already wrapped for rings), two sites per step so that
//     each tap row is loaded once for both; they release each accumulator buffer as soon
//     as they have read it.  The band sums are formed in the
//     same order (site n ascending, fmaf(tap, z, acc)) as the separate band kernel, so
//     the fused result equals the two-kernel one.
//   Registers move from the staging and control warpgroups to the band warpgroups
//   (setmaxnreg): 512 threads x 128 at launch = 128 x 72 + 256 x 200 + 128 x 40.
// Every mbarrier wait is bounded; a wait that gives up raises bit 8 of the cache flag,
// every role stops, the copies already issued are waited for (bounded), the tensor
// memory is freed and nothing is written.
#include "dn_internal.cuh"
#include "tc_common.cuh"

namespace dn {

namespace {

constexpr int kDbD = 32;                             // channels
constexpr int kDbCols = 128;                         // source columns per CTA
constexpr int kDbStages = 4;                         // depth of the input ring
constexpr int kDbBufs = 4;                           // operand buffers and accumulators in flight
constexpr int kDbAPl = 2;                            // BF16 planes of the A operand (the hop output)
constexpr int kDbThreads = 512;                      // warpgroups: 0 staging, 1-2 band sums, 3 loads + MMAs
constexpr int kDbStageRegs = 72, kDbBandRegs = 200, kDbCtlRegs = 40;   // x 128, 256, 128 threads = 512 x 128
constexpr uint32_t kDbUBytes = kDbD * kDbCols * 4;   // Y[:, n, tile]: 16 KB
constexpr uint32_t kDbDBytes = kDbD * kDbD * 4;      // D0_n: 4 KB
constexpr uint32_t kDbStage = kDbUBytes + kDbDBytes;
constexpr uint32_t kDbBSlab = kDbD * 32;
constexpr uint32_t kDbBPlane = 2 * kDbBSlab;
constexpr uint32_t kDbBBuf = 3 * kDbBPlane;
constexpr uint32_t kDbFixed = kDbBufs * kDbBBuf + kDbStages * kDbStage;
// Tensor-memory columns: A operands (kDbAPl planes x K = 32 BF16, two per column) and accumulators.
constexpr uint32_t kDbACols = kDbAPl * 16;
constexpr uint32_t kDbZCol0 = kDbBufs * kDbACols;                  // accumulators after the A operands
constexpr uint32_t kDbTmemCols = 256;                               // >= kDbZCol0 + kDbBufs * 32
constexpr uint32_t kDbTail = (2 * kDbStages + 3 * kDbBufs) * 8 + 16;   // mbarriers, TMEM slot, status

__device__ __forceinline__ void arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Eight 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// MMA with the A operand in tensor memory (BF16, row i in lane i, two K values per column).
__device__ __forceinline__ void mma_bf16_ta(uint32_t dt, uint32_t at, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
                 "r"(at), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tma_slice(void *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
                 : "memory");
}

}  // namespace

template <int NB>
__global__ void __launch_bounds__(kDbThreads, 1)
    k_dband_tc(int N, int periodic, int P, const float *__restrict__ taps, const float *__restrict__ Dm,
               long long dm_ss, const float *__restrict__ Y, float *__restrict__ band, long long bss, long long brs,
               long long bos, long long b0, unsigned *__restrict__ flag, const __grid_constant__ CUtensorMap ymap) {
    constexpr int R = (NB - 1) / 2;
    extern __shared__ __align__(1024) unsigned char smb[];
    unsigned char *ring = smb;                                   // [stages][Y slice | D0_n]
    unsigned char *Bbuf = ring + kDbStages * kDbStage;           // [bufs][3 planes][2 slabs]
    float *tap_s = reinterpret_cast<float *>(Bbuf + kDbBufs * kDbBBuf);   // [N + 3 + 2R][32]
    const int ntap = N + 3 + 2 * R;
    uint64_t *full = reinterpret_cast<uint64_t *>(tap_s + (size_t)ntap * kDbD);   // [S] stage loaded
    uint64_t *empty = full + kDbStages;                                            // [S] stage read
    uint64_t *staged = empty + kDbStages;                                          // [bufs] operands of a site
    uint64_t *mmad = staged + kDbBufs;                                             // [bufs] its MMAs done
    uint64_t *zfree = mmad + kDbBufs;                                              // [bufs] accumulator read
    uint32_t *tslot = reinterpret_cast<uint32_t *>(zfree + kDbBufs);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = (P + kDbCols - 1) / kDbCols;
    const long long blk = blockIdx.x;
    const int p0 = (int)(blk % tiles) * kDbCols;
    const long long bl = blk / tiles;
    const int k0 = p0 / kDbD;
    const int ncol = P - p0 < kDbCols ? P - p0 : kDbCols;           // a multiple of 32
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
    if (tid == 0) {
        for (int st = 0; st < kDbStages; ++st) {
            tc::mbar_init(&full[st], 1);
            tc::mbar_init(&empty[st], 4);
        }
        for (int j = 0; j < kDbBufs; ++j) {
            tc::mbar_init(&staged[j], 4);
            tc::mbar_init(&mmad[j], 1);
            tc::mbar_init(&zfree[j], 8);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, kDbTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    auto alive = [&]() { return *((volatile int *)s_ok) != 0; };

    if (warp < 4) {
        // ---------------------------------------------------- warpgroup 0: operand planes --
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kDbStageRegs));
        const uint32_t trow = (uint32_t)(32 * warp) << 16;            // this thread's lane = row p = tid
        for (int n = 0; n < N; ++n) {
            const int st = n % kDbStages, j = n % kDbBufs;
            bool ok = alive();
            // buffer j was read by the MMAs of site n - bufs; the stage holds site n
            if (ok && n >= kDbBufs) ok = tc::wait(&mmad[j], (uint32_t)((n / kDbBufs - 1) & 1));
            if (ok) ok = tc::wait(&full[st], (uint32_t)((n / kDbStages) & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) *s_ok = 0;
                break;
            }
            tc::fence_after();
            const unsigned char *src = ring + st * kDbStage;
            // A operand (tensor memory): row p = tid of the tile, K = input channel a; each
            // 16-wide K slab as BF16 planes of 8 columns (element 2c in the low half).
            const float *us = reinterpret_cast<const float *>(src) + tid;
            const uint32_t abase = tmem + trow + (uint32_t)(j * kDbACols);
#pragma unroll
            for (int a16 = 0; a16 < kDbD; a16 += 16) {
                float r[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) r[u] = us[(a16 + u) * kDbCols];
#pragma unroll
                for (int pl = 0; pl < kDbAPl; ++pl) {
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
                        w[i] = *reinterpret_cast<const uint32_t *>(&h);
                        if (pl < kDbAPl - 1) {
                            r[2 * i] -= __low2float(h);
                            r[2 * i + 1] -= __high2float(h);
                        }
                    }
                    tmem_st8(abase + (uint32_t)(pl * 16 + (a16 >> 1)), w);
                }
            }
            // B operand (shared memory): row = output channel c, K = input channel a.
            {
                unsigned char *Bp = Bbuf + j * kDbBBuf;
                const int c = tid >> 2, k8 = (tid & 3) * 8;
                const float *ds = reinterpret_cast<const float *>(src + kDbUBytes) + c * kDbD + k8;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ds[u];
                tc::stage8_planes<3>(Bp, kDbBPlane, (uint32_t)(k8 >> 4) * kDbBSlab + tc::canon(c, k8 & 15), v);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc::fence_async_smem();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) {
                arrive(&staged[j]);
                arrive(&empty[st]);
            }
        }
    } else if (warp < 12) {
        // ---------------------------------------------------- warpgroups 1-2: band sums --
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kDbBandRegs));
        const int q4 = warp & 3, ch = (warp - 4) >> 2;
        const uint32_t tlane = (uint32_t)(32 * q4) << 16;
        float acc[NB][16];
#pragma unroll
        for (int dl = 0; dl < NB; ++dl)
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[dl][c] = 0.f;
        bool good = true;
        // One site per step; the accumulator columns of site n + 1 are loaded (tcgen05.ld, no
        // wait) before the band sums of site n and waited for after them, so the tensor-memory
        // load latency hides behind the FMAs.  Sites go in ascending order, as in the band kernel.
        auto issue = [&](int n, uint32_t (&dst)[16]) -> bool {
            const int j = n % kDbBufs;
            bool ok = alive() && tc::wait(&mmad[j], (uint32_t)((n / kDbBufs) & 1));
            if (!__all_sync(0xffffffffu, ok)) return false;
            tc::fence_after();
            const uint32_t zc = tmem + tlane + kDbZCol0 + (uint32_t)(j * kDbD + 16 * ch);
            tc::tmem_ld8_async(zc, dst);
            tc::tmem_ld8_async(zc + 8, dst + 8);
            return true;
        };
        auto release = [&](int n, uint32_t (&r)[16]) {
            tc::tmem_wait_ld(r, 16);
            tc::fence_before();
            __syncwarp();
            if (lane == 0) arrive(&zfree[n % kDbBufs]);
        };
        uint32_t zc[16];
        if (!issue(0, zc)) {
            if (lane == 0) *s_ok = 0;
            good = false;
        } else {
            release(0, zc);
        }
        for (int n = 0; n < N && good; ++n) {
            uint32_t zn[16];
            const bool nxt = n + 1 < N;
            if (nxt && !issue(n + 1, zn)) {
                if (lane == 0) *s_ok = 0;
                good = false;
                break;
            }
            // tap of (site n, offset dl): tap_s row q4 + N - 1 - n + dl
            const float *tr = tap_s + (size_t)(q4 + N - 1 - n) * kDbD + 16 * ch;
#pragma unroll
            for (int dl = 0; dl < NB; ++dl) {
                const float4 *t4 = reinterpret_cast<const float4 *>(tr + dl * kDbD);
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const float4 g = t4[c4];
                    acc[dl][4 * c4 + 0] = fmaf(g.x, __uint_as_float(zc[4 * c4 + 0]), acc[dl][4 * c4 + 0]);
                    acc[dl][4 * c4 + 1] = fmaf(g.y, __uint_as_float(zc[4 * c4 + 1]), acc[dl][4 * c4 + 1]);
                    acc[dl][4 * c4 + 2] = fmaf(g.z, __uint_as_float(zc[4 * c4 + 2]), acc[dl][4 * c4 + 2]);
                    acc[dl][4 * c4 + 3] = fmaf(g.w, __uint_as_float(zc[4 * c4 + 3]), acc[dl][4 * c4 + 3]);
                }
            }
            if (nxt) {
                release(n + 1, zn);
#pragma unroll
                for (int c = 0; c < 16; ++c) zc[c] = zn[c];
            }
        }
        const int k = k0 + q4;
        if (good && alive() && k < N && 32 * q4 < ncol) {
            float *colb = band + (b0 + bl) * bss + (long long)(16 * ch) * kDbD + lane;
#pragma unroll
            for (int dl = 0; dl < NB; ++dl) {
                int i = k + dl - R;
                if (periodic) i = ((i % N) + N) % N;
                else if (i < 0 || i >= N) continue;
                float *dst = colb + (long long)i * brs + (long long)(2 * R - dl) * bos;
#pragma unroll
                for (int c = 0; c < 16; ++c) dst[c * kDbD] = acc[dl][c];
            }
        }
    } else {
        // ------------------------------------------------ warpgroup 3: loads and MMAs --
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kDbCtlRegs));
        if (warp == 12 && lane == 0) {
            // loader: site n into stage n % S once the staging warps have read site n - S
            int n = 0;
            for (; n < N; ++n) {
                const int st = n % kDbStages;
                if (!alive()) break;
                if (n >= kDbStages && !tc::wait(&empty[st], (uint32_t)((n / kDbStages - 1) & 1))) {
                    *s_ok = 0;
                    break;
                }
                unsigned char *dst = ring + st * kDbStage;
                arrive_tx(&full[st], kDbStage);   // the whole box counts, zero-filled past P
                tma_slice(dst, &ymap, p0, n, (int)bl * kDbD, &full[st]);
                bulk_g2s(dst + kDbUBytes, Db + (long long)n * (kDbD * kDbD), kDbDBytes, &full[st]);
            }
            // copies still in flight (only after a failure) land before the CTA exits
            for (int q = n - kDbStages > 0 ? n - kDbStages : 0; q < n; ++q)
                (void)tc::wait(&full[q % kDbStages], (uint32_t)((q / kDbStages) & 1));
        } else if (warp == 13 && lane == 0) {
            // MMA issue: site n's operands into accumulator n % bufs once it has been read
            const uint32_t idesc = tc::idesc_bf16(128, kDbD);
            for (int n = 0; n < N; ++n) {
                const int j = n % kDbBufs;
                bool go = alive() && tc::wait(&staged[j], (uint32_t)((n / kDbBufs) & 1));
                if (go && n >= kDbBufs) go = tc::wait(&zfree[j], (uint32_t)((n / kDbBufs - 1) & 1));
                if (!go) {
                    *s_ok = 0;
                    break;
                }
                tc::fence_after();
                const uint32_t at = tmem + (uint32_t)(j * kDbACols);
                const unsigned char *Bp = Bbuf + j * kDbBBuf;
#pragma unroll 1
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int pa = 0; pa < kDbAPl; ++pa)
#pragma unroll
                        for (int pb = 0; pa + pb < 3; ++pb)
                            mma_bf16_ta(tmem + kDbZCol0 + (uint32_t)(j * kDbD), at + (uint32_t)(pa * 16 + s * 8),
                                        tc::desc(tc::smem_u32(Bp + pb * kDbBPlane + s * kDbBSlab)), idesc,
                                        (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
                tc::commit(&mmad[j]);
            }
        }
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && !*s_ok && flag) atomicOr(flag, 8u);
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, kDbTmemCols);
}

template <int NB>
static cudaError_t launch_dband_nb(int N, int periodic, int P, const float *taps, const float *Dm, long long dm_ss,
                                   const float *Y, float *band, long long bss, long long brs, long long bos,
                                   long long b0, int nb, unsigned *flag, cudaStream_t st) {
    constexpr int R = (NB - 1) / 2;
    const size_t smem = kDbFixed + (size_t)(N + 3 + 2 * R) * kDbD * 4 + kDbTail;
    if (smem > 225 * 1024) return cudaErrorNotSupported;
    cudaError_t err = cudaFuncSetAttribute(k_dband_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const long long blocks = (long long)nb * ((P + kDbCols - 1) / kDbCols);
    alignas(64) CUtensorMap ymap;
    if (!dband_input_map(&ymap, Y, N, P, (long long)nb * kDbD)) return cudaErrorNotSupported;
    ProfScope _ps("k_dband", st);
    k_dband_tc<NB><<<(unsigned)blocks, kDbThreads, smem, st>>>(N, periodic, P, taps, Dm, dm_ss, Y, band, bss, brs,
                                                                bos, b0, flag, ymap);
    return cudaGetLastError();
}

int g_fused_links = 1;

// The register split of k_dband_tc (setmaxnreg) assumes the launch allocation of
// kDbThreads x 168 registers; a build that allocates another count is never launched
// (the chain ends then run as two kernels).
template <int NB>
static bool dband_regs_ok() {
    static int regs = -1;
    if (regs < 0) {
        cudaFuncAttributes fa;
        regs = cudaFuncGetAttributes(&fa, k_dband_tc<NB>) == cudaSuccess ? fa.numRegs : 0;
        cudaGetLastError();
    }
    return regs * kDbThreads == 128 * kDbStageRegs + 256 * kDbBandRegs + 128 * kDbCtlRegs;
}

bool dband_tc_ok(int d, int N, int periodic, int P, int nsrc, int R) {
    if (d != kDbD || nsrc != kDbD || P != N * kDbD || N < 1) return false;
    if (periodic && N < 2 * R + 1) return false;
    if (kDbFixed + (size_t)(N + 3 + 2 * R) * kDbD * 4 + kDbTail > 225 * 1024) return false;
    switch (R) {
        case 2: return dband_regs_ok<5>();
        case 3: return dband_regs_ok<7>();
        case 4: return dband_regs_ok<9>();
        default: return false;
    }
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
