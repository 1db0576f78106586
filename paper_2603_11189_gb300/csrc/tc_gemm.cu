// Toeplitz hop of the link construction on the tcgen05 tensor cores (FP32 path).
//
// Y[b][a][i][p] = sum_n g_{i-n,a} X[b][a][n][p] for one channel a, 128 rows i and
// 256 columns p per CTA.  Operands are FP32; each is split into two BF16 terms
// (x = x_hi + x_lo, x_hi = bf16(x), x_lo = bf16(x - x_hi)) and the product is
// accumulated in FP32 in tensor memory as A_hi B_hi + A_hi B_lo + A_lo B_hi, which
// keeps about 16 mantissa bits (plain TF32 or BF16 products are not accurate
// enough for the FP32 path's 1e-4 bound on log-amplitude ratios).
//
// Shared-memory operands use the no-swizzle K-major canonical layout: a slab of
// 16 K values holds 8-row x 16-byte core matrices, K-adjacent cores 128 B apart
// (leading byte offset) and row-group-adjacent cores 256 B apart (stride byte
// offset).  The Toeplitz operand is stored as a Hankel matrix instead: running the
// contraction over each 64-site chunk in reverse order makes A(r, k) depend on
// r + k only, so a 128 x 64 chunk has 23 distinct core matrices, stored once and
// addressed with both offsets equal to 128 B.  One thread issues the MMAs (M=128, N=256, K=16 each) and commits
// them to an mbarrier; every wait is bounded, and a timeout raises bit 8 of the
// error flag, skips the epilogue and still releases the tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <mutex>

#include "dn_internal.cuh"
#include "tc_common.cuh"

namespace dn {

namespace {

constexpr int kTcM = 128, kTcK = 64;     // K staged 64 sites (4 MMA slabs) at a time
constexpr int kHankel = kTcM / 8 + kTcK / 8 - 1;   // distinct core matrices of a Toeplitz chunk
constexpr int kHankelBytes = ((kHankel * 128 + 1023) / 1024) * 1024;
constexpr int kNBuf = 1;                 // operand buffers per CTA
constexpr int kEpiBytes = 8 * 32 * 33 * 4; // epilogue staging: one 32 x 33 float tile per warp
constexpr long kTcSpin = 1L << 24;

__device__ __forceinline__ uint32_t sm_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;     // K-adjacent core matrices
    d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;     // row-group-adjacent core matrices
    d |= (uint64_t)1 << 46;
    return d;
}

// Descriptor of a Hankel operand: core matrices one 128-B step apart along both rows and K,
// so that core (rg, kg) is read from start + 128 (rg + kg).
__device__ __forceinline__ uint64_t umma_desc_hankel(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (row r, k within a 16-wide slab) in the canonical layout.
__device__ __forceinline__ uint32_t canon(int r, int k16) {
    return (uint32_t)((r >> 3) * 256 + (k16 >> 3) * 128 + (r & 7) * 16 + (k16 & 7) * 2);
}

__device__ __forceinline__ int tap_row_tc(int r, int N, int periodic) {
    return periodic ? (r < 0 ? r + N : (r >= N ? r - N : r)) : r + N - 1;
}

__device__ __forceinline__ int ring_delta_tc(int dl, int N, int periodic) {
    if (periodic) {
        if (dl > N / 2) dl -= N;
        else if (dl <= -((N + 1) / 2)) dl += N;
    }
    return dl;
}

__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < kTcSpin; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(sm_u32(mbar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace

template <bool GEN, int TN, int NPL>
__global__ void __launch_bounds__(256, 3) k_tgemm_tc(Geom g, const float *__restrict__ taps, int P,
                                                  const float *__restrict__ X, const float *__restrict__ gtaps,
                                                  const float *__restrict__ gDm, long long dm_ss, float *__restrict__ Y,
                                                  float *__restrict__ band, long long bss, long long brs, long long bos,
                                                  int bR, int bns, long long b0, unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smtc[];
    constexpr int kTcN = TN, kSlabB = TN * 16 * 2, kTpc = 256 / TN;   // threads per B column
    const int N = g.N, d = g.d;
    // One operand buffer (a second one would cost an SM a resident CTA, which measured slower):
    // chunk c waits for the MMAs of chunk c - 1 before it overwrites the operands.
    // Operand planes (NPL BF16 terms per value): A planes, then B planes.  The epilogue reuses
    // the start of shared memory as 8 staging tiles of 32 x 33 floats, so everything else
    // starts after the larger of the two regions.
    constexpr int kBuf = NPL * (kHankelBytes + 4 * kSlabB);
    constexpr int kFront = kNBuf * kBuf > kEpiBytes ? kNBuf * kBuf : kEpiBytes;
    float *gx = reinterpret_cast<float *>(smtc + kFront);   // taps of channel a: gx[r + N - 1]
    float *Dms = gx + ((2 * N + 1) & ~1);                       // [32][d]   (generated operand only)
    float *Tps = Dms + (GEN ? 32 * d : 0);                      // [32 + nk - 1][d]
    const int nk = (kTcN + d - 1) / d + 1;                      // source sites a column tile touches
    const bool gstage = GEN && (kTcN % d == 0) && d <= 64;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Tps + (GEN ? ((32 + nk - 1) * d + 1) / 2 * 2 : 0));   // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * kTcN, i0 = blockIdx.y * kTcM;
    const long long za = blockIdx.z;
    const int a = (int)(za % d);
    const long long bl = za / d;
    for (int q = tid; q < 2 * N - 1; q += blockDim.x) gx[q] = taps[(long long)tap_row_tc(q - (N - 1), N, g.periodic) * d + a];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(tslot)), "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
    // This thread stages column p0 + pp of B for its share (1 / kTpc) of the sites of a chunk.
    const int pp = tid % TN, part = tid / TN;
    const int pcol = p0 + pp;
    const bool pok = pcol < P;
    int kq = 0, cq = 0;
    if (GEN) {
        kq = pcol / d;
        cq = pcol - kq * d;
    }
    const int kfirst = p0 / d;                  // first source site of the tile
    const float *xcol = (!GEN) ? X + (bl * d + a) * (long long)N * P + pcol : nullptr;
    const float *dmcol = GEN ? gDm + bl * dm_ss + (long long)a * d + cq : nullptr;
    const long long dd = (long long)d * d;
    uint32_t waits[2] = {0u, 0u};
    const int nchunks = (N + kTcK - 1) / kTcK;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int n0 = ch * kTcK, buf = ch % kNBuf;
        unsigned char *Ap = smtc + buf * kBuf;                // NPL planes of kHankel cores of 128 B
        unsigned char *Bp = Ap + NPL * kHankelBytes;          // NPL planes of 4 slabs x kSlabB
        if (ch >= kNBuf) {
            // The MMAs that last read this buffer (chunk ch - kNBuf) must be done; one warp waits.
            if (warp == 0 && !tc_wait(mbar + buf, waits[buf] & 1u) && lane == 0) *s_ok = 0;
            waits[buf]++;
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (!*s_ok) break;
        }
        // A: the chunk's K order is reversed (position k <-> site n0 + kTcK - 1 - k), which
        // makes A(r, k) = g(base + r + k) a Hankel matrix: core matrix (row group rg, K group
        // kg) depends on rg + kg only, so the kHankel distinct cores are stored once and the
        // descriptors step 128 B in both directions.
        for (int q = tid; q < kHankel * 8; q += blockDim.x) {
            const int D = q >> 3, rr = q & 7;
            const int t0 = i0 - n0 - kTcK + 1 + 8 * D + rr;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u;
                v[u] = (t > -N && t < N) ? gx[t + N - 1] : 0.f;
            }
            tc::stage8_planes<NPL>(Ap, kHankelBytes, (uint32_t)(D * 128 + rr * 16), v);
        }
        if (GEN && gstage) {
            // Generated operand: the vertex rows D0_n[a][:] and the tap rows g_{n-k} the tile needs
            // are staged in shared memory (coalesced), 32 sites at a time.
            for (int h = 0; h < kTcK; h += 32) {
                __syncthreads();
                for (int nn = warp; nn < 32; nn += 8) {
                    const int n = n0 + h + nn;
                    for (int cc = lane; cc < d; cc += 32)
                        Dms[nn * d + cc] = n < N ? gDm[bl * dm_ss + ((long long)n * d + a) * d + cc] : 0.f;
                }
                const int rmin = n0 + h - (kfirst + nk - 1), nrow = 32 + nk - 1;
                for (int rr = warp; rr < nrow; rr += 8) {
                    const int r = rmin + rr;
                    const bool rok = r > -N && r < N;
                    const float *src = gtaps + (long long)(rok ? tap_row_tc(r, N, g.periodic) : 0) * d;
                    for (int cc = lane; cc < d; cc += 32) Tps[rr * d + cc] = rok ? src[cc] : 0.f;
                }
                __syncthreads();
#pragma unroll
                for (int kx = 0; kx < 4 / kTpc; ++kx) {
                    const int kc = part * (4 / kTpc) + kx;
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int nn = kc * 8 + 7 - u, n = n0 + h + nn;
                        v[u] = (pok && n < N) ? Dms[nn * d + cq] * Tps[(n - kq - rmin) * d + cq] : 0.f;
                    }
                    const int kk = kTcK - 8 - h - kc * 8;
                    tc::stage8_planes<NPL>(Bp, 4 * kSlabB, (uint32_t)(kk >> 4) * kSlabB + canon(pp, kk & 15), v);
                }
            }
        } else {
            // Column pcol of B for this thread's share of the 64 sites: every load issued before any is used.
            constexpr int KS = kTcK / kTpc;
            float v[KS];
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const int n = n0 + part * KS + kk;
                float x = 0.f;
                if (pok && n < N) {
                    if (GEN) x = dmcol[(long long)n * dd] * gtaps[(long long)tap_row_tc(n - kq, N, g.periodic) * d + cq];
                    else x = xcol[(long long)n * P];
                }
                v[kk] = x;
            }
#pragma unroll
            for (int kc = 0; kc < KS / 8; ++kc) {
                float w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) w[u] = v[8 * kc + 7 - u];
                const int kk = kTcK - 8 - part * KS - kc * 8;
                tc::stage8_planes<NPL>(Bp, 4 * kSlabB, (uint32_t)(kk >> 4) * kSlabB + canon(pp, kk & 15), w);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int s = 0; s < kTcK / 16; ++s) {
#pragma unroll
                for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                    for (int pb = 0; pa + pb < NPL; ++pb) {
                        const uint64_t ad = umma_desc_hankel(sm_u32(Ap + pa * kHankelBytes + 2 * s * 128));
                        const uint64_t bd = umma_desc(sm_u32(Bp + pb * 4 * kSlabB + s * kSlabB));
                        tc::mma_bf16(tmem, ad, bd, idesc, (ch == 0 && s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
                    }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(mbar + buf)));
        }
    }
    // The last commit covers every MMA issued before it.
    if (*s_ok && nchunks > 0) {
        const int lb = (nchunks - 1) % kNBuf;
        if (warp == 0 && !tc_wait(mbar + lb, waits[lb] & 1u) && lane == 0) *s_ok = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    const bool ok = *s_ok != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!ok) {
        if (tid == 0) atomicOr(flag, 8u);
    } else {
        // Epilogue: warp w owns TMEM lanes 32 (w % 4).. (rows) and columns (TN / 2) (w / 4)..; each
        // 32 x 32 piece goes through shared memory (the operand buffers are free now) so that a
        // lane then owns a column and the global stores of a row are contiguous.
        const int quad = warp & 3, half = warp >> 2;
        float *stage = reinterpret_cast<float *>(smtc) + warp * (32 * 33);
        const int prow0 = i0 + quad * 32;
        const int nrows = N - prow0 < 32 ? N - prow0 : 32;
        for (int c0 = 0; c0 < kTcN / 2; c0 += 32) {
            uint32_t r[32];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * (kTcN / 2) + c0 + 8 * q);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[8 * q + 0]), "=r"(r[8 * q + 1]), "=r"(r[8 * q + 2]), "=r"(r[8 * q + 3]),
                               "=r"(r[8 * q + 4]), "=r"(r[8 * q + 5]), "=r"(r[8 * q + 6]), "=r"(r[8 * q + 7])
                             : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const int p = p0 + half * (kTcN / 2) + c0 + lane;
            if (p < P && nrows > 0) {
                if (Y) {
                    float *yp = Y + ((bl * d + a) * N + prow0) * (long long)P + p;
                    for (int rr = 0; rr < nrows; ++rr, yp += P) *yp = stage[rr * 33 + lane];
                }
                if (band) {
                    // Only the rows within bR of the column's source site hold band entries.
                    const int k = p / bns, cc = p - k * bns;
                    float *bp = band + (b0 + bl) * bss + (long long)a * bns + cc;
                    for (int dl = -bR; dl <= bR; ++dl) {
                        int i = k + dl;
                        if (g.periodic) i = i < 0 ? i + N : (i >= N ? i - N : i);
                        else if (i < 0 || i >= N) continue;
                        if (i < prow0 || i >= prow0 + nrows) continue;
                        if (g.periodic && ring_delta_tc(i - k, N, 1) != dl) continue;
                        bp[(long long)i * brs + (long long)(bR - dl) * bos] = stage[(i - prow0) * 33 + lane];
                    }
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// Persistent variant for the generated operand (first hop of a source chain) when the
// whole chain fits in shared memory (N <= 256): one CTA per (sample, channel a, 128-row
// site tile) loops over column tiles.  The source-layer vertex rows D0_n[a][:], the
// source-layer taps g_r[:] for r in (-N, N) and the Hankel operand of every K chunk are
// staged once per CTA, so a column tile costs its operand generation, MMAs and epilogue
// only.  Chunks share one B buffer: chunk c waits for the MMAs of chunk c - 1.
constexpr int kGpMaxChunks = 4;

template <int NPL, int DD>
__global__ void __launch_bounds__(256, 2) k_tgemm_genp(Geom g, const float *__restrict__ taps, int P,
                                                       const float *__restrict__ gtaps, const float *__restrict__ gDm,
                                                       long long dm_ss, const __grid_constant__ CUtensorMap tmY,
                                                       float *__restrict__ band, long long bss, long long brs,
                                                       long long bos, int bR, int bns, long long b0,
                                                       unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smtc[];
    constexpr int TN = 128, kSlabB = TN * 16 * 2;
    constexpr int kBbytes = NPL * 4 * kSlabB;
    constexpr int kFront = kBbytes > kEpiBytes ? kBbytes : kEpiBytes;
    const int N = g.N;
    constexpr int d = DD;   // channels: compile-time, so site strides fold into immediates
    const int nch = (N + kTcK - 1) / kTcK;
    unsigned char *Bp = smtc;                                       // NPL planes x 4 slabs
    unsigned char *Aall = smtc + kFront;                            // [nch][NPL][kHankelBytes]
    float *gx = reinterpret_cast<float *>(Aall + (size_t)nch * NPL * kHankelBytes);   // gx[r + N - 1], channel a
    float *Dfull = gx + ((2 * N + 1) & ~1);                         // [N][d]: D0_n[a][c']
    float *Tfull = Dfull + (size_t)N * d;                           // [2N - 1][d]: g_r[c'], row r + N - 1
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Tfull + ((size_t)(2 * N - 1) * d + 1) / 2 * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * kTcM;
    const long long za = blockIdx.z;
    const int a = (int)(za % d);
    const long long bl = za / d;
    for (int q = tid; q < 2 * N - 1; q += blockDim.x) gx[q] = taps[(long long)tap_row_tc(q - (N - 1), N, g.periodic) * d + a];
    for (int q = tid; q < N * d; q += blockDim.x) {
        const int n = q / d, c = q - n * d;
        Dfull[q] = gDm[bl * dm_ss + ((long long)n * d + a) * d + c];
    }
    for (int q = tid; q < (2 * N - 1) * d; q += blockDim.x) {
        const int rr = q / d, c = q - rr * d;
        Tfull[q] = gtaps[(long long)tap_row_tc(rr - (N - 1), N, g.periodic) * d + c];
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, TN);
    __syncthreads();
    // Hankel operand of every chunk (reversed K order, as in k_tgemm_tc).
    for (int ch = 0; ch < nch; ++ch) {
        const int n0 = ch * kTcK;
        unsigned char *Ap = Aall + (size_t)ch * NPL * kHankelBytes;
        for (int q = tid; q < kHankel * 8; q += blockDim.x) {
            const int D = q >> 3, rr = q & 7;
            const int t0 = i0 - n0 - kTcK + 1 + 8 * D + rr;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u;
                v[u] = (t > -N && t < N) ? gx[t + N - 1] : 0.f;
            }
            tc::stage8_planes<NPL>(Ap, kHankelBytes, (uint32_t)(D * 128 + rr * 16), v);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(kTcM, TN);
    const int pp = tid % TN, part = tid / TN;        // column of the tile, half of a chunk's sites
    const int ntiles = (P + TN - 1) / TN;
    uint32_t phase = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int p0 = t * TN, pcol = p0 + pp;
        const bool pok = pcol < P;
        const int kq = pcol / d, cq = pcol - kq * d;
        bool ok = true;
        for (int ch = 0; ch < nch; ++ch) {
            const int n0 = ch * kTcK;
            if (ch > 0) {
                // The MMAs of chunk ch - 1 read the B buffer this chunk overwrites.
                if (warp == 0 && !tc::wait(mbar, phase) && lane == 0) *s_ok = 0;
                phase ^= 1u;
                __syncthreads();
                if (!*s_ok) {
                    ok = false;
                    break;
                }
            }
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const int base = part * 32 + kc * 8;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int n = n0 + base + 7 - u;
                    v[u] = (pok && n < N) ? Dfull[n * d + cq] * Tfull[(n - kq + N - 1) * d + cq] : 0.f;
                }
                const int kk = kTcK - 8 - base;
                tc::stage8_planes<NPL>(Bp, 4 * kSlabB, (uint32_t)(kk >> 4) * kSlabB + tc::canon(pp, kk & 15), v);
            }
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                const unsigned char *Ap = Aall + (size_t)ch * NPL * kHankelBytes;
                for (int s = 0; s < kTcK / 16; ++s)
#pragma unroll
                    for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                        for (int pb = 0; pa + pb < NPL; ++pb)
                            tc::mma_bf16(tmem, umma_desc_hankel(sm_u32(Ap + pa * kHankelBytes + 2 * s * 128)),
                                         umma_desc(sm_u32(Bp + pb * 4 * kSlabB + s * kSlabB)), idesc,
                                         (ch == 0 && s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
                tc::commit(mbar);
            }
        }
        if (ok) {
            if (warp == 0 && !tc::wait(mbar, phase) && lane == 0) *s_ok = 0;
            phase ^= 1u;
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (!*s_ok) break;
        // Epilogue: thread = row i (TMEM lane), 32 columns per pass in registers.  Y leaves
        // through a 32 x 32 staging tile per warp (128-byte rows, 16-byte chunks XOR-swizzled
        // by row, the layout of the tensor map's 128B swizzle) and one TMA store; the band
        // entries of the row are written straight from the registers (4 columns per store,
        // which share a source site since the source count per site is a multiple of 4).
        const int quad = warp & 3, half = warp >> 2;
        unsigned char *stg = smtc + warp * 4096;
        const uint32_t stg_s = sm_u32(stg);
        const int prow0 = i0 + quad * 32, i = prow0 + lane;
        const long long zc = bl * d + a;
        for (int c0 = 0; c0 < TN / 2; c0 += 32) {
            float r[32];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tc::tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * (TN / 2) + c0 + 8 * q), r + 8 * q);
            const int pb = p0 + half * (TN / 2) + c0;
            if (pb >= P || prow0 >= N) continue;       // warp-uniform
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<float4 *>(stg + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                    make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                asm volatile(
                    "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                        reinterpret_cast<uint64_t>(&tmY)),
                    "r"(pb), "r"(prow0), "r"((int)zc), "r"(stg_s)
                    : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            if (band && i < N) {
                // (k, cc) of column pb, then stepped by 4 columns without dividing again
                int k = pb / bns, cc = pb - k * bns;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (pb + 4 * j >= P) break;
                    const int dl = g.periodic ? ring_delta_tc(i - k, N, 1) : i - k;
                    if (dl >= -bR && dl <= bR) {
                        float *bp = band + (b0 + bl) * bss + (long long)i * brs + (long long)(bR - dl) * bos +
                                    (long long)a * bns + cc;
                        *reinterpret_cast<float4 *>(bp) =
                            make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
                    }
                    cc += 4;
                    if (cc == bns) {
                        cc = 0;
                        ++k;
                    }
                }
            }
        }
        // The staging tiles are read before the next tile's operands overwrite them.
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
        // The next tile overwrites the staging area (B buffer) and the accumulator.
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (!*s_ok && tid == 0) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TN);
}

// Warp-specialised form of k_tgemm_genp (used when its shared memory fits): the operand
// generation of the next chunk, the MMAs of the current one and the epilogue of the
// previous column tile run at the same time instead of one after the other.
//  * warps 0-7 generate the B operand (column pp = thread mod 128, 32 of the 64 sites of a
//    chunk each, NPL BF16 planes) into one of three buffers;
//  * the last warp (one thread) issues the MMAs of a chunk once its buffer is full, into one of
//    four 128-column accumulators in tensor memory, and commits them to the buffer's empty
//    barrier and, after the last chunk of a tile, to the accumulator's full barrier;
//  * warps 8-23 drain an accumulator (TMEM lanes 32 (w mod 4) .., a quarter of the columns
//    each): hop output through a 128B-swizzled staging tile per warp and a TMA tensor
//    store, band rows from registers; they release the accumulator after their last
//    tensor-memory load.
// The products, their order and the epilogue's values are those of k_tgemm_genp.  Every
// wait is bounded; a wait that gives up raises bit 8 of the flag, every role leaves its
// loop, the MMAs issued are waited for and the tensor memory is released.
constexpr int kGwEpi = 16;  // epilogue warps: kGwEpi / 4 per tensor-memory lane quadrant
constexpr int kGwThreads = 32 * (8 + kGwEpi + 1);
constexpr int kGwStg = 1;   // staging tiles per epilogue warp (TMA stores in flight)
constexpr int kGwB = 3;     // operand buffers
constexpr int kGwAcc = 4;   // accumulators (128 tensor-memory columns each)

template <int NPL>
static size_t tgemm_genp_ws_smem(int N, int d) {
    const int nch = (N + kTcK - 1) / kTcK;
    const size_t B = (size_t)kGwB * NPL * 4 * 128 * 32, stg = (size_t)kGwEpi * kGwStg * 4096;
    return B + stg + (size_t)nch * NPL * kHankelBytes +
           ((size_t)((2 * N + 1) & ~1) + (size_t)N * d + ((size_t)(2 * N - 1) * d + 1) / 2 * 2) * sizeof(float) +
           2 * (kGwB + kGwAcc) * sizeof(uint64_t) + 16;
}

template <int NPL, int DD>
__global__ void __launch_bounds__(kGwThreads, 1) k_tgemm_genp_ws(Geom g, const float *__restrict__ taps, int P,
                                                                 const float *__restrict__ gtaps,
                                                                 const float *__restrict__ gDm, long long dm_ss,
                                                                 const __grid_constant__ CUtensorMap tmY,
                                                                 float *__restrict__ band, long long bss,
                                                                 long long brs, long long bos, int bR, int bns,
                                                                 long long b0, unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smgw[];
    constexpr int TN = 128, kSlabB = TN * 16 * 2;
    constexpr int kBbytes = NPL * 4 * kSlabB;
    const int N = g.N;
    constexpr int d = DD;
    const int nch = (N + kTcK - 1) / kTcK;
    unsigned char *Bbuf = smgw;                                   // [kGwB][kBbytes]
    unsigned char *Stg = smgw + kGwB * kBbytes;                      // [kGwEpi][kGwStg][4096]
    unsigned char *Aall = Stg + kGwEpi * kGwStg * 4096;           // [nch][NPL][kHankelBytes]
    float *gx = reinterpret_cast<float *>(Aall + (size_t)nch * NPL * kHankelBytes);   // gx[r + N - 1], channel a
    float *Dfull = gx + ((2 * N + 1) & ~1);                       // [N][d]: D0_n[a][c']
    float *Tfull = Dfull + (size_t)N * d;                         // [2N - 1][d]: g_r[c'], row r + N - 1
    uint64_t *bar = reinterpret_cast<uint64_t *>(Tfull + ((size_t)(2 * N - 1) * d + 1) / 2 * 2);
    uint64_t *bfull = bar, *bempty = bar + kGwB, *afull = bar + 2 * kGwB, *aempty = afull + kGwAcc;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(aempty + kGwAcc);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * kTcM;
    const long long za = blockIdx.z;
    const int a = (int)(za % d);
    const long long bl = za / d;
#pragma unroll 4
    for (int q = tid; q < 2 * N - 1; q += blockDim.x) gx[q] = taps[(long long)tap_row_tc(q - (N - 1), N, g.periodic) * d + a];
#pragma unroll 4
    for (int q = tid; q < N * d; q += blockDim.x) {
        const int n = q / d, c = q - n * d;
        Dfull[q] = gDm[bl * dm_ss + ((long long)n * d + a) * d + c];
    }
#pragma unroll 4
    for (int q = tid; q < (2 * N - 1) * d; q += blockDim.x) {
        const int rr = q / d, c = q - rr * d;
        Tfull[q] = gtaps[(long long)tap_row_tc(rr - (N - 1), N, g.periodic) * d + c];
    }
    if (tid == 0) {
        for (int j = 0; j < kGwB; ++j) {
            tc::mbar_init(bfull + j, 256);
            tc::mbar_init(bempty + j, 1);
        }
        for (int j = 0; j < kGwAcc; ++j) {
            tc::mbar_init(afull + j, 1);
            tc::mbar_init(aempty + j, 32 * kGwEpi);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, kGwAcc * TN);
    __syncthreads();
    // Hankel operand of every chunk (reversed K order, as in k_tgemm_tc).
    for (int ch = 0; ch < nch; ++ch) {
        const int n0 = ch * kTcK;
        unsigned char *Ap = Aall + (size_t)ch * NPL * kHankelBytes;
        for (int q = tid; q < kHankel * 8; q += blockDim.x) {
            const int D = q >> 3, rr = q & 7;
            const int t0 = i0 - n0 - kTcK + 1 + 8 * D + rr;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0 + u;
                v[u] = (t > -N && t < N) ? gx[t + N - 1] : 0.f;
            }
            tc::stage8_planes<NPL>(Ap, kHankelBytes, (uint32_t)(D * 128 + rr * 16), v);
        }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const int ntiles = (P + TN - 1) / TN;
    const int nt = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto alive = [&]() { return *((volatile int *)s_ok) != 0; };
    if (warp < 8) {
        // ------------------------------------------------------------- B operand --
        const int pp = tid & 127, part = tid >> 7;
        int use = 0;
        bool ok = true;
        for (int k = 0; k < nt && ok; ++k) {
            const int p0 = ((int)blockIdx.x + k * (int)gridDim.x) * TN, pcol = p0 + pp;
            const bool pok = pcol < P;
            const int kq = pcol / d, cq = pcol - kq * d;
            for (int ch = 0; ch < nch; ++ch, ++use) {
                const int bb = use % kGwB, n0 = ch * kTcK;
                ok = alive();
                if (ok && use >= kGwB) ok = tc::wait(bempty + bb, (uint32_t)(((use - kGwB) / kGwB) & 1));
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    if (lane == 0) *s_ok = 0;
                    break;
                }
                unsigned char *Bp = Bbuf + bb * kBbytes;
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    const int base = part * 32 + kc * 8;
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int n = n0 + base + 7 - u;
                        v[u] = (pok && n < N) ? Dfull[n * d + cq] * Tfull[(n - kq + N - 1) * d + cq] : 0.f;
                    }
                    const int kk = kTcK - 8 - base;
                    tc::stage8_planes<NPL>(Bp, 4 * kSlabB, (uint32_t)(kk >> 4) * kSlabB + tc::canon(pp, kk & 15), v);
                }
                tc::fence_async_smem();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(bfull + bb)) : "memory");
            }
        }
    } else if (warp < 8 + kGwEpi) {
        // --------------------------------------------------------------- epilogue --
        constexpr int kCols = TN / (kGwEpi / 4);                     // columns per epilogue warp
        const int quad = (warp - 8) & 3, part = (warp - 8) >> 2;    // TMEM lanes, column part
        const int prow0 = i0 + quad * 32, i = prow0 + lane;
        const long long zc = bl * d + a;
        int nst = 0;   // stores committed by this warp: staging tile nst mod kGwStg is next
        for (int k = 0; k < nt; ++k) {
            const int ab = k % kGwAcc;
            bool ok = alive() && tc::wait(afull + ab, (uint32_t)((k / kGwAcc) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *s_ok = 0;
                break;
            }
            tc::fence_after();
            const int p0 = ((int)blockIdx.x + k * (int)gridDim.x) * TN;
            for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += 32) {
                uint32_t rr[32];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    tc::tmem_ld8_async(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ab * TN + c0 + 8 * q), rr + 8 * q);
                tc::tmem_wait_ld(rr, 32);
                if (c0 + 32 == (part + 1) * kCols) {
                    tc::fence_before();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_u32(aempty + ab)) : "memory");
                }
                float r[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = __uint_as_float(rr[j]);
                const int pb = p0 + c0;
                if (pb >= P || prow0 >= N) continue;       // warp-uniform
                unsigned char *stg = Stg + ((warp - 8) * kGwStg + nst % kGwStg) * 4096;
                // the store kGwStg back, which used this staging tile, has read it
                if (lane == 0) asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kGwStg - 1) : "memory");
                __syncwarp();
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4 *>(stg + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                        make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    asm volatile(
                        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                            reinterpret_cast<uint64_t>(&tmY)),
                        "r"(pb), "r"(prow0), "r"((int)zc), "r"(sm_u32(stg))
                        : "memory");
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
                ++nst;
                if (band && i < N) {
                    // (k, cc) of column pb, then stepped by 4 columns without dividing again
                    int ks = pb / bns, cc = pb - ks * bns;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (pb + 4 * j >= P) break;
                        const int dl = g.periodic ? ring_delta_tc(i - ks, N, 1) : i - ks;
                        if (dl >= -bR && dl <= bR) {
                            float *bp = band + (b0 + bl) * bss + (long long)i * brs + (long long)(bR - dl) * bos +
                                        (long long)a * bns + cc;
                            *reinterpret_cast<float4 *>(bp) =
                                make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
                        }
                        cc += 4;
                        if (cc == bns) {
                            cc = 0;
                            ++ks;
                        }
                    }
                }
            }
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    } else if (lane == 0) {
        // ------------------------------------------------------------- MMA issue --
        const uint32_t idesc = tc::idesc_bf16(kTcM, TN);
        int use = 0;
        bool ok = true;
        for (int k = 0; k < nt && ok; ++k) {
            const int ab = k % kGwAcc;
            ok = alive();
            if (ok && k >= kGwAcc) ok = tc::wait(aempty + ab, (uint32_t)(((k - kGwAcc) / kGwAcc) & 1));
            if (!ok) break;
            tc::fence_after();
            const uint32_t tacc = tmem + (uint32_t)(ab * TN);
            for (int ch = 0; ch < nch; ++ch, ++use) {
                const int bb = use % kGwB;
                ok = alive() && tc::wait(bfull + bb, (uint32_t)((use / kGwB) & 1));
                if (!ok) break;
                tc::fence_after();
                const unsigned char *Ap = Aall + (size_t)ch * NPL * kHankelBytes;
                const unsigned char *Bp = Bbuf + bb * kBbytes;
                for (int s = 0; s < kTcK / 16; ++s)
#pragma unroll
                    for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                        for (int pb = 0; pa + pb < NPL; ++pb)
                            tc::mma_bf16(tacc, umma_desc_hankel(sm_u32(Ap + pa * kHankelBytes + 2 * s * 128)),
                                         umma_desc(sm_u32(Bp + pb * 4 * kSlabB + s * kSlabB)), idesc,
                                         (ch == 0 && s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
                tc::commit(bempty + bb);
            }
            if (ok) tc::commit(afull + ab);
        }
        if (!ok) *s_ok = 0;
        // every MMA issued has completed before the tensor memory is released: wait for the
        // commit of the last B buffer used (commits complete in order)
        if (use > 0) (void)tc::wait(bempty + ((use - 1) % kGwB), (uint32_t)(((use - 1) / kGwB) & 1));
    }
    tc::fence_before();
    __syncthreads();
    if (!*s_ok && tid == 0) atomicOr(flag, 8u);
    if (warp == 0) tc::tmem_free(tmem, kGwAcc * TN);
}

// Vertex hop on the tensor cores: X[b][c][n][p] = sum_a D0_n[c][a] Y[b][a][n][p].  Per site n it is
// a GEMM with the columns p as rows (M = 128 per tile), the output channels as N and the input
// channels as K; D0_n is the B operand, staged once per CTA, which then loops over column tiles.
// Each FP32 value of D0 is split into NPL BF16 planes (3 for FP32 accuracy, 1 for BF16), each
// value of Y into 2 (FP32) or 1.
template <int D, int NPL>
__global__ void __launch_bounds__(128) k_dhop_tc(int N, int P, const float *__restrict__ Dm, long long dm_ss,
                                                 const float *__restrict__ Yin, float *__restrict__ Xo,
                                                 unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smd[];
    constexpr int ns = D / 16;
    constexpr uint32_t aslab = 128 * 32, bslab = D * 32, aplane = ns * aslab, bplane = ns * bslab;
    constexpr uint32_t cols = D < 32 ? 32 : D;
    // The input Y carries the Toeplitz hop's own error (two BF16 planes, about 2^-17
    // relative), so two planes of it suffice: products (0,0) (0,1) (0,2) (1,0) (1,1).
    constexpr int NPA = NPL == 3 ? 2 : NPL;
    unsigned char *Ap = smd;                       // NPL planes (NPA used): rows p, K a
    unsigned char *Bp = Ap + NPL * aplane;         // NPL planes: rows c, K a
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Bp + NPL * bplane);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = blockIdx.y;
    const long long bl = blockIdx.z;
    const float *Dn = Dm + bl * dm_ss + (long long)n * D * D;
    for (int q = tid; q < D * (D / 8); q += blockDim.x) {
        const int c = q / (D / 8), k8 = (q % (D / 8)) * 8;
        tc::stage8_planes<NPL>(Bp, bplane, (uint32_t)(k8 >> 4) * bslab + tc::canon(c, k8 & 15), Dn + (long long)c * D + k8);
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, D);
    const int ntiles = (P + 127) / 128;
    const long long cs = (long long)N * P;            // channel stride of Y and X
    const float *ybase = Yin + (bl * D * N + n) * (long long)P;
    // Input columns (all D channels of one column per thread) are loaded into registers
    // ahead of use - two tiles ahead for D <= 32, one for D = 64 - so the HBM reads of later
    // tiles are in flight while the current tile's MMAs and stores run.
    auto load_col = [&](float (&buf)[D], int tt) {
        const int pp = tt * 128 + tid;
        const bool ok = pp < P;
        const float *yg = ybase + (ok ? pp : 0);
#pragma unroll
        for (int u = 0; u < D; ++u) buf[u] = ok ? yg[u * cs] : 0.f;
    };
    constexpr int depth = D <= 32 ? 2 : 1;
    uint32_t phase = 0;
    // One tile: stage its inputs from buf, refill buf with the tile `depth` steps later,
    // then MMAs and the stores of X.  Returns false when the MMA wait gave up.
    auto tile = [&](int t, float (&buf)[D]) -> bool {
        const int p = t * 128 + tid;
        const bool valid = p < P;
#pragma unroll
        for (int a16 = 0; a16 < D; a16 += 16) {
            tc::stage8_planes<NPA>(Ap, aplane, (uint32_t)(a16 >> 4) * aslab + tc::canon(tid, 0), buf + a16);
            tc::stage8_planes<NPA>(Ap, aplane, (uint32_t)(a16 >> 4) * aslab + tc::canon(tid, 8), buf + a16 + 8);
        }
        if (t + depth * (int)gridDim.x < ntiles) load_col(buf, t + depth * gridDim.x);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            // Descriptors are formed per slab (not hoisted out of the tile loop: 2 * ns * NPL^2
            // 64-bit values would take the registers the staging needs).
#pragma unroll 1
            for (int s = 0; s < ns; ++s)
#pragma unroll
                for (int pa = 0; pa < NPA; ++pa)
#pragma unroll
                    for (int pb = 0; pa + pb < NPL; ++pb)
                        tc::mma_bf16(tmem, tc::desc(tc::smem_u32(Ap + pa * aplane + s * aslab)),
                                     tc::desc(tc::smem_u32(Bp + pb * bplane + s * bslab)), idesc,
                                     (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
            tc::commit(mbar);
        }
        if (warp == 0 && !tc::wait(mbar, phase) && lane == 0) *s_ok = 0;
        phase ^= 1u;
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (!*s_ok) return false;
        float *xg = Xo + (bl * D * N + n) * (long long)P + (valid ? p : 0);
#pragma unroll 1
        for (int c8 = 0; c8 < D; c8 += 8, xg += 8 * cs) {
            float f[8];
            tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c8, f);
            if (valid)
#pragma unroll
                for (int u = 0; u < 8; ++u) xg[u * cs] = f[u];
        }
        // The next tile overwrites the A operand and the accumulator.
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        return true;
    };
    const int g0 = (int)gridDim.x;
    if constexpr (depth == 2) {
        float va[D], vb[D];
        if ((int)blockIdx.x < ntiles) load_col(va, blockIdx.x);
        if ((int)blockIdx.x + g0 < ntiles) load_col(vb, blockIdx.x + g0);
        for (int t = blockIdx.x; t < ntiles; t += 2 * g0) {
            if (!tile(t, va)) break;
            if (t + g0 >= ntiles) break;
            if (!tile(t + g0, vb)) break;
        }
    } else {
        float va[D];
        if ((int)blockIdx.x < ntiles) load_col(va, blockIdx.x);
        for (int t = blockIdx.x; t < ntiles; t += g0)
            if (!tile(t, va)) break;
    }
    if (!*s_ok && tid == 0 && flag) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, cols);
}

// Vertex hop for a column count of at most one tile (the embedding chain, P = N <= 128): a
// CTA loops over sites n = blockIdx.y, + gridDim.y, ... of one configuration, so the tensor
// memory and barrier set-up are paid once, and the next site's input column is loaded into
// registers while the current site's operands are staged, multiplied and stored.  Products,
// planes and order as in k_dhop_tc.
template <int D, int NPL>
__global__ void __launch_bounds__(128) k_dhop_tc_sites(int N, int P, const float *__restrict__ Dm, long long dm_ss,
                                                       const float *__restrict__ Yin, float *__restrict__ Xo,
                                                       unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smd[];
    constexpr int ns = D / 16;
    constexpr uint32_t aslab = 128 * 32, bslab = D * 32, aplane = ns * aslab, bplane = ns * bslab;
    constexpr uint32_t cols = D < 32 ? 32 : D;
    constexpr int NPA = NPL == 3 ? 2 : NPL;
    unsigned char *Ap = smd;
    unsigned char *Bp = Ap + NPL * aplane;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Bp + NPL * bplane);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long bl = blockIdx.z;
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, D);
    const long long cs = (long long)N * P;
    const bool valid = tid < P;
    auto load_col = [&](float (&buf)[D], int n) {
        const float *yg = Yin + (bl * D * N + n) * (long long)P + (valid ? tid : 0);
#pragma unroll
        for (int u = 0; u < D; ++u) buf[u] = valid ? yg[u * cs] : 0.f;
    };
    float va[D];
    const int n0 = blockIdx.y, ng = gridDim.y;
    if (n0 < N) load_col(va, n0);
    uint32_t phase = 0;
    for (int n = n0; n < N; n += ng) {
        const float *Dn = Dm + bl * dm_ss + (long long)n * D * D;
        for (int q = tid; q < D * (D / 8); q += blockDim.x) {
            const int c = q / (D / 8), k8 = (q % (D / 8)) * 8;
            tc::stage8_planes<NPL>(Bp, bplane, (uint32_t)(k8 >> 4) * bslab + tc::canon(c, k8 & 15), Dn + (long long)c * D + k8);
        }
#pragma unroll
        for (int a16 = 0; a16 < D; a16 += 16) {
            tc::stage8_planes<NPA>(Ap, aplane, (uint32_t)(a16 >> 4) * aslab + tc::canon(tid, 0), va + a16);
            tc::stage8_planes<NPA>(Ap, aplane, (uint32_t)(a16 >> 4) * aslab + tc::canon(tid, 8), va + a16 + 8);
        }
        if (n + ng < N) load_col(va, n + ng);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
#pragma unroll 1
            for (int s = 0; s < ns; ++s)
#pragma unroll
                for (int pa = 0; pa < NPA; ++pa)
#pragma unroll
                    for (int pb = 0; pa + pb < NPL; ++pb)
                        tc::mma_bf16(tmem, tc::desc(tc::smem_u32(Ap + pa * aplane + s * aslab)),
                                     tc::desc(tc::smem_u32(Bp + pb * bplane + s * bslab)), idesc,
                                     (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
            tc::commit(mbar);
        }
        if (warp == 0 && !tc::wait(mbar, phase) && lane == 0) *s_ok = 0;
        phase ^= 1u;
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (!*s_ok) break;
        float *xg = Xo + (bl * D * N + n) * (long long)P + (valid ? tid : 0);
#pragma unroll 1
        for (int c8 = 0; c8 < D; c8 += 8, xg += 8 * cs) {
            float f[8];
            tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c8, f);
            if (valid)
#pragma unroll
                for (int u = 0; u < 8; ++u) xg[u * cs] = f[u];
        }
        // the next site overwrites both operands and the accumulator
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (!*s_ok && tid == 0 && flag) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, cols);
}

template <int D, int NPL>
static cudaError_t launch_dhop_tc_dp(int N, int P, const float *Dm, long long dm_ss, const float *Y, float *Xo, int nb,
                                     unsigned *flag, cudaStream_t st) {
    constexpr int ns = D / 16;
    const size_t smem = (size_t)NPL * ns * (128 * 32 + D * 32) + 32;
    const int ntiles = (P + 127) / 128;
    if (ntiles == 1) {
        // one tile per site: CTAs loop over sites, about seven per SM over the whole grid
        long long ng = (7LL * 152 + nb - 1) / nb;
        ng = ng < 1 ? 1 : (ng > N ? N : ng);
        cudaError_t err =
            cudaFuncSetAttribute(k_dhop_tc_sites<D, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        {
            ProfScope _ps("k_dhop", st);
            k_dhop_tc_sites<D, NPL><<<dim3(1, (unsigned)ng, (unsigned)nb), 128, smem, st>>>(N, P, Dm, dm_ss, Y, Xo, flag);
        }
        return cudaGetLastError();
    }
    const int cg = ntiles < 4 ? ntiles : 4;      // column tiles split over at most 4 CTAs per site
    dim3 grid((unsigned)cg, (unsigned)N, (unsigned)nb);
    cudaError_t err = cudaFuncSetAttribute(k_dhop_tc<D, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_dhop", st);
        k_dhop_tc<D, NPL><<<grid, 128, smem, st>>>(N, P, Dm, dm_ss, Y, Xo, flag);
    }
    return cudaGetLastError();
}

cudaError_t launch_dhop_tc(int d, int N, int P, const float *Dm, long long dm_ss, const float *Y, float *Xo, int nb,
                           int planes, unsigned *flag, cudaStream_t st) {
    if (d == 32 && planes == 3) return launch_dhop_tc_dp<32, 3>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    if (d == 32 && planes == 1) return launch_dhop_tc_dp<32, 1>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    if (d == 64 && planes == 3) return launch_dhop_tc_dp<64, 3>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    if (d == 64 && planes == 1) return launch_dhop_tc_dp<64, 1>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    if (d == 16 && planes == 3) return launch_dhop_tc_dp<16, 3>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    if (d == 16 && planes == 1) return launch_dhop_tc_dp<16, 1>(N, P, Dm, dm_ss, Y, Xo, nb, flag, st);
    return cudaErrorNotSupported;
}

// Sample-space SR Gram on the tensor cores: partial[split][tile] = Xc[a0:a0+128] Xc[c0:c0+128]^T over
// one K range, Xc = X - m (centred in FP32), X [n][K] row-major.  One CTA per (upper-triangle
// 128 x 128 tile, K split); K streams in chunks of 64 through two operand stages (the next
// chunk is converted into BF16 planes while the MMAs of the current one run); the FP32
// accumulator stays in TMEM for the whole K range and is written as an FP32 tile.  Diagonal
// tiles stage one operand and use it on both sides.  With NPL planes per value the products
// of planes pa + pb < NPL are accumulated (NPL = 3: FP32-grade products).
constexpr int kGcK = 64;
// Chunks per tensor-memory partial: the accumulator's FP32 additions carry a small one-sided
// rounding bias (measured: 1e-4 relative after 16384 terms), so every kGcFold chunks (1024
// terms) the partial is added into per-thread FP32 totals (round to nearest) and restarted.
constexpr int kGcFold = 16;

template <int NPL>
__global__ void __launch_bounds__(256, 1) k_gram_tc(const float *__restrict__ X, int n, long long K,
                                                    const float *__restrict__ m, long long kspan, float *__restrict__ part,
                                                    unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smg[];
    constexpr uint32_t slab = 128 * 32, plane = 4 * slab, opnd = NPL * plane, stage_b = 2 * opnd;
    unsigned char *st0 = smg;                                       // [2 stages][A | B][NPL planes][4 slabs]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smg + 2 * stage_b);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = (n + 127) / 128;
    int t = blockIdx.x, ta = 0;
    while (t >= nt - ta) {
        t -= nt - ta;
        ++ta;
    }
    const int tc_ = ta + t;
    const bool diag = tc_ == ta;
    const int a0 = ta * 128, c0 = tc_ * 128;
    const long long kb = (long long)blockIdx.y * kspan;
    const long long ke = kb + kspan < K ? kb + kspan : K;
    const int nch = (int)((ke - kb + kGcK - 1) / kGcK);
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        tc::mbar_init(mbar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, 128);
    const int r = tid & 127, kh = tid >> 7;          // row of the tile, half of the chunk's K
    const bool ra = a0 + r < n, rc = c0 + r < n;
    const float *xa = X + (long long)(ra ? a0 + r : 0) * K;
    const float *xc = X + (long long)(rc ? c0 + r : 0) * K;
    const bool vec = (K & 3) == 0;   // rows 16-byte aligned: two 16-byte loads per 8 values
    // The 32 values of this thread's half row of chunk k0 (centred), into registers.
    auto load = [&](float (&v)[32], const float *row, bool ok, long long k0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long k = k0 + kh * 32 + 8 * j;
            if (ok && vec && k + 8 <= ke) {
                const float4 x0 = __ldg(reinterpret_cast<const float4 *>(row + k));
                const float4 x1 = __ldg(reinterpret_cast<const float4 *>(row + k + 4));
                const float4 m0 = __ldg(reinterpret_cast<const float4 *>(m + k));
                const float4 m1 = __ldg(reinterpret_cast<const float4 *>(m + k + 4));
                v[8 * j + 0] = x0.x - m0.x; v[8 * j + 1] = x0.y - m0.y; v[8 * j + 2] = x0.z - m0.z;
                v[8 * j + 3] = x0.w - m0.w; v[8 * j + 4] = x1.x - m1.x; v[8 * j + 5] = x1.y - m1.y;
                v[8 * j + 6] = x1.z - m1.z; v[8 * j + 7] = x1.w - m1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) v[8 * j + u] = (ok && k + u < ke) ? row[k + u] - m[k + u] : 0.f;
            }
        }
    };
    auto store = [&](unsigned char *dst, const float (&v)[32]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = kh * 32 + 8 * j;
            tc::stage8_planes<NPL>(dst, plane, (uint32_t)(kk >> 4) * slab + tc::canon(r, kk & 15), v + 8 * j);
        }
    };
    float va[32], vc[32];
    if (nch > 0) {
        load(va, xa, ra, kb);
        if (!diag) load(vc, xc, rc, kb);
    }
    // Running totals of this thread's 64 cells (rows quad*32 + lane, columns half*64 .. +63).
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t tcell = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 64);
    float tot[64];
#pragma unroll
    for (int u = 0; u < 64; ++u) tot[u] = 0.f;
    auto fold = [&]() {
#pragma unroll
        for (int c8 = 0; c8 < 64; c8 += 8) {
            float v[8];
            tc::tmem_ld8(tcell + (uint32_t)c8, v);
#pragma unroll
            for (int u = 0; u < 8; ++u) tot[c8 + u] += v[u];
        }
    };
    for (int c = 0; c < nch; ++c) {
        const int sidx = c & 1;
        unsigned char *A = st0 + sidx * stage_b, *Bm = A + opnd;
        if (c >= 2) {
            // the MMAs of chunk c - 2 read this stage
            if (!tc::wait(mbar + sidx, (uint32_t)((c >> 1) + 1) & 1u) && lane == 0) *s_ok = 0;
            __syncwarp();
        }
        if (c % kGcFold == 0 && c > 0) {
            // the partial of chunks c - kGcFold .. c - 1 is complete once chunk c - 1's MMAs are
            uint32_t done = 1u;
            if (lane == 0) done = tc::wait(mbar + ((c - 1) & 1), (uint32_t)(((c - 1) >> 1) & 1)) ? 1u : 0u;
            done = __shfl_sync(0xffffffffu, done, 0);
            if (!done) {
                if (lane == 0) *s_ok = 0;
            } else {
                tc::fence_after();
                fold();
            }
        }
        store(A, va);
        if (!diag) store(Bm, vc);
        // the next chunk's loads are in flight during the barrier and the MMAs
        if (c + 1 < nch) {
            const long long k1 = kb + (long long)(c + 1) * kGcK;
            load(va, xa, ra, k1);
            if (!diag) load(vc, xc, rc, k1);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (!*s_ok) break;
        if (tid == 0) {
            const unsigned char *Bu = diag ? A : Bm;
#pragma unroll 1
            for (int sl = 0; sl < 4; ++sl)
#pragma unroll
                for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                    for (int pb = 0; pa + pb < NPL; ++pb)
                        tc::mma_bf16(tmem, tc::desc(tc::smem_u32(A + pa * plane + sl * slab)),
                                     tc::desc(tc::smem_u32(Bu + pb * plane + sl * slab)), idesc,
                                     (c % kGcFold == 0 && sl == 0 && pa == 0 && pb == 0) ? 0u : 1u);
            tc::commit(mbar + sidx);
        }
    }
    // the last commit covers every earlier MMA
    if (nch > 0 && *s_ok) {
        const int cl = nch - 1;
        if (!tc::wait(mbar + (cl & 1), (uint32_t)(cl >> 1) & 1u) && lane == 0) *s_ok = 0;
        __syncwarp();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const bool ok = *s_ok != 0;
    // epilogue: warp (quad, half) -> rows quad*32 + lane, columns half*64 .. +63
    if (ok && nch > 0) fold();
    float *pt = part + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * 128 * 128 + (long long)(quad * 32 + lane) * 128 +
                half * 64;
#pragma unroll
    for (int u = 0; u < 64; ++u) pt[u] = (ok && nch > 0) ? tot[u] : (nch > 0 ? __int_as_float(0x7fc00000) : 0.f);
    if (!ok && tid == 0 && flag) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 128);
}

// S[a][c] = scale sum over the K splits of the tile partials (FP64), both triangles.
__global__ void k_gram_reduce(const float *__restrict__ part, int n, int nsplit, int ntri, double scale,
                              double *__restrict__ S) {
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)n * n) return;
    const int a = (int)(x / n), c = (int)(x % n);
    const int lo = a < c ? a : c, hi = a < c ? c : a;
    const int ta = lo / 128, tc_ = hi / 128, nt = (n + 127) / 128;
    const int tile = ta * nt - ta * (ta - 1) / 2 + (tc_ - ta);     // row-major upper triangle
    // inside the tile: the row index comes from the tile's first block, the column from its second
    const bool a_row = a / 128 == ta;
    const int ri = a_row ? a % 128 : c % 128, ci = a_row ? c % 128 : a % 128;
    double acc = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) acc += (double)part[((long long)sp * ntri + tile) * 128 * 128 + ri * 128 + ci];
    S[x] = acc * scale;
}

template <int NPL>
static cudaError_t launch_gram_tc_p(const float *X, int n, long long K, const float *m, double scale, double *S,
                                    float *part, int nsplit, unsigned *flag, cudaStream_t st) {
    constexpr size_t smem = 2 * 2 * (size_t)NPL * 4 * 128 * 32 + 64;
    cudaError_t err = cudaFuncSetAttribute(k_gram_tc<NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int nt = (n + 127) / 128, ntri = nt * (nt + 1) / 2;
    const long long kspan = ((K + nsplit - 1) / nsplit + kGcK - 1) / kGcK * kGcK;
    {
        ProfScope _ps("k_gram_tc", st);
        k_gram_tc<NPL><<<dim3((unsigned)ntri, (unsigned)nsplit), 256, smem, st>>>(X, n, K, m, kspan, part, flag);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    {
        ProfScope _ps("k_gram_reduce", st);
        k_gram_reduce<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, st>>>(part, n, nsplit, ntri, scale, S);
    }
    return cudaGetLastError();
}

size_t gram_tc_partial_elems(int n, long long K, int *nsplit) {
    const int nt = (n + 127) / 128, ntri = nt * (nt + 1) / 2;
    // at most 16384 terms per split (each split accumulates in FP32 in TMEM; the splits are
    // summed in FP64), and enough CTAs for four waves
    int ns = (int)((K + 16383) / 16384);
    const int waves = (4 * 152 + ntri - 1) / ntri;
    if (ns < waves) ns = waves;
    const long long maxs = (K + kGcK - 1) / kGcK;
    if (ns > maxs) ns = (int)maxs;
    if (ns < 1) ns = 1;
    *nsplit = ns;
    return (size_t)ns * ntri * 128 * 128;
}

cudaError_t launch_gram_tc(const float *X, int n, long long K, const float *m, double scale, double *S, float *part,
                           int nsplit, unsigned *flag, cudaStream_t st) {
    return launch_gram_tc_p<3>(X, n, K, m, scale, S, part, nsplit, flag, st);
}

static size_t tgemm_genp_smem(int N, int d, int npl) {
    const int nch = (N + kTcK - 1) / kTcK;
    const size_t B = (size_t)npl * 4 * 128 * 32;
    const size_t front = B > (size_t)kEpiBytes ? B : (size_t)kEpiBytes;
    return front + (size_t)nch * npl * kHankelBytes +
           ((size_t)((2 * N + 1) & ~1) + (size_t)N * d + ((size_t)(2 * N - 1) * d + 1) / 2 * 2) * sizeof(float) + 32;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a hop output Y [zs][N][P] (float), 32 x 32 boxes with the 128B swizzle.
static bool hop_output_map(CUtensorMap *tm, float *Y, int N, int P, long long zs) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || P % 4 != 0 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)N, (cuuint64_t)zs};
    const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)P * N * 4};
    const cuuint32_t box[3] = {32, 32, 1}, estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a hop output Y [z][N][P] (float, z = configuration x channel) for the fused
// chain end: boxes of 128 columns x 1 site x 32 channels, no swizzle, zero fill past P.
bool dband_input_map(CUtensorMap *tm, const float *Y, int N, int P, long long zs) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || P % 4 != 0 || zs < 1 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)P, (cuuint64_t)N, (cuuint64_t)zs};
    const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)P * N * 4};
    const cuuint32_t box[3] = {128, 1, 32}, estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(Y), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a cache's link array viewed as rows of d floats (d = 32 or 64): boxes of
// 32 columns x box_rows rows with the 128B swizzle.  Row indices must fit in int.
bool link_rows_map(CUtensorMap *tm, const float *base, unsigned long long rows, int d, int box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || rows == 0 || rows > 0x7fffffffull || (d != 32 && d != 64) || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)d * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows}, estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NPL, int DD>
static cudaError_t launch_tgemm_genp_d(const Geom &g, const float *taps, int P, const float *gtaps, const float *gDm,
                                       long long dm_ss, float *Y, float *band, long long bss, long long brs,
                                       long long bos, int bR, int bns, long long b0, int nb, unsigned *flag,
                                       cudaStream_t st) {
    alignas(64) CUtensorMap tmY;
    if (!Y || bns % 4 != 0 || !hop_output_map(&tmY, Y, g.N, P, (long long)nb * g.d)) return cudaErrorNotSupported;
    const int itiles = (g.N + kTcM - 1) / kTcM, ntiles = (P + 127) / 128;
    const long long ctas = (long long)itiles * nb * g.d;
    const size_t smw = tgemm_genp_ws_smem<NPL>(g.N, g.d);
    if (smw <= 227 * 1024) {
        // one CTA per SM; column tiles per CTA: all of them when the CTAs fill the GPU twice over
        long long cg = (2 * 152 + ctas - 1) / ctas;
        if (cg < 1) cg = 1;
        if (cg > ntiles) cg = ntiles;
        dim3 grid((unsigned)cg, (unsigned)itiles, (unsigned)((long long)nb * g.d));
        cudaError_t err =
            cudaFuncSetAttribute(k_tgemm_genp_ws<NPL, DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
        if (err != cudaSuccess) return err;
        {
            ProfScope _ps("k_tgemm_tc", st);
            k_tgemm_genp_ws<NPL, DD><<<grid, kGwThreads, smw, st>>>(g, taps, P, gtaps, gDm, dm_ss, tmY, band, bss, brs,
                                                                    bos, bR, bns, b0, flag);
        }
        return cudaGetLastError();
    }
    const size_t smem = tgemm_genp_smem(g.N, g.d, NPL);
    // Column tiles per CTA: all of them when there are enough CTAs to fill the GPU twice over.
    long long cg = (2 * 2 * 152 + ctas - 1) / ctas;
    if (cg < 1) cg = 1;
    if (cg > ntiles) cg = ntiles;
    dim3 grid((unsigned)cg, (unsigned)itiles, (unsigned)((long long)nb * g.d));
    cudaError_t err =
        cudaFuncSetAttribute(k_tgemm_genp<NPL, DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_tgemm_tc", st);
        k_tgemm_genp<NPL, DD><<<grid, 256, smem, st>>>(g, taps, P, gtaps, gDm, dm_ss, tmY, band, bss, brs, bos, bR,
                                                       bns, b0, flag);
    }
    return cudaGetLastError();
}

template <int NPL>
static cudaError_t launch_tgemm_genp(const Geom &g, const float *taps, int P, const float *gtaps, const float *gDm,
                                     long long dm_ss, float *Y, float *band, long long bss, long long brs,
                                     long long bos, int bR, int bns, long long b0, int nb, unsigned *flag,
                                     cudaStream_t st) {
    switch (g.d) {
    case 16: return launch_tgemm_genp_d<NPL, 16>(g, taps, P, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb, flag, st);
    case 32: return launch_tgemm_genp_d<NPL, 32>(g, taps, P, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb, flag, st);
    case 64: return launch_tgemm_genp_d<NPL, 64>(g, taps, P, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb, flag, st);
    default: return cudaErrorNotSupported;
    }
}

template <int TN, int NPL>
static size_t tgemm_tc_smem(int N, int d, bool gen) {
    const int nk = (TN + d - 1) / d + 1;
    const size_t stage = gen ? (size_t)32 * d + ((size_t)(32 + nk - 1) * d + 1) / 2 * 2 : 0;
    const size_t ops = (size_t)kNBuf * NPL * (kHankelBytes + 4 * TN * 32);
    const size_t front = ops > (size_t)kEpiBytes ? ops : (size_t)kEpiBytes;
    return front + ((size_t)((2 * N + 1) & ~1) + stage) * sizeof(float) + 32;
}

template <int TN, int NPL>
static cudaError_t launch_tgemm_tc_tn(const Geom &g, const float *taps, int P, const float *X, const float *gtaps,
                                      const float *gDm, long long dm_ss, float *Y, float *band, long long bss,
                                      long long brs, long long bos, int bR, int bns, long long b0, int nb,
                                      unsigned *flag, cudaStream_t st) {
    const size_t smem = tgemm_tc_smem<TN, NPL>(g.N, g.d, gtaps != nullptr);
    if (smem > 220 * 1024) return cudaErrorNotSupported;
    dim3 grid((P + TN - 1) / TN, (g.N + kTcM - 1) / kTcM, (unsigned)nb * g.d);
    cudaError_t err;
    if (gtaps) {
        err = cudaFuncSetAttribute(k_tgemm_tc<true, TN, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm_tc", st);
        k_tgemm_tc<true, TN, NPL><<<grid, 256, smem, st>>>(g, taps, P, nullptr, gtaps, gDm, dm_ss, Y, band, bss, brs,
                                                             bos, bR, bns, b0, flag);
    } else {
        err = cudaFuncSetAttribute(k_tgemm_tc<false, TN, NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm_tc", st);
        k_tgemm_tc<false, TN, NPL><<<grid, 256, smem, st>>>(g, taps, P, X, nullptr, nullptr, 0, Y, band, bss, brs,
                                                              bos, bR, bns, b0, flag);
    }
    return cudaGetLastError();
}

// 128-column tiles, 128 TMEM columns per CTA, 3 CTAs per SM.  planes = BF16 terms per
// operand value: 1 (plain BF16), 2 (3 products, about 2^-18 relative), 3 (6 products,
// FP32-grade).
cudaError_t launch_tgemm_tc(const Geom &g, const float *taps, int P, const float *X, const float *gtaps,
                            const float *gDm, long long dm_ss, float *Y, float *band, long long bss, long long brs,
                            long long bos, int bR, int bns, long long b0, int nb, unsigned *flag, cudaStream_t st,
                            int planes) {
    // Generated operand with the whole chain in shared memory: the persistent kernel.
    if (gtaps && g.N <= kGpMaxChunks * kTcK && g.d <= 64 && 128 % g.d == 0 && (planes == 1 || planes == 2) &&
        tgemm_genp_smem(g.N, g.d, planes) <= 110 * 1024) {
        const cudaError_t e = planes == 1 ? launch_tgemm_genp<1>(g, taps, P, gtaps, gDm, dm_ss, Y, band, bss, brs, bos,
                                                                 bR, bns, b0, nb, flag, st)
                                          : launch_tgemm_genp<2>(g, taps, P, gtaps, gDm, dm_ss, Y, band, bss, brs, bos,
                                                                 bR, bns, b0, nb, flag, st);
        if (e != cudaErrorNotSupported) return e;
    }
    switch (planes) {
    case 1:
        return launch_tgemm_tc_tn<128, 1>(g, taps, P, X, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb,
                                          flag, st);
    case 2:
        return launch_tgemm_tc_tn<128, 2>(g, taps, P, X, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb,
                                          flag, st);
    case 3:
        return launch_tgemm_tc_tn<128, 3>(g, taps, P, X, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb,
                                          flag, st);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace dn
