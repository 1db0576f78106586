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
// offset).  One thread issues the MMAs (M=128, N=256, K=16 each) and commits
// them to an mbarrier; every wait is bounded, and a timeout raises bit 8 of the
// error flag, skips the epilogue and still releases the tensor memory.
#include <cuda_bf16.h>

#include "dn_internal.cuh"

namespace dn {

namespace {

constexpr int kTcM = 128, kTcK = 64;     // K staged 64 sites (4 MMA slabs) at a time
constexpr int kSlabA = kTcM * 16 * 2;    // bytes per 16-wide K slab of A (B: TN * 32)
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

// Eight consecutive K values of one row -> their BF16 hi and lo parts, one 16-byte store each.
__device__ __forceinline__ void split_store8(unsigned char *hi, unsigned char *lo, uint32_t off, const float *v) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        h[u] = __float2bfloat16_rn(v[u]);
        l[u] = __float2bfloat16_rn(v[u] - __bfloat162float(h[u]));
    }
    *reinterpret_cast<uint4 *>(hi + off) = *reinterpret_cast<const uint4 *>(h);
    *reinterpret_cast<uint4 *>(lo + off) = *reinterpret_cast<const uint4 *>(l);
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

template <bool GEN, int TN>
__global__ void __launch_bounds__(256) k_tgemm_tc(Geom g, const float *__restrict__ taps, int P,
                                                  const float *__restrict__ X, const float *__restrict__ gtaps,
                                                  const float *__restrict__ gDm, long long dm_ss, float *__restrict__ Y,
                                                  float *__restrict__ band, long long bss, long long brs, long long bos,
                                                  int bR, int bns, long long b0, unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smtc[];
    constexpr int kTcN = TN, kSlabB = TN * 16 * 2, kTpc = 256 / TN;   // threads per B column
    const int N = g.N, d = g.d;
    unsigned char *Ahi = smtc;                            // 4 slabs x kSlabA
    unsigned char *Alo = Ahi + 4 * kSlabA;
    unsigned char *Bhi = Alo + 4 * kSlabA;                // 4 slabs x kSlabB
    unsigned char *Blo = Bhi + 4 * kSlabB;
    float *gx = reinterpret_cast<float *>(Blo + 4 * kSlabB);   // taps of channel a: gx[r + N - 1]
    float *Dms = gx + ((2 * N + 1) & ~1);                       // [32][d]   (generated operand only)
    float *Tps = Dms + (GEN ? 32 * d : 0);                      // [32 + nk - 1][d]
    const int nk = (kTcN + d - 1) / d + 1;                      // source sites a column tile touches
    const bool gstage = GEN && (kTcN % d == 0) && d <= 64;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Tps + (GEN ? ((32 + nk - 1) * d + 1) / 2 * 2 : 0));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * kTcN, i0 = blockIdx.y * kTcM;
    const long long za = blockIdx.z;
    const int a = (int)(za % d);
    const long long bl = za / d;
    for (int q = tid; q < 2 * N - 1; q += blockDim.x) gx[q] = taps[(long long)tap_row_tc(q - (N - 1), N, g.periodic) * d + a];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
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
    bool ok = true;
    uint32_t phase = 0;
    const int nchunks = (N + kTcK - 1) / kTcK;
    for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int n0 = ch * kTcK;
        if (ch > 0) {
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();           // the previous chunk's MMAs have completed (waited below)
        }
        // A: Toeplitz rows i0..i0+127, sites n0..n0+63; a task is one row and 8 sites.
        for (int q = tid; q < kTcM * (kTcK / 8); q += blockDim.x) {
            const int r = q % kTcM, kc = q / kTcM;
            const int i = i0 + r;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int n = n0 + kc * 8 + u;
                v[u] = (i < N && n < N) ? gx[i - n + N - 1] : 0.f;
            }
            split_store8(Ahi, Alo, (uint32_t)(kc >> 1) * kSlabA + canon(r, (kc & 1) * 8), v);
        }
        if (GEN && gstage) {
            // Generated operand: the vertex rows D0_n[a][:] and the tap rows g_{n-k} the tile needs
            // are staged in shared memory (coalesced), 32 sites at a time.
            for (int h = 0; h < kTcK; h += 32) {
                __syncthreads();
                for (int q = tid; q < 32 * d; q += blockDim.x) {
                    const int nn = q / d, cc = q % d, n = n0 + h + nn;
                    Dms[q] = n < N ? gDm[bl * dm_ss + ((long long)n * d + a) * d + cc] : 0.f;
                }
                const int rmin = n0 + h - (kfirst + nk - 1), nrow = 32 + nk - 1;
                for (int q = tid; q < nrow * d; q += blockDim.x) {
                    const int rr = q / d, cc = q % d, r = rmin + rr;
                    Tps[q] = (r > -N && r < N) ? gtaps[(long long)tap_row_tc(r, N, g.periodic) * d + cc] : 0.f;
                }
                __syncthreads();
#pragma unroll
                for (int kx = 0; kx < 4 / kTpc; ++kx) {
                    const int kc = part * (4 / kTpc) + kx;
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int nn = kc * 8 + u, n = n0 + h + nn;
                        v[u] = (pok && n < N) ? Dms[nn * d + cq] * Tps[(n - kq - rmin) * d + cq] : 0.f;
                    }
                    const int kk = h + kc * 8;
                    split_store8(Bhi, Blo, (uint32_t)(kk >> 4) * kSlabB + canon(pp, kk & 15), v);
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
                const int kk = part * KS + kc * 8;
                split_store8(Bhi, Blo, (uint32_t)(kk >> 4) * kSlabB + canon(pp, kk & 15), v + 8 * kc);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int s = 0; s < kTcK / 16; ++s) {
                const uint64_t ah = umma_desc(sm_u32(Ahi + s * kSlabA)), al = umma_desc(sm_u32(Alo + s * kSlabA));
                const uint64_t bh = umma_desc(sm_u32(Bhi + s * kSlabB)), blo = umma_desc(sm_u32(Blo + s * kSlabB));
                const uint32_t first = (ch == 0 && s == 0) ? 0u : 1u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ah), "l"(bh), "r"(idesc), "r"(first));
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ah), "l"(blo), "r"(idesc), "r"(1u));
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(al), "l"(bh), "r"(idesc), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(mbar)));
        }
        if (!tc_wait(mbar, phase)) ok = false;
        phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!ok) {
        if (tid == 0) atomicOr(flag, 8u);
    } else {
        // Epilogue: warp w owns TMEM lanes 32 (w % 4).. (rows) and columns 128 (w / 4)..; each
        // 32 x 32 piece goes through shared memory (the operand buffers are free now) so that a
        // lane then owns a column and the global stores of a row are contiguous.
        const int quad = warp & 3, half = warp >> 2;
        float *stage = reinterpret_cast<float *>(smtc) + warp * (32 * 33);
        const int prow0 = i0 + quad * 32;
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
            if (p < P) {
                const int k = p / bns, cc = p - k * bns;
                for (int rr = 0; rr < 32; ++rr) {
                    const int i = prow0 + rr;
                    if (i >= N) break;
                    const float v = stage[rr * 33 + lane];
                    if (Y) Y[((bl * d + a) * N + i) * (long long)P + p] = v;
                    if (band) {
                        const int dl = ring_delta_tc(i - k, N, g.periodic);
                        if (dl >= -bR && dl <= bR)
                            band[(b0 + bl) * bss + (long long)i * brs + (long long)(bR - dl) * bos + (long long)a * bns + cc] = v;
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

template <int TN>
static size_t tgemm_tc_smem(int N, int d, bool gen) {
    const int nk = (TN + d - 1) / d + 1;
    const size_t stage = gen ? (size_t)32 * d + ((size_t)(32 + nk - 1) * d + 1) / 2 * 2 : 0;
    return (size_t)8 * kSlabA + (size_t)8 * TN * 32 + ((size_t)((2 * N + 1) & ~1) + stage) * sizeof(float) + 16;
}

template <int TN>
static cudaError_t launch_tgemm_tc_tn(const Geom &g, const float *taps, int P, const float *X, const float *gtaps,
                                      const float *gDm, long long dm_ss, float *Y, float *band, long long bss,
                                      long long brs, long long bos, int bR, int bns, long long b0, int nb,
                                      unsigned *flag, cudaStream_t st) {
    const size_t smem = tgemm_tc_smem<TN>(g.N, g.d, gtaps != nullptr);
    if (smem > 220 * 1024) return cudaErrorNotSupported;
    dim3 grid((P + TN - 1) / TN, (g.N + kTcM - 1) / kTcM, (unsigned)nb * g.d);
    cudaError_t err;
    if (gtaps) {
        err = cudaFuncSetAttribute(k_tgemm_tc<true, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm_tc", st);
        k_tgemm_tc<true, TN><<<grid, 256, smem, st>>>(g, taps, P, nullptr, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR,
                                                      bns, b0, flag);
    } else {
        err = cudaFuncSetAttribute(k_tgemm_tc<false, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm_tc", st);
        k_tgemm_tc<false, TN><<<grid, 256, smem, st>>>(g, taps, P, X, nullptr, nullptr, 0, Y, band, bss, brs, bos, bR,
                                                       bns, b0, flag);
    }
    return cudaGetLastError();
}

// 128-column tiles (3 CTAs per SM: 64 KB of operands, 128 TMEM columns each).
cudaError_t launch_tgemm_tc(const Geom &g, const float *taps, int P, const float *X, const float *gtaps,
                            const float *gDm, long long dm_ss, float *Y, float *band, long long bss, long long brs,
                            long long bos, int bR, int bns, long long b0, int nb, unsigned *flag, cudaStream_t st) {
    return launch_tgemm_tc_tn<128>(g, taps, P, X, gtaps, gDm, dm_ss, Y, band, bss, brs, bos, bR, bns, b0, nb, flag, st);
}

}  // namespace dn
