// Helpers for the hand-written tcgen05 kernels (sm_103a): shared-memory matrix
// descriptors for the no-swizzle K-major canonical layout, BF16 operand staging
// (plain or split into hi + lo for FP32-accurate products), MMA issue, commit and
// bounded mbarrier waits, and tensor-memory loads.
//
// Canonical layout of one 16-wide K slab of an R-row operand: 8-row x 16-byte core
// matrices, the two K-adjacent cores of a row group 128 B apart (leading byte
// offset) and consecutive row groups 256 B apart (stride byte offset); a slab takes
// R * 32 bytes.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace dn {
namespace tc {

constexpr long kSpin = 1L << 24;   // bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo = 128, uint32_t sbo = 256) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (row r, k within a 16-wide slab) in the canonical layout.
__device__ __forceinline__ uint32_t canon(int r, int k16) {
    return (uint32_t)((r >> 3) * 256 + (k16 >> 3) * 128 + (r & 7) * 16 + (k16 & 7) * 2);
}

// Instruction descriptor: BF16 A and B, FP32 accumulation, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Eight consecutive K values of one row -> BF16 hi (and, with lo != null, the BF16
// rounding of the remainder), one 16-byte store each.
__device__ __forceinline__ void stage8(unsigned char *hi, unsigned char *lo, uint32_t off, const float *v) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        h[u] = __float2bfloat16_rn(v[u]);
        l[u] = __float2bfloat16_rn(v[u] - __bfloat162float(h[u]));
    }
    *reinterpret_cast<uint4 *>(hi + off) = *reinterpret_cast<const uint4 *>(h);
    if (lo) *reinterpret_cast<uint4 *>(lo + off) = *reinterpret_cast<const uint4 *>(l);
}

// Eight consecutive K values of one row split into NPL BF16 planes
// (v = p0 + p1 + p2 + remainder, each plane the BF16 rounding of what is left),
// plane p at base + p * pstride + off.  Products of planes pa, pb with
// pa + pb <= NPL - 1 reproduce the FP32 product to about 2^-(9 NPL) relative.
template <int NPL>
__device__ __forceinline__ void stage8_planes(unsigned char *base, uint32_t pstride, uint32_t off, const float *v) {
    float r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = v[u];
#pragma unroll
    for (int p = 0; p < NPL; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // one conversion rounds a pair (element 2i in the low half, as in memory)
            const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t *>(&h);
            if (p + 1 < NPL) {
                r[2 * i] -= __low2float(h);
                r[2 * i + 1] -= __high2float(h);
            }
        }
        *reinterpret_cast<uint4 *>(base + p * pstride + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ bool wait(uint64_t *mbar, uint32_t parity) {
    uint32_t done = 0;
    for (long it = 0; it < kSpin; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(mbar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Warp-wide (warp 0): allocate / release `cols` tensor-memory columns (a power of two >= 32).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// Eight consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Issue a load of 8 columns into raw registers without waiting; tmem_wait_ld() waits for
// every load issued before it, after which the registers may be read.
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t *r, int n) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // the registers are live across the wait: a no-op that ties them to it
    for (int j = 0; j < n; ++j) asm volatile("" : "+r"(r[j]));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tc
}  // namespace dn
