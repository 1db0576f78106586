// Forward pass on the tcgen05 tensor cores (the BF16 precision, d a multiple of 16,
// d <= 128; the kernels also take 2 or 3 BF16 planes per operand value).
//
// Activations are kept channel-major, h[c][r] with row r = n B + b, so that both
// contractions of a layer are plain GEMMs over coalesced rows:
//  * the S4 convolution u = G^(l) h (Sec. "Architecture", a channel-diagonal
//    Toeplitz operator) is the Toeplitz GEMM of the link build with the samples as
//    columns (k_tgemm_tc);
//  * the channel mixing and gate y = V u, h' = U (chi . y) (Eq. for h^(l)) is
//    k_mix_tc below: two chained MMAs per 128-row tile, the gate applied in the
//    epilogue of the first and fed back through shared memory as the A operand of
//    the second; y is written to the cache on the way.
// With NPL planes per operand value the products of planes pa + pb < NPL are
// accumulated in FP32; BF16 precision uses NPL = 1.  Pooled readout sums are
// accumulated in FP64.
#include "dn_internal.cuh"
#include "tc_common.cuh"

namespace dn {

namespace {

__host__ __device__ inline uint32_t tmem_cols_for(int n) {
    uint32_t c = 32;
    while (c < (uint32_t)n) c <<= 1;
    return c;
}

}  // namespace

// h0[c][n B + b] = e_c sigma_{b,n}
__global__ void k_h0_cm(int d, int N, int B, const int8_t *__restrict__ spins, const float *__restrict__ e,
                        float *__restrict__ h) {
    const long long R = (long long)N * B;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < R * d; x += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(x / R);
        const long long r = x - (long long)c * R;
        const int n = (int)(r / B), b = (int)(r - (long long)n * B);
        h[x] = e[c] * (float)spins[(long long)b * N + n];
    }
}

// pooled[b][l][c] = sum_n omega_{n,c} h[c][n B + b] (readout sums of layer l, FP64 result).
__global__ void k_pool_cm(int d, int N, int B, int l, const float *__restrict__ h, const float *__restrict__ omega,
                          double *__restrict__ pooled, long long pstride) {
    const long long R = (long long)N * B;
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)d * B) return;
    const int c = (int)(x / B), b = (int)(x - (long long)c * B);
    const float *hc = h + (long long)c * R + b;
    // products and partial sums of 16 sites in FP32, the partials added in FP64 (FP64
    // arithmetic is slow on this part; 16-term partials are far inside the BF16 error)
    double s = 0.0;
    for (int n0 = 0; n0 < N; n0 += 16) {
        float p = 0.f;
        const int n1 = n0 + 16 < N ? n0 + 16 : N;
        for (int n = n0; n < n1; ++n) p = fmaf(omega[(long long)n * d + c], hc[(long long)n * B], p);
        s += (double)p;
    }
    pooled[(long long)b * pstride + (long long)l * d + c] = s;
}

// y = V u, h' = U (chi . y) for 128 rows r = n B + b; u, h' channel-major [d][R];
// chi, y sample-major caches [B][L][N][d] (y may be null).  One thread per row.
template <int NPL>
__global__ void __launch_bounds__(128) k_mix_tc(int d, int N, int B, int L, int l, const float *__restrict__ V,
                                                const float *__restrict__ U, const float *__restrict__ ucm,
                                                const float *__restrict__ chi, float *__restrict__ y,
                                                float *__restrict__ hcm, unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smx[];
    const int ns = d / 16;
    const long long R = (long long)N * B;
    const uint32_t wslab = (uint32_t)d * 32, aslab = 128 * 32;
    const uint32_t wplane = ns * wslab, aplane = ns * aslab;
    unsigned char *Vp = smx;                     // NPL planes, B operand of MMA 1 (rows c, K a)
    unsigned char *Up = Vp + NPL * wplane;       // NPL planes, B operand of MMA 2 (rows c', K c)
    unsigned char *Ap = Up + NPL * wplane;       // NPL planes, A operand (u, then chi . y)
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Ap + NPL * aplane);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long r = (long long)blockIdx.x * 128 + tid;
    const bool valid = r < R;
    const uint32_t cols = tmem_cols_for(2 * d);
    const int d8 = d / 8;
    for (int q = tid; q < d * d8; q += blockDim.x) {
        const int c = q / d8, k8 = (q - c * d8) * 8;
        const uint32_t off = (uint32_t)(k8 >> 4) * wslab + tc::canon(c, k8 & 15);
        tc::stage8_planes<NPL>(Vp, wplane, off, V + (long long)c * d + k8);
        tc::stage8_planes<NPL>(Up, wplane, off, U + (long long)c * d + k8);
    }
    for (int k8 = 0; k8 < d; k8 += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = valid ? ucm[(long long)(k8 + u) * R + r] : 0.f;
        tc::stage8_planes<NPL>(Ap, aplane, (uint32_t)(k8 >> 4) * aslab + tc::canon(tid, k8 & 15), v);
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, cols);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, d);
    auto gemm = [&](uint32_t dst, const unsigned char *bw) {
        for (int s = 0; s < ns; ++s)
#pragma unroll
            for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                for (int pb = 0; pa + pb < NPL; ++pb)
                    tc::mma_bf16(dst, tc::desc(tc::smem_u32(Ap + pa * aplane + s * aslab)),
                                 tc::desc(tc::smem_u32(bw + pb * wplane + s * wslab)), idesc,
                                 (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
        tc::commit(mbar);
    };
    if (tid == 0) gemm(tmem, Vp);
    if (warp == 0 && !tc::wait(mbar, 0) && (tid & 31) == 0) *s_ok = 0;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const int n = (int)(r / B), b = (int)(r - (long long)n * B);
    const long long crow = (((long long)b * L + (l - 1)) * N + n) * d;
    if (*s_ok) {
        // Epilogue 1: y to the cache, z = chi . y back into the A operand.
        for (int c8 = 0; c8 < d; c8 += 8) {
            float yv[8], z[8];
            tc::tmem_ld8(lane_base + (uint32_t)c8, yv);
            if (valid) {
                const float4 x0 = *reinterpret_cast<const float4 *>(chi + crow + c8);
                const float4 x1 = *reinterpret_cast<const float4 *>(chi + crow + c8 + 4);
                if (y) {
                    *reinterpret_cast<float4 *>(y + crow + c8) = make_float4(yv[0], yv[1], yv[2], yv[3]);
                    *reinterpret_cast<float4 *>(y + crow + c8 + 4) = make_float4(yv[4], yv[5], yv[6], yv[7]);
                }
                z[0] = x0.x * yv[0]; z[1] = x0.y * yv[1]; z[2] = x0.z * yv[2]; z[3] = x0.w * yv[3];
                z[4] = x1.x * yv[4]; z[5] = x1.y * yv[5]; z[6] = x1.z * yv[6]; z[7] = x1.w * yv[7];
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) z[u] = 0.f;
            }
            tc::stage8_planes<NPL>(Ap, aplane, (uint32_t)(c8 >> 4) * aslab + tc::canon(tid, c8 & 15), z);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) gemm(tmem + (uint32_t)d, Up);
        if (warp == 0 && !tc::wait(mbar, 1) && (tid & 31) == 0) *s_ok = 0;
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    // Epilogue 2 (a timed-out tile writes NaN, so the error reaches the outputs).
    const bool ok = *s_ok != 0;
    for (int c8 = 0; c8 < d; c8 += 8) {
        float hv[8];
        if (ok) tc::tmem_ld8(lane_base + (uint32_t)(d + c8), hv);
        if (valid)
#pragma unroll
            for (int u = 0; u < 8; ++u) hcm[(long long)(c8 + u) * R + r] = ok ? hv[u] : __int_as_float(0x7fc00000);
    }
    if (!ok && tid == 0 && flag) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, cols);
}

// Persistent form of k_mix_tc for d in {16, 32, 64}: a CTA stages V and U once and loops over
// row tiles; the u rows of its next tile are loaded into registers while the current tile
// is staged, multiplied and written, and the tile's chi rows are loaded before its first MMA
// is waited for.  Same products, order and outputs as k_mix_tc.
template <int NPL, int D>
__global__ void __launch_bounds__(128) k_mix_tcp(int N, int B, int L, int l, const float *__restrict__ V,
                                                 const float *__restrict__ U, const float *__restrict__ ucm,
                                                 const float *__restrict__ chi, float *__restrict__ y,
                                                 float *__restrict__ hcm, unsigned *__restrict__ flag) {
    extern __shared__ __align__(1024) unsigned char smx[];
    constexpr int d = D, ns = D / 16;
    const long long R = (long long)N * B;
    constexpr uint32_t wslab = (uint32_t)D * 32, aslab = 128 * 32;
    constexpr uint32_t wplane = ns * wslab, aplane = ns * aslab;
    unsigned char *Vp = smx;
    unsigned char *Up = Vp + NPL * wplane;
    unsigned char *Ap = Up + NPL * wplane;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Ap + NPL * aplane);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_ok = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr uint32_t cols = D * 2 <= 32 ? 32 : (D * 2 <= 64 ? 64 : 128);
    constexpr int d8 = D / 8;
    for (int q = tid; q < D * d8; q += blockDim.x) {
        const int c = q / d8, k8 = (q - c * d8) * 8;
        const uint32_t off = (uint32_t)(k8 >> 4) * wslab + tc::canon(c, k8 & 15);
        tc::stage8_planes<NPL>(Vp, wplane, off, V + (long long)c * d + k8);
        tc::stage8_planes<NPL>(Up, wplane, off, U + (long long)c * d + k8);
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, cols);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, D);
    auto gemm = [&](uint32_t dst, const unsigned char *bw) {
        for (int s = 0; s < ns; ++s)
#pragma unroll
            for (int pa = 0; pa < NPL; ++pa)
#pragma unroll
                for (int pb = 0; pa + pb < NPL; ++pb)
                    tc::mma_bf16(dst, tc::desc(tc::smem_u32(Ap + pa * aplane + s * aslab)),
                                 tc::desc(tc::smem_u32(bw + pb * wplane + s * wslab)), idesc,
                                 (s == 0 && pa == 0 && pb == 0) ? 0u : 1u);
        tc::commit(mbar);
    };
    auto load_u = [&](float (&buf)[D], long long t) {
        const long long r = t * 128 + tid;
        const bool ok = r < R;
#pragma unroll
        for (int u = 0; u < D; ++u) buf[u] = ok ? ucm[(long long)u * R + (ok ? r : 0)] : 0.f;
    };
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const long long ntiles = (R + 127) / 128;
    float un[D];
    if ((long long)blockIdx.x < ntiles) load_u(un, blockIdx.x);
    uint32_t phase = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long r = t * 128 + tid;
        const bool valid = r < R;
#pragma unroll
        for (int k8 = 0; k8 < D; k8 += 8)
            tc::stage8_planes<NPL>(Ap, aplane, (uint32_t)(k8 >> 4) * aslab + tc::canon(tid, k8 & 15), un + k8);
        if (t + gridDim.x < ntiles) load_u(un, t + gridDim.x);
        const int n = (int)(r / B), b = (int)(r - (long long)n * B);
        const long long crow = (((long long)b * L + (l - 1)) * N + n) * d;
        float xc[D];
#pragma unroll
        for (int c4 = 0; c4 < D; c4 += 4) {
            const float4 x = valid ? *reinterpret_cast<const float4 *>(chi + crow + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
            xc[c4] = x.x; xc[c4 + 1] = x.y; xc[c4 + 2] = x.z; xc[c4 + 3] = x.w;
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) gemm(tmem, Vp);
        if (warp == 0 && !tc::wait(mbar, phase) && (tid & 31) == 0) *s_ok = 0;
        phase ^= 1u;
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        ok = *s_ok != 0;
        if (ok) {
            // Epilogue 1: y to the cache, z = chi . y back into the A operand.
#pragma unroll
            for (int c8 = 0; c8 < D; c8 += 8) {
                float yv[8], z[8];
                tc::tmem_ld8(lane_base + (uint32_t)c8, yv);
                if (valid && y) {
                    *reinterpret_cast<float4 *>(y + crow + c8) = make_float4(yv[0], yv[1], yv[2], yv[3]);
                    *reinterpret_cast<float4 *>(y + crow + c8 + 4) = make_float4(yv[4], yv[5], yv[6], yv[7]);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) z[u] = valid ? xc[c8 + u] * yv[u] : 0.f;
                tc::stage8_planes<NPL>(Ap, aplane, (uint32_t)(c8 >> 4) * aslab + tc::canon(tid, c8 & 15), z);
            }
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) gemm(tmem + (uint32_t)D, Up);
            if (warp == 0 && !tc::wait(mbar, phase) && (tid & 31) == 0) *s_ok = 0;
            phase ^= 1u;
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            ok = *s_ok != 0;
        }
        // Epilogue 2 (a timed-out tile writes NaN, so the error reaches the outputs).
#pragma unroll
        for (int c8 = 0; c8 < D; c8 += 8) {
            float hv[8];
            if (ok) tc::tmem_ld8(lane_base + (uint32_t)(D + c8), hv);
            if (valid)
#pragma unroll
                for (int u = 0; u < 8; ++u) hcm[(long long)(c8 + u) * R + r] = ok ? hv[u] : __int_as_float(0x7fc00000);
        }
        // the next tile overwrites the A operand and the accumulators
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (!ok) break;
    }
    if (!ok && tid == 0 && flag) atomicOr(flag, 8u);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, cols);
}

bool forward_tc_ok(const Geom &g) { return g.d % 16 == 0 && g.d >= 16 && g.d <= 128; }

cudaError_t launch_h0_cm(const Geom &g, const int8_t *spins, const float *e, int B, float *h, cudaStream_t st) {
    const long long n = (long long)g.N * B * g.d;
    const int blocks = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    {
        ProfScope _ps("k_h0_cm", st);
        k_h0_cm<<<blocks, 256, 0, st>>>(g.d, g.N, B, spins, e, h);
    }
    return cudaGetLastError();
}

cudaError_t launch_pool_cm(const Geom &g, int l, const float *h, const float *omega, int B, double *pooled,
                           long long pstride, cudaStream_t st) {
    const long long n = (long long)g.d * B;
    {
        ProfScope _ps("k_pool_cm", st);
        k_pool_cm<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g.d, g.N, B, l, h, omega, pooled, pstride);
    }
    return cudaGetLastError();
}

template <int NPL>
static cudaError_t launch_mix_tc_p(const Geom &g, int l, const float *V, const float *U, const float *ucm,
                                   const float *chi, float *y, float *hcm, int B, unsigned *flag, cudaStream_t st) {
    const int d = g.d, ns = d / 16;
    const size_t smem = (size_t)NPL * (2 * ns * d * 32 + ns * 128 * 32) + 32;
    const long long R = (long long)g.N * B;
    const unsigned grid = (unsigned)((R + 127) / 128);
    if (d == 16 || d == 32 || d == 64) {
        // persistent: up to three CTAs per SM (shared memory and registers)
        const unsigned pgrid = grid < 3 * 152 ? grid : 3 * 152;
        cudaError_t err;
        auto go = [&](auto kern) {
            err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return;
            ProfScope _ps("k_mix_tc", st);
            kern<<<pgrid, 128, smem, st>>>(g.N, B, g.L, l, V, U, ucm, chi, y, hcm, flag);
            err = cudaGetLastError();
        };
        if (d == 16) go(k_mix_tcp<NPL, 16>);
        else if (d == 32) go(k_mix_tcp<NPL, 32>);
        else go(k_mix_tcp<NPL, 64>);
        return err;
    }
    cudaError_t err = cudaFuncSetAttribute(k_mix_tc<NPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps("k_mix_tc", st);
        k_mix_tc<NPL><<<grid, 128, smem, st>>>(d, g.N, B, g.L, l, V, U, ucm, chi, y, hcm, flag);
    }
    return cudaGetLastError();
}

cudaError_t launch_mix_tc(const Geom &g, int l, const Weights<float> &w, const float *ucm, const float *chi, float *y,
                          float *hcm, int B, int planes, unsigned *flag, cudaStream_t st) {
    if (!forward_tc_ok(g)) return cudaErrorNotSupported;
    const long long dd = (long long)g.d * g.d;
    const float *V = w.V + (long long)(l - 1) * dd, *U = w.U + (long long)(l - 1) * dd;
    switch (planes) {
    case 1: return launch_mix_tc_p<1>(g, l, V, U, ucm, chi, y, hcm, B, flag, st);
    case 2: return launch_mix_tc_p<2>(g, l, V, U, ucm, chi, y, hcm, B, flag, st);
    case 3: return launch_mix_tc_p<3>(g, l, V, U, ucm, chi, y, hcm, B, flag, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dn
