// Interlayer link tensors (Eq. Lmn; App. "Exact algorithm to construct link
// tensors", Eqs. B_def, X_def, L_def) by exact propagation of unit sources.
//
// A source is placed at the output of layer m at site k:
//   m = 0:  the embedding e at site k          (P = N sources per sample, p = k);
//   m >= 1: the unit vector e_c' at site k     (P = N d sources, p = k d + c').
// The sources of one sample form a matrix X with rows (channel a, site n) and
// columns p, stored channel-major [a][n][p].  Propagation through the frozen
// background B^(n) = D0^(n) G^(n) is two GEMMs per layer:
//   Toeplitz hop  Y[a] = T^(n)_a X[a]            T_a[i][j] = g^(n)_{i-j,a}: an
//                                                  N x N by N x P product per channel
//   vertex hop    X[:, i, :] = D0^(n)_i Y[:, i, :]  a d x d by d x P product per site
// After every G^(l) with l >= m+2 the band rows |i - k| <= R of Y are stored:
//   m = 0  -> ell^(l)_{i,k}        = [G^(l) X_{1,l-1} (e delta_k)]_i
//   m >= 1 -> L^(l,m)_{i,k}[:, c'] = [G^(l) X_{m+1,l-1} (e_c' delta_k)]_i
// For m >= 1 the first G is the analytic kernel column, so the first hop's
// input X[a][n][(k,c')] = D0^(m+1)_n[a][c'] g^(m+1)_{n-k,c'} is generated inside
// the kernel that consumes it; the last layer's G is evaluated on the band only.
#include "dn_internal.cuh"

namespace dn {

__device__ __forceinline__ int tap_row(int r, int N, int periodic) {
    return periodic ? (r < 0 ? r + N : (r >= N ? r - N : r)) : r + N - 1;
}

// Site offset i - k reduced to (-N/2, N/2] on a ring.
__device__ __forceinline__ int ring_delta(int dl, int N, int periodic) {
    if (periodic) {
        if (dl > N / 2) dl -= N;
        else if (dl <= -((N + 1) / 2)) dl += N;
    }
    return dl;
}

// Where band rows go: element (sample b, row i, offset o = R - (i - k), output
// channel a, source channel c') is base[b*ss + i*rs + o*os + a*nsrc + c'].
struct BandDst {
    long long ss, rs, os;
    int R, nsrc;
};

// Generated first-hop input (sources at layer m >= 1): X[a][n][k d + c'] =
// D0^(m+1)_n[a][c'] g^(m+1)_{n-k,c'}.
template <typename T>
struct GenSrc {
    const T *taps;   // layer m+1 taps [R][d]
    const T *Dm;     // D0^(m+1) of sample 0 of the chunk: [n][a][c'], sample stride dm_ss
    long long dm_ss;
};

template <typename T>
__device__ __forceinline__ T gen_x(const GenSrc<T> &gs, int N, int d, int periodic, long long bl, int a, int n, int p) {
    const int k = p / d, c = p - k * d;
    return gs.Dm[bl * gs.dm_ss + ((long long)n * d + a) * d + c] * gs.taps[(long long)tap_row(n - k, N, periodic) * d + c];
}

// ------------------------------------------------------------ site vertices --
// Dm[b][l-1][n] = U diag(chi_n) V (row-major d x d) for layers 1..L-1.  One CTA per
// (sample, layer, tile of kDmTile sites): U, V and the tile's chi (transposed, [e][site])
// are staged in shared memory; a thread owns output entries (a, c) and forms
// U[a][e] V[e][c] once per e for all sites of the tile.
constexpr int kDmTile = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_dmat(Geom g, Weights<T> w, const T *__restrict__ chi, long long b0,
                                              T *__restrict__ Dm) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, L = g.L;
    const long long dd = (long long)d * d;
    T *Us = reinterpret_cast<T *>(smraw);     // [a][e]
    T *Vs = Us + dd;                          // [e][c]
    T *xs = Vs + dd;                          // [e][kDmTile]
    const int ntile = (N + kDmTile - 1) / kDmTile;
    const long long blk = blockIdx.x;
    const int n0 = (int)(blk % ntile) * kDmTile;
    const int l = (int)((blk / ntile) % (L - 1)) + 1;
    const long long bl = blk / ((long long)ntile * (L - 1));
    const int ns = N - n0 < kDmTile ? N - n0 : kDmTile;
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        Us[q] = w.U[(l - 1) * dd + q];
        Vs[q] = w.V[(l - 1) * dd + q];
    }
    const T *x = chi + (((b0 + bl) * L + (l - 1)) * N + n0) * d;
    for (int q = threadIdx.x; q < kDmTile * d; q += blockDim.x) {
        const int s = q / d, e = q % d;
        xs[e * kDmTile + s] = s < ns ? x[(long long)s * d + e] : (T)0;
    }
    __syncthreads();
    T *dst = Dm + ((bl * (L - 1) + (l - 1)) * N + n0) * dd;
    for (int q = threadIdx.x; q < dd; q += blockDim.x) {
        const int a = q / d, c = q % d;
        T acc[kDmTile];
#pragma unroll
        for (int s = 0; s < kDmTile; ++s) acc[s] = 0;
        for (int e = 0; e < d; ++e) {
            const T wv = Us[a * d + e] * Vs[e * d + c];
            const T *xe = xs + e * kDmTile;
#pragma unroll
            for (int s = 0; s < kDmTile; ++s) acc[s] += wv * xe[s];
        }
#pragma unroll
        for (int s = 0; s < kDmTile; ++s)
            if (s < ns) dst[s * dd + q] = acc[s];
    }
}

// Same entries, one CTA per (sample, layer, site), weights read through L1 (channel
// counts whose staged weights exceed shared memory).
template <typename T>
__global__ void k_dmat_site(Geom g, Weights<T> w, const T *__restrict__ chi, long long b0, T *__restrict__ Dm) {
    const int N = g.N, d = g.d, L = g.L;
    const long long blk = blockIdx.x;
    const int n = (int)(blk % N);
    const int l = (int)((blk / N) % (L - 1)) + 1;
    const long long bl = blk / ((long long)N * (L - 1));
    const long long dd = (long long)d * d;
    const T *U = w.U + (l - 1) * dd, *V = w.V + (l - 1) * dd;
    const T *x = chi + (((b0 + bl) * L + (l - 1)) * N + n) * d;
    T *dst = Dm + ((bl * (L - 1) + (l - 1)) * N + n) * dd;
    for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
        const int a = idx / d, c = idx % d;
        T acc = 0;
        for (int e = 0; e < d; ++e) acc += U[a * d + e] * x[e] * V[e * d + c];
        dst[idx] = acc;
    }
}

// Embedding sources through layer 1: X[b][a][n][k] = (D0^(1)_n (g^(1)_{n-k} * e))_a.
// One CTA per (sample, site n): D0_n (transposed, [c][a]) and the tap rows of 128 sources
// at a time are staged in shared memory (rows padded to d+1 floats); thread (half, kk)
// forms 16 outputs a at a time for source kk, reading 16 D0 entries per channel as four
// 16-byte broadcasts.
constexpr int kEmbChunk = 128;   // source sites staged per pass

template <typename T>
__global__ void __launch_bounds__(256) k_embed_src(Geom g, const T *__restrict__ taps1, const T *__restrict__ e,
                                                   const T *__restrict__ Dm, T *__restrict__ X) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, L = g.L, dp = d + 1;
    T *Ds = reinterpret_cast<T *>(smraw);      // [c][a]
    T *Gs = Ds + d * d;                        // [kEmbChunk][d+1]: sources k0 .. k0 + kEmbChunk - 1
    const long long blk = blockIdx.x;
    const int n = (int)(blk % N);
    const long long bl = blk / N;
    const long long dd = (long long)d * d;
    const T *D = Dm + ((bl * (L - 1)) * N + n) * dd;
    for (int q = threadIdx.x; q < d * d; q += blockDim.x) Ds[(q % d) * d + q / d] = D[q];
    const int kk = threadIdx.x % kEmbChunk, half = threadIdx.x / kEmbChunk;
    const int ah = (d + 1) / 2;                // output channels per half
    for (int k0 = 0; k0 < N; k0 += kEmbChunk) {
        const int kn = N - k0 < kEmbChunk ? N - k0 : kEmbChunk;
        __syncthreads();
        for (int q = threadIdx.x; q < kn * d; q += blockDim.x) {
            const int k = q / d, c = q % d;
            Gs[k * dp + c] = taps1[(long long)tap_row(n - (k0 + k), N, g.periodic) * d + c] * e[c];
        }
        __syncthreads();
        if (kk >= kn) continue;
        const T *gk = Gs + kk * dp;
        for (int a0 = half * ah; a0 < (half + 1) * ah && a0 < d; a0 += 16) {
            T acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
            if (a0 + 16 <= d) {
                for (int c = 0; c < d; ++c) {
                    const T gv = gk[c];
                    const T *dc = Ds + c * d + a0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] += dc[j] * gv;
                }
            } else {
                for (int c = 0; c < d; ++c) {
                    const T gv = gk[c];
                    const T *dc = Ds + c * d + a0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] += (a0 + j < d ? dc[j] : (T)0) * gv;
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (a0 + j < d && a0 + j < (half + 1) * ah) X[((bl * d + a0 + j) * N + n) * (long long)N + k0 + kk] = acc[j];
        }
    }
}

// Same sources, several sites per CTA: the scaled tap rows g^(1)_r * e for every offset
// r in (-N, N) are staged once per CTA ([2N-1][d+1]); site n's rows are then the
// window starting at row n - k.  D0_n is staged transposed ([c][a], row stride d + 4 so
// that its 16-byte reads stay aligned), double-buffered across the CTA's sites.
constexpr int kEmbSites = 8;   // sites per CTA of k_embed_src_multi

template <typename T>
__global__ void __launch_bounds__(256) k_embed_src_multi(Geom g, const T *__restrict__ taps1, const T *__restrict__ e,
                                                         const T *__restrict__ Dm, T *__restrict__ X) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, L = g.L, dp = d + 1, ds = d + 4;
    T *Ds = reinterpret_cast<T *>(smraw);      // [2][d][d + 4]
    T *Ga = Ds + 2 * d * ds;                   // [2N - 1][d + 1]: row r + N - 1 = g^(1)_r * e
    const int groups = (N + kEmbSites - 1) / kEmbSites;
    const long long blk = blockIdx.x;
    const int n0 = (int)(blk % groups) * kEmbSites;
    const long long bl = blk / groups;
    const long long dd = (long long)d * d;
    const int nn = N - n0 < kEmbSites ? N - n0 : kEmbSites;
    for (int q = threadIdx.x; q < (2 * N - 1) * d; q += blockDim.x) {
        const int r = q / d, c = q % d;
        Ga[r * dp + c] = taps1[(long long)tap_row(r - (N - 1), N, g.periodic) * d + c] * e[c];
    }
    auto stage = [&](int j) {
        const T *D = Dm + ((bl * (L - 1)) * N + n0 + j) * dd;
        T *dst = Ds + (j & 1) * d * ds;
        for (int q = threadIdx.x; q < d * d; q += blockDim.x) dst[(q % d) * ds + q / d] = D[q];
    };
    stage(0);
    const int kk = threadIdx.x % kEmbChunk, half = threadIdx.x / kEmbChunk;
    const int ah = (d + 1) / 2;                // output channels per half
    for (int j = 0; j < nn; ++j) {
        __syncthreads();                       // site j's D0 (and the tap rows) staged; site j - 1 done
        if (j + 1 < nn) stage(j + 1);          // into the other buffer, read by nobody now
        const int n = n0 + j;
        const T *Dj = Ds + (j & 1) * d * ds;
        for (int k0 = 0; k0 < N; k0 += kEmbChunk) {
            const int k = k0 + kk;
            if (k >= N) break;
            const T *gk = Ga + (long long)(n - k + N - 1) * dp;
            for (int a0 = half * ah; a0 < (half + 1) * ah && a0 < d; a0 += 16) {
                T acc[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) acc[u] = 0;
                if (a0 + 16 <= d) {
                    for (int c = 0; c < d; ++c) {
                        const T gv = gk[c];
                        T dv[8], dw[8];
                        lds8<T>(Dj + c * ds + a0, dv);
                        lds8<T>(Dj + c * ds + a0 + 8, dw);
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            acc[u] += dv[u] * gv;
                            acc[u + 8] += dw[u] * gv;
                        }
                    }
                } else {
                    for (int c = 0; c < d; ++c) {
                        const T gv = gk[c];
                        const T *dc = Dj + c * ds + a0;
#pragma unroll
                        for (int u = 0; u < 16; ++u) acc[u] += (a0 + u < d ? dc[u] : (T)0) * gv;
                    }
                }
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (a0 + u < d && a0 + u < (half + 1) * ah) X[((bl * d + a0 + u) * N + n) * (long long)N + k] = acc[u];
            }
        }
    }
}

// ------------------------------------------------------------ Toeplitz hop --
// Y[b][a][i][p] = sum_n g_{i-n,a} X[b][a][n][p] on a 128 x 128 (i, p) tile per
// CTA; 256 threads, each an 8 x 8 register tile (rows ty*8.., columns tx*4..
// and 64 + tx*4..).  The Toeplitz operand is read from the channel's taps in
// shared memory; X is staged 16 sites at a time, the next 16 sites' loads in
// flight (in registers) while the current ones are multiplied.
constexpr int kTgTile = 128, kTgK = 16, kTgOff = 16;

template <typename T, bool GEN>
__global__ void __launch_bounds__(256) k_tgemm(Geom g, const T *__restrict__ taps, int P, const T *__restrict__ X,
                                               GenSrc<T> gs, T *__restrict__ Y, T *__restrict__ band, BandDst bd,
                                               long long b0) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d;
    T *gx = reinterpret_cast<T *>(smraw);                       // [kTgOff + 2N + kTgTile]
    const int gx_len = kTgOff + 2 * N + kTgTile;
    T *Bs = gx + ((gx_len + 3) & ~3);                           // [kTgK][kTgTile]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int p0 = blockIdx.x * kTgTile;
    const int i0 = blockIdx.y * kTgTile;
    const long long za = blockIdx.z;
    const int a = (int)(za % d);
    const long long bl = za / d;
    for (int q = tid; q < gx_len; q += blockDim.x) {
        const int r = q - kTgOff - (N - 1);
        T v = 0;
        if (r > -N && r < N) v = taps[(long long)tap_row(r, N, g.periodic) * d + a];
        gx[q] = v;
    }
    // This thread stages column pp of rows kr0 + 2r (r = 0..7) of every chunk.
    const int pp = tid & (kTgTile - 1), kr0 = tid >> 7;
    const int pl = p0 + pp;
    const bool pok = pl < P;
    int kq = 0, cq = 0;
    if (GEN && pok) {
        kq = pl / d;
        cq = pl - kq * d;
    }
    const long long dd = (long long)d * d;
    const T *dmcol = GEN ? gs.Dm + bl * gs.dm_ss + (long long)a * d + cq : nullptr;
    const T *xcol = (!GEN && X) ? X + (bl * d + a) * (long long)N * P + pl : nullptr;
    T st[8];
    auto fetch = [&](int n0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int n = n0 + kr0 + 2 * r;
            T v = 0;
            if (pok && n < N) {
                if (GEN) v = dmcol[(long long)n * dd] * gs.taps[(long long)tap_row(n - kq, N, g.periodic) * d + cq];
                else v = xcol[(long long)n * P];
            }
            st[r] = v;
        }
    };
    T acc[8][8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[q][j] = 0;
    const int rbase = kTgOff + i0 + ty * 8 + N - 1;
    fetch(0);
    for (int n0 = 0; n0 < N; n0 += kTgK) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; ++r) Bs[(kr0 + 2 * r) * kTgTile + pp] = st[r];
        __syncthreads();
        if (n0 + kTgK < N) fetch(n0 + kTgK);
#pragma unroll 4
        for (int kk = 0; kk < kTgK; ++kk) {
            const int n = n0 + kk;
            T av[8], bv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) av[q] = gx[rbase + q - n];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bv[j] = Bs[kk * kTgTile + tx * 4 + j];
                bv[4 + j] = Bs[kk * kTgTile + 64 + tx * 4 + j];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[q][j] += av[q] * bv[j];
        }
    }
    // Epilogue: full output and/or its band rows.
    int kc[8], cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int p = p0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        kc[j] = p / bd.nsrc;
        cc[j] = p - kc[j] * bd.nsrc;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int i = i0 + ty * 8 + q;
        if (i >= N) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int p = p0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (p >= P) continue;
            if (Y) Y[((bl * d + a) * N + i) * (long long)P + p] = acc[q][j];
            if (band) {
                const int dl = ring_delta(i - kc[j], N, g.periodic);
                if (dl >= -bd.R && dl <= bd.R)
                    band[(b0 + bl) * bd.ss + (long long)i * bd.rs + (long long)(bd.R - dl) * bd.os +
                         (long long)a * bd.nsrc + cc[j]] = acc[q][j];
            }
        }
    }
}

// -------------------------------------------------------------- vertex hop --
// Xo[b][c][i][p] = sum_a D[b][i][c][a] Y[b][a][i][p]; one CTA per (sample,
// site, column tile).  Fast path (d a multiple of 8, d <= 64): thread owns 8
// output channels x 4 columns; D is staged transposed so that both operands
// come as 16-byte shared-memory vectors.  Other d: one output per thread.
template <typename T, bool FAST>
__global__ void __launch_bounds__(256) k_dhop(Geom g, int P, int cols, const T *__restrict__ Dm, long long dm_ss,
                                              const T *__restrict__ Yin, T *__restrict__ Xo) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d;
    T *DsT = reinterpret_cast<T *>(smraw);      // [a][c] = D[c][a] (rows padded to d+1 off the fast path)
    T *Ys = DsT + ((d * (d + 1) + 3) / 4 * 4);  // [a][cols], 16-byte aligned
    const int p0 = blockIdx.x * cols;
    const int i = blockIdx.y;
    const long long bl = blockIdx.z;
    const T *D = Dm + bl * dm_ss + (long long)i * d * d;
    const int dp = FAST ? d : d + 1;            // fast path reads 8 consecutive rows as two 16-byte vectors
    // Transposed on the read side: consecutive threads write consecutive words of a DsT
    // row (no bank conflicts); D (4 KB per site) is read from L1/L2.
    for (int q = threadIdx.x; q < d * d; q += blockDim.x) {
        const int a = q / d, c = q % d;
        DsT[a * dp + c] = D[(long long)c * d + a];
    }
    if (sizeof(T) == 4 && P % 4 == 0 && cols % 4 == 0 && p0 + cols <= P) {
        // 16-byte loads, several in flight per thread.
        const int nv = d * cols / 4;
#pragma unroll 8
        for (int q = threadIdx.x; q < nv; q += blockDim.x) {
            const int a = (4 * q) / cols, pp = (4 * q) % cols;
            const float4 v = *reinterpret_cast<const float4 *>(Yin + ((bl * d + a) * N + i) * (long long)P + p0 + pp);
            *reinterpret_cast<float4 *>(Ys + (size_t)a * cols + pp) = v;
        }
    } else {
#pragma unroll 4
        for (int q = threadIdx.x; q < d * cols; q += blockDim.x) {
            const int a = q / cols, pp = q % cols, p = p0 + pp;
            Ys[q] = p < P ? Yin[((bl * d + a) * N + i) * (long long)P + p] : (T)0;
        }
    }
    __syncthreads();
    if (FAST) {
        const int rg = d / 8, cgs = 256 / rg;
        const int ty = threadIdx.x / cgs, tx = threadIdx.x % cgs;
        if (ty >= rg) return;
        T acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[r][j] = 0;
#pragma unroll 4
        for (int a = 0; a < d; ++a) {
            T dv[8], yv[4];
            if constexpr (sizeof(T) == 4) {
                const float4 d0 = *reinterpret_cast<const float4 *>(DsT + a * dp + ty * 8);
                const float4 d1 = *reinterpret_cast<const float4 *>(DsT + a * dp + ty * 8 + 4);
                const float4 y0 = *reinterpret_cast<const float4 *>(Ys + a * cols + tx * 4);
                dv[0] = d0.x; dv[1] = d0.y; dv[2] = d0.z; dv[3] = d0.w;
                dv[4] = d1.x; dv[5] = d1.y; dv[6] = d1.z; dv[7] = d1.w;
                yv[0] = y0.x; yv[1] = y0.y; yv[2] = y0.z; yv[3] = y0.w;
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r) dv[r] = DsT[a * dp + ty * 8 + r];
#pragma unroll
                for (int j = 0; j < 4; ++j) yv[j] = Ys[a * cols + tx * 4 + j];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[r][j] += dv[r] * yv[j];
        }
        const int pb = p0 + tx * 4;
        const bool vec = sizeof(T) == 4 && P % 4 == 0 && pb + 3 < P;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int c = ty * 8 + r;
            T *dst = Xo + ((bl * d + c) * N + i) * (long long)P + pb;
            if (vec) {
                // one 16-byte store per row: a warp writes 512 contiguous bytes
                float4 v;
                v.x = (float)acc[r][0];
                v.y = (float)acc[r][1];
                v.z = (float)acc[r][2];
                v.w = (float)acc[r][3];
                *reinterpret_cast<float4 *>(dst) = v;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (pb + j < P) dst[j] = acc[r][j];
            }
        }
    } else {
        for (int q = threadIdx.x; q < d * cols; q += blockDim.x) {
            const int c = q / cols, pp = q % cols, p = p0 + pp;
            if (p >= P) continue;
            T acc = 0;
            for (int a = 0; a < d; ++a) acc += DsT[a * dp + c] * Ys[a * cols + pp];
            Xo[((bl * d + c) * N + i) * (long long)P + p] = acc;
        }
    }
}

// ------------------------------------------------------- last-layer band --
// band[b][k+dl][R-dl][a][c'] = sum_n g^(L)_{k+dl-n,a} X[b][a][n][k nsrc + c'].
// One warp per (sample, channel a, 32 consecutive source columns p = k nsrc + c'):
// lane = column; it streams its column of X over n and keeps the 2R+1 taps
// g_{k+dl-n} it needs in a register window that slides by one tap per site.
constexpr int kBcMaxBand = 31;
constexpr int kBcU = 8;   // sites per tap window in k_bandconv4

template <typename T, bool GEN, int NB>
__global__ void __launch_bounds__(256) k_bandconv(Geom g, const T *__restrict__ taps, int P, const T *__restrict__ X,
                                                  GenSrc<T> gs, T *__restrict__ band, BandDst bd, long long b0) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, R = bd.R, ns = bd.nsrc;
    const int pad = kBcMaxBand + 1;
    T *gx = reinterpret_cast<T *>(smraw);       // gx[pad + r + N - 1] = g_{r,a}, zero outside (-N, N)
    const int gx_len = 2 * N - 1 + 2 * pad;
    const int chunks = (P + 255) / 256;         // 8 warps x 32 columns per CTA
    const long long blk = blockIdx.x;
    const int ch = (int)(blk % chunks);
    const int a = (int)((blk / chunks) % d);
    const long long bl = blk / ((long long)chunks * d);
    for (int q = threadIdx.x; q < gx_len; q += blockDim.x) {
        const int r = q - pad - (N - 1);
        gx[q] = (r > -N && r < N) ? taps[(long long)tap_row(r, N, g.periodic) * d + a] : (T)0;
    }
    __syncthreads();
    const int p = ch * 256 + threadIdx.x;
    if (p >= P) return;
    const int k = p / ns, c = p - k * ns;
    const T *Xa = X ? X + (bl * d + a) * (long long)N * P + p : nullptr;
    T acc[NB], win[NB];
    // win[q] = g_{k - R + q - n} for the current n; on a ring the taps are circulant
    // and the window index is reduced mod N by the tap table itself.
    auto G = [&](int r) -> T {
        if (g.periodic) r = ((r % N) + N) % N;
        return gx[pad + r + N - 1];
    };
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        acc[q] = 0;
        win[q] = (q <= 2 * R) ? G(k - R + q) : (T)0;
    }
#pragma unroll 4
    for (int n = 0; n < N; ++n) {
        const T xv = GEN ? gen_x<T>(gs, N, d, g.periodic, bl, a, n, p) : Xa[(long long)n * P];
#pragma unroll
        for (int q = 0; q < NB; ++q) acc[q] += win[q] * xv;
#pragma unroll
        for (int q = NB - 1; q > 0; --q) win[q] = win[q - 1];
        win[0] = G(k - R - n - 1);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (q > 2 * R) break;
        const int dl = q - R;
        int i = k + dl;
        if (g.periodic) i = ((i % N) + N) % N;
        else if (i < 0 || i >= N) continue;
        band[(b0 + bl) * bd.ss + (long long)i * bd.rs + (long long)(R - dl) * bd.os + (long long)a * ns + c] = acc[q];
    }
}

// Same band, FP32, four adjacent source columns per lane (they share the source site k,
// so they share the taps): one 16-byte load of X per site, taps from a shared table
// already wrapped for rings (no index arithmetic in the loop), one 16-byte store per
// band entry.  Requires nsrc % 4 == 0 and P % 4 == 0.
template <bool GEN, int NB>
__global__ void __launch_bounds__(256) k_bandconv4(Geom g, const float *__restrict__ taps, int P,
                                                   const float *__restrict__ X, GenSrc<float> gs,
                                                   float *__restrict__ band, BandDst bd, long long b0) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, R = bd.R, ns = bd.nsrc;
    const int pad = kBcMaxBand + 1;
    float *gx = reinterpret_cast<float *>(smraw);   // gx[pad + r + N - 1] = g_{r,a} (wrapped on a ring)
    const int gx_len = 2 * N - 1 + 2 * pad;
    // Generated operand: D0_n[a][:] for every n and the source-layer taps g_r[:] for
    // r in (-N, N), both staged in shared memory.
    float *Dsm = gx + ((gx_len + 3) & ~3);          // [N][d]
    float *Tsm = Dsm + (GEN ? N * d : 0);           // [2N-1][d], row r + N - 1
    const int chunks = (P + 1023) / 1024;           // 256 threads x 4 columns per CTA
    const long long blk = blockIdx.x;
    const int ch = (int)(blk % chunks);
    const int a = (int)((blk / chunks) % d);
    const long long bl = blk / ((long long)chunks * d);
    for (int q = threadIdx.x; q < gx_len; q += blockDim.x) {
        int r = q - pad - (N - 1);
        float v = 0.f;
        if (g.periodic) {
            r = ((r % N) + N) % N;
            v = taps[(long long)tap_row(r, N, 1) * d + a];
        } else if (r > -N && r < N) {
            v = taps[(long long)tap_row(r, N, 0) * d + a];
        }
        gx[q] = v;
    }
    if (GEN) {
        for (int q = threadIdx.x; q < N * d; q += blockDim.x) {
            const int n = q / d, cc = q - n * d;
            Dsm[q] = gs.Dm[bl * gs.dm_ss + ((long long)n * d + a) * d + cc];
        }
        for (int q = threadIdx.x; q < (2 * N - 1) * d; q += blockDim.x) {
            const int rr = q / d, cc = q - rr * d;
            Tsm[q] = gs.taps[(long long)tap_row(rr - (N - 1), N, g.periodic) * d + cc];
        }
    }
    __syncthreads();
    const int p = ch * 1024 + 4 * threadIdx.x;
    if (p >= P) return;
    const int k = p / ns, c = p - k * ns;
    const float *Xa = GEN ? nullptr : X + (bl * d + a) * (long long)N * P + p;
    // Generated operand (first hop of a source chain): X[n][(k, c..c+3)] = D0_n[a][c..c+3] g_{n-k, c..c+3}.
    const float *Dma = GEN ? Dsm + c : nullptr;
    const float *Tk = GEN ? Tsm + (long long)(N - 1 - k) * d + c : nullptr;   // row of g_{n-k} at Tk[n d]
    const float *gk = gx + pad + (k - R) + (N - 1);   // tap of (q, n) at gk[q - n]
    float acc[NB][4];
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[q][j] = 0.f;
    // Sites in blocks of kBcU: the taps of a block are a window of NB + kBcU - 1 values,
    // win[m] = gk[m - (n0 + kBcU - 1)], loaded once, so that (q, n0 + u) reads
    // win[q - u + kBcU - 1] at a compile-time index.  Taps for q > 2R are never used.
    auto site = [&](int n, const float *win, int u) {
        float4 xv;
        if (GEN) {
            const float4 dm = *reinterpret_cast<const float4 *>(Dma + n * d);
            const float4 tp = *reinterpret_cast<const float4 *>(Tk + n * d);
            xv = make_float4(dm.x * tp.x, dm.y * tp.y, dm.z * tp.z, dm.w * tp.w);
        } else {
            xv = __ldg(reinterpret_cast<const float4 *>(Xa + (long long)n * P));
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const float w = win[q - u + kBcU - 1];
            acc[q][0] = fmaf(w, xv.x, acc[q][0]);
            acc[q][1] = fmaf(w, xv.y, acc[q][1]);
            acc[q][2] = fmaf(w, xv.z, acc[q][2]);
            acc[q][3] = fmaf(w, xv.w, acc[q][3]);
        }
    };
    int n0 = 0;
    for (; n0 + kBcU <= N; n0 += kBcU) {
        float win[NB + kBcU - 1];
#pragma unroll
        for (int m = 0; m < NB + kBcU - 1; ++m) win[m] = gk[m - (n0 + kBcU - 1)];
#pragma unroll
        for (int u = 0; u < kBcU; ++u) site(n0 + u, win, u);
    }
    for (; n0 < N; ++n0) {
        float win[NB + kBcU - 1];
#pragma unroll
        for (int m = 0; m < NB + kBcU - 1; ++m) win[m] = gk[m - (n0 + kBcU - 1)];
        site(n0, win, 0);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (q > 2 * R) break;
        const int dl = q - R;
        int i = k + dl;
        if (g.periodic) i = ((i % N) + N) % N;
        else if (i < 0 || i >= N) continue;
        float *dst = band + (b0 + bl) * bd.ss + (long long)i * bd.rs + (long long)(R - dl) * bd.os + (long long)a * ns + c;
        *reinterpret_cast<float4 *>(dst) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
}

// Generated-operand band (first hop of a source chain), two adjacent source sites k and
// k + 1 per lane with the same four source channels: they share the D0 row loads, and the
// tap window of k + 1 is that of k shifted by one, so the shared-memory loads per FMA are
// about halved.  Every band sum is formed in the same order as in k_bandconv4<true, NB>.
// Requires nsrc % 4 == 0 and 1024 % nsrc == 0.
template <int NB>
__global__ void __launch_bounds__(256) k_bandconv4g(Geom g, const float *__restrict__ taps, GenSrc<float> gs,
                                                    float *__restrict__ band, BandDst bd, long long b0) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = g.N, d = g.d, R = bd.R, ns = bd.nsrc;
    const int pad = kBcMaxBand + 1;
    float *gx = reinterpret_cast<float *>(smraw);   // gx[pad + r + N - 1] = g_{r,a} (wrapped on a ring)
    const int gx_len = 2 * N - 1 + 2 * pad;
    float *Dsm = gx + ((gx_len + 3) & ~3);          // [N][d]: D0_n[a][:]
    float *Tsm = Dsm + N * d;                       // [2N-1][d], row r + N - 1: source-layer taps g_r[:]
    const int kpc = 2 * (1024 / ns);                // source sites per CTA
    const int chunks = (N + kpc - 1) / kpc;
    const long long blk = blockIdx.x;
    const int ch = (int)(blk % chunks);
    const int a = (int)((blk / chunks) % d);
    const long long bl = blk / ((long long)chunks * d);
#pragma unroll 4
    for (int q = threadIdx.x; q < gx_len; q += blockDim.x) {
        int r = q - pad - (N - 1);
        float v = 0.f;
        if (g.periodic) {
            r = ((r % N) + N) % N;
            v = taps[(long long)tap_row(r, N, 1) * d + a];
        } else if (r > -N && r < N) {
            v = taps[(long long)tap_row(r, N, 0) * d + a];
        }
        gx[q] = v;
    }
#pragma unroll 8
    for (int q = threadIdx.x; q < N * d; q += blockDim.x) {
        const int n = q / d, cc = q - n * d;
        Dsm[q] = gs.Dm[bl * gs.dm_ss + ((long long)n * d + a) * d + cc];
    }
#pragma unroll 8
    for (int q = threadIdx.x; q < (2 * N - 1) * d; q += blockDim.x) {
        const int rr = q / d, cc = q - rr * d;
        Tsm[q] = gs.taps[(long long)tap_row(rr - (N - 1), N, g.periodic) * d + cc];
    }
    __syncthreads();
    const int k = ch * kpc + 2 * (int)(threadIdx.x / (ns / 4)), c = 4 * (int)(threadIdx.x % (ns / 4));
    if (k >= N) return;
    const bool has1 = k + 1 < N;
    const float *Dma = Dsm + c;
    const float *Tk0 = Tsm + (long long)(N - 1 - k) * d + c;   // row of g_{n-k} at Tk0[n d]
    const float *Tk1 = has1 ? Tk0 - d : Tk0;                    // g_{n-k-1} (a copy of k's when k + 1 = N)
    const float *gk = gx + pad + (k - R) + (N - 1);             // tap of (q, n) at gk[q - n]; k + 1: gk[q - n + 1]
    float acc0[NB][4], acc1[NB][4];
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc0[q][j] = acc1[q][j] = 0.f;
    // win[m] = gk[m - (n0 + kBcU - 1)]: (q, n0 + u) of k reads win[q - u + kBcU - 1], of k + 1
    // win[q - u + kBcU].
    auto site = [&](int n, const float *win, int u) {
        const float4 dm = *reinterpret_cast<const float4 *>(Dma + n * d);
        const float4 t0 = *reinterpret_cast<const float4 *>(Tk0 + n * d);
        const float4 t1 = *reinterpret_cast<const float4 *>(Tk1 + n * d);
        const float4 x0 = make_float4(dm.x * t0.x, dm.y * t0.y, dm.z * t0.z, dm.w * t0.w);
        const float4 x1 = make_float4(dm.x * t1.x, dm.y * t1.y, dm.z * t1.z, dm.w * t1.w);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const float w0 = win[q - u + kBcU - 1], w1 = win[q - u + kBcU];
            acc0[q][0] = fmaf(w0, x0.x, acc0[q][0]);
            acc1[q][0] = fmaf(w1, x1.x, acc1[q][0]);
            acc0[q][1] = fmaf(w0, x0.y, acc0[q][1]);
            acc1[q][1] = fmaf(w1, x1.y, acc1[q][1]);
            acc0[q][2] = fmaf(w0, x0.z, acc0[q][2]);
            acc1[q][2] = fmaf(w1, x1.z, acc1[q][2]);
            acc0[q][3] = fmaf(w0, x0.w, acc0[q][3]);
            acc1[q][3] = fmaf(w1, x1.w, acc1[q][3]);
        }
    };
    int n0 = 0;
    for (; n0 + kBcU <= N; n0 += kBcU) {
        float win[NB + kBcU];
#pragma unroll
        for (int m = 0; m < NB + kBcU; ++m) win[m] = gk[m - (n0 + kBcU - 1)];
#pragma unroll
        for (int u = 0; u < kBcU; ++u) site(n0 + u, win, u);
    }
    for (; n0 < N; ++n0) {
        float win[NB + kBcU];
#pragma unroll
        for (int m = 0; m < NB + kBcU; ++m) win[m] = gk[m - (n0 + kBcU - 1)];
        site(n0, win, 0);
    }
    auto store = [&](int kk, const float (&acc)[NB][4]) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if (q > 2 * R) break;
            const int dl = q - R;
            int i = kk + dl;
            if (g.periodic) i = ((i % N) + N) % N;
            else if (i < 0 || i >= N) continue;
            float *dst = band + (b0 + bl) * bd.ss + (long long)i * bd.rs + (long long)(R - dl) * bd.os +
                         (long long)a * ns + c;
            *reinterpret_cast<float4 *>(dst) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
        }
    };
    store(k, acc0);
    if (has1) store(k + 1, acc1);
}

// ------------------------------------------------------------------- host --
static size_t links_per_sample_elems(const dn_model *m, int N) {
    const long long d = m->desc.d, L = m->desc.L;
    const long long P = N * d;
    return (size_t)(2 * d * N * P + (L > 1 ? (L - 1) : 0) * N * d * d);
}

size_t links_scratch_elems(const dn_model *m, int N, int B) {
    // Up to 6 GiB of probe fields (at 4 bytes per element), at least one sample.
    const size_t per = links_per_sample_elems(m, N);
    size_t nb = (size_t(6) << 30) / 4 / per;
    if (nb < 1) nb = 1;
    if (nb > (size_t)B) nb = (size_t)B;
    return nb * per;
}

template <typename T>
static cudaError_t launch_tgemm_ffma(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> *gs, T *Y,
                                     T *band, const BandDst &bd, long long b0, int nb, cudaStream_t st);

// FP32/BF16: tensor cores (BF16 planes per operand value); FP64: the FMA kernel.
template <typename T>
static cudaError_t launch_tgemm(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> *gs, T *Y, T *band,
                                const BandDst &bd, long long b0, int nb, unsigned *flag, cudaStream_t st,
                                int planes = 2) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t err = launch_tgemm_tc(g, reinterpret_cast<const float *>(taps), P,
                                          reinterpret_cast<const float *>(X),
                                          gs ? reinterpret_cast<const float *>(gs->taps) : nullptr,
                                          gs ? reinterpret_cast<const float *>(gs->Dm) : nullptr, gs ? gs->dm_ss : 0,
                                          reinterpret_cast<float *>(Y), reinterpret_cast<float *>(band), bd.ss, bd.rs,
                                          bd.os, bd.R, bd.nsrc, b0, nb, flag, st, planes);
        if (err != cudaErrorNotSupported) return err;
        cudaGetLastError();
    }
    return launch_tgemm_ffma<T>(g, taps, P, X, gs, Y, band, bd, b0, nb, st);
}

template <typename T>
static cudaError_t launch_tgemm_ffma(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> *gs, T *Y,
                                     T *band, const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    const int gx_len = kTgOff + 2 * g.N + kTgTile;
    const size_t smem = (((size_t)gx_len + 3) & ~size_t(3)) * sizeof(T) + (size_t)kTgK * kTgTile * sizeof(T);
    cudaError_t err;
    dim3 grid((P + kTgTile - 1) / kTgTile, (g.N + kTgTile - 1) / kTgTile, (unsigned)nb * g.d);
    if (gs) {
        err = cudaFuncSetAttribute(k_tgemm<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm", st);
        k_tgemm<T, true><<<grid, 256, smem, st>>>(g, taps, P, nullptr, *gs, Y, band, bd, b0);
    } else {
        err = cudaFuncSetAttribute(k_tgemm<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_tgemm", st);
        k_tgemm<T, false><<<grid, 256, smem, st>>>(g, taps, P, X, GenSrc<T>{nullptr, nullptr, 0}, Y, band, bd, b0);
    }
    return cudaGetLastError();
}

template <typename T, bool GEN, int NB>
static cudaError_t launch_bandconv_nb(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> &gs, T *band,
                                      const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    const size_t smem = ((size_t)2 * g.N - 1 + 2 * (kBcMaxBand + 1)) * sizeof(T);
    const int chunks = (P + 255) / 256;
    const unsigned blocks = (unsigned)((long long)nb * g.d * chunks);
    cudaError_t err = cudaFuncSetAttribute(k_bandconv<T, GEN, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        // traced apart: the generated-operand variant is FMA-bound, the other reads its operand
        ProfScope _ps(GEN ? "k_bandconv_gen" : "k_bandconv", st);
        k_bandconv<T, GEN, NB><<<blocks, 256, smem, st>>>(g, taps, P, X, gs, band, bd, b0);
    }
    return cudaGetLastError();
}

template <typename T, bool GEN>
static cudaError_t launch_bandconv_gen(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> &gs, T *band,
                                       const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    const int nbw = 2 * bd.R + 1;
    if (nbw <= 5) return launch_bandconv_nb<T, GEN, 5>(g, taps, P, X, gs, band, bd, b0, nb, st);
    if (nbw <= 9) return launch_bandconv_nb<T, GEN, 9>(g, taps, P, X, gs, band, bd, b0, nb, st);
    if (nbw <= 13) return launch_bandconv_nb<T, GEN, 13>(g, taps, P, X, gs, band, bd, b0, nb, st);
    if (nbw <= kBcMaxBand) return launch_bandconv_nb<T, GEN, kBcMaxBand>(g, taps, P, X, gs, band, bd, b0, nb, st);
    return cudaErrorInvalidConfiguration;
}

template <bool GEN, int NB>
static cudaError_t launch_bandconv4_nb(const Geom &g, const float *taps, int P, const float *X, const GenSrc<float> &gs,
                                       float *band, const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    const size_t gx_len = (((size_t)2 * g.N - 1 + 2 * (kBcMaxBand + 1)) + 3) & ~(size_t)3;
    const size_t smem = (gx_len + (GEN ? (size_t)g.N * g.d + (size_t)(2 * g.N - 1) * g.d : 0)) * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorNotSupported;
    if (GEN && bd.nsrc % 4 == 0 && 1024 % bd.nsrc == 0 && P == g.N * bd.nsrc) {
        const int kpc = 2 * (1024 / bd.nsrc);
        const unsigned blocks = (unsigned)((long long)nb * g.d * ((g.N + kpc - 1) / kpc));
        cudaError_t err = cudaFuncSetAttribute(k_bandconv4g<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_bandconv_gen", st);
        k_bandconv4g<NB><<<blocks, 256, smem, st>>>(g, taps, gs, band, bd, b0);
        return cudaGetLastError();
    }
    const int chunks = (P + 1023) / 1024;
    const unsigned blocks = (unsigned)((long long)nb * g.d * chunks);
    cudaError_t err =
        cudaFuncSetAttribute(k_bandconv4<GEN, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    {
        ProfScope _ps(GEN ? "k_bandconv_gen" : "k_bandconv", st);
        k_bandconv4<GEN, NB><<<blocks, 256, smem, st>>>(g, taps, P, X, gs, band, bd, b0);
    }
    return cudaGetLastError();
}

template <bool GEN>
static cudaError_t launch_bandconv4(const Geom &g, const float *taps, int P, const float *X, const GenSrc<float> &gs,
                                    float *band, const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    const int nbw = 2 * bd.R + 1;
    if (nbw <= 5) return launch_bandconv4_nb<GEN, 5>(g, taps, P, X, gs, band, bd, b0, nb, st);
    if (nbw <= 9) return launch_bandconv4_nb<GEN, 9>(g, taps, P, X, gs, band, bd, b0, nb, st);
    if (nbw <= 13) return launch_bandconv4_nb<GEN, 13>(g, taps, P, X, gs, band, bd, b0, nb, st);
    return cudaErrorNotSupported;
}

template <typename T>
static cudaError_t launch_bandconv(const Geom &g, const T *taps, int P, const T *X, const GenSrc<T> *gs, T *band,
                                   const BandDst &bd, long long b0, int nb, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        // Four source columns per lane (FP32, channel count a multiple of 4).
        if (bd.nsrc % 4 == 0 && P % 4 == 0 && g.d % 4 == 0) {
            const float *tf = reinterpret_cast<const float *>(taps), *xf = reinterpret_cast<const float *>(X);
            float *bf = reinterpret_cast<float *>(band);
            GenSrc<float> gf{nullptr, nullptr, 0};
            if (gs)
                gf = GenSrc<float>{reinterpret_cast<const float *>(gs->taps), reinterpret_cast<const float *>(gs->Dm),
                                   gs->dm_ss};
            cudaError_t err = gs ? launch_bandconv4<true>(g, tf, P, nullptr, gf, bf, bd, b0, nb, st)
                                 : launch_bandconv4<false>(g, tf, P, xf, gf, bf, bd, b0, nb, st);
            if (err != cudaErrorNotSupported) return err;
            cudaGetLastError();
        }
    }
    if (gs) return launch_bandconv_gen<T, true>(g, taps, P, nullptr, *gs, band, bd, b0, nb, st);
    return launch_bandconv_gen<T, false>(g, taps, P, X, GenSrc<T>{nullptr, nullptr, 0}, band, bd, b0, nb, st);
}

template <typename T>
static cudaError_t launch_dhop(const Geom &g, int P, const T *Dm, long long dm_ss, const T *Y, T *Xo, int nb,
                               cudaStream_t st, int planes = 3, unsigned *flag = nullptr) {
    if constexpr (sizeof(T) == 4) {
        cudaError_t e = launch_dhop_tc(g.d, g.N, P, reinterpret_cast<const float *>(Dm), dm_ss,
                                       reinterpret_cast<const float *>(Y), reinterpret_cast<float *>(Xo), nb, planes,
                                       flag, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
    }
    const bool fast = g.d % 8 == 0 && g.d <= 64;
    const int cols = fast ? (256 / (g.d / 8)) * 4 : 128;
    const size_t smem = (((size_t)g.d * (g.d + 1) + 3) / 4 * 4 + (size_t)g.d * cols) * sizeof(T);
    dim3 grid((P + cols - 1) / cols, g.N, nb);
    cudaError_t err;
    if (fast) {
        err = cudaFuncSetAttribute(k_dhop<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_dhop", st);
        k_dhop<T, true><<<grid, 256, smem, st>>>(g, P, cols, Dm, dm_ss, Y, Xo);
    } else {
        err = cudaFuncSetAttribute(k_dhop<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope _ps("k_dhop", st);
        k_dhop<T, false><<<grid, 256, smem, st>>>(g, P, cols, Dm, dm_ss, Y, Xo);
    }
    return cudaGetLastError();
}

// Band links of a one-intermediate pair by FFT (g_fft_links: 0 never, 1 where the direct
// sum has no fast kernel or N >= 512, 2 always).  The direct generated-operand sum on four
// columns per lane (FP32) is faster up to a few hundred sites: at N = 128, d = 32 it took
// 10.1 ms per 1024 configurations against 19.1 ms for the radix-2 FFT.
template <typename T>
static bool use_fft_links(const Geom &g, int Rk) {
    if (g_fft_links == 0) return false;
    if (g_fft_links == 2) return true;
    const size_t gx_len = (((size_t)2 * g.N - 1 + 2 * (kBcMaxBand + 1)) + 3) & ~(size_t)3;
    const size_t smem = (gx_len + (size_t)g.N * g.d + (size_t)(2 * g.N - 1) * g.d) * sizeof(float);
    const bool fast_direct = sizeof(T) == 4 && g.d % 4 == 0 && 1024 % g.d == 0 && 2 * Rk + 1 <= 13 &&
                             smem <= 200 * 1024;
    return !fast_direct || g.N >= 512;
}

template <typename T>
cudaError_t build_links(const dn_model *m, const Plan<T> &pl, const Weights<T> &w, dn_cache *c, T *scratch,
                        size_t scratch_elems, cudaStream_t st) {
    const Geom g = geom_of(m, c->N);
    const int N = g.N, d = g.d, L = g.L;
    if (L < 2) return cudaSuccess;
    const size_t per = links_per_sample_elems(m, N);
    const int nb_max = (int)(scratch_elems / per);
    if (nb_max < 1) return cudaErrorInvalidValue;
    const long long Pm = (long long)N * d;                 // sources per sample, m >= 1
    const long long dd = (long long)d * d;
    const long long dm_ss = (long long)(L - 1) * N * dd;   // Dm sample stride
    const T *chi = static_cast<const T *>(c->chi);
    T *ell = static_cast<T *>(c->ell);
    T *K = static_cast<T *>(c->K);
    const int nRl = 2 * c->Rl + 1, nRk = 2 * c->Rk + 1;
    // The link tensors are built at FP32 accuracy for FP32 and BF16 caches alike (BF16 is
    // confined to the forward pass's convolutions and channel mixing): Toeplitz hops as
    // hi*hi + hi*lo + lo*hi of two BF16 planes, vertex hops (K = d) with three planes.
    const int planes = 2;
    const int dplanes = 3;
    cudaError_t err;
    for (int b0 = 0; b0 < c->B; b0 += nb_max) {
        const int nb = (c->B - b0 < nb_max) ? c->B - b0 : nb_max;
        T *U = scratch;
        T *F = U + (size_t)nb * d * N * Pm;
        T *Dm = F + (size_t)nb * d * N * Pm;
        {
            const size_t smem = ((size_t)2 * dd + (size_t)kDmTile * d) * sizeof(T);
            ProfScope _ps("k_dmat", st);
            if (smem <= 200 * 1024) {
                if ((err = cudaFuncSetAttribute(k_dmat<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                    cudaSuccess)
                    return err;
                const long long ntile = (N + kDmTile - 1) / kDmTile;
                k_dmat<T><<<(unsigned)((long long)nb * (L - 1) * ntile), 256, smem, st>>>(g, w, chi, b0, Dm);
            } else {
                k_dmat_site<T><<<(unsigned)((long long)nb * (L - 1) * N), 128, 0, st>>>(g, w, chi, b0, Dm);
            }
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        // Embedding sources (m = 0), P = N.
        {
            const size_t msm = ((size_t)2 * d * (d + 4) + (size_t)(2 * N - 1) * (d + 1)) * sizeof(T);
            ProfScope _ps("k_embed_src", st);
            if (d % 8 == 0 && msm <= 160 * 1024) {
                if ((err = cudaFuncSetAttribute(k_embed_src_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)msm)) != cudaSuccess)
                    return err;
                const long long groups = (N + kEmbSites - 1) / kEmbSites;
                k_embed_src_multi<T><<<(unsigned)((long long)nb * groups), 256, msm, st>>>(g, pl.taps, w.e, Dm, F);
            } else {
                const size_t smem = ((size_t)d * d + (size_t)(N < kEmbChunk ? N : kEmbChunk) * (d + 1)) * sizeof(T);
                if ((err = cudaFuncSetAttribute(k_embed_src<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem)) != cudaSuccess)
                    return err;
                k_embed_src<T><<<(unsigned)((long long)nb * N), 256, smem, st>>>(g, pl.taps, w.e, Dm, F);
            }
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        for (int n = 2; n <= L; ++n) {
            BandDst bd{(long long)(L - 1) * N * nRl * d, (long long)nRl * d, (long long)d, c->Rl, 1};
            T *dst = ell + (long long)(n - 2) * N * nRl * d;
            const T *taps_n = pl.taps + (long long)(n - 1) * g.R * d;
            if (n < L) {
                if ((err = launch_tgemm<T>(g, taps_n, N, F, nullptr, U, dst, bd, b0, nb, c->flag, st, planes)) != cudaSuccess)
                    return err;
                if ((err = launch_dhop<T>(g, N, Dm + (long long)(n - 1) * N * dd, dm_ss, U, F, nb, st, dplanes, c->flag)) != cudaSuccess)
                    return err;
            } else {
                if ((err = launch_bandconv<T>(g, taps_n, N, F, nullptr, dst, bd, b0, nb, st)) != cudaSuccess) return err;
            }
        }
        // Interlayer sources (m >= 1), P = N d.
        for (int msrc = 1; msrc <= L - 2; ++msrc) {
            GenSrc<T> gs{pl.taps + (long long)msrc * g.R * d, Dm + (long long)msrc * N * dd, dm_ss};
            // The chain's last vertex hop and the band of G^(L) run as one kernel where it applies
            // (FP32, d = 32): the hop output Y = G^(L-1) ... then never round-trips HBM.
            const bool fuse_end = sizeof(T) == 4 && dplanes == 3 && g_fused_links && msrc + 2 < L &&
                                  dband_tc_ok(d, N, g.periodic, (int)Pm, d, c->Rk);
            for (int n = msrc + 2; n <= L; ++n) {
                BandDst bd{(long long)c->P * N * nRk * dd, (long long)nRk * dd, dd, c->Rk, d};
                T *dst = K + (long long)pair_index(n, msrc) * N * nRk * dd;
                const T *taps_n = pl.taps + (long long)(n - 1) * g.R * d;
                const bool first = n == msrc + 2;
                if (n < L) {
                    err = launch_tgemm<T>(g, taps_n, (int)Pm, first ? nullptr : F, first ? &gs : nullptr, U, dst, bd,
                                          b0, nb, c->flag, st, planes);
                    if (err != cudaSuccess) return err;
                    if (fuse_end && n == L - 1) continue;
                    if ((err = launch_dhop<T>(g, (int)Pm, Dm + (long long)(n - 1) * N * dd, dm_ss, U, F, nb, st, dplanes, c->flag)) !=
                        cudaSuccess)
                        return err;
                } else if (fuse_end) {
                    if constexpr (sizeof(T) == 4) {
                        err = launch_dband_tc(d, N, g.periodic, (int)Pm, d, c->Rk, reinterpret_cast<const float *>(taps_n),
                                              reinterpret_cast<const float *>(Dm + (long long)(L - 2) * N * dd), dm_ss,
                                              reinterpret_cast<const float *>(U), reinterpret_cast<float *>(dst), bd.ss,
                                              bd.rs, bd.os, b0, nb, c->flag, st);
                        if (err == cudaErrorNotSupported) {
                            // the two-kernel end of the chain: vertex hop of layer L - 1, then the band
                            cudaGetLastError();
                            err = launch_dhop<T>(g, (int)Pm, Dm + (long long)(L - 2) * N * dd, dm_ss, U, F, nb, st,
                                                 dplanes, c->flag);
                            if (err == cudaSuccess)
                                err = launch_bandconv<T>(g, taps_n, (int)Pm, F, nullptr, dst, bd, b0, nb, st);
                        }
                        if (err != cudaSuccess) return err;
                    }
                } else {
                    // A chain with one intermediate layer: its band by FFT where the shape allows
                    // (the probe fields are unused here and hold the spectra), else summed directly.
                    err = cudaErrorNotSupported;
                    if (first && use_fft_links<T>(g, c->Rk))
                        err = launch_link_fft<T>(N, g.periodic, d, c->Rk, taps_n, gs.taps, gs.Dm, dm_ss, dst, bd.ss,
                                                 bd.rs, bd.os, b0, nb, F, (size_t)nb * d * N * Pm, st);
                    if (err == cudaErrorNotSupported) {
                        cudaGetLastError();
                        err = launch_bandconv<T>(g, taps_n, (int)Pm, first ? nullptr : F, first ? &gs : nullptr, dst,
                                                 bd, b0, nb, st);
                    }
                    if (err != cudaSuccess) return err;
                }
            }
        }
    }
    return cudaSuccess;
}

template cudaError_t build_links<double>(const dn_model *, const Plan<double> &, const Weights<double> &, dn_cache *,
                                         double *, size_t, cudaStream_t);
template cudaError_t build_links<float>(const dn_model *, const Plan<float> &, const Weights<float> &, dn_cache *,
                                        float *, size_t, cudaStream_t);

}  // namespace dn
