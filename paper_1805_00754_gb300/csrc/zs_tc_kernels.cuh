// zs_tc_kernels.cuh - truncated SVD of many tall matrices X_j (rows_j x n) on
// tensor cores.  Used for the blocks of the storage phase (Section 3.2) and for
// the stacked Sigma V^T matrix of each query's Stitched-SVD (Algorithm 2).
//
// The SVD is computed through a Gram matrix, split so that tensor cores carry
// the O(rows n^2) work without giving up FP32 accuracy:
//   1. k_gram_lo    G~ = bf16(X)^T bf16(X), fp32 accumulate (mma.sync bf16).
//                   Only used to locate the dominant subspace (~1e-3 accurate).
//   2. k_subspace   m columns Q of G~'s dominant subspace: pivoted columns of G~
//                   and power steps with Gram-Schmidt (SIMT), stored as bf16 Q~.
//   3. k_project    Y = X Q~ with X split into bf16 hi + lo parts: two bf16
//                   tensor products give X Q~ to ~2^-17 relative (Q~ is exact in
//                   bf16, so nothing of Q is lost).
//   4. k_rr         Rayleigh-Ritz on span(Q~): Y^T Y z = theta (Q~^T Q~) z via a
//                   Cholesky of Q~^T Q~ and the small Jacobi core; then
//                   sigma = sqrt(theta), V = Q~ Z, U = Y Z Sigma^{-1}.
// Accuracy of sigma, U, V is set by step 3-4 (FP32 products of the exact data
// against an exact basis); steps 1-2 only decide how good the subspace is,
// which subspace iteration makes exponentially good in
// (lambda_{m+1} / lambda_k).
#pragma once

#include <cuda_bf16.h>

#include "zs_internal.h"
#include "zs_linalg.cuh"
#include "zs_tc.cuh"

namespace zs {

// Row stride (elements) of a bf16 tile of width w so that 8 consecutive rows
// hit distinct 16-byte bank groups under ldmatrix.
__host__ __device__ __forceinline__ int bf16_ld(int w) { return w + (((w / 8) % 2 == 0) ? 8 : 16); }

// ---------------------------------------------------------------------------
// Sources: how item j of a launch maps to (X, ld, rows) and scratch slots.
// ---------------------------------------------------------------------------
struct SrcCompress {
    CompressChunk c;
    __device__ __forceinline__ int count() const { return c.nblk; }
    __device__ __forceinline__ int rows(int j) const {
        return (int)min((int64_t)c.b, c.rows_total - (int64_t)j * c.b);
    }
    __device__ __forceinline__ int64_t ld() const { return c.lda; }
    __device__ __forceinline__ const void* X(int j, int elem) const {
        return (const char*)c.A + (size_t)j * c.b * c.lda * elem;
    }
    __device__ __forceinline__ int64_t ybase(int j) const { return (int64_t)j * c.b; }   // Y row offset
};

struct SrcQuery {
    QueryArgs a;
    __device__ __forceinline__ int count() const { return a.hdr->nq; }
    __device__ __forceinline__ int rows(int q) const { return a.plans[q].nslab * a.k; }
    __device__ __forceinline__ int64_t ld() const { return a.n; }
    __device__ __forceinline__ const void* X(int q, int elem) const {
        return (const char*)a.M + (size_t)a.plans[q].slab0 * a.k * a.n * elem;
    }
    __device__ __forceinline__ int64_t ybase(int q) const { return a.plans[q].slab0 * a.k; }
};

// Scratch for the tensor path (per launch).
struct TcScratch {
    float* G;               // items x n x n
    __nv_bfloat16* Qb;      // items x n x m
    float* Y;               // (sum of rows) x m, row offsets from Src::ybase
    void* ews;              // per-CTA workspace (subspace Y block), ews_ctas x n x (m+1) floats
    int ews_ctas;
    int m;                  // subspace width (multiple of 8, <= 64)
    int power_its;          // power steps on G~
};

template <typename Tin>
__device__ __forceinline__ float4 ld4(const Tin* p);
template <>
__device__ __forceinline__ float4 ld4<float>(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// ---------------------------------------------------------------------------
// 1. G~ = bf16(X)^T bf16(X): one 128 x 128 output tile per CTA (upper triangle
//    of tiles), rows streamed in chunks of 32 through shared memory.
// ---------------------------------------------------------------------------
template <class Src, typename Tin>
__global__ void __launch_bounds__(256, 2) k_gram_lo(Src src, TcScratch sc, int n) {
    constexpr int LDS = 136;                        // bf16_ld(128)
    __shared__ __align__(16) __nv_bfloat16 XI[32 * LDS];
    __shared__ __align__(16) __nv_bfloat16 XJ[32 * LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wi = warp >> 2, wj = warp & 3;
    const int ntile = (n + 127) / 128;
    int ti = 0, p = blockIdx.x;
    while (p >= ntile - ti) { p -= ntile - ti; ++ti; }
    const int tj = ti + p;
    const int I0 = ti * 128, J0 = tj * 128;
    const bool diag = (ti == tj);
    const int64_t ld = src.ld();
    const bool vec = std::is_same<Tin, float>::value && (ld % 4 == 0) && (n % 4 == 0);
    for (int item = blockIdx.y; item < src.count(); item += gridDim.y) {
        const Tin* X = (const Tin*)src.X(item, sizeof(Tin));
        const bool xal = vec && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
        const int rows = src.rows(item);
        float acc[4][4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
        for (int r0 = 0; r0 < rows; r0 += 32) {
            __syncthreads();
            // stage two column panels of 32 rows as bf16
            for (int pnl = 0; pnl < (diag ? 1 : 2); ++pnl) {
                const int P0 = pnl ? J0 : I0;
                __nv_bfloat16* D = pnl ? XJ : XI;
                for (int f = tid; f < 32 * 32; f += 256) {
                    const int r = f >> 5, c = (f & 31) * 4, gr = r0 + r, gc = P0 + c;
                    float v[4] = {0.f, 0.f, 0.f, 0.f};
                    if (gr < rows) {
                        const Tin* src_p = X + (int64_t)gr * ld + gc;
                        if constexpr (std::is_same<Tin, float>::value) {
                            if (xal && gc + 3 < n) {
                                const float4 q = ld4<float>(src_p);
                                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (gc + e < n) v[e] = (float)src_p[e];
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (gc + e < n) v[e] = __bfloat162float(src_p[e]);
                        }
                    }
                    uint32_t* dp = reinterpret_cast<uint32_t*>(D + r * LDS + c);
                    dp[0] = pack_bf16(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
                    dp[1] = pack_bf16(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
                }
            }
            __syncthreads();
            const __nv_bfloat16* BJ = diag ? XI : XJ;
#pragma unroll
            for (int kk = 0; kk < 32; kk += 16) {
                uint32_t af[4][4], bf[4][2];
                const int mat = lane >> 3, rr = lane & 7;
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    const int t = kk + rr + ((mat >> 1) ? 8 : 0);
                    const int i = wi * 64 + mt * 16 + ((mat & 1) ? 8 : 0);
                    ldsm_x4_t(smem_u32(XI + t * LDS + i), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
                }
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    const int t = kk + rr + ((mat & 1) ? 8 : 0);
                    const int j = wj * 32 + np * 16 + ((mat >> 1) ? 8 : 0);
                    ldsm_x4_t(smem_u32(BJ + t * LDS + j), bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0],
                              bf[2 * np + 1][1]);
                }
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bf[nt][0], bf[nt][1]);
            }
        }
        float* G = sc.G + (size_t)item * n * n;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = I0 + wi * 64 + mt * 16 + (lane >> 2) + ((e >> 1) ? 8 : 0);
                    const int j = J0 + wj * 32 + nt * 8 + 2 * (lane & 3) + (e & 1);
                    if (i < n && j < n) {
                        G[(size_t)i * n + j] = acc[mt][nt][e];
                        if (!diag) G[(size_t)j * n + i] = acc[mt][nt][e];
                    }
                }
    }
}

// ---------------------------------------------------------------------------
// 2. Dominant m-dimensional subspace of G~ (rough): pivoted columns, then
//    power steps, each followed by Gram-Schmidt; stored as bf16 (n x m).
// ---------------------------------------------------------------------------
template <class Src>
__global__ void __launch_bounds__(256) k_subspace(Src src, TcScratch sc, int n, int yglob) {
    extern __shared__ __align__(16) char dsm[];
    __shared__ int piv[ZS_MAXM];
    __shared__ float red[32];
    __shared__ float coef[ZS_MAXM];
    const int m = sc.m, ldq = m + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    float* Q = (float*)dsm;
    float* Y = yglob ? (float*)sc.ews + (size_t)blockIdx.x * n * ldq : Q + (size_t)n * ldq;
    for (int item = blockIdx.x; item < src.count(); item += gridDim.x) {
        const float* G = sc.G + (size_t)item * n * n;
        __syncthreads();
        for (int i = tid; i < n; i += nt) Y[i] = G[(size_t)i * n + i];
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            const float v = Y[i];
            int rk = 0;
            for (int j = 0; j < n; ++j) {
                const float u = Y[j];
                rk += (u > v) || (u == v && j < i);
            }
            if (rk < m) piv[rk] = i;
        }
        __syncthreads();
        for (int e = tid; e < n * m; e += nt) {
            const int c = e / n, i = e - (e / n) * n;
            Q[i * ldq + c] = G[(size_t)piv[c] * n + i];
        }
        __syncthreads();
        mgs_orth<float>(Q, ldq, n, m, red, coef);
        for (int it = 0; it < sc.power_its; ++it) {
            for (int i = tid; i < n; i += nt) {
                float acc[ZS_MAXM];
#pragma unroll
                for (int c = 0; c < ZS_MAXM; ++c) acc[c] = 0.f;
                for (int l = 0; l < n; ++l) {
                    const float g = G[(size_t)l * n + i];
                    const float* qr = Q + l * ldq;
#pragma unroll
                    for (int c = 0; c < ZS_MAXM; ++c)
                        if (c < m) acc[c] += g * qr[c];
                }
#pragma unroll
                for (int c = 0; c < ZS_MAXM; ++c)
                    if (c < m) Y[i * ldq + c] = acc[c];
            }
            __syncthreads();
            for (int e = tid; e < n * m; e += nt) {
                const int i = e / m, c = e - (e / m) * m;
                Q[i * ldq + c] = Y[i * ldq + c];
            }
            __syncthreads();
            mgs_orth<float>(Q, ldq, n, m, red, coef);
        }
        __nv_bfloat16* Qb = sc.Qb + (size_t)item * n * m;
        for (int e = tid; e < n * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            Qb[e] = __float2bfloat16_rn(Q[i * ldq + c]);
        }
    }
}

// ---------------------------------------------------------------------------
// 3. Y = X Q~ for 128-row tiles: X split into bf16 hi + lo (two products).
// ---------------------------------------------------------------------------
template <class Src, typename Tin>
__global__ void __launch_bounds__(256) k_project(Src src, TcScratch sc, int n) {
    extern __shared__ __align__(16) char dsm[];
    constexpr int KC = 64, LDX = 72;               // bf16_ld(64)
    const int m = sc.m, ldqs = bf16_ld(m);
    __nv_bfloat16* Qs = (__nv_bfloat16*)dsm;                      // n x ldqs
    __nv_bfloat16* Xh = Qs + (size_t)((n + 15) / 16 * 16) * ldqs;    // 128 x LDX
    __nv_bfloat16* Xl = Xh + 128 * LDX;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ld = src.ld();
    const int ntn = m / 8;
    int loaded = -1;
    for (int item = blockIdx.y; item < src.count(); item += gridDim.y) {
        const int rows = src.rows(item);
        const int r0 = blockIdx.x * 128;
        if (r0 >= rows) continue;
        const Tin* X = (const Tin*)src.X(item, sizeof(Tin));
        __syncthreads();
        if (loaded != item) {
            const __nv_bfloat16* Qg = sc.Qb + (size_t)item * n * m;
            const int npad = (n + 15) / 16 * 16;
            for (int e = tid; e < npad * m; e += 256) {
                const int l = e / m, c = e - (e / m) * m;
                Qs[l * ldqs + c] = (l < n) ? Qg[(size_t)l * m + c] : __float2bfloat16_rn(0.f);
            }
            loaded = item;
        }
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int k0 = 0; k0 < n; k0 += KC) {
            __syncthreads();
            for (int e = tid; e < 128 * KC; e += 256) {
                const int r = e / KC, c = e - (e / KC) * KC;
                float v = 0.f;
                if (r0 + r < rows && k0 + c < n) {
                    const Tin* p = X + (int64_t)(r0 + r) * ld + k0 + c;
                    if constexpr (std::is_same<Tin, float>::value) v = __ldg(p);
                    else v = __bfloat162float(*p);
                }
                __nv_bfloat16 hi, lo;
                split_bf16(v, hi, lo);
                Xh[r * LDX + c] = hi;
                Xl[r * LDX + c] = lo;
            }
            __syncthreads();
            const int kmax = min(KC, ((n - k0) + 15) / 16 * 16);
            for (int kk = 0; kk < kmax; kk += 16) {
                const int mat = lane >> 3, rr = lane & 7;
                const int arow = warp * 16 + ((mat & 1) ? 8 : 0) + rr, acol = kk + ((mat >> 1) ? 8 : 0);
                uint32_t ah[4], al[4];
                ldsm_x4(smem_u32(Xh + arow * LDX + acol), ah[0], ah[1], ah[2], ah[3]);
                ldsm_x4(smem_u32(Xl + arow * LDX + acol), al[0], al[1], al[2], al[3]);
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    if (2 * np >= ntn) break;
                    const int t = k0 + kk + rr + ((mat & 1) ? 8 : 0);
                    const int c = np * 16 + ((mat >> 1) ? 8 : 0);
                    uint32_t b0, b1, b2, b3;
                    if (2 * np + 1 < ntn) {
                        ldsm_x4_t(smem_u32(Qs + t * ldqs + c), b0, b1, b2, b3);
                    } else {
                        ldsm_x2_t(smem_u32(Qs + t * ldqs + np * 16), b0, b1);
                        b2 = b3 = 0;
                    }
                    mma_bf16(acc[2 * np], ah[0], ah[1], ah[2], ah[3], b0, b1);
                    mma_bf16(acc[2 * np], al[0], al[1], al[2], al[3], b0, b1);
                    if (2 * np + 1 < ntn) {
                        mma_bf16(acc[2 * np + 1], ah[0], ah[1], ah[2], ah[3], b2, b3);
                        mma_bf16(acc[2 * np + 1], al[0], al[1], al[2], al[3], b2, b3);
                    }
                }
            }
        }
        float* Y = sc.Y + (size_t)src.ybase(item) * m;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntn) break;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = r0 + warp * 16 + (lane >> 2) + ((e >> 1) ? 8 : 0);
                const int c = nt * 8 + 2 * (lane & 3) + (e & 1);
                if (r < rows) Y[(size_t)r * m + c] = acc[nt][e];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 4. Rayleigh-Ritz on span(Q~) and the outputs.
// ---------------------------------------------------------------------------
template <typename TR>
__device__ void sym_pairs_accumulate(const float* __restrict__ A, int64_t lda, const __nv_bfloat16* __restrict__ Ab,
                                     int rows, int m, float* st, TR* out, int ldo) {
    // out[a][c] = sum_r A[r][a] A[r][c]  (upper triangle computed, mirrored)
    const int tid = threadIdx.x, nt = blockDim.x, lds = m + 1;
    constexpr int NS = (ZS_MAXM * (ZS_MAXM + 1) / 2 + 255) / 256;
    const int np = m * (m + 1) / 2;
    TR acc[NS];
    int pa[NS], pc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        acc[s] = 0;
        int e = tid + s * nt, aa = 0;
        while (aa < m && e >= m - aa) { e -= m - aa; ++aa; }
        pa[s] = aa;
        pc[s] = aa + e;
    }
    for (int r0 = 0; r0 < rows; r0 += 32) {
        const int nr = min(32, rows - r0);
        __syncthreads();
        for (int e = tid; e < nr * m; e += nt) {
            const int r = e / m, c = e - (e / m) * m;
            st[r * lds + c] = A ? A[(int64_t)(r0 + r) * lda + c] : __bfloat162float(Ab[(int64_t)(r0 + r) * lda + c]);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (tid + s * nt < np) {
                TR t = 0;
                for (int r = 0; r < nr; ++r) t += (TR)st[r * lds + pa[s]] * (TR)st[r * lds + pc[s]];
                acc[s] += t;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (tid + s * nt < np) {
            out[pa[s] * ldo + pc[s]] = acc[s];
            out[pc[s] * ldo + pa[s]] = acc[s];
        }
    __syncthreads();
}

template <class Src, bool REF, bool QUERY>
__global__ void __launch_bounds__(256) k_rr(Src src, TcScratch sc, int n, int kw) {
    using TR = typename std::conditional<REF, double, float>::type;
    extern __shared__ __align__(16) char dsm[];
    __shared__ JacobiScratch<float> js;
    __shared__ JacobiScratch<double> jd;
    __shared__ int perm[ZS_MAXM];
    __shared__ TR theta[ZS_MAXM];
    __shared__ float sig[ZS_MAXM];
    __shared__ int sgn[ZS_MAXM];
    __shared__ int s_rank;
    const int m = sc.m, ld = m + 1;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    TR* Hb = (TR*)dsm;                     // H, then H'
    TR* Cb = Hb + (size_t)m * ld;          // C, then L, then W (REF)
    TR* Li = Cb + (size_t)m * ld;          // L^{-1}, then Z
    TR* Tb = Li + (size_t)m * ld;          // temp, then X (REF)
    float* A_T = (float*)(Tb + (size_t)m * ld);
    float* Z_T = A_T + (size_t)m * ld;
    float* stg = A_T;                      // staging aliases the Jacobi buffers
    for (int item = blockIdx.x; item < src.count(); item += gridDim.x) {
        const int rows = src.rows(item);
        const float* Y = sc.Y + (size_t)src.ybase(item) * m;
        const __nv_bfloat16* Qb = sc.Qb + (size_t)item * n * m;
        sym_pairs_accumulate<TR>(Y, m, nullptr, rows, m, stg, Hb, ld);
        sym_pairs_accumulate<TR>(nullptr, m, Qb, n, m, stg, Cb, ld);
        // Cholesky C = L L^T in place (lower)
        for (int j = 0; j < m; ++j) {
            if (tid == 0) {
                TR d = Cb[j * ld + j];
                for (int p = 0; p < j; ++p) d -= Cb[j * ld + p] * Cb[j * ld + p];
                Cb[j * ld + j] = d > TR(1e-12) ? (TR)sqrt((double)d) : TR(1e-6);
            }
            __syncthreads();
            for (int i = j + 1 + tid; i < m; i += nt) {
                TR d = Cb[i * ld + j];
                for (int p = 0; p < j; ++p) d -= Cb[i * ld + p] * Cb[j * ld + p];
                Cb[i * ld + j] = d / Cb[j * ld + j];
            }
            __syncthreads();
        }
        // L^{-1} by forward substitution, one column per thread
        for (int c = tid; c < m; c += nt) {
            for (int i = 0; i < m; ++i) {
                if (i < c) { Li[i * ld + c] = 0; continue; }
                TR d = (i == c) ? TR(1) : TR(0);
                for (int p = c; p < i; ++p) d -= Cb[i * ld + p] * Li[p * ld + c];
                Li[i * ld + c] = d / Cb[i * ld + i];
            }
        }
        __syncthreads();
        // H' = L^{-1} H L^{-T}
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            TR d = 0;
            for (int p = 0; p <= i; ++p) d += Li[i * ld + p] * Hb[p * ld + c];
            Tb[i * ld + c] = d;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            TR d = 0;
            for (int p = 0; p <= c; ++p) d += Tb[i * ld + p] * Li[c * ld + p];
            Hb[i * ld + c] = d;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            const TR v = (Hb[i * ld + c] + Hb[c * ld + i]) * TR(0.5);
            A_T[i * ld + c] = (float)v;
        }
        __syncthreads();
        if constexpr (REF) {
            for (int e = tid; e < m * m; e += nt) {
                const int i = e / m, c = e - (e / m) * m;
                Tb[i * ld + c] = (Hb[i * ld + c] + Hb[c * ld + i]) * 0.5;
            }
            __syncthreads();
            for (int e = tid; e < m * m; e += nt) Hb[(e / m) * ld + e % m] = Tb[(e / m) * ld + e % m];
            __syncthreads();
        }
        // small core: FP32 Jacobi, then (REF) one FP64 refinement on Z^T H' Z
        SmallEig<float, REF> se;
        se.A_T = A_T;
        se.Z_T = Z_T;
        se.A_R = REF ? (double*)Hb : nullptr;
        se.X = REF ? (double*)Tb : nullptr;
        se.W = REF ? (double*)Cb : nullptr;
        se.ld = ld;
        TR* Zo;
        small_eig<float, REF>(se, m, js, jd, theta, perm, Zo);
        // Z = L^{-T} W(:, perm) for the kw wanted pairs -> Li (its own rows free as we go? use Tb/Hb)
        TR* Zc = REF ? (TR*)Hb : Tb;           // m x kw (ld)
        if (REF) {
            // Hb held A_R (consumed); Zo = X = Tb
            for (int e = tid; e < m * kw; e += nt) {
                const int a = e / kw, c = e - (e / kw) * kw;
                TR d = 0;
                for (int p = a; p < m; ++p) d += Li[p * ld + a] * Zo[p * ld + perm[c]];
                Zc[a * ld + c] = d;
            }
        } else {
            for (int e = tid; e < m * kw; e += nt) {
                const int a = e / kw, c = e - (e / kw) * kw;
                TR d = 0;
                for (int p = a; p < m; ++p) d += Li[p * ld + a] * (TR)Zo[p * ld + perm[c]];
                Zc[a * ld + c] = d;
            }
        }
        __syncthreads();
        int kcap = kw;
        if constexpr (QUERY) kcap = src.a.plans[item].kcap;
        else kcap = min(kw, min(rows, n));
        if (tid == 0) s_rank = 0;
        __syncthreads();
        const float s0 = sqrtf(fmaxf((float)theta[0], 0.f));
        for (int c = tid; c < kw; c += nt) {
            float s = sqrtf(fmaxf((float)theta[c], 0.f));
            if (!(c < kcap && s > kRankTolF32 * s0)) s = 0.f;
            sig[c] = s;
            if (s > 0.f) atomicAdd(&s_rank, 1);
        }
        // sign: largest-|.| entry of v_c = Q~ z_c positive (lowest index on ties)
        for (int c = wid; c < kw; c += nw) {
            float best = -1.f;
            int bi = 0x7fffffff;
            for (int l = lane; l < n; l += 32) {
                float v = 0.f;
                for (int a = 0; a < m; ++a) v += __bfloat162float(Qb[(size_t)l * m + a]) * (float)Zc[a * ld + c];
                const float av = fabsf(v);
                if (av > best || (av == best && l < bi)) { best = av; bi = l; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                float v = 0.f;
                for (int a = 0; a < m; ++a) v += __bfloat162float(Qb[(size_t)bi * m + a]) * (float)Zc[a * ld + c];
                sgn[c] = v < 0.f ? -1 : 1;
            }
        }
        __syncthreads();
        // V^T (kw x n) and U = Y Z Sigma^-1 (rows x kw)
        float* vt_out;
        float* u_out;
        int64_t urows;
        if constexpr (QUERY) {
            const QPlan& P = src.a.plans[item];
            vt_out = (float*)src.a.vr + (size_t)item * src.a.kq * n;
            u_out = (float*)src.a.C + (size_t)P.slab0 * src.a.k * src.a.kq;
            urows = rows;
            float* sr = (float*)src.a.sr + (size_t)item * src.a.kq;
            for (int c = tid; c < src.a.kout; c += nt) {
                const float s = c < kw ? sig[c] : 0.f;
                if (c < kw) sr[c] = s;
                ((float*)P.S_out)[c] = s;
            }
            if (tid == 0 && P.rank) *P.rank = s_rank;
        } else {
            const int slot = src.c.slot0 + item;
            vt_out = (float*)src.c.vt + (size_t)slot * src.c.k * n;
            u_out = (float*)src.c.U + (size_t)slot * src.c.b * src.c.k;
            urows = src.c.b;
            float* so = (float*)src.c.sig + (size_t)slot * src.c.k;
            for (int c = tid; c < src.c.k; c += nt) so[c] = c < kw ? sig[c] : 0.f;
        }
        for (int e = tid; e < kw * n; e += nt) {
            const int c = e / n, l = e - (e / n) * n;
            float v = 0.f;
            if (sig[c] > 0.f) {
                for (int a = 0; a < m; ++a) v += __bfloat162float(Qb[(size_t)l * m + a]) * (float)Zc[a * ld + c];
                v *= (float)sgn[c];
            }
            vt_out[e] = v;
        }
        __syncthreads();
        if constexpr (QUERY) {
            const QPlan& P = src.a.plans[item];
            for (int e = tid; e < n * src.a.kout; e += nt) {
                const int l = e / src.a.kout, c = e - (e / src.a.kout) * src.a.kout;
                ((float*)P.V_out)[(size_t)l * P.ldv + c] = c < kw ? vt_out[(size_t)c * n + l] : 0.f;
            }
        }
        for (int e = tid; e < urows * kw; e += nt) {
            const int r = e / kw, c = e - (e / kw) * kw;
            float v = 0.f;
            if (r < rows && sig[c] > 0.f) {
                const float* yr = Y + (size_t)r * m;
                TR d = 0;
                for (int a = 0; a < m; ++a) d += (TR)yr[a] * Zc[a * ld + c];
                v = (float)d / sig[c] * (float)sgn[c];
            }
            u_out[e] = v;
        }
        __syncthreads();
    }
}

// Query boundary slabs: C_slab <- (Sigma V~ Sigma~^{-1}) C_slab  (k x kq), in place.
__global__ void __launch_bounds__(256) k_bfix(QueryArgs a) {
    extern __shared__ __align__(16) char dsm[];
    const int k = a.k, kq = a.kq;
    float* Tc = (float*)dsm;          // k x k
    float* Us = Tc + (size_t)k * k;   // k x kq
    const int nq = a.hdr->nq;
    for (int p = blockIdx.x; p < 2 * nq; p += gridDim.x) {
        const int q = p >> 1, side = p & 1;
        const QPlan& P = a.plans[q];
        if (side == 1 && P.nslab == 1) continue;
        const int t = side ? P.nslab - 1 : 0;
        float* Cg = (float*)a.C + (size_t)(P.slab0 + t) * k * kq;
        const float* tg = (const float*)a.tco + (size_t)p * k * k;
        __syncthreads();
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) Tc[e] = tg[e];
        for (int e = threadIdx.x; e < k * kq; e += blockDim.x) Us[e] = Cg[e];
        __syncthreads();
        for (int e = threadIdx.x; e < k * kq; e += blockDim.x) {
            const int aa = e / kq, c = e - (e / kq) * kq;
            float acc = 0.f;
            for (int j = 0; j < k; ++j) acc += Tc[aa * k + j] * Us[j * kq + c];
            Cg[e] = acc;
        }
    }
}

}  // namespace zs
