// zs_tc_kernels.cuh - truncated SVD of many tall matrices X_j (rows_j x n) on
// tensor cores.  Used for the blocks of the storage phase (Section 3.2) and for
// the stacked Sigma V^T matrix of each query's Stitched-SVD (Algorithm 2).
//
// The SVD is a Rayleigh-Ritz step on a sketched subspace, arranged so that
// tensor cores carry the O(rows n m) work without giving up FP32 accuracy:
//   1. k_sketch     S = X^T (X Omega), Omega random signs (bf16 operands, fp32
//                   accumulate), by a cluster of CTAs per item; only locates
//                   the dominant subspace.  (k_gram_lo + k_subspace: the same
//                   from the bf16 Gram, for shapes outside the sketch's limits.)
//   2. k_orth       Q~ = orthonormal basis of S (two-pass Gram-Schmidt),
//                   rounded to tf32, and Q~^T Q~.
//   3. k_project    Y = X Q~ with X split into two tf32 terms: Y to FP32
//                   accuracy (Q~ is exact in tf32, so nothing of Q is lost).
//   4. k_rr_core    Rayleigh-Ritz on span(Q~): Y^T Y z = theta (Q~^T Q~) z
//                   (register core for m <= 32, else the shared-memory core);
//      k_rr_out     sigma = sqrt(theta), V = Q~ Z, U = Y Z Sigma^{-1}.
// Accuracy of sigma, U, V is set by steps 3-4 (FP32 products of the exact data
// against an exact basis); steps 1-2 only decide how good the subspace is,
// which is exponentially good in lambda_{m+1} / lambda_k.
#pragma once

#include <cooperative_groups.h>
#include <cuda.h>
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
    // row r of item j and the factor its values are scaled by; `Ctx` holds
    // what is fixed per item (loaded once, outside the row loops)
    struct Ctx { const char* base; };
    __device__ __forceinline__ Ctx ctx(int j, int elem) const {
        return Ctx{(const char*)c.A + (size_t)j * c.b * c.lda * elem};
    }
    template <typename Tin>
    __device__ __forceinline__ const Tin* row(const Ctx& x, int r, float& scale) const {
        scale = 1.f;
        return (const Tin*)x.base + (size_t)r * c.lda;
    }
    // the factors the storage step wrote for item j: U rows (row stride kw),
    // sigma (kw), V^T (kw x n); kcap = columns that can be nonzero
    __device__ __forceinline__ float* u_out(int j, int kw) const {
        return (float*)c.U + (size_t)(c.slot0 + j) * c.b * kw;
    }
    __device__ __forceinline__ float* sig_out(int j, int kw) const {
        return (float*)c.sig + (size_t)(c.slot0 + j) * kw;
    }
    __device__ __forceinline__ float* vt_out(int j, int kw) const {
        return (float*)c.vt + (size_t)(c.slot0 + j) * kw * c.n;
    }
    __device__ __forceinline__ float* w_out(int j, int kw) const {
        return c.w ? (float*)c.w + (size_t)(c.slot0 + j) * kw * c.n : nullptr;
    }
    __device__ __forceinline__ int kcap(int j, int kw) const { return min(kw, min(rows(j), c.n)); }
    __device__ __forceinline__ int64_t tile0(int j) const { return (int64_t)j * ((c.b + 127) / 128); }
    __device__ __forceinline__ int64_t ntiles() const { return (int64_t)c.nblk * ((c.b + 127) / 128); }
    __device__ __forceinline__ void tile_item(int64_t t, int& item, int& rt) const {
        const int tpi = (c.b + 127) / 128;
        item = (int)(t / tpi);
        rt = (int)(t - (int64_t)item * tpi);
    }
};

struct SrcQuery {
    QueryArgs a;
    __device__ __forceinline__ int count() const { return a.hdr->nq; }
    // ragged stacks (a.rowmap): the stacked row count that k_ragged_map
    // recorded in the plan; otherwise k rows per slab
    __device__ __forceinline__ int rows(int q) const {
        return a.rowmap ? a.plans[q].pad1 : a.plans[q].nslab * a.k;
    }
    __device__ __forceinline__ int64_t ld() const { return a.n; }
    __device__ __forceinline__ const void* X(int q, int elem) const {
        return (const char*)a.M + (size_t)a.plans[q].slab0 * a.k * a.n * elem;
    }
    __device__ __forceinline__ int64_t ybase(int q) const { return a.plans[q].slab0 * a.k; }
    // row r of query q's stacked matrix M (Algorithm 2, stack step).  The two
    // boundary slabs are written to M by the Partial-SVD kernel; the interior
    // slabs are the store's Sigma_i V_i^T, read in place when the store keeps
    // them (wst) and otherwise copied into M by the stack kernel.
    // kmagic = ceil(2^32 / k): the slab of row r is umulhi(r, kmagic), exact
    // for r < 2^32 / k (no integer division per row)
    struct Ctx { const char* base; const char* wbase; int nslab; uint32_t kmagic; const int* map; };
    __device__ __forceinline__ Ctx ctx(int q, int elem) const {
        const QPlan& P = a.plans[q];
        return Ctx{(const char*)a.M + (size_t)P.slab0 * a.k * a.n * elem,
                   a.wst ? (const char*)a.wst + (size_t)P.S * a.k * a.n * elem : nullptr, P.nslab,
                   (uint32_t)((0x100000000ull + (uint64_t)a.k - 1) / (uint64_t)a.k),
                   a.rowmap ? a.rowmap + P.slab0 * a.k : nullptr};
    }
    template <typename Tin>
    __device__ __forceinline__ const Tin* row(const Ctx& x, int r, float& scale) const {
        scale = 1.f;
        if (x.map) {              // ragged: the row map names the source row
            const int v = x.map[r];
            return v >= 0 ? (const Tin*)a.wst + (size_t)v * a.n : (const Tin*)a.M + (size_t)(-1 - v) * a.n;
        }
        if (x.wbase) {
            const int t = (int)__umulhi((uint32_t)r, x.kmagic);
            if (t > 0 && t < x.nslab - 1) return (const Tin*)x.wbase + (size_t)r * a.n;
        }
        return (const Tin*)x.base + (size_t)r * a.n;
    }
    // the stitched factors of query q: U_r rows = the lift coefficients C
    // (row stride kq), sigma (kq), V_r^T (kq x n); kcap from the plan
    __device__ __forceinline__ float* u_out(int q, int kw) const {
        return (float*)(a.rowmap ? a.Cc : a.C) + (size_t)a.plans[q].slab0 * a.k * kw;
    }
    __device__ __forceinline__ float* sig_out(int q, int kw) const { return (float*)a.sr + (size_t)q * kw; }
    __device__ __forceinline__ float* vt_out(int q, int kw) const { return (float*)a.vr + (size_t)q * kw * a.n; }
    __device__ __forceinline__ float* w_out(int, int) const { return nullptr; }
    __device__ __forceinline__ int kcap(int q, int kw) const { return min(kw, a.plans[q].kcap); }
    __device__ __forceinline__ int64_t tile0(int q) const { return a.plans[q].pad0; }
    __device__ __forceinline__ int64_t ntiles() const { return a.hdr->ntiles_total; }
    __device__ __forceinline__ void tile_item(int64_t t, int& item, int& rt) const {
        int lo = 0, hi = a.hdr->nq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.plans[mid].pad0 <= t) lo = mid; else hi = mid - 1;
        }
        item = lo;
        rt = (int)(t - a.plans[lo].pad0);
    }
};

// Scratch for the tensor path (per launch).
struct TcScratch {
    float* G;               // items x n x n
    float* Qf;              // items x n x m: Q~, values exact in tf32
    float* Qt;              // items x round16(m) x n: Q~^T for the tcgen05 projection (or null)
    float* Y;               // (sum of rows) x m, row offsets from Src::ybase
    void* ews;              // per-CTA workspace (subspace Y block), ews_ctas x n x (m+1) floats
    int ews_ctas;
    int m;                  // subspace width (multiple of 8, <= 64)
    int power_its;          // power steps on G~
    float* Hp;              // per 128-row tile of Y: Y_t^T Y_t (m x m)
    float* Cq;              // items x m x m: Q~^T Q~
    float* Zs;              // items x m x kw: Ritz coefficients
    float* th;              // items x kw: Ritz values (sigma^2)
    float* thm;             // items x m: all m Ritz values, descending (accuracy test)
    int* list;              // 2 + items ints: count, work counter, then the items that failed the accuracy test
    int* cplan;             // 2 items + 1 ints: k_check's part plan for stacked query matrices (or null)
    int* noconv;            // incremented per item whose refinement stopped at its pass cap (or null)
    int* refined;           // incremented per item refined (or null)
    double xi;              // storage phase, xi > 0: energy rule (Eq. 1); only ranks < k_i are tested
    const double* energy;   // xi > 0: each item's squared Frobenius norm
    int* kxi;               // xi > 0: each item's rank k_i, recorded for the truncation
    int* fault;             // set to 1 by a kernel whose bounded wait gave up (or null)
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
__global__ void __launch_bounds__(256, 1) k_gram_lo(Src src, TcScratch sc, int n) {
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
    const bool vecb = std::is_same<Tin, __nv_bfloat16>::value && (ld % 4 == 0) && (n % 4 == 0);
    for (int item = blockIdx.y; item < src.count(); item += gridDim.y) {
        const Tin* X = (const Tin*)src.X(item, sizeof(Tin));
        const bool xal = vec && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
        // bf16 rows: four values as one 8-byte load, kept as they are (exact in bf16)
        const bool xalb = vecb && ((reinterpret_cast<uintptr_t>(X) & 7) == 0);
        const auto cx = src.ctx(item, sizeof(Tin));
        const int rows = src.rows(item);
        float acc[4][4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
        // Each thread owns 4 groups of 4 consecutive columns per panel and keeps
        // the next 32-row chunk in registers while the current one is multiplied.
        const int npnl = diag ? 1 : 2;
        float pre[2][4][4];
        uint2 preb[2][4];
        auto fetch = [&](int r0) {
#pragma unroll
            for (int pnl = 0; pnl < 2; ++pnl) {
                if (pnl >= npnl) break;
                const int P0 = pnl ? J0 : I0;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int f = tid + g * 256;
                    const int r = f >> 5, c = (f & 31) * 4, gr = r0 + r, gc = P0 + c;
                    float* v = pre[pnl][g];
                    v[0] = v[1] = v[2] = v[3] = 0.f;
                    if constexpr (std::is_same<Tin, __nv_bfloat16>::value) {
                        if (xalb) {
                            uint2 q = make_uint2(0u, 0u);
                            if (gr < rows && gc < n) {
                                float sc = 1.f;
                                q = *reinterpret_cast<const uint2*>(src.template row<Tin>(cx, gr, sc) + gc);
                            }
                            preb[pnl][g] = q;
                            continue;
                        }
                    }
                    if (gr < rows) {
                        float sc = 1.f;
                        const Tin* src_p = src.template row<Tin>(cx, gr, sc) + gc;
                        if constexpr (std::is_same<Tin, float>::value) {
                            if (xal && gc + 3 < n) {
                                const float4 q = ld4<float>(src_p);
                                v[0] = q.x * sc; v[1] = q.y * sc; v[2] = q.z * sc; v[3] = q.w * sc;
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (gc + e < n) v[e] = (float)src_p[e] * sc;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (gc + e < n) v[e] = __bfloat162float(src_p[e]) * sc;
                        }
                    }
                }
            }
        };
        fetch(0);
        for (int r0 = 0; r0 < rows; r0 += 32) {
            __syncthreads();
#pragma unroll
            for (int pnl = 0; pnl < 2; ++pnl) {
                if (pnl >= npnl) break;
                __nv_bfloat16* D = pnl ? XJ : XI;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int f = tid + g * 256;
                    const int r = f >> 5, c = (f & 31) * 4;
                    const float* v = pre[pnl][g];
                    uint32_t* dp = reinterpret_cast<uint32_t*>(D + r * LDS + c);
                    if (std::is_same<Tin, __nv_bfloat16>::value && xalb) {
                        dp[0] = preb[pnl][g].x;
                        dp[1] = preb[pnl][g].y;
                        continue;
                    }
                    dp[0] = pack_bf16(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
                    dp[1] = pack_bf16(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
                }
            }
            __syncthreads();
            if (r0 + 32 < rows) fetch(r0 + 32);     // in flight during the MMAs
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
template <class Src, int MB>
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
        // the pivoted columns of G~, eight loads in flight per thread
        for (int e0 = tid; e0 < n * m; e0 += 8 * nt) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * nt;
                const int c = e / n, i = e - (e / n) * n;
                v[u] = e < n * m ? __ldg(G + (size_t)piv[c] * n + i) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * nt;
                const int c = e / n, i = e - (e / n) * n;
                if (e < n * m) Q[i * ldq + c] = v[u];
            }
        }
        __syncthreads();
        mgs_orth<float>(Q, ldq, n, m, red, coef);
        for (int it = 0; it < sc.power_its; ++it) {
            // Y = G~ Q~ in register tiles of 4 rows x 8 columns per thread.
            // G~ is symmetric, so row l of G~ holds the l-th coefficient of
            // rows i0..i0+3: one 16-byte load feeds 32 fused multiply-adds.
            const int cgn = (m + 7) >> 3, tasks = ((n + 3) >> 2) * cgn;
            const bool vec = (n & 3) == 0;
            for (int t = tid; t < tasks; t += nt) {
                const int rg = t / cgn, c0 = (t - rg * cgn) * 8, i0 = rg * 4;
                float acc[4][8];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
                const float* Gc = G + i0;
                // eight rows of G~ in flight per thread: the loop is bound by
                // the latency of these loads, not by the multiply-adds
                for (int l0 = 0; l0 < n; l0 += 8) {
                    const int lim = min(8, n - l0);
                    float g[8][4];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float* gr = Gc + (size_t)(l0 + u) * n;
                        if (vec) {
                            const float4 v = u < lim ? __ldg(reinterpret_cast<const float4*>(gr))
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                            g[u][0] = v.x; g[u][1] = v.y; g[u][2] = v.z; g[u][3] = v.w;
                        } else {
#pragma unroll
                            for (int r = 0; r < 4; ++r) g[u][r] = (u < lim && i0 + r < n) ? __ldg(gr + r) : 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (u < lim) {
                            const float* qr = Q + (l0 + u) * ldq + c0;
                            float q[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) q[c] = (c0 + c < m) ? qr[c] : 0.f;
#pragma unroll
                            for (int r = 0; r < 4; ++r)
#pragma unroll
                                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(g[u][r], q[c], acc[r][c]);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (i0 + r < n && c0 + c < m) Y[(i0 + r) * ldq + c0 + c] = acc[r][c];
            }
            __syncthreads();
            for (int e = tid; e < n * m; e += nt) {
                const int i = e / m, c = e - (e / m) * m;
                Q[i * ldq + c] = Y[i * ldq + c];
            }
            __syncthreads();
            mgs_orth<float>(Q, ldq, n, m, red, coef);
        }
        float* Qf = sc.Qf + (size_t)item * n * m;
        __syncthreads();
        for (int e = tid; e < n * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            const float h = __uint_as_float(to_tf32(Q[i * ldq + c]));
            Qf[e] = h;
            Q[i * ldq + c] = h;                         // Q~ as it will be used
        }
        __syncthreads();
        if (sc.Qt) {
            const int np = (m + 15) / 16 * 16;
            float* Qt = sc.Qt + (size_t)item * np * n;
            for (int e = tid; e < n * np; e += nt) {
                const int i = e / np, c = e - (e / np) * np;
                Qt[(size_t)(i >> 5) * np * 32 + tc5_canon(c, i & 31, 32)] = c < m ? Q[i * ldq + c] : 0.f;
            }
        }
        // C = Q~^T Q~ (exact products of bf16 values, fp32 sums)
        float* Cq = sc.Cq + (size_t)item * m * m;
        for (int e = tid; e < m * m; e += nt) {
            const int a = e / m, c = e - (e / m) * m;
            if (c < a) continue;
            float acc = 0.f;
            for (int i = 0; i < n; ++i) acc += Q[i * ldq + a] * Q[i * ldq + c];
            Cq[a * m + c] = acc;
            Cq[c * m + a] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// 3. Y = X Q~ for 128-row tiles on tf32 tensor cores: X = X_hi + X_lo with both
//    terms tf32 (~21 significant bits; bf16 inputs are exact in X_hi alone) and
//    Q~ exact in tf32, so Y carries FP32 accuracy.  X and Q~ arrive in 32-column
//    chunks by cp.async into a double buffer; fragments are split in registers.
// ---------------------------------------------------------------------------
constexpr int kPjKC = 32;              // columns per chunk
constexpr int kPjLDX = kPjKC + 4;      // X stage row stride (floats): conflict-free A fragments
constexpr int kPjStages = 3;
__host__ __device__ __forceinline__ int pj_ldq(int m) { return (m + 31) / 32 * 32 + 8; }   // = 8 mod 32
__host__ __device__ __forceinline__ size_t pj_stage_floats(int m) {
    return (size_t)128 * kPjLDX + (size_t)kPjKC * pj_ldq(m);
}
__host__ __device__ __forceinline__ size_t project_smem_bytes(int m) {
    const size_t st = kPjStages * pj_stage_floats(m) * 4;
    const size_t ys = (size_t)128 * pj_ldq(m) * 4;          // Y tile for Y^T Y, reuses the stages
    return st > ys ? st : ys;
}

// tf32 split of one fragment value: x = hi + lo with both terms tf32
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// Cheaper split for streamed data: hi = x with the 13 low mantissa bits
// cleared, lo = x - hi (exact in fp32) likewise truncated; x - (hi + lo) is
// below 2^-20 |x|.  Plain bit operations, no conversion instructions.
__device__ __forceinline__ void tf32_split_trunc(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u;
}

template <class Src, typename Tin>
__global__ void __launch_bounds__(256, 3) k_project(Src src, TcScratch sc, int n) {
    extern __shared__ __align__(16) float fsm[];
    const int m = sc.m, ldq = pj_ldq(m), ntn = m / 8;
    const size_t sf = pj_stage_floats(m);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int64_t ld = src.ld();
    const int nch = (n + kPjKC - 1) / kPjKC;
    constexpr bool kF32 = std::is_same<Tin, float>::value;
    const int64_t ntiles = src.ntiles();
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int item, rt;
        src.tile_item(tile, item, rt);
        const int rows = src.rows(item);
        const int r0 = rt * 128;
        if (r0 >= rows) continue;
        const char* X = (const char*)src.X(item, sizeof(Tin));
        const auto cx = src.ctx(item, sizeof(Tin));
        const float* Qg = sc.Qf + (size_t)item * n * m;
        const bool async_x = kF32 && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
        const bool async_q = (m % 4 == 0) && ((reinterpret_cast<uintptr_t>(Qg) & 15) == 0);
        // stage chunk c into buffer b: X rows r0.., columns 32c..; Q~ rows 32c..
        auto issue = [&](int c, int b) {
            float* Xs = fsm + (size_t)b * sf;
            float* Qs = Xs + 128 * kPjLDX;
            const int k0 = c * kPjKC;
            for (int f = tid; f < 128 * (kPjKC / 4); f += 256) {
                const int r = f / (kPjKC / 4), c4 = (f - r * (kPjKC / 4)) * 4;
                const int gr = r0 + r, gc = k0 + c4;
                float* dst = Xs + r * kPjLDX + c4;
                float rs;
                if (async_x) {
                    const int nb = (gr < rows && gc < n) ? 4 * min(4, n - gc) : 0;
                    const float* sp = nb ? (const float*)src.template row<Tin>(cx, gr, rs) + gc : (const float*)X;
                    cp_async16(dst, sp, nb);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float v = 0.f;
                        if (gr < rows && gc + e < n) {
                            const Tin* p = src.template row<Tin>(cx, gr, rs) + gc + e;
                            if constexpr (kF32) v = __ldg(p);
                            else v = __bfloat162float(*p);
                        }
                        dst[e] = v;
                    }
                }
            }
            for (int f = tid; f < kPjKC * (ldq / 4); f += 256) {
                const int r = f / (ldq / 4), c4 = (f - r * (ldq / 4)) * 4;
                const int gr = k0 + r;
                float* dst = Qs + r * ldq + c4;
                if (async_q) {
                    const int nb = (gr < n && c4 < m) ? 16 : 0;
                    cp_async16(dst, nb ? Qg + (size_t)gr * m + c4 : Qg, nb);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) dst[e] = (gr < n && c4 + e < m) ? Qg[(size_t)gr * m + c4 + e] : 0.f;
                }
            }
            cp_async_commit();
        };
        float acc[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        __syncthreads();                    // previous tile's readers are done with the stages
        issue(0, 0);
        if (nch > 1) issue(1, 1);
        for (int c = 0; c < nch; ++c) {
            if (c + 2 < nch) {
                issue(c + 2, (c + 2) % kPjStages);
                cp_async_wait<2>();
            } else if (c + 1 < nch) {
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float* Xs = fsm + (size_t)(c % kPjStages) * sf;
            const float* Qs = Xs + 128 * kPjLDX;
            const int kk_max = min(kPjKC, n - c * kPjKC);
            for (int kk = 0; kk < kk_max; kk += 8) {
                const float* xa = Xs + (warp * 16 + g) * kPjLDX + kk + t4;
                uint32_t h0, h1, h2, h3, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
                if constexpr (kF32) {
                    tf32_split_trunc(xa[0], h0, l0);
                    tf32_split_trunc(xa[8 * kPjLDX], h1, l1);
                    tf32_split_trunc(xa[4], h2, l2);
                    tf32_split_trunc(xa[8 * kPjLDX + 4], h3, l3);
                } else {                    // bf16 values are exact in tf32
                    h0 = __float_as_uint(xa[0]);
                    h1 = __float_as_uint(xa[8 * kPjLDX]);
                    h2 = __float_as_uint(xa[4]);
                    h3 = __float_as_uint(xa[8 * kPjLDX + 4]);
                }
                const float* qb = Qs + (kk + t4) * ldq + g;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    if (nt >= ntn) break;
                    const uint32_t b0 = __float_as_uint(qb[nt * 8]), b1 = __float_as_uint(qb[4 * ldq + nt * 8]);
                    if constexpr (kF32) mma_tf32(acc[nt], l0, l1, l2, l3, b0, b1);
                    mma_tf32(acc[nt], h0, h1, h2, h3, b0, b1);
                }
            }
            __syncthreads();                // buffer (c % kPjStages) is refilled two chunks later
        }
        float* Y = sc.Y + (size_t)src.ybase(item) * m;
        float* Ys = fsm;                    // 128 x ldq, zero past row `rows` and column m
        const int mp = (m + 15) / 16 * 16;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= ntn) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rl = warp * 16 + g + 8 * h;
                const int cc = nt * 8 + 2 * t4;
                const int r = r0 + rl;
                const float v0 = r < rows ? acc[nt][2 * h] : 0.f, v1 = r < rows ? acc[nt][2 * h + 1] : 0.f;
                if (r < rows) *reinterpret_cast<float2*>(Y + (size_t)r * m + cc) = make_float2(v0, v1);
                Ys[rl * ldq + cc] = v0;
                Ys[rl * ldq + cc + 1] = v1;
            }
        }
        if (mp > m)
            for (int e = tid; e < 128 * (mp - m); e += 256) Ys[(e / (mp - m)) * ldq + m + e % (mp - m)] = 0.f;
        __syncthreads();
        // this tile's Y^T Y on tensor cores, Y split into two tf32 terms (three
        // products); each warp owns 16 x 8 output tiles in a fixed order
        float* Hp = sc.Hp + (size_t)tile * m * m;
        const int nmt = mp / 16;
        for (int ot = warp; ot < nmt * ntn; ot += 8) {
            const int mt = ot / ntn, nt = ot - (ot / ntn) * ntn;
            float h[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k0 = 0; k0 < 128; k0 += 8) {
                const float* ya = Ys + (k0 + t4) * ldq + mt * 16 + g;
                const float* yb = Ys + (k0 + t4) * ldq + nt * 8 + g;
                uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3, bh0, bl0, bh1, bl1;
                tf32_split(ya[0], ah0, al0);
                tf32_split(ya[8], ah1, al1);
                tf32_split(ya[4 * ldq], ah2, al2);
                tf32_split(ya[4 * ldq + 8], ah3, al3);
                tf32_split(yb[0], bh0, bl0);
                tf32_split(yb[4 * ldq], bh1, bl1);
                mma_tf32(h, al0, al1, al2, al3, bh0, bh1);
                mma_tf32(h, ah0, ah1, ah2, ah3, bl0, bl1);
                mma_tf32(h, ah0, ah1, ah2, ah3, bh0, bh1);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = mt * 16 + g + ((e >> 1) ? 8 : 0);
                const int j = nt * 8 + 2 * t4 + (e & 1);
                if (i < m) Hp[i * m + j] = h[e];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 3'. Y = X Q~ on Blackwell tensor cores (tcgen05, kind::tf32, accumulator in
//     TMEM), float inputs with n % 32 == 0, warp-specialised.  A CTA walks its
//     128-row tiles (tile row r <-> TMEM lane r) as one stream of 32-column
//     chunks through a ring of kT5Stages shared-memory stages:
//       warp 5 (loads)  X by TMA into the 128-byte swizzled K-major layout
//                       (one 128-row box, or 8-row boxes that follow a query's
//                       row sources) and the chunk of Q~^T - stored by the
//                       basis kernel in the canonical K-major layout - by one
//                       bulk copy, both completing on the stage's mbarrier;
//       warps 0-3       one tile row per thread: X_lo = X - tf32(X) in
//                       registers (zero past the item) into one of two TMEM
//                       buffers; at a tile's end the epilogue (one Y row per
//                       thread from TMEM, the tile's Y^T Y on mma.sync tensor
//                       cores as in k_project);
//       warp 4, lane 0  the MMAs: Y += X_hi Q~ with A = X from shared memory
//                       (the tensor core reads it as tf32, dropping the 13
//                       low mantissa bits: X_hi with no work) and Y += X_lo Q~
//                       with A from TMEM - FP32 accuracy from eight MMAs of
//                       K = 8 per chunk, into one of two TMEM accumulators so
//                       the next tile's MMAs need not wait for the epilogue.
//     The roles hand over through mbarriers only.  A tf32 MMA of M = 128
//     costs about the same for any N <= 128, so with N = m the tensor pipe sets
//     the pace; two CTAs per SM keep it fed.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kT5Stages = 4;
constexpr int kT5MaxPoll = 1 << 20;
constexpr int kT5Threads = 192;
// Tensor maps of the row sources (32 x 128 or 32 x 8 float boxes, 128-byte
// swizzle): SrcCompress reads x0 (the chunk's rows); SrcQuery reads x0 (the
// stacked M) and x1 (the store's Sigma V^T).
struct alignas(128) T5Maps {
    CUtensorMap x0, x1;
};
__host__ __device__ __forceinline__ int t5_np(int m) { return (m + 15) / 16 * 16; }      // MMA N
__host__ __device__ __forceinline__ uint32_t t5_stage_bytes(int m) { return 128 * 128 + t5_np(m) * 128; }
__host__ __device__ __forceinline__ uint32_t t5_ys_bytes(int m) {   // the epilogue's Y tile
    return (128 * pj_ldq(m) * 4 + 1023) / 1024 * 1024;
}
__host__ __device__ __forceinline__ size_t t5_smem_bytes(int m) {
    return (size_t)kT5Stages * t5_stage_bytes(m) + t5_ys_bytes(m) + 8 * (2 * kT5Stages + 6) + 16;
}
// TMEM columns: accumulators (np <= 64) at 0 and 64, X_lo buffers at 128 and 160
constexpr uint32_t kT5Cols = 256;

template <class Src>
__global__ void __launch_bounds__(kT5Threads, 1) k_project_tc5(Src src, TcScratch sc, int n,
                                                            const __grid_constant__ T5Maps maps) {
    extern __shared__ __align__(1024) unsigned char t5raw[];
    const int m = sc.m, np = t5_np(m), ldq = pj_ldq(m), ntn = m / 8, mp = (m + 15) / 16 * 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t stb = t5_stage_bytes(m);
    float* Ys = reinterpret_cast<float*>(t5raw + kT5Stages * stb);   // 128 x ldq
    uint64_t* full = reinterpret_cast<uint64_t*>(t5raw + kT5Stages * stb + t5_ys_bytes(m));
    uint64_t* done = full + kT5Stages;      // the MMAs of the stage's chunk have completed
    uint64_t* lo_ready = done + kT5Stages;  // [2] X_lo of a chunk is in TMEM (4 warp arrivals)
    uint64_t* acc_full = lo_ready + 2;      // [2] the tile's accumulator is complete
    uint64_t* acc_empty = acc_full + 2;     // [2] the epilogue has read the accumulator (4 warp arrivals)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    if (smem_u32(t5raw) & 1023) {           // the swizzle atoms need a 1024-byte aligned base
        if (tid == 0 && sc.fault) atomicExch(sc.fault, 1);
        return;
    }
    if (warp == 0) tc5_alloc(tmem_slot, kT5Cols);
    if (tid == 0) {
        for (int q = 0; q < kT5Stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&lo_ready[i], 4);
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4);
        }
    }
    fence_proxy_async();
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nch = n / 32;
    const int64_t ntiles = src.ntiles();
    // the CTA's tiles, those without rows skipped
    auto next_tile = [&](int64_t t) {
        for (; t < ntiles; t += gridDim.x) {
            int item, rt;
            src.tile_item(t, item, rt);
            if (rt * 128 < src.rows(item)) break;
        }
        return t;
    };
    bool ok = true;                         // after a failed wait no further waits: the roles run out quickly
    int64_t last_commit = -1;               // MMA thread: the last chunk it committed
    int64_t issued = 0;                     // load warp: chunks issued
    if (warp == 5) {
        // ---------------- loads
        int64_t q = 0;
        for (int64_t tile = next_tile(blockIdx.x); tile < ntiles; tile = next_tile(tile + gridDim.x)) {
            int item, rt;
            src.tile_item(tile, item, rt);
            const int r0 = rt * 128, valid = min(128, src.rows(item) - r0);
            const float* qt = sc.Qt + (size_t)item * np * n;
            for (int c = 0; c < nch; ++c, ++q) {
                const int s = (int)(q % kT5Stages);
                // the stage's previous chunk (q - stages) has been read by its MMAs
                if (ok && q >= kT5Stages &&
                    !mbar_wait(&done[s], (uint32_t)((q - kT5Stages) / kT5Stages) & 1, kT5MaxPoll))
                    ok = false;
                unsigned char* Xs = t5raw + (size_t)s * stb;
                const uint32_t bbytes = (uint32_t)np * 128;
                const float* bsrc = qt + (size_t)c * np * 32;
                if constexpr (std::is_same<Src, SrcCompress>::value) {
                    if (lane == 0) {
                        mbar_expect_tx(&full[s], 128 * 128 + bbytes);
                        tma_load_2d(Xs, &maps.x0, c * 32, (int)((int64_t)item * src.c.b + r0), &full[s]);
                        bulk_load(Xs + 128 * 128, bsrc, bbytes, &full[s]);
                    }
                } else {
                    // 8-row boxes (k % 8 == 0: a box lies in one slab); interior
                    // slabs from the store's Sigma V^T, the boundary slabs from M
                    const QPlan& P = src.a.plans[item];
                    const int kk = src.a.k;
                    const uint32_t kmagic = (uint32_t)((0x100000000ull + (uint64_t)kk - 1) / (uint64_t)kk);
                    const int npc = (valid + 7) / 8;
                    if (lane == 0) mbar_expect_tx(&full[s], (uint32_t)npc * 1024 + bbytes);
                    __syncwarp();
                    if (lane < npc) {
                        const int r = r0 + 8 * lane;
                        const int t = (int)__umulhi((uint32_t)r, kmagic);
                        const bool inner = src.a.wst && t > 0 && t < P.nslab - 1;
                        const int y = inner ? (int)(P.S * kk + r) : (int)(P.slab0 * kk + r);
                        tma_load_2d(Xs + lane * 1024, inner ? (const void*)&maps.x1 : (const void*)&maps.x0, c * 32,
                                    y, &full[s]);
                    }
                    if (lane == 31) bulk_load(Xs + 128 * 128, bsrc, bbytes, &full[s]);
                }
                issued = q + 1;
            }
        }
    } else if (warp == 4) {
        // ---------------- MMAs (one thread)
        if (lane == 0) {
            const uint32_t idesc = tc5_idesc_tf32(128, np);
            int64_t q = 0, t = 0;
            for (int64_t tile = next_tile(blockIdx.x); tile < ntiles; tile = next_tile(tile + gridDim.x), ++t) {
                const int a = (int)(t & 1);
                const uint32_t acc = tmem + 64 * a;
                // the epilogue of tile t - 2 has read this accumulator
                if (ok && t >= 2 && !mbar_wait(&acc_empty[a], (uint32_t)((t - 2) / 2) & 1, kT5MaxPoll)) ok = false;
                for (int c = 0; c < nch; ++c, ++q) {
                    const int s = (int)(q % kT5Stages), b = (int)(q & 1);
                    if (ok && !mbar_wait(&full[s], (uint32_t)(q / kT5Stages) & 1, kT5MaxPoll)) ok = false;
                    if (ok && !mbar_wait(&lo_ready[b], (uint32_t)(q / 2) & 1, kT5MaxPoll)) ok = false;
                    tc5_fence_after();
                    if (!ok) continue;
                    const uint32_t xa = smem_u32(t5raw + (size_t)s * stb), ba = xa + 128 * 128;
                    const uint32_t la = tmem + 128 + 32 * b;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc5_mma_tf32(acc, tc5_desc_sw128(xa + ks * 32), tc5_desc(ba + ks * 256, 128, 1024), idesc,
                                     (c > 0 || ks > 0) ? 1u : 0u);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc5_mma_tf32_ta(acc, la + ks * 8, tc5_desc(ba + ks * 256, 128, 1024), idesc, 1u);
                    tc5_commit(&done[s]);
                    last_commit = q;
                    if (c == nch - 1) tc5_commit(&acc_full[a]);
                }
            }
        }
    } else {
        // ---------------- X_lo and the epilogue (warps 0-3, thread = tile row).
        // A tile's epilogue runs once X_lo of the next tile's first two chunks
        // is in TMEM, so the MMAs have work while it runs.
        const int row = tid, g = lane >> 2, t4 = lane & 3;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        bool pending = false;               // a finished tile waits for its epilogue
        int64_t e_tile = 0, e_t = 0;
        int e_item = 0, e_r0 = 0, e_valid = 0;
        auto epilogue = [&]() {
            const int a = (int)(e_t & 1);
            if (ok && !mbar_wait(&acc_full[a], (uint32_t)(e_t / 2) & 1, kT5MaxPoll)) ok = false;
            tc5_fence_after();
            float y0[32], y1[32];
            tc5_ld32(lane_base + 64 * a, y0);
            if (np > 32) tc5_ld32(lane_base + 64 * a + 32, y1);
            else {
#pragma unroll
                for (int i = 0; i < 32; ++i) y1[i] = 0.f;
            }
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[a]);
            // Ys: 128 x ldq, zero past the item and column m
            const bool live = row < e_valid;
#pragma unroll
            for (int c4 = 0; c4 < 16; ++c4) {
                if (4 * c4 >= mp) break;
                float4 v = c4 < 8 ? make_float4(y0[4 * c4], y0[4 * c4 + 1], y0[4 * c4 + 2], y0[4 * c4 + 3])
                                  : make_float4(y1[4 * c4 - 32], y1[4 * c4 - 31], y1[4 * c4 - 30], y1[4 * c4 - 29]);
                if (4 * c4 >= m || !live) v = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4*>(Ys + row * ldq + 4 * c4) = v;
            }
            named_sync(1, 128);
            // the tile's Y rows, coalesced (16-byte pieces, consecutive threads on consecutive pieces)
            {
                float* Y = sc.Y + ((size_t)src.ybase(e_item) + e_r0) * m;
                const int pr = m / 4;       // pieces per row
                for (int p = tid; p < e_valid * pr; p += 128) {
                    const int r = p / pr, c4 = p - (p / pr) * pr;
                    *reinterpret_cast<float4*>(Y + (size_t)r * m + 4 * c4) =
                        *reinterpret_cast<const float4*>(Ys + r * ldq + 4 * c4);
                }
            }
            // this tile's Y^T Y on tensor cores (two tf32 terms, three products),
            // fixed order; two output tiles per pass give two independent chains
            float* Hp = sc.Hp + (size_t)e_tile * m * m;
            const int nmt = mp / 16, tot = nmt * ntn;
            for (int o0 = warp; o0 < tot; o0 += 8) {
                const bool two = o0 + 4 < tot;
                float h[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                for (int k0 = 0; k0 < 128; k0 += 8) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (u == 1 && !two) continue;
                        const int ot = o0 + 4 * u;
                        const int mt = ot / ntn, nt = ot - (ot / ntn) * ntn;
                        const float* ya = Ys + (k0 + t4) * ldq + mt * 16 + g;
                        const float* yb = Ys + (k0 + t4) * ldq + nt * 8 + g;
                        uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3, bh0, bl0, bh1, bl1;
                        tf32_split(ya[0], ah0, al0);
                        tf32_split(ya[8], ah1, al1);
                        tf32_split(ya[4 * ldq], ah2, al2);
                        tf32_split(ya[4 * ldq + 8], ah3, al3);
                        tf32_split(yb[0], bh0, bl0);
                        tf32_split(yb[4 * ldq], bh1, bl1);
                        mma_tf32(h[u], al0, al1, al2, al3, bh0, bh1);
                        mma_tf32(h[u], ah0, ah1, ah2, ah3, bl0, bl1);
                        mma_tf32(h[u], ah0, ah1, ah2, ah3, bh0, bh1);
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (u == 1 && !two) continue;
                    const int ot = o0 + 4 * u;
                    const int mt = ot / ntn, nt = ot - (ot / ntn) * ntn;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = mt * 16 + g + ((e >> 1) ? 8 : 0);
                        const int j = nt * 8 + 2 * t4 + (e & 1);
                        if (i < m) Hp[i * m + j] = h[u][e];
                    }
                }
            }
            named_sync(1, 128);             // Ys is rewritten by the next epilogue
            pending = false;
        };
        int64_t q = 0, t = 0;
        for (int64_t tile = next_tile(blockIdx.x); tile < ntiles; tile = next_tile(tile + gridDim.x), ++t) {
            int item, rt;
            src.tile_item(tile, item, rt);
            const int r0 = rt * 128, valid = min(128, src.rows(item) - r0);
            for (int c = 0; c < nch; ++c, ++q) {
                const int s = (int)(q % kT5Stages), b = (int)(q & 1);
                if (ok && !mbar_wait(&full[s], (uint32_t)(q / kT5Stages) & 1, kT5MaxPoll)) ok = false;
                // the MMAs of chunk q - 2 have read this X_lo buffer
                if (ok && q >= 2 &&
                    !mbar_wait(&done[(q - 2) % kT5Stages], (uint32_t)((q - 2) / kT5Stages) & 1, kT5MaxPoll))
                    ok = false;
                tc5_fence_after();
                // this thread's row: its 16-byte pieces sit at j ^ (row % 8) (128-byte swizzle)
                float* xr = reinterpret_cast<float*>(t5raw + (size_t)s * stb) + row * 32;
                float lo[32];
                if (row < valid) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 v = *reinterpret_cast<const float4*>(xr + 4 * (j ^ (row & 7)));
                        lo[4 * j] = v.x - __uint_as_float(__float_as_uint(v.x) & 0xffffe000u);
                        lo[4 * j + 1] = v.y - __uint_as_float(__float_as_uint(v.y) & 0xffffe000u);
                        lo[4 * j + 2] = v.z - __uint_as_float(__float_as_uint(v.z) & 0xffffe000u);
                        lo[4 * j + 3] = v.w - __uint_as_float(__float_as_uint(v.w) & 0xffffe000u);
                    }
                } else {                    // past the item: zero in both terms
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4*>(xr + 4 * j) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 32; ++j) lo[j] = 0.f;
                }
                tc5_st32(lane_base + 128 + 32 * b, lo);
                fence_proxy_async();
                tc5_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&lo_ready[b]);
                if (pending && c == (nch > 1 ? 1 : 0)) epilogue();
            }
            pending = true;
            e_tile = tile;
            e_t = t;
            e_item = item;
            e_r0 = r0;
            e_valid = valid;
        }
        if (pending) epilogue();
    }
    if (__syncthreads_or(!ok)) {
        // a wait gave up: let the MMAs (the last commit tracks all of them)
        // and the copies already issued finish, bounded, before the
        // accumulators and the shared memory are released
        if (warp == 4 && lane == 0 && last_commit >= 0)
            mbar_wait(&done[last_commit % kT5Stages], (uint32_t)(last_commit / kT5Stages) & 1, kT5MaxPoll);
        if (warp == 5 && lane == 0)
            for (int64_t c = issued > kT5Stages ? issued - kT5Stages : 0; c < issued; ++c)
                mbar_wait(&full[c % kT5Stages], (uint32_t)(c / kT5Stages) & 1, kT5MaxPoll);
        if (tid == 0 && sc.fault) atomicExch(sc.fault, 1);
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    if (warp == 0) tc5_dealloc(tmem, kT5Cols);
}

// ---------------------------------------------------------------------------
// 2'. Subspace sketch of one item by a cluster of kSketchCL CTAs that split the
//     item's 128-row tiles round-robin: S = X^T (X Omega), Omega an n x m
//     matrix of random signs (bf16 operands, fp32 accumulation) - one step of
//     the randomized range finder of Halko, Martinsson & Tropp (SIAM Review 53,
//     2011) applied to the rows' Gram matrix without forming it.  The CTAs'
//     partial S are summed through distributed shared memory in a fixed order
//     (each CTA reduces a slice of rows and stores it): S to sc.G as n x m.
//     Costs O(rows n m) tensor work and one read of X.
// ---------------------------------------------------------------------------
constexpr int kSketchCL = 4;

// Random signs of row i of Omega: bit c of the SplitMix64 output function
// (Steele, Lea & Flood, OOPSLA 2014) of the counter i gives Omega(i, c), c < 64.
__device__ __forceinline__ uint64_t omega_row_bits(uint32_t i) {
    uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Shared-memory plan of k_sketch (bytes from the dynamic base):
// [Rx: the bf16 X tile, later the fp32 partial S and the reduced slice |
//  Bs: bf16 Omega, npad x bf16_ld(m) | Ws: bf16 W, 128 x bf16_ld(m)]
struct SketchSmem {
    size_t rx, bs, ws, total;
};
__host__ __device__ __forceinline__ SketchSmem sketch_smem(int n, int m) {
    auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t npad = (size_t)(n + 15) / 16 * 16;
    const size_t chunk = (npad + kSketchCL - 1) / kSketchCL;
    size_t rx = r16((size_t)128 * bf16_ld((int)npad) * 2);
    const size_t sred = r16((npad + chunk) * (m + 1) * 4);
    rx = rx > sred ? rx : sred;
    SketchSmem s;
    s.rx = rx;
    s.bs = r16(npad * bf16_ld(m) * 2);
    s.ws = r16((size_t)128 * bf16_ld(m) * 2);
    s.total = s.rx + s.bs + s.ws;
    return s;
}

// NMT: 16-row tiles of S per warp (n <= 128 NMT); MB: bound on m.
template <class Src, typename Tin, int NMT, int MB>
__global__ void __cluster_dims__(kSketchCL, 1, 1) __launch_bounds__(256, (NMT * MB <= 64) ? 2 : 1)
    k_sketch(Src src, TcScratch sc, int n) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) char dsm[];
    const int item = blockIdx.x / kSketchCL;
    const int cr = (int)cl.block_rank();
    if (item >= src.count()) return;                 // the whole cluster leaves together
    const int m = sc.m, rows = src.rows(item);
    const int ntl = (rows + 127) / 128;
    const int npad = (n + 15) / 16 * 16;
    const int ldx = bf16_ld(npad), ldb = bf16_ld(m), lds = m + 1;
    const SketchSmem L = sketch_smem(n, m);
    __nv_bfloat16* Xs = (__nv_bfloat16*)dsm;
    float* Sp = (float*)dsm;                          // npad x lds (after the tiles)
    const int chunk = (npad + kSketchCL - 1) / kSketchCL;
    __nv_bfloat16* Bs = (__nv_bfloat16*)(dsm + L.rx);
    __nv_bfloat16* Ws = (__nv_bfloat16*)(dsm + L.rx + L.bs);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mat = lane >> 3, rr = lane & 7;
    const int ntn = m / 8;
    const int64_t ld = src.ld();
    const Tin* X = (const Tin*)src.X(item, sizeof(Tin));
    const bool xal = std::is_same<Tin, float>::value && (ld % 4 == 0) && (n % 4 == 0) &&
                     ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const auto cx = src.ctx(item, sizeof(Tin));

    for (int l = tid; l < npad; l += 256) {
        const uint64_t bits = omega_row_bits((uint32_t)l);
        for (int c = 0; c < m; c += 2) {
            const float a = l < n ? (((bits >> c) & 1) ? 1.f : -1.f) : 0.f;
            const float b = l < n ? (((bits >> (c + 1)) & 1) ? 1.f : -1.f) : 0.f;
            *reinterpret_cast<uint32_t*>(Bs + l * ldb + c) = pack_bf16(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
        }
    }
    float sacc[NMT][MB / 8][4];
#pragma unroll
    for (int a = 0; a < NMT; ++a)
#pragma unroll
        for (int b = 0; b < MB / 8; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) sacc[a][b][c] = 0.f;
    for (int t = cr; t < ntl; t += kSketchCL) {
        const int r0 = t * 128;
        __syncthreads();
        // X tile -> bf16 Xs (zero rows past `rows`, columns past n); element
        // group f = tid + 256 j sits at row f / q4, column 4 (f % q4), advanced
        // incrementally (no division in the loop)
        const int q4 = npad / 4;
        const int dr = 256 / q4, dc = 256 - dr * q4;
        int r_i = tid / q4, c_i = tid - r_i * q4;
        for (int f0 = 0; f0 < 128 * q4; f0 += 256 * 8) {
            float v[8][4];
            int rs[8], cs[8];
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                rs[gg] = r_i;
                cs[gg] = c_i * 4;
                r_i += dr;
                c_i += dc;
                if (c_i >= q4) { c_i -= q4; ++r_i; }
            }
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                const int f = f0 + tid + gg * 256;
                const int r = rs[gg], c = cs[gg];
                v[gg][0] = v[gg][1] = v[gg][2] = v[gg][3] = 0.f;
                if (f < 128 * q4 && r0 + r < rows) {
                    float s = 1.f;
                    const Tin* p = src.template row<Tin>(cx, r0 + r, s) + c;
                    if constexpr (std::is_same<Tin, float>::value) {
                        if (xal && c + 3 < n) {
                            const float4 q = __ldg(reinterpret_cast<const float4*>(p));
                            v[gg][0] = q.x * s; v[gg][1] = q.y * s; v[gg][2] = q.z * s; v[gg][3] = q.w * s;
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (c + e < n) v[gg][e] = __ldg(p + e) * s;
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (c + e < n) v[gg][e] = __bfloat162float(p[e]) * s;
                    }
                }
            }
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                const int f = f0 + tid + gg * 256;
                if (f >= 128 * q4) break;
                const int r = rs[gg], c = cs[gg];
                uint32_t* dp = reinterpret_cast<uint32_t*>(Xs + r * ldx + c);
                dp[0] = pack_bf16(__float2bfloat16_rn(v[gg][0]), __float2bfloat16_rn(v[gg][1]));
                dp[1] = pack_bf16(__float2bfloat16_rn(v[gg][2]), __float2bfloat16_rn(v[gg][3]));
            }
        }
        __syncthreads();
        // W = Xs Omega (warp: rows 16 warp .. +15, all m columns) -> bf16 Ws
        {
            float wacc[MB / 8][4];
#pragma unroll
            for (int b = 0; b < MB / 8; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) wacc[b][c] = 0.f;
            const int arow = warp * 16 + ((mat & 1) ? 8 : 0) + rr;
            for (int kk = 0; kk < npad; kk += 16) {
                uint32_t a0, a1, a2, a3;
                ldsm_x4(smem_u32(Xs + arow * ldx + kk + ((mat >> 1) ? 8 : 0)), a0, a1, a2, a3);
#pragma unroll
                for (int np = 0; np < MB / 16; ++np) {
                    if (2 * np >= ntn) break;
                    const int tt = kk + rr + ((mat & 1) ? 8 : 0);
                    uint32_t b0, b1, b2, b3;
                    if (2 * np + 1 < ntn) {
                        ldsm_x4_t(smem_u32(Bs + tt * ldb + np * 16 + ((mat >> 1) ? 8 : 0)), b0, b1, b2, b3);
                    } else {
                        ldsm_x2_t(smem_u32(Bs + tt * ldb + np * 16), b0, b1);
                        b2 = b3 = 0;
                    }
                    mma_bf16(wacc[2 * np], a0, a1, a2, a3, b0, b1);
                    if (2 * np + 1 < ntn) mma_bf16(wacc[2 * np + 1], a0, a1, a2, a3, b2, b3);
                }
            }
#pragma unroll
            for (int nt = 0; nt < MB / 8; ++nt) {
                if (nt >= ntn) break;
                const int rl = warp * 16 + (lane >> 2);
                const int c = nt * 8 + 2 * (lane & 3);
                *reinterpret_cast<uint32_t*>(Ws + rl * ldb + c) =
                    pack_bf16(__float2bfloat16_rn(wacc[nt][0]), __float2bfloat16_rn(wacc[nt][1]));
                *reinterpret_cast<uint32_t*>(Ws + (rl + 8) * ldb + c) =
                    pack_bf16(__float2bfloat16_rn(wacc[nt][2]), __float2bfloat16_rn(wacc[nt][3]));
            }
        }
        __syncthreads();
        // S += Xs^T Ws (warp: S rows 16 NMT warp .. , K = the tile's 128 rows)
        {
            const int i0 = warp * 16 * NMT;
            if (i0 < npad) {
                for (int kk = 0; kk < 128; kk += 16) {
                    uint32_t bf[MB / 8][2];
#pragma unroll
                    for (int np = 0; np < MB / 16; ++np) {
                        if (2 * np >= ntn) break;
                        const int tt = kk + rr + ((mat & 1) ? 8 : 0);
                        if (2 * np + 1 < ntn) {
                            ldsm_x4_t(smem_u32(Ws + tt * ldb + np * 16 + ((mat >> 1) ? 8 : 0)), bf[2 * np][0],
                                      bf[2 * np][1], bf[2 * np + 1][0], bf[2 * np + 1][1]);
                        } else {
                            ldsm_x2_t(smem_u32(Ws + tt * ldb + np * 16), bf[2 * np][0], bf[2 * np][1]);
                        }
                    }
#pragma unroll
                    for (int mt = 0; mt < NMT; ++mt) {
                        const int ib = i0 + mt * 16;
                        if (ib >= npad) break;
                        uint32_t a0, a1, a2, a3;
                        const int tt = kk + rr + ((mat >> 1) ? 8 : 0);
                        ldsm_x4_t(smem_u32(Xs + tt * ldx + ib + ((mat & 1) ? 8 : 0)), a0, a1, a2, a3);
#pragma unroll
                        for (int nt = 0; nt < MB / 8; ++nt) {
                            if (nt >= ntn) break;
                            mma_bf16(sacc[mt][nt], a0, a1, a2, a3, bf[nt][0], bf[nt][1]);
                        }
                    }
                }
            }
        }
    }
    // cluster sum of S in a fixed order: CTA cr reduces rows [cr chunk, ..) and stores them
    __syncthreads();
    {
        const int i0 = warp * 16 * NMT;
#pragma unroll
        for (int mt = 0; mt < NMT; ++mt) {
            const int ib = i0 + mt * 16;
            if (ib >= npad) break;
#pragma unroll
            for (int nt = 0; nt < MB / 8; ++nt) {
                if (nt >= ntn) break;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = ib + (lane >> 2) + ((e >> 1) ? 8 : 0);
                    const int c = nt * 8 + 2 * (lane & 3) + (e & 1);
                    Sp[i * lds + c] = sacc[mt][nt][e];
                }
            }
        }
    }
    cl.sync();
    {
        const int lo = cr * chunk, hi = min(n, lo + chunk);
        const float* rp[kSketchCL];
#pragma unroll
        for (int q = 0; q < kSketchCL; ++q) rp[q] = cl.map_shared_rank(Sp, q);
        float* Sg = sc.G + (size_t)item * n * m;
        for (int e = tid; e < (hi - lo) * m; e += 256) {
            const int i = lo + e / m, c = e - (e / m) * m;
            float v[kSketchCL];
#pragma unroll
            for (int q = 0; q < kSketchCL; ++q) v[q] = rp[q][i * lds + c];
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < kSketchCL; ++q) s += v[q];
            Sg[(size_t)i * m + c] = s;
        }
    }
    cl.sync();                                     // peers may still read this CTA's partial until here
}

// ---------------------------------------------------------------------------
// 2''. Orthonormal basis of the sketch, one CTA of 16 warps per item: warp w
//      owns columns w, w + 16, ... of S (n x m, sc.G) with RPL rows per lane
//      in registers.  Right-looking modified Gram-Schmidt: the owner
//      normalises column c and publishes it, then every warp removes its
//      component from its later columns (warp-shuffle dots).  One pass leaves
//      Q~ orthonormal to ~eps kappa(S); the Rayleigh-Ritz step uses the exact
//      Q~^T Q~, so only the conditioning of Q~ matters here.  A column whose
//      norm falls below 1e-5 of its starting norm is dependent and becomes
//      zero: its direction carries rounding error of order eps / 1e-5, and
//      such directions (lambda_j < 1e-5 lambda_1) lie below what the fp32
//      Gram route resolves anyway.  Q~ is rounded to tf32 (exact operand of the
//      projection); C = Q~^T Q~ follows.
// ---------------------------------------------------------------------------
constexpr int kOrthWarps = 16;

template <class Src, int RPL, int CPW>
__global__ void __launch_bounds__(32 * kOrthWarps) k_orth(Src src, TcScratch sc, int n) {
    extern __shared__ __align__(16) float osm[];     // Q~, n x (m+1), for C
    __shared__ float qc[2 * 32 * RPL];                // the published column (two buffers)
    const int m = sc.m, lds = m + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = blockIdx.x;
    if (item >= src.count()) return;
    const float* Sg = sc.G + (size_t)item * n * m;
    // S through shared memory: coalesced reads of its rows, then columns per lane
    for (int e = threadIdx.x; e < n * m; e += 32 * kOrthWarps) {
        const int row = e / m, col = e - (e / m) * m;
        osm[row * lds + col] = Sg[e];
    }
    __syncthreads();
    float s[CPW][RPL], nrm0[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
        const int col = warp + kOrthWarps * j;
        float ss = 0.f;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int row = lane + 32 * r;
            s[j][r] = (col < m && row < n) ? osm[row * lds + col] : 0.f;
            ss = fmaf(s[j][r], s[j][r], ss);
        }
        nrm0[j] = sqrtf(warp_sum(ss));
    }
    __syncthreads();                                  // osm is rewritten with Q~ below
    // one pass; the published column alternates between two buffers so that a
    // single barrier per column separates its writer from its readers
    for (int c = 0; c < m; ++c) {
        const int ow = c % kOrthWarps, oj = c / kOrthWarps;
        float* qb = qc + (c & 1) * 32 * RPL;
        if (warp == ow) {
            float v[RPL];
            float base = 0.f;
#pragma unroll
            for (int j = 0; j < CPW; ++j)
                if (j == oj) {
#pragma unroll
                    for (int r = 0; r < RPL; ++r) v[r] = s[j][r];
                    base = nrm0[j];
                }
            float ss = 0.f;
#pragma unroll
            for (int r = 0; r < RPL; ++r) ss = fmaf(v[r], v[r], ss);
            const float nn = sqrtf(warp_sum(ss));
            const float inv = (nn > 0.f && nn > 1e-5f * base) ? 1.f / nn : 0.f;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                v[r] *= inv;
                qb[lane + 32 * r] = v[r];
            }
#pragma unroll
            for (int j = 0; j < CPW; ++j)
                if (j == oj) {
#pragma unroll
                    for (int r = 0; r < RPL; ++r) s[j][r] = v[r];
                }
        }
        __syncthreads();
        float q[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) q[r] = qb[lane + 32 * r];
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
            const int d = warp + kOrthWarps * j;
            if (d > c && d < m) {
                float dot = 0.f;
#pragma unroll
                for (int r = 0; r < RPL; ++r) dot = fmaf(q[r], s[j][r], dot);
                dot = warp_sum(dot);
#pragma unroll
                for (int r = 0; r < RPL; ++r) s[j][r] = fmaf(-dot, q[r], s[j][r]);
            }
        }
    }
    // Q~ = tf32(Q): to the projection's scratch and, for C, to shared memory
    float* Qf = sc.Qf + (size_t)item * n * m;
    const int np = (m + 15) / 16 * 16;
    float* Qt = sc.Qt ? sc.Qt + (size_t)item * np * n : nullptr;
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
        const int col = warp + kOrthWarps * j;
        if (col >= m) {
            // zero columns m..round16(m) of the transposed copy (MMA N padding)
            if (Qt && col < np)
#pragma unroll
                for (int r = 0; r < RPL; ++r)
                    if (lane + 32 * r < n) Qt[(size_t)r * np * 32 + tc5_canon(col, lane, 32)] = 0.f;
            continue;
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int row = lane + 32 * r;
            s[j][r] = __uint_as_float(to_tf32(s[j][r]));
            if (row < n) {
                Qf[(size_t)row * m + col] = s[j][r];
                osm[row * lds + col] = s[j][r];
                // Q~^T, 32-row chunk r, canonical K-major position (col, lane)
                if (Qt) Qt[(size_t)r * np * 32 + tc5_canon(col, lane, 32)] = s[j][r];
            }
        }
    }
    __syncthreads();
    // C = Q~^T Q~ (exact products of tf32 values, fp32 sums; the same
    // summation tree for C[a][c] and C[c][a], so C is exactly symmetric)
    float* Cq = sc.Cq + (size_t)item * m * m;
    if (m <= 32) {
        // each lane's partial dots with all m columns, then one butterfly
        // reduce-scatter (lane c ends with column c; 31 shuffles).  Every
        // element is summed over the same tree of lanes, so C stays symmetric.
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
            const int a = warp + kOrthWarps * j;
            if (a >= m) continue;
            float p[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) p[c] = 0.f;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int row = lane + 32 * r;
                if (row < n) {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (c < m) p[c] = fmaf(s[j][r], osm[row * lds + c], p[c]);
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const bool up = (lane & off) != 0;
#pragma unroll
                for (int i = 0; i < off; ++i) {
                    const float send = up ? p[i] : p[i + off];
                    const float keep = up ? p[i + off] : p[i];
                    p[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            if (lane < m) Cq[a * m + lane] = p[0];
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
        const int a = warp + kOrthWarps * j;
        if (a >= m) continue;
        for (int c = 0; c < m; ++c) {
            float dot = 0.f;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int row = lane + 32 * r;
                if (row < n) dot = fmaf(s[j][r], osm[row * lds + c], dot);
            }
            dot = warp_sum(dot);
            if (lane == 0) Cq[a * m + c] = dot;
        }
    }
}

// ---------------------------------------------------------------------------
// 4a. Rayleigh-Ritz core, one CTA per item: H = sum of the tiles' Y^T Y,
//     C = Q~^T Q~ = L L^T, H' = L^-1 H L^-T, Jacobi H' = W Theta W^T
//     (FP32 sweeps; with REF one FP64 refinement on W^T H' W), Z = L^-T W.
// ---------------------------------------------------------------------------
template <bool REF>
__host__ __device__ __forceinline__ size_t rr_warp_bytes(int m) {
    const size_t ld = m + 1;
    const size_t tr = REF ? 8 : 4;
    // Hs, Cs(L), Li in TR; A_T, Z_T in float (+ 4 bytes to align X); REF: X in
    // double (W shares Cs, which is free once H' is formed); perm, theta
    size_t b = 3 * tr * m * ld + 2 * 4 * m * ld + 8 + (REF ? 8 * m * ld : 0) + 4 * 64 + 8 * 64;
    return (b + 15) & ~size_t(15);
}

template <class Src, bool REF>
__global__ void __launch_bounds__(128) k_rr_core(Src src, TcScratch sc, int kw) {
    using TR = typename std::conditional<REF, double, float>::type;
    extern __shared__ __align__(16) char dsm[];
    const int m = sc.m, ld = m + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ JacobiScratch<float> jsf;
    char* base = dsm;
    TR* Hs = (TR*)base;
    TR* Cs = Hs + (size_t)m * ld;
    TR* Li = Cs + (size_t)m * ld;
    float* A_T = (float*)(Li + (size_t)m * ld);
    float* Z_T = A_T + (size_t)m * ld;
    double* X = (double*)(Z_T + (size_t)m * ld + ((m * ld) & 1));
    double* W = REF ? (double*)Cs : nullptr;       // refinement rotations, after H' is formed
    int* perm = (int*)(base + rr_warp_bytes<REF>(m) - 4 * 64 - 8 * 64);
    double* thd = (double*)(base + rr_warp_bytes<REF>(m) - 8 * 64);
    const int count = src.count();
    for (int item = blockIdx.x; item < count; item += gridDim.x) {
        const int rows = src.rows(item);
        const int ntiles = (rows + 127) / 128;
        const float* Hp = sc.Hp + (size_t)src.tile0(item) * m * m;
        const float* Cq = sc.Cq + (size_t)item * m * m;
        for (int e = tid; e < m * m; e += nt) {
            TR h = 0;
            // tile partials in fixed order, eight loads in flight
            for (int t0 = 0; t0 < ntiles; t0 += 8) {
                float hv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) hv[u] = t0 + u < ntiles ? __ldg(Hp + (size_t)(t0 + u) * m * m + e) : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (t0 + u < ntiles) h += (TR)hv[u];
            }
            Hs[(e / m) * ld + e % m] = h;
            Cs[(e / m) * ld + e % m] = (TR)Cq[e];
        }
        __syncthreads();
        // Cholesky C = L L^T (lower, in place), right-looking: step j takes the
        // pivot's square root, scales column j, then updates the trailing
        // triangle in parallel.  Each entry receives its updates in the order
        // p = 0, 1, ..., as in the dot-product form.
        for (int j = 0; j < m; ++j) {
            if (tid == 0) {
                const TR d = Cs[j * ld + j];
                Cs[j * ld + j] = d > TR(1e-12) ? (TR)sqrt((double)d) : TR(1e-6);
            }
            __syncthreads();
            for (int i = j + 1 + tid; i < m; i += nt) Cs[i * ld + j] = Cs[i * ld + j] / Cs[j * ld + j];
            __syncthreads();
            const int w = m - 1 - j;                      // trailing order
            for (int e = tid; e < w * w; e += nt) {
                const int i = j + 1 + e / w, k = j + 1 + (e - (e / w) * w);
                if (k <= i) Cs[i * ld + k] -= Cs[i * ld + j] * Cs[k * ld + j];
            }
            __syncthreads();
        }
        // L^-1 by right-looking forward substitution on all columns at once:
        // step p divides row p, then removes it from the rows below
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            Li[i * ld + c] = (i == c) ? TR(1) : TR(0);
        }
        __syncthreads();
        for (int p = 0; p < m; ++p) {
            for (int c = tid; c <= p; c += nt) Li[p * ld + c] = Li[p * ld + c] / Cs[p * ld + p];
            __syncthreads();
            const int rws = m - 1 - p, cls = p + 1;
            for (int e = tid; e < rws * cls; e += nt) {
                const int i = p + 1 + e / cls, c = e - (e / cls) * cls;
                Li[i * ld + c] -= Cs[i * ld + p] * Li[p * ld + c];
            }
            __syncthreads();
        }
        // H' = L^-1 H L^-T  (temp in Cs, L no longer needed)
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e % m;
            TR d = 0;
            for (int p = 0; p <= i; ++p) d += Li[i * ld + p] * Hs[p * ld + c];
            Cs[i * ld + c] = d;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e % m;
            TR d = 0;
            for (int p = 0; p <= c; ++p) d += Cs[i * ld + p] * Li[c * ld + p];
            Hs[i * ld + c] = d;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e % m;
            const TR v = (Hs[i * ld + c] + Hs[c * ld + i]) * TR(0.5);
            A_T[i * ld + c] = (float)v;
            if (REF) X[i * ld + c] = (double)v;
        }
        __syncthreads();
        jacobi_eig<float>(A_T, ld, Z_T, ld, m, jsf, 30, true);
        const double* Zsrc_d = nullptr;
        if constexpr (REF) {
            // B = Z^T H' Z in FP64 (X holds H'), then FP64 Jacobi (refinement)
            double* Hd = (double*)Hs;                    // reuse: Hs is double when REF
            for (int e = tid; e < m * m; e += nt) {
                const int i = e / m, c = e % m;
                double d = 0;
                for (int l = 0; l < m; ++l) d += X[i * ld + l] * (double)Z_T[l * ld + c];
                Hd[i * ld + c] = d;                       // H' Z
            }
            __syncthreads();
            for (int e = tid; e < m * m; e += nt) {
                const int a = e / m, c = e % m;
                double d = 0;
                for (int i = 0; i < m; ++i) d += (double)Z_T[i * ld + a] * Hd[i * ld + c];
                X[a * ld + c] = d;                        // B
            }
            __syncthreads();
            // one FP64 refinement sweep (closed form: B is diagonal to FP32 rounding)
            refine_sweep<double>(X, ld, W, ld, m, tid, nt, thd, [] { __syncthreads(); });
            for (int e = tid; e < m * m; e += nt) {
                const int i = e / m, c = e % m;
                double d = 0;
                for (int a = 0; a < m; ++a) d += (double)Z_T[i * ld + a] * W[a * ld + c];
                Hd[i * ld + c] = d;                       // Z W
            }
            __syncthreads();
            sort_desc<double>(X, ld, m, perm);
            for (int c = tid; c < m; c += nt) thd[c] = X[perm[c] * ld + perm[c]];
            Zsrc_d = Hd;
        } else {
            sort_desc<float>(A_T, ld, m, perm);
            for (int c = tid; c < m; c += nt) thd[c] = (double)A_T[perm[c] * ld + perm[c]];
        }
        __syncthreads();
        // Z = L^-T W(:, perm) for the kw wanted pairs
        float* Zg = sc.Zs + (size_t)item * m * kw;
        for (int e = tid; e < m * kw; e += nt) {
            const int a = e / kw, c = e % kw;
            const int pc = perm[c];
            double d = 0;
            for (int p = a; p < m; ++p)
                d += (double)Li[p * ld + a] * (REF ? Zsrc_d[p * ld + pc] : (double)Z_T[p * ld + pc]);
            Zg[e] = (float)d;
        }
        for (int c = tid; c < kw; c += nt) sc.th[(size_t)item * kw + c] = (float)thd[c];
        if (sc.thm)
            for (int c = tid; c < m; c += nt) sc.thm[(size_t)item * m + c] = (float)thd[c];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 4a'. Rayleigh-Ritz core in registers (m <= 32, FP32 cores): one warp per
//      item, lane l owning column l of each m x m matrix (padded to 32):
//        C = Q~^T Q~ = L L^T          Cholesky, pivots broadcast by shuffle
//        H' = L^-1 H L^-T             two forward substitutions (H symmetric)
//        H' = G G^T                   Cholesky
//        G J = W Theta^(1/2)          one-sided (Hestenes) Jacobi on G's columns
//      G is R^T for R^T R = H', so the orthogonalised columns of G are the
//      eigenvectors of H' scaled by sqrt(theta): no rotation accumulator.
//      Then Z = L^-T W for the kw largest theta.  Pairing is the round-robin
//      schedule of zs_linalg.cuh (index 0 fixed, 1..31 rotating), in closed
//      form so that each lane finds its partner without a table.
// ---------------------------------------------------------------------------
template <class Src>
__global__ void __launch_bounds__(128) k_rr_core_reg(Src src, TcScratch sc, int kw) {
    __shared__ float tl[4][32 * 33];                  // per warp: Cholesky factor of C
    __shared__ float tw[4][32 * 33];                  // per warp: work tile
    const int m = sc.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    float* TL = tl[warp];
    float* TW = tw[warp];
    // one item per warp (the launch covers every item): the register arrays
    // below stay in registers only while no loop encloses the unrolled code
    const int item = blockIdx.x * wpc + warp;
    if (item >= src.count()) return;
    {
        const int rows = src.rows(item);
        const int ntiles = (rows + 127) / 128;
        const float* Hp = sc.Hp + (size_t)src.tile0(item) * m * m;
        const float* Cq = sc.Cq + (size_t)item * m * m;
        float lc[32], v[32], x[32];
        // columns of H (sum of the tiles, fixed order) and of C, identity-padded
        // unconditional loads from clamped addresses (then a select), so that
        // each group of 32 loads is issued at once rather than one by one
        const int lc_ = min(lane, m - 1);
        const bool lok = lane < m;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float cv = __ldg(Cq + min(i, m - 1) * m + lc_);
            v[i] = 0.f;
            lc[i] = (i < m && lok) ? cv : (i == lane ? 1.f : 0.f);
        }
        for (int t = 0; t < ntiles; ++t) {
            const float* hp = Hp + (size_t)t * m * m;
            float hv[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) hv[i] = __ldg(hp + min(i, m - 1) * m + lc_);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += (i < m && lok) ? hv[i] : 0.f;
        }
        warp_chol32(lc, TL, lane);                     // C = L L^T, L in TL
        warp_fsub32(TL, v, x, TW, lane);               // X = L^-1 H, column `lane` (also in TW)
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = TW[lane * 33 + i];   // row `lane` of X
        __syncwarp();
        warp_fsub32(TL, v, x, TW, lane);               // H' = L^-1 X^T, column `lane`
        __syncwarp();
        warp_chol32(x, TW, lane);                      // H' = G G^T, column `lane` of G
        const float al = warp_hestenes32(x, v, lane);
        // rank of this lane's theta (descending, lower lane first on ties)
        int rk = 0;
#pragma unroll
        for (int o = 0; o < 32; ++o) {
            const float ot = __shfl_sync(0xffffffffu, al, o);
            rk += (ot > al) || (ot == al && o < lane);
        }
        __syncwarp();
        warp_bsub32(TL, x, v, TW, lane);               // z = L^-T w
        if (rk < kw) {
            float* Zg = sc.Zs + (size_t)item * m * kw;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < m) Zg[i * kw + rk] = v[i];
            sc.th[(size_t)item * kw + rk] = al;
        }
        if (sc.thm && rk < m) sc.thm[(size_t)item * m + rk] = al;
    }
}

// ---------------------------------------------------------------------------
// 4b. Outputs per item: sigma = sqrt(theta), V = Q~ Z (signed), U = Y Z Sigma^-1.
// ---------------------------------------------------------------------------
// Shared-memory plan of k_rr_out: Z (m x ldz) then V (n x (kwp + 1)), with
// kwp = kw rounded up to 8 and ldz = 8 mod 32 (conflict-free B fragments).
__host__ __device__ __forceinline__ int rro_kwp(int kw) { return (kw + 7) / 8 * 8; }
__host__ __device__ __forceinline__ int rro_ldz(int kw) { return (rro_kwp(kw) + 31) / 32 * 32 + 8; }
__host__ __device__ __forceinline__ size_t rr_out_smem_bytes(int n, int m, int kw) {
    return sizeof(float) * ((size_t)m * rro_ldz(kw) + (size_t)n * (rro_kwp(kw) + 1));
}

// D(16 x kwp rows r0..) = A(rows x m, global fp32, row stride m) . Zs(m x kwp)
// on tf32 tensor cores; A_EXACT: A is already tf32 (one product), else A and
// Z are split into two terms each (three products).  Rows >= nrows read as 0.
template <bool A_EXACT>
__device__ __forceinline__ void rro_tile(const float* A, int r0, int nrows, int m, const float* Zs, int ldz,
                                         int nnt, float (&acc)[8][4], int lane) {
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int ra = r0 + g, rb = r0 + g + 8;
    const float* pa = A + (size_t)ra * m;
    const float* pb = A + (size_t)rb * m;
    for (int k0 = 0; k0 < m; k0 += 8) {
        const float x0 = ra < nrows ? __ldg(pa + k0 + t4) : 0.f;
        const float x1 = rb < nrows ? __ldg(pb + k0 + t4) : 0.f;
        const float x2 = ra < nrows ? __ldg(pa + k0 + t4 + 4) : 0.f;
        const float x3 = rb < nrows ? __ldg(pb + k0 + t4 + 4) : 0.f;
        uint32_t h0, h1, h2, h3, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
        if constexpr (A_EXACT) {
            h0 = __float_as_uint(x0); h1 = __float_as_uint(x1); h2 = __float_as_uint(x2); h3 = __float_as_uint(x3);
        } else {
            tf32_split(x0, h0, l0); tf32_split(x1, h1, l1); tf32_split(x2, h2, l2); tf32_split(x3, h3, l3);
        }
        const float* zb = Zs + (k0 + t4) * ldz + g;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= nnt) break;
            uint32_t bh0, bl0, bh1, bl1;
            tf32_split(zb[nt * 8], bh0, bl0);
            tf32_split(zb[4 * ldz + nt * 8], bh1, bl1);
            if constexpr (!A_EXACT) mma_tf32(acc[nt], l0, l1, l2, l3, bh0, bh1);
            mma_tf32(acc[nt], h0, h1, h2, h3, bl0, bl1);
            mma_tf32(acc[nt], h0, h1, h2, h3, bh0, bh1);
        }
    }
}

template <class Src, bool QUERY>
__global__ void __launch_bounds__(256) k_rr_out(Src src, TcScratch sc, int n, int kw) {
    extern __shared__ __align__(16) char dsm[];
    const int m = sc.m, kwp = rro_kwp(kw), ldz = rro_ldz(kw), ldv = kwp + 1, nnt = kwp / 8;
    float* Zsm = (float*)dsm;                  // m x ldz
    float* Vs = Zsm + (size_t)m * ldz;         // n x ldv
    __shared__ float sig[ZS_MAXM];
    __shared__ float sgnf[ZS_MAXM];
    __shared__ int s_rank;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    for (int item = blockIdx.x; item < src.count(); item += gridDim.x) {
        const int rows = src.rows(item);
        const float* Y = sc.Y + (size_t)src.ybase(item) * m;
        const float* Qf = sc.Qf + (size_t)item * n * m;
        __syncthreads();
        for (int e = tid; e < m * kwp; e += nt) {
            const int a = e / kwp, c = e - (e / kwp) * kwp;
            Zsm[a * ldz + c] = c < kw ? sc.Zs[(size_t)item * m * kw + a * kw + c] : 0.f;
        }
        int kcap;
        if constexpr (QUERY) kcap = src.a.plans[item].kcap;
        else kcap = min(kw, min(rows, n));
        if (tid == 0) s_rank = 0;
        __syncthreads();
        const float s0 = sqrtf(fmaxf(sc.th[(size_t)item * kw], 0.f));
        for (int c = tid; c < kw; c += nt) {
            float sv = sqrtf(fmaxf(sc.th[(size_t)item * kw + c], 0.f));
            if (!(c < kcap && sv > kRankTolF32 * s0)) sv = 0.f;
            sig[c] = sv;
            if (sv > 0.f) atomicAdd(&s_rank, 1);
        }
        // V = Q~ Z on tensor cores (Q~ exact in tf32), 16-row tiles per warp
        for (int rt = wid; rt * 16 < n; rt += nw) {
            float acc[8][4];
            rro_tile<true>(Qf, rt * 16, n, m, Zsm, ldz, nnt, acc, lane);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= nnt) break;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int l = rt * 16 + g + ((e >> 1) ? 8 : 0), c = q * 8 + 2 * t4 + (e & 1);
                    if (l < n) Vs[l * ldv + c] = acc[q][e];
                }
            }
        }
        __syncthreads();
        for (int c = wid; c < kw; c += nw) {
            float best = -1.f;
            int bi = 0x7fffffff;
            for (int l = lane; l < n; l += 32) {
                const float av = fabsf(Vs[l * ldv + c]);
                if (av > best || (av == best && l < bi)) { best = av; bi = l; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) sgnf[c] = (bi < n && Vs[bi * ldv + c] < 0.f) ? -1.f : 1.f;
        }
        __syncthreads();
        float* vt_out;
        float* u_out;
        int64_t urows;
        if constexpr (QUERY) {
            const QPlan& P = src.a.plans[item];
            vt_out = (float*)src.a.vr + (size_t)item * src.a.kq * n;
            u_out = src.u_out(item, src.a.kq);        // C, or the compact Cc of a ragged stack
            urows = rows;
            float* sr = (float*)src.a.sr + (size_t)item * src.a.kq;
            for (int c = tid; c < src.a.kout; c += nt) {
                const float sv = c < kw ? sig[c] : 0.f;
                if (c < kw) sr[c] = sv;
                ((float*)P.S_out)[c] = sv;
            }
            if (tid == 0 && P.rank) *P.rank = s_rank;
            for (int e = tid; e < n * src.a.kout; e += nt) {
                const int l = e / src.a.kout, c = e - (e / src.a.kout) * src.a.kout;
                const float v = (c < kw && sig[c] > 0.f) ? sgnf[c] * Vs[l * ldv + c] : 0.f;
                ((float*)P.V_out)[(size_t)l * P.ldv + c] = v;
            }
        } else {
            const int slot = src.c.slot0 + item;
            vt_out = (float*)src.c.vt + (size_t)slot * src.c.k * n;
            u_out = (float*)src.c.U + (size_t)slot * src.c.b * src.c.k;
            urows = src.c.b;
            float* so = (float*)src.c.sig + (size_t)slot * src.c.k;
            for (int c = tid; c < src.c.k; c += nt) so[c] = c < kw ? sig[c] : 0.f;
        }
        float* w_out = nullptr;
        if constexpr (!QUERY) {
            if (src.c.w) w_out = (float*)src.c.w + (size_t)(src.c.slot0 + item) * src.c.k * n;
        }
        for (int e = tid; e < kw * n; e += nt) {
            const int c = e / n, l = e - (e / n) * n;
            const float vv = sig[c] > 0.f ? sgnf[c] * Vs[l * ldv + c] : 0.f;
            vt_out[e] = vv;
            if (w_out) w_out[e] = sig[c] * vv;      // Sigma V^T, the stack-ready slab
        }
        // fold sign / sigma into Z so that U = Y Zsm
        __syncthreads();
        for (int e = tid; e < m * kwp; e += nt) {
            const int a = e / kwp, c = e - (e / kwp) * kwp;
            float& z = Zsm[a * ldz + c];
            z = (c < kw && sig[c] > 0.f) ? z * sgnf[c] / sig[c] : 0.f;
        }
        __syncthreads();
        // U = Y Zsm on tensor cores (both split), 16-row tiles per warp
        const bool pair = (kw % 2) == 0;
        for (int rt = wid; rt * 16 < urows; rt += nw) {
            float acc[8][4];
            rro_tile<false>(Y, rt * 16, rows, m, Zsm, ldz, nnt, acc, lane);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= nnt) break;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = rt * 16 + g + 8 * h, c = q * 8 + 2 * t4;
                    if (r >= urows || c >= kw) continue;
                    float* up = u_out + (size_t)r * kw + c;
                    if (pair) {
                        *reinterpret_cast<float2*>(up) = make_float2(acc[q][2 * h], acc[q][2 * h + 1]);
                    } else {
                        up[0] = acc[q][2 * h];
                        if (c + 1 < kw) up[1] = acc[q][2 * h + 1];
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 5. Lift on tf32 tensor cores (float stores): the rows of U_{S:E} are the
//    stored U_i rows times each slab's coefficients C (k x kq) (Algorithm 2,
//    last step; Eq. 9), one warp per slab, 32 rows per step.  U rows and C are
//    split into two tf32 terms each (three products: FP32-grade results); C is
//    split once per slab into two shared tiles.
// ---------------------------------------------------------------------------
template <int QMAX>
// C tile row stride: 4 * LDC = 8 (mod 32) keeps the permuted B loads (rows 4 t4 + .., column g) on distinct banks
__host__ __device__ constexpr int lift_ldc() { return (QMAX + 31) / 32 * 32 + 2; }
template <int KMAX, int QMAX>
__host__ __device__ __forceinline__ size_t lift_tc_warp_floats() { return (size_t)2 * KMAX * lift_ldc<QMAX>(); }

template <int KMAX, int QMAX>
__global__ void __launch_bounds__(256) k_lift_tc(QueryArgs a) {
    extern __shared__ __align__(16) float lsm[];
    constexpr int LDC = lift_ldc<QMAX>();
    const int k = a.k, kq = a.kq, kout = a.kout;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    float* Ch = lsm + (size_t)warp * lift_tc_warp_floats<KMAX, QMAX>();
    float* Cl = Ch + KMAX * LDC;
    const int nq = a.hdr->nq;
    const int64_t total = a.hdr->nslab_total, Trows = a.hdr->T;
    const int nnt = (kout + 7) / 8;
    // each warp takes a contiguous range of slabs, so the owning query only
    // advances (one search per warp instead of one per slab)
    const int64_t nw = (int64_t)gridDim.x * wpc, wid = (int64_t)blockIdx.x * wpc + warp;
    const int64_t per = (total + nw - 1) / nw;
    const int64_t s_lo = wid * per, s_hi = min(total, s_lo + per);
    int q = s_lo < s_hi ? find_query(a.slab_prefix, nq, s_lo) : 0;
    for (int64_t s = s_lo; s < s_hi; ++s) {
        while (q + 1 < nq && a.slab_prefix[q + 1] <= s) ++q;
        const QPlan& P = a.plans[q];
        const int t = (int)(s - P.slab0);
        const BlockRange br = slab_rows(P, t, a.b, Trows);
        const float* U = (const float*)a.U + (int64_t)br.blk * a.b * k;
        const float* Cg = (const float*)a.C + s * k * kq;
        __syncwarp();
        for (int e = lane; e < KMAX * QMAX; e += 32) {
            const int aa = e / QMAX, c = e % QMAX;
            const float v = (aa < k && c < kq) ? Cg[aa * kq + c] : 0.f;
            uint32_t h, l;
            tf32_split(v, h, l);
            Ch[aa * LDC + c] = __uint_as_float(h);
            Cl[aa * LDC + c] = __uint_as_float(l);
        }
        __syncwarp();
        float* out = (float*)P.U;
        const int64_t o0 = (int64_t)br.blk * a.b - P.ts;
        const bool pair = (kout % 2 == 0) && (P.ldu % 2 == 0) && ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
        // The MMA's K order is permuted so that each thread reads its U row
        // segments as 16-byte pieces: in column group gi (16 columns), thread
        // t4 holds columns 16 gi + 4 t4 + {0, 1} as K slots (t4, t4 + 4) of
        // step 2 gi and + {2, 3} as those of step 2 gi + 1; the B fragments
        // take C's rows in the same order.  32 rows per step, the next 32
        // prefetched (two 16-row halves).
        constexpr int NG = KMAX / 16;
        const int ngv = (k + 15) / 16;
        const bool vec = (k % 4) == 0;      // 16-byte aligned row segments
        float nx[2][NG][2][4];
        auto fetch = [&](int r0, float (&dst)[NG][2][4]) {
            const int ra = r0 + g, rb = r0 + g + 8;
            const bool va = ra < br.hi, vb = rb < br.hi;
            const float* pa = U + (int64_t)ra * k;
            const float* pb = U + (int64_t)rb * k;
#pragma unroll
            for (int gi = 0; gi < NG; ++gi) {
                const int c = gi * 16 + 4 * t4;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
                if (gi < ngv) {
                    if (vec) {
                        if (va && c < k) x = __ldg(reinterpret_cast<const float4*>(pa + c));
                        if (vb && c < k) y = __ldg(reinterpret_cast<const float4*>(pb + c));
                    } else {
                        if (va) {
                            x.x = c < k ? __ldg(pa + c) : 0.f;
                            x.y = c + 1 < k ? __ldg(pa + c + 1) : 0.f;
                            x.z = c + 2 < k ? __ldg(pa + c + 2) : 0.f;
                            x.w = c + 3 < k ? __ldg(pa + c + 3) : 0.f;
                        }
                        if (vb) {
                            y.x = c < k ? __ldg(pb + c) : 0.f;
                            y.y = c + 1 < k ? __ldg(pb + c + 1) : 0.f;
                            y.z = c + 2 < k ? __ldg(pb + c + 2) : 0.f;
                            y.w = c + 3 < k ? __ldg(pb + c + 3) : 0.f;
                        }
                    }
                }
                // fragment order a0 (row g, slot t4), a1 (row g+8, slot t4), a2 (row g, slot t4+4), a3
                dst[gi][0][0] = x.x; dst[gi][0][1] = y.x; dst[gi][0][2] = x.y; dst[gi][0][3] = y.y;
                dst[gi][1][0] = x.z; dst[gi][1][1] = y.z; dst[gi][1][2] = x.w; dst[gi][1][3] = y.w;
            }
        };
        if (br.lo < br.hi) {
            fetch(br.lo, nx[0]);
            fetch(br.lo + 16, nx[1]);
        }
        // B fragments of the slab (fixed over its rows) held in registers when they fit
        constexpr bool HOIST = NG * (QMAX / 8) <= 4;
        uint32_t bf[HOIST ? NG : 1][2][HOIST ? QMAX / 8 : 1][4];
        if constexpr (HOIST) {
#pragma unroll
            for (int gi = 0; gi < NG; ++gi)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int cr = gi * 16 + 4 * t4 + 2 * j;
#pragma unroll
                    for (int nt = 0; nt < QMAX / 8; ++nt) {
                        bf[gi][j][nt][0] = __float_as_uint(Ch[cr * LDC + nt * 8 + g]);
                        bf[gi][j][nt][1] = __float_as_uint(Ch[(cr + 1) * LDC + nt * 8 + g]);
                        bf[gi][j][nt][2] = __float_as_uint(Cl[cr * LDC + nt * 8 + g]);
                        bf[gi][j][nt][3] = __float_as_uint(Cl[(cr + 1) * LDC + nt * 8 + g]);
                    }
                }
        }
        for (int r0 = br.lo; r0 < br.hi; r0 += 32) {
            float cx[2][NG][2][4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
                for (int gi = 0; gi < NG; ++gi)
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int e = 0; e < 4; ++e) cx[h2][gi][j][e] = nx[h2][gi][j][e];
            if (r0 + 32 < br.hi) {
                fetch(r0 + 32, nx[0]);
                fetch(r0 + 48, nx[1]);
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int rs = r0 + 16 * h2;
                if (rs >= br.hi) break;
                float acc[QMAX / 8][4];
#pragma unroll
                for (int x = 0; x < QMAX / 8; ++x) acc[x][0] = acc[x][1] = acc[x][2] = acc[x][3] = 0.f;
#pragma unroll
                for (int gi = 0; gi < NG; ++gi) {
                    if (gi >= ngv) break;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        uint32_t h0, h1, h2v, h3, l0, l1, l2, l3;
                        tf32_split_trunc(cx[h2][gi][j][0], h0, l0);
                        tf32_split_trunc(cx[h2][gi][j][1], h1, l1);
                        tf32_split_trunc(cx[h2][gi][j][2], h2v, l2);
                        tf32_split_trunc(cx[h2][gi][j][3], h3, l3);
                        // K slot t4 <-> C row 16 gi + 4 t4 + 2 j, slot t4 + 4 <-> the row after it
                        const int cr = gi * 16 + 4 * t4 + 2 * j;
                        const float* bh = Ch + cr * LDC + g;
                        const float* bl = Cl + cr * LDC + g;
#pragma unroll
                        for (int nt = 0; nt < QMAX / 8; ++nt) {
                            if (nt >= nnt) break;
                            uint32_t bh0, bh1, bl0, bl1;
                            if constexpr (HOIST) {
                                bh0 = bf[gi][j][nt][0];
                                bh1 = bf[gi][j][nt][1];
                                bl0 = bf[gi][j][nt][2];
                                bl1 = bf[gi][j][nt][3];
                            } else {
                                bh0 = __float_as_uint(bh[nt * 8]);
                                bh1 = __float_as_uint(bh[LDC + nt * 8]);
                                bl0 = __float_as_uint(bl[nt * 8]);
                                bl1 = __float_as_uint(bl[LDC + nt * 8]);
                            }
                            mma_tf32(acc[nt], l0, l1, l2, l3, bh0, bh1);
                            mma_tf32(acc[nt], h0, h1, h2v, h3, bl0, bl1);
                            mma_tf32(acc[nt], h0, h1, h2v, h3, bh0, bh1);
                        }
                    }
                }
                const int ra = rs + g, rb = rs + g + 8;
#pragma unroll
                for (int nt = 0; nt < QMAX / 8; ++nt) {
                    if (nt >= nnt) break;
                    const int c = nt * 8 + 2 * t4;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int r = hh ? rb : ra;
                        if (r >= br.hi || c >= kout) continue;
                        float* orow = out + (o0 + r) * P.ldu + c;
                        if (pair) {
                            *reinterpret_cast<float2*>(orow) = make_float2(acc[nt][2 * hh], acc[nt][2 * hh + 1]);
                        } else {
                            orow[0] = acc[nt][2 * hh];
                            if (c + 1 < kout) orow[1] = acc[nt][2 * hh + 1];
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 5'. Lift for k not a multiple of 16 (the K order of k_lift_tc would waste a
//    step on a partly filled 16-column group): the same product in natural K
//    order: the stored U_i rows times each slab's coefficients C (k x kq)
//    (Algorithm 2, last step; Eq. 9), one warp per slab, 16 rows per step, U
//    fragments of the next step loaded before the current step's products.
//    U rows and C are split into two tf32 terms each (three products); C is
//    split once per slab into two shared tiles.
// ---------------------------------------------------------------------------
template <int QMAX>
__host__ __device__ constexpr int lift_ldc_nat() { return (QMAX + 31) / 32 * 32 + 8; }
template <int KMAX, int QMAX>
__host__ __device__ __forceinline__ size_t lift_nat_warp_floats() { return (size_t)2 * KMAX * lift_ldc_nat<QMAX>(); }

template <int KMAX, int QMAX>
__global__ void __launch_bounds__(256) k_lift_tc_nat(QueryArgs a) {
    extern __shared__ __align__(16) float lsm[];
    constexpr int LDC = lift_ldc_nat<QMAX>();
    const int k = a.k, kq = a.kq, kout = a.kout;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    float* Ch = lsm + (size_t)warp * lift_nat_warp_floats<KMAX, QMAX>();
    float* Cl = Ch + KMAX * LDC;
    const int nq = a.hdr->nq;
    const int64_t total = a.hdr->nslab_total, Trows = a.hdr->T;
    const int nkt = (k + 7) / 8, nnt = (kout + 7) / 8;
    // each warp takes a contiguous range of slabs, so the owning query only
    // advances (one search per warp instead of one per slab)
    const int64_t nw = (int64_t)gridDim.x * wpc, wid = (int64_t)blockIdx.x * wpc + warp;
    const int64_t per = (total + nw - 1) / nw;
    const int64_t s_lo = wid * per, s_hi = min(total, s_lo + per);
    int q = s_lo < s_hi ? find_query(a.slab_prefix, nq, s_lo) : 0;
    for (int64_t s = s_lo; s < s_hi; ++s) {
        while (q + 1 < nq && a.slab_prefix[q + 1] <= s) ++q;
        const QPlan& P = a.plans[q];
        const int t = (int)(s - P.slab0);
        const BlockRange br = slab_rows(P, t, a.b, Trows);
        const float* U = (const float*)a.U + (int64_t)br.blk * a.b * k;
        const float* Cg = (const float*)a.C + s * k * kq;
        __syncwarp();
        for (int e = lane; e < KMAX * QMAX; e += 32) {
            const int aa = e / QMAX, c = e % QMAX;
            const float v = (aa < k && c < kq) ? Cg[aa * kq + c] : 0.f;
            uint32_t h, l;
            tf32_split(v, h, l);
            Ch[aa * LDC + c] = __uint_as_float(h);
            Cl[aa * LDC + c] = __uint_as_float(l);
        }
        __syncwarp();
        float* out = (float*)P.U;
        const int64_t o0 = (int64_t)br.blk * a.b - P.ts;
        const bool pair = (kout % 2 == 0) && (P.ldu % 2 == 0) && ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
        // U fragments of the next 16-row step are loaded before the current
        // step's products (software pipeline over the slab's rows)
        float nx[KMAX / 8][4];
        auto fetch = [&](int r0, float (&dst)[KMAX / 8][4]) {
            const int ra = r0 + g, rb = r0 + g + 8;
            const bool va = ra < br.hi, vb = rb < br.hi;
            const float* pa = U + (int64_t)ra * k;
            const float* pb = U + (int64_t)rb * k;
#pragma unroll
            for (int kt = 0; kt < KMAX / 8; ++kt) {
                const int c0 = kt * 8 + t4, c1 = c0 + 4;
                dst[kt][0] = (kt < nkt && va && c0 < k) ? __ldg(pa + c0) : 0.f;
                dst[kt][1] = (kt < nkt && vb && c0 < k) ? __ldg(pb + c0) : 0.f;
                dst[kt][2] = (kt < nkt && va && c1 < k) ? __ldg(pa + c1) : 0.f;
                dst[kt][3] = (kt < nkt && vb && c1 < k) ? __ldg(pb + c1) : 0.f;
            }
        };
        if (br.lo < br.hi) fetch(br.lo, nx);
        for (int r0 = br.lo; r0 < br.hi; r0 += 16) {
            float cx[KMAX / 8][4];
#pragma unroll
            for (int kt = 0; kt < KMAX / 8; ++kt)
#pragma unroll
                for (int e = 0; e < 4; ++e) cx[kt][e] = nx[kt][e];
            if (r0 + 16 < br.hi) fetch(r0 + 16, nx);
            float acc[QMAX / 8][4];
#pragma unroll
            for (int x = 0; x < QMAX / 8; ++x) acc[x][0] = acc[x][1] = acc[x][2] = acc[x][3] = 0.f;
            const int ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
            for (int kt = 0; kt < KMAX / 8; ++kt) {
                if (kt >= nkt) break;
                const int c0 = kt * 8 + t4;
                uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
                tf32_split_trunc(cx[kt][0], h0, l0);
                tf32_split_trunc(cx[kt][1], h1, l1);
                tf32_split_trunc(cx[kt][2], h2, l2);
                tf32_split_trunc(cx[kt][3], h3, l3);
                const float* bh = Ch + c0 * LDC + g;
                const float* bl = Cl + c0 * LDC + g;
#pragma unroll
                for (int nt = 0; nt < QMAX / 8; ++nt) {
                    if (nt >= nnt) break;
                    const uint32_t bh0 = __float_as_uint(bh[nt * 8]), bh1 = __float_as_uint(bh[4 * LDC + nt * 8]);
                    const uint32_t bl0 = __float_as_uint(bl[nt * 8]), bl1 = __float_as_uint(bl[4 * LDC + nt * 8]);
                    mma_tf32(acc[nt], l0, l1, l2, l3, bh0, bh1);
                    mma_tf32(acc[nt], h0, h1, h2, h3, bl0, bl1);
                    mma_tf32(acc[nt], h0, h1, h2, h3, bh0, bh1);
                }
            }
#pragma unroll
            for (int nt = 0; nt < QMAX / 8; ++nt) {
                if (nt >= nnt) break;
                const int c = nt * 8 + 2 * t4;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int r = hh ? rb : ra;
                    if (r >= br.hi || c >= kout) continue;
                    float* orow = out + (o0 + r) * P.ldu + c;
                    if (pair) {
                        *reinterpret_cast<float2*>(orow) = make_float2(acc[nt][2 * hh], acc[nt][2 * hh + 1]);
                    } else {
                        orow[0] = acc[nt][2 * hh];
                        if (c + 1 < kout) orow[1] = acc[nt][2 * hh + 1];
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Partial-SVD (Algorithm 3; Eq. 5-6) of one boundary slab per warp, float
// stores with k <= KB <= 32:
//   H = Sigma (X U)^T (X U) Sigma over the slab's rows on tf32 tensor cores
//       (U split in two terms, three products; each row segment loaded once
//       serves both operands),
//   H = G G^T, one-sided Jacobi on G's columns -> V~, Sigma~^2 (sorted),
//   slab rows Sigma~ V~^T V^T of M (another small tensor-core product) and
//   the lift coefficient Sigma V~ Sigma~^{-1}.
// ---------------------------------------------------------------------------
template <int KB>
__global__ void __launch_bounds__(128) k_partial_warp(QueryArgs a) {
    constexpr int MT = KB / 16, NT = KB / 8, KT = KB / 8;
    __shared__ float tiles[4][2][32 * 33];            // per warp: work tile, sorted V~
    __shared__ float sts[4][32];                      // per warp: sorted Sigma~
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int p = blockIdx.x * 4 + warp;
    const int nq = a.hdr->nq;
    if (p >= 2 * nq) return;
    const int q = p >> 1, side = p & 1;
    const QPlan& P = a.plans[q];
    if (side == 1 && P.nslab == 1) return;
    const int t = side ? P.nslab - 1 : 0;
    const int k = a.k, n = a.n;
    const BlockRange br = slab_rows(P, t, a.b, a.hdr->T);
    const int ki = min(k, min(br.rows_i, n));
    const float* U = (const float*)a.U + (int64_t)br.blk * a.b * k;
    const float* sg = (const float*)a.sig + (int64_t)br.blk * k;
    const float* vt = (const float*)a.vt + (int64_t)br.blk * k * n;
    float* T = tiles[warp][0];
    float* Zs = tiles[warp][1];
    float* st = sts[warp];
    // 1. Gram of the slab's rows of U
    float h[MT][NT][4];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < NT; ++y) h[x][y][0] = h[x][y][1] = h[x][y][2] = h[x][y][3] = 0.f;
    float n0[NT], n1[NT];
    auto fetch = [&](int r0) {
        const int ra = r0 + t4, rb = r0 + t4 + 4;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int c = g + 8 * j;
            n0[j] = (ra < br.hi && c < ki) ? __ldg(U + (int64_t)ra * k + c) : 0.f;
            n1[j] = (rb < br.hi && c < ki) ? __ldg(U + (int64_t)rb * k + c) : 0.f;
        }
    };
    if (br.lo < br.hi) fetch(br.lo);
    for (int r0 = br.lo; r0 < br.hi; r0 += 8) {
        uint32_t h0[NT], l0[NT], h1[NT], l1[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            tf32_split(n0[j], h0[j], l0[j]);
            tf32_split(n1[j], h1[j], l1[j]);
        }
        if (r0 + 8 < br.hi) fetch(r0 + 8);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                mma_tf32(h[mt][nt], l0[2 * mt], l0[2 * mt + 1], l1[2 * mt], l1[2 * mt + 1], h0[nt], h1[nt]);
                mma_tf32(h[mt][nt], h0[2 * mt], h0[2 * mt + 1], h1[2 * mt], h1[2 * mt + 1], l0[nt], l1[nt]);
                mma_tf32(h[mt][nt], h0[2 * mt], h0[2 * mt + 1], h1[2 * mt], h1[2 * mt + 1], h0[nt], h1[nt]);
            }
    }
    // H -> column `lane` in registers, scaled by sigma_i sigma_j
    float sgl = lane < ki ? sg[lane] : 0.f;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = mt * 16 + g + ((e >> 1) ? 8 : 0), j = nt * 8 + 2 * t4 + (e & 1);
                T[i * 33 + j] = h[mt][nt][e];
            }
    __syncwarp();
    float x[32], v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float si = __shfl_sync(0xffffffffu, sgl, i);
        x[i] = (i < ki && lane < ki) ? T[i * 33 + lane] * si * sgl : 0.f;
    }
    __syncwarp();
    // 2. eigenpairs of H
    warp_chol32(x, T, lane);
    const float th = warp_hestenes32(x, v, lane);
    int rk = 0;
#pragma unroll
    for (int o = 0; o < 32; ++o) {
        const float ot = __shfl_sync(0xffffffffu, th, o);
        rk += (ot > th) || (ot == th && o < lane);
    }
    // keep r = min(rows, ki) pairs (the rank of X U Sigma), above the rank tolerance
    const int r = min(br.hi - br.lo, ki);
    float sv = rk < r ? sqrtf(fmaxf(th, 0.f)) : 0.f;
    float s0 = sv;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s0 = fmaxf(s0, __shfl_xor_sync(0xffffffffu, s0, o));
    if (!(sv > kRankTolF32 * s0)) sv = 0.f;
    st[rk] = sv;
#pragma unroll
    for (int i = 0; i < 32; ++i) Zs[i * 33 + rk] = x[i];
    __syncwarp();
    // 3. lift coefficient Sigma V~ Sigma~^{-1} (k x k)
    float* tc = (float*)a.tco + (int64_t)p * k * k;
    for (int e = lane; e < k * k; e += 32) {
        const int aa = e / k, j = e - (e / k) * k;
        const float sj = st[j];
        tc[e] = (aa < ki && sj > 0.f) ? sg[aa] * Zs[aa * 33 + j] / sj : 0.f;
    }
    // 4. slab rows of M: Ms[j][l] = Sigma~_j sum_aa V~[aa][j] Vt[aa][l]
    uint32_t ah[KT][MT][4], al[KT][MT][4];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int r0 = kt * 8 + t4, jr = mt * 16 + g;
            tf32_split(Zs[r0 * 33 + jr], ah[kt][mt][0], al[kt][mt][0]);
            tf32_split(Zs[r0 * 33 + jr + 8], ah[kt][mt][1], al[kt][mt][1]);
            tf32_split(Zs[(r0 + 4) * 33 + jr], ah[kt][mt][2], al[kt][mt][2]);
            tf32_split(Zs[(r0 + 4) * 33 + jr + 8], ah[kt][mt][3], al[kt][mt][3]);
        }
    float* Ms = (float*)a.M + (P.slab0 + t) * k * n;
    for (int l0 = 0; l0 < n; l0 += 8) {
        float c[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) c[mt][0] = c[mt][1] = c[mt][2] = c[mt][3] = 0.f;
        const int l = l0 + g;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const int r0 = kt * 8 + t4;
            const float b0 = (r0 < ki && l < n) ? __ldg(vt + (int64_t)r0 * n + l) : 0.f;
            const float b1 = (r0 + 4 < ki && l < n) ? __ldg(vt + (int64_t)(r0 + 4) * n + l) : 0.f;
            uint32_t bh0, bl0, bh1, bl1;
            tf32_split(b0, bh0, bl0);
            tf32_split(b1, bh1, bl1);
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                mma_tf32(c[mt], al[kt][mt][0], al[kt][mt][1], al[kt][mt][2], al[kt][mt][3], bh0, bh1);
                mma_tf32(c[mt], ah[kt][mt][0], ah[kt][mt][1], ah[kt][mt][2], ah[kt][mt][3], bl0, bl1);
                mma_tf32(c[mt], ah[kt][mt][0], ah[kt][mt][1], ah[kt][mt][2], ah[kt][mt][3], bh0, bh1);
            }
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = mt * 16 + g + ((e >> 1) ? 8 : 0), ll = l0 + 2 * t4 + (e & 1);
                if (j < k && ll < n) {
                    const float sj = st[j];
                    Ms[(int64_t)j * n + ll] = sj > 0.f ? sj * c[mt][e] : 0.f;
                }
            }
    }
}

// ---------------------------------------------------------------------------
// Ragged stacks (energy rule, Eq. 1): the stacked matrix of a query takes the
// two boundary slabs' k rows (Partial-SVD output in M) and only the live rows
// of the interior slabs - block s contributes kpre[s + 1] - kpre[s] rows of
// its stored Sigma_s V_s^T, the rest being zero rows that change no result.
// k_ragged_map writes each query's row map (>= 0: row of the store's
// Sigma V^T, < 0: -1 - row of M) and its row count (plan.pad1); after the
// stitched SVD, k_ragged_expand spreads the compact U_r rows back to k rows
// per slab (zero for the dropped rows) for the boundary fix and the lift.
// One CTA per query.
// ---------------------------------------------------------------------------
// kpre[i] = live ranks (nonzero sigma: the energy rule and R5 zero the rest)
// of blocks 0 .. i-1 of the store's T rows; one CTA, a block-wide scan per
// 1,024 blocks.
static __global__ void __launch_bounds__(1024) k_ragged_prefix(QueryArgs a) {
    __shared__ int64_t s_carry;
    __shared__ int s_warp[32];
    const int k = a.k;
    const int64_t nblk = (a.hdr->T + a.b - 1) / a.b;
    const float* sig = (const float*)a.sig;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        s_carry = 0;
        a.kpre[0] = 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < nblk; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int v = 0;
        if (i < nblk)
            for (int j = 0; j < k; ++j) v += sig[i * k + j] > 0.f;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nwarp ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? s_warp[warp - 1] : 0);
        if (i < nblk) a.kpre[i + 1] = s_carry + incl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += incl;
        __syncthreads();
    }
}

static __global__ void __launch_bounds__(256) k_ragged_map(QueryArgs a) {
    const int k = a.k, nq = a.hdr->nq;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        QPlan& P = const_cast<QPlan&>(a.plans[q]);
        const int64_t base = P.slab0 * k;
        int* map = a.rowmap + base;
        const int ns = P.nslab;
        int R = k;
        if (ns == 1) {
            for (int r = threadIdx.x; r < k; r += blockDim.x) map[r] = (int)(-1 - (base + r));
        } else {
            const int64_t K0 = a.kpre[P.S + 1];
            R = 2 * k + (int)(a.kpre[P.S + ns - 1] - K0);
            for (int r = threadIdx.x; r < k; r += blockDim.x) {
                map[r] = (int)(-1 - (base + r));
                map[R - k + r] = (int)(-1 - (base + (int64_t)(ns - 1) * k + r));
            }
            for (int e = threadIdx.x; e < (ns - 2) * k; e += blockDim.x) {
                const int t = 1 + e / k, j = e - (e / k) * k;
                const int64_t s = P.S + t;
                const int64_t lo = a.kpre[s];
                if (j < (int)(a.kpre[s + 1] - lo)) map[k + (lo - K0) + j] = (int)(s * k + j);
            }
        }
        if (threadIdx.x == 0) P.pad1 = R;
    }
}

static __global__ void __launch_bounds__(256) k_ragged_expand(QueryArgs a) {
    const int k = a.k, kq = a.kq, nq = a.hdr->nq;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const QPlan& P = a.plans[q];
        const int64_t base = P.slab0 * k;
        float* C = (float*)a.C + base * kq;
        const float* Cc = (const float*)a.Cc + base * kq;
        const int* map = a.rowmap + base;
        const int R = P.pad1;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)P.nslab * k * kq; e += blockDim.x) C[e] = 0.f;
        __syncthreads();
        for (int e = threadIdx.x; e < R * kq; e += blockDim.x) {
            const int r = e / kq, c = e - (e / kq) * kq;
            const int v = map[r];
            int64_t dst;                                 // the row's place in the slab layout
            if (v >= 0) dst = (int64_t)(v / k - P.S) * k + v % k;
            else dst = (int64_t)(-1 - v) - base;
            C[dst * kq + c] = Cc[(int64_t)r * kq + c];
        }
    }
}

// Query boundary slabs: C_slab <- (Sigma V~ Sigma~^{-1}) C_slab  (k x kq), in place.
static __global__ void __launch_bounds__(256) k_bfix(QueryArgs a) {
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
