// zs_certify.cuh - a-posteriori accuracy test of the float path's truncated
// SVDs (each stored block of the storage phase, Section 3.2 / Algorithm 1, and
// each query's Stitched-SVD, Algorithm 2), and bounded subspace iteration for
// the items that fail it.
//
// The sketch + Rayleigh-Ritz step of zs_tc_kernels.cuh returns the exact
// truncated SVD (Eckart-Young, Section 2.1) only when the sketched subspace
// holds the top k singular directions, which a spectrum without a gap after k
// does not guarantee.  So every item is tested on the device instead of
// trusting the input:
//
//   k_check   R = X^T U from the factors as written (split tf32 operands:
//             FP32-grade products), then for each kept pair the residual
//             rho_j = |X^T u_j - sigma_j v_j| (X v_j = sigma_j u_j holds by
//             construction, U = X V Sigma^-1) and the bound
//                 beta_j = min(rho_j, rho_j^2 / eta_j),  eta_j = sigma_j - s_m,
//             on |sigma_j - sigma_j(X)|: the residual bound for a singular
//             triplet, and its quadratic form, with the gap to the smallest
//             Ritz value s_m of the subspace standing for the gap to the part
//             of the spectrum the subspace does not hold.  An item passes when
//             beta_j <= kCertTol max(sigma_j, 1e-2 sigma_1) for every kept
//             pair; the others are listed for refinement.
//   k_refine  one CTA (16 warps) per listed item: subspace iteration of width
//             kRefineM on X^T X, started from the sketch's basis plus random
//             sign columns.  One pass over the item's rows per iteration gives
//             Y = X Q, W = X^T Y and H = Y^T Y (split tf32 operands); then
//             Rayleigh-Ritz on H (FP32 Jacobi), the residual
//             r_j = W z_j - theta_j Q z_j (|r_j| / sigma_j is rho_j above) and
//             the same test decide whether to stop, else Q = orth(W).  The
//             outputs are rewritten from the last iterate (U by one more pass,
//             U = X V Sigma^-1).  An item that has not passed after
//             kRefineMaxPasses passes keeps that last iterate and increments
//             the status word `noconv`, which the library reports as an error.
#pragma once

#include "zs_tc_kernels.cuh"

namespace zs {

constexpr float kCertTol = 1e-5f;       // bound on |sigma_j - sigma_j(X)| / max(sigma_j, 1e-2 sigma_1)
constexpr int kRefineMaxPasses = 16;    // passes over an item's rows in k_refine
constexpr int kRefineM = 64;            // width of the refinement subspace (<= n on the tensor path)
constexpr int kRefineThreads = 512;
constexpr int kRefineTR = 32;           // rows per tile in k_refine

// k_check tiles: TR rows of X (fp32, row stride ldx) and of U (row stride ldb)
__host__ __device__ __forceinline__ int ck_rows(int n) {
    int t = 8192 / (n > 0 ? n : 1);
    t = t < 32 ? 32 : (t > 128 ? 128 : t);
    return t / 8 * 8;
}
// strides = 8 mod 32: the transposed-operand fragments (rows t4, columns g) are conflict-free
__host__ __device__ __forceinline__ int ck_ldx(int n) { return (n + 31) / 32 * 32 + 8; }
__host__ __device__ __forceinline__ int ck_ldb(int w) {        // = 8 or 24 mod 32
    const int wp = (w + 7) / 8 * 8;
    return wp + (((wp / 8) % 2 == 0) ? 8 : 16);
}
__host__ __device__ __forceinline__ size_t ck_stage_floats(int n, int kw) {
    return (size_t)ck_rows(n) * ck_ldx(n) + (size_t)ck_rows(n) * ck_ldb(kw);
}
__host__ __device__ __forceinline__ int ck_stages(int n, int kw) {
    return 2 * ck_stage_floats(n, kw) * 4 <= 200 * 1024 ? 2 : 1;
}
// bf16 rows are copied raw (TR x round32(n) bf16) and their scale factors
// (TR floats) per stage, then widened into the stage's fp32 tile
__host__ __device__ __forceinline__ size_t ck_raw_floats(int n) {
    return (size_t)ck_rows(n) * ((n + 31) / 32 * 32) / 2 + ck_rows(n);
}
__host__ __device__ __forceinline__ size_t ck_smem_bytes(int n, int kw, bool raw16 = false) {
    const size_t st = (size_t)ck_stages(n, kw) * ck_stage_floats(n, kw);
    const size_t rs = (size_t)(n < 512 ? (n + 15) / 16 * 16 : 512) * ((kw + 7) / 8 * 8 + 1);
    return 4 * ((st > rs ? st : rs) + (raw16 ? (size_t)ck_stages(n, kw) * ck_raw_floats(n) : 0));
}
// k_refine: Q (round32(n) x ldq), then a region holding either the X and Y
// tiles of a pass or H and Z of the Rayleigh-Ritz step
__host__ __device__ __forceinline__ int rf_ldq() { return kRefineM + 8; }
__host__ __device__ __forceinline__ size_t rf_smem_bytes(int n) {
    const size_t q = (size_t)((n + 31) / 32 * 32) * rf_ldq();
    const size_t tile = (size_t)kRefineTR * ck_ldx(n) + (size_t)kRefineTR * rf_ldq();
    const size_t rr = 2 * (size_t)kRefineM * (kRefineM + 1);
    return 4 * (q + (tile > rr ? tile : rr));
}

// Rows [r0, r0 + nr) of an item into Xs (fp32, row stride ldx); rows past
// `rows` and columns [n, ncp) are zero.  Aligned float rows go by cp.async
// (the caller commits and waits); other inputs are loaded, converted to fp32
// and stored.
template <class Src, typename Tin>
__device__ __forceinline__ void ld_xtile(const Src& src, const typename Src::Ctx& cx, int r0, int nr, int rows,
                                         int n, int ncp, float* Xs, int ldx, bool vec) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if constexpr (std::is_same<Tin, float>::value) {
        if (vec && nt % (ncp / 4) == 0) {
            // each thread keeps one 16-byte column piece and steps through the rows
            const int q4 = ncp / 4, c = (tid % q4) * 4, rstep = nt / q4;
            const bool live_c = c < n;
            for (int r = tid / q4; r < nr; r += rstep) {
                float* d = Xs + r * ldx + c;
                if (r0 + r < rows && live_c) {
                    float s;
                    cp_async16(d, src.template row<float>(cx, r0 + r, s) + c, 16);
                } else {
                    *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            return;
        }
        if (vec) {
            const int q4 = ncp / 4;
            for (int f = tid; f < nr * q4; f += nt) {
                const int r = f / q4, c = (f - r * q4) * 4;
                float* d = Xs + r * ldx + c;
                if (r0 + r < rows && c < n) {
                    float s;
                    cp_async16(d, src.template row<float>(cx, r0 + r, s) + c, 16);
                } else {
                    *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            return;
        }
    }
    for (int f = tid; f < nr * ncp; f += nt) {
        const int r = f / ncp, c = f - r * ncp;
        float v = 0.f;
        if (r0 + r < rows && c < n) {
            float s;
            v = ld_in(src.template row<Tin>(cx, r0 + r, s) + c) * s;
        }
        Xs[r * ldx + c] = v;
    }
}

// bf16 rows with 16-byte aligned starts (n % 8 == 0): rows [r0, r0 + nr) of
// an item copied as they are into Rw (nr x ncp bf16) by cp.async, zero past
// `rows` and past column n, with each row's scale factor in rs (0 for rows
// past the item); cvt_xtile widens them into the fp32 tile once they landed.
template <class Src>
__device__ __forceinline__ void ld_xtile_raw16(const Src& src, const typename Src::Ctx& cx, int r0, int nr, int rows,
                                               int n, int ncp, __nv_bfloat16* Rw, float* rs) {
    const int q8 = ncp / 8;
    for (int f = threadIdx.x; f < nr * q8; f += blockDim.x) {
        const int r = f / q8, c = (f - r * q8) * 8;
        const bool live = r0 + r < rows && c < n;
        float sc = 0.f;
        const __nv_bfloat16* pr = src.template row<__nv_bfloat16>(cx, min(r0 + r, rows - 1), sc);
        cp_async16(Rw + (size_t)r * ncp + c, pr + (live ? c : 0), live ? 16 : 0);
        if (c == 0) rs[r] = r0 + r < rows ? sc : 0.f;
    }
}
__device__ __forceinline__ void cvt_xtile(const __nv_bfloat16* Rw, const float* rs, int nr, int ncp, float* Xs,
                                          int ldx) {
    const int q8 = ncp / 8;
    for (int f = threadIdx.x; f < nr * q8; f += blockDim.x) {
        const int r = f / q8, c = (f - r * q8) * 8;
        const uint4 v = *reinterpret_cast<const uint4*>(Rw + (size_t)r * ncp + c);
        const float sc = rs[r];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        float o[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = __uint_as_float(w[i] << 16) * sc;
            o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u) * sc;
        }
        *reinterpret_cast<float4*>(Xs + r * ldx + c) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4*>(Xs + r * ldx + c + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
}
template <class Src, typename Tin>
__device__ __forceinline__ bool rows_raw16(const Src& src, int item, int n) {
    if constexpr (std::is_same<Tin, __nv_bfloat16>::value)
        return (n % 8 == 0) && (src.ld() % 8 == 0) && ((reinterpret_cast<uintptr_t>(src.X(item, 2)) & 15) == 0);
    return false;
}

// Rows [r0, r0 + nr) of a row-major rows x w matrix B (row stride ldg) into
// Bs (row stride ldb, wp >= w columns, zero past w and past `rows`), by
// cp.async (16-byte pieces when w and ldg are multiples of 4 and B is
// 16-byte aligned, else 4-byte elements); the caller commits and waits.
__device__ __forceinline__ void ld_btile(const float* B, int ldg, int r0, int nr, int rows, int w, int wp,
                                         float* Bs, int ldb) {
    if (w % 4 == 0 && ldg % 4 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0) {
        const int q4 = wp / 4;
        for (int f = threadIdx.x; f < nr * q4; f += blockDim.x) {
            const int r = f / q4, c = (f - r * q4) * 4;
            const bool live = r0 + r < rows && c < w;
            cp_async16(Bs + r * ldb + c, B + (live ? (size_t)(r0 + r) * ldg + c : 0), live ? 16 : 0);
        }
        return;
    }
    for (int f = threadIdx.x; f < nr * wp; f += blockDim.x) {
        const int r = f / wp, c = f - r * wp;
        const bool live = r0 + r < rows && c < w;
        cp_async4(Bs + r * ldb + c, B + (live ? (size_t)(r0 + r) * ldg + c : 0), live ? 4 : 0);
    }
}

template <class Src, typename Tin>
__device__ __forceinline__ bool rows_vec16(const Src& src, int item, int n) {
    if constexpr (std::is_same<Tin, float>::value)
        return (n % 4 == 0) && (src.ld() % 4 == 0) && ((reinterpret_cast<uintptr_t>(src.X(item, 4)) & 15) == 0);
    return false;
}

// Pass/fail rule shared by both kernels (thread 0): sig[j] the kept singular
// values (0 = dropped, sig[0] the largest), rho[j] the residual norms, sm the
// smallest Ritz value.  The bound must stay below kCertTol max(sigma_j,
// 1e-2 sigma_1): relative for sigma_j >= 1e-2 sigma_1, and 1e-7 sigma_1
// absolute below that, where FP32 products of the rows (error ~ eps sigma_1)
// leave no relative accuracy to certify.
__device__ __forceinline__ bool cert_pass(const float* sig, const float* rho, int kc, float sm) {
    bool ok = true;
    const float floor_ = 1e-2f * sig[0];
    for (int j = 0; j < kc; ++j) {
        const float sj = sig[j];
        if (!(sj > 0.f)) continue;
        const float r = rho[j], eta = sj - sm;
        const float beta = eta > 0.f ? fminf(r, r * r / eta) : r;
        if (!(beta <= kCertTol * fmaxf(sj, floor_))) ok = false;          // a NaN fails
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Work units of k_check on stacked query matrices, whose rows differ by 30x
// within a batch: a matrix of more than kCheckPartRows rows is cut into up to
// n / kwp parts of whole 32-row tiles, so that the largest query no longer
// runs alone on one SM.  Each part's partial X^T U (n x kwp) goes to the
// item's n x n scratch G (free once the basis is formed; the refinement that
// reuses it runs after the test), and the CTA that finishes an item's last
// part sums the parts in part order and applies the test.  cplan: the
// exclusive prefix of the items' part counts (count + 1 entries), then one
// arrival counter per item, zeroed here.
// ---------------------------------------------------------------------------
constexpr int kCheckPartRows = 512;
template <class Src>
__global__ void __launch_bounds__(1024) k_check_plan(Src src, TcScratch sc, int n, int kw) {
    __shared__ int s_carry, s_warp[32];
    const int count = src.count();
    const int kwp = (kw + 7) / 8 * 8, pmax = max(1, n / kwp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int* pre = sc.cplan;
    int* arrive = sc.cplan + count + 1;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < count; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int v = 0;
        if (i < count) {
            const int rows = src.rows(i);
            v = rows > kCheckPartRows ? min(pmax, (rows + kCheckPartRows - 1) / kCheckPartRows) : 1;
            arrive[i] = 0;
        }
        int x = v;                                    // inclusive scan: warp, then across warps
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
        if (i < count) pre[i] = s_carry + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[count] = s_carry;
}

// ---------------------------------------------------------------------------
// k_check: R = X^T U by column blocks of X of up to 512 (NTW <= 4 16-row tiles
// of R per warp, KT <= 8 column tiles of 8: kw <= 8 KT), each block one sweep
// over the unit's rows; rho_j^2 accumulates over the blocks.  A unit is an
// item, or (stacked query matrices, sc.cplan set) a part of one.
// ---------------------------------------------------------------------------
template <class Src, typename Tin, int NTW, int KT>
__global__ void __launch_bounds__(256, (NTW * KT <= 4) ? 3 : ((NTW * KT <= 8) ? 2 : 1))
    k_check(Src src, TcScratch sc, int n, int kw) {
    extern __shared__ __align__(16) float cks[];
    __shared__ float s_sig[ZS_MAXM];
    __shared__ float s_rho[ZS_MAXM];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int TR = ck_rows(n), ldx = ck_ldx(n), ldb = ck_ldb(kw);
    const int kwp = (kw + 7) / 8 * 8, nkt = kwp / 8, ncp = (n + 31) / 32 * 32;
    const int nmt = (n + 15) / 16;
    const int nst = ck_stages(n, kw);
    const size_t sf = ck_stage_floats(n, kw);
    const int m = sc.m;
    __shared__ int s_item, s_last;
    const bool split = std::is_same<Src, SrcQuery>::value && sc.cplan != nullptr;
    for (;;) {
        // units are handed out one at a time (item sizes differ by 30x in a query batch)
        __syncthreads();                                  // the previous unit's shared data are consumed
        if (tid == 0) s_item = atomicAdd(sc.list + 1, 1);
        __syncthreads();
        int item = s_item, part = 0, nparts = 1;
        if (split) {
            const int u = s_item, count = src.count();
            if (u >= sc.cplan[count]) break;
            int lo = 0, hi = count - 1;                   // the last item whose first unit is <= u
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sc.cplan[mid] <= u) lo = mid; else hi = mid - 1;
            }
            item = lo;
            part = u - sc.cplan[item];
            nparts = sc.cplan[item + 1] - sc.cplan[item];
        } else if (item >= src.count()) {
            break;
        }
        const int rows_all = src.rows(item);
        // this unit's rows [r_lo, rows): whole TR-row tiles per part
        const int prr = nparts > 1 ? ((rows_all + nparts - 1) / nparts + TR - 1) / TR * TR : rows_all;
        const int r_lo = min(rows_all, part * prr);
        const int rows = min(rows_all, r_lo + prr);
        const int kc = src.kcap(item, kw);
        const auto cx = src.ctx(item, sizeof(Tin));
        const float* U = src.u_out(item, kw);
        const float* vt = src.vt_out(item, kw);
        const bool vec = rows_vec16<Src, Tin>(src, item, n);
        const bool raw = rows_raw16<Src, Tin>(src, item, n);
        if (tid < kw) {
            s_sig[tid] = src.sig_out(item, kw)[tid];
            s_rho[tid] = 0.f;
        }
        const int ntl = (rows - r_lo + TR - 1) / TR;
        float* Rpart = split ? sc.G + (size_t)item * n * n + (size_t)part * n * kwp : nullptr;
        // this block of R rows through shared memory, then its share of rho_j^2
        auto rho_block = [&](int i0, int i1) {
            const float* Rs = cks;
            const int ldr = kwp + 1;
            for (int j = warp; j < kw; j += 8) {
                const float sj = s_sig[j];
                float ss = 0.f;
                for (int l = i0 + lane; l < i1; l += 32) {
                    const float d = Rs[(l - i0) * ldr + j] - sj * vt[(size_t)j * n + l];
                    ss = fmaf(d, d, ss);
                }
                ss = warp_sum(ss);
                if (lane == 0) s_rho[j] += ss;
            }
        };
        for (int mt0 = 0; mt0 < nmt; mt0 += 8 * NTW) {
            float acc[NTW][KT][4], acx[NTW][KT][4];
#pragma unroll
            for (int a = 0; a < NTW; ++a)
#pragma unroll
                for (int b = 0; b < KT; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][b][c] = acx[a][b][c] = 0.f;
            auto issue = [&](int t) {
                float* Xs = cks + (size_t)(t % nst) * sf;
                if (raw) {
                    float* rw = cks + (size_t)nst * sf + (size_t)(t % nst) * ck_raw_floats(n);
                    ld_xtile_raw16<Src>(src, cx, r_lo + t * TR, TR, rows, n, ncp,
                                        reinterpret_cast<__nv_bfloat16*>(rw), rw + (size_t)TR * ncp / 2);
                } else {
                    ld_xtile<Src, Tin>(src, cx, r_lo + t * TR, TR, rows, n, ncp, Xs, ldx, vec);
                }
                ld_btile(U, kw, r_lo + t * TR, TR, rows, kw, kwp, Xs + (size_t)TR * ldx, ldb);
                cp_async_commit();
            };
            __syncthreads();                              // the residual step below has read the stages
            issue(0);
            for (int t = 0; t < ntl; ++t) {
                if (nst == 2) {
                    if (t + 1 < ntl) issue(t + 1);
                    else cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                if (raw) {                                // widen the raw bf16 rows
                    const float* rw = cks + (size_t)nst * sf + (size_t)(t % nst) * ck_raw_floats(n);
                    cvt_xtile(reinterpret_cast<const __nv_bfloat16*>(rw), rw + (size_t)TR * ncp / 2, TR, ncp,
                              cks + (size_t)(t % nst) * sf, ldx);
                    __syncthreads();
                }
                const float* Xs = cks + (size_t)(t % nst) * sf;
                const float* Bs = Xs + (size_t)TR * ldx;
#pragma unroll 2
                for (int k0 = 0; k0 < TR; k0 += 8) {
                    uint32_t bh[KT][2], bl[KT][2];
#pragma unroll
                    for (int nt = 0; nt < KT; ++nt) {
                        if (nt >= nkt) break;
                        tf32_split_trunc(Bs[(k0 + t4) * ldb + nt * 8 + g], bh[nt][0], bl[nt][0]);
                        tf32_split_trunc(Bs[(k0 + t4 + 4) * ldb + nt * 8 + g], bh[nt][1], bl[nt][1]);
                    }
#pragma unroll
                    for (int mi = 0; mi < NTW; ++mi) {
                        const int mt = mt0 + warp + 8 * mi;
                        if (mt >= nmt) break;
                        // A = X^T: A[g][t4] = X[k0 + t4][16 mt + g]
                        const float* xa = Xs + (k0 + t4) * ldx + mt * 16 + g;
                        uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
                        tf32_split_trunc(xa[0], ah0, al0);
                        tf32_split_trunc(xa[8], ah1, al1);
                        tf32_split_trunc(xa[4 * ldx], ah2, al2);
                        tf32_split_trunc(xa[4 * ldx + 8], ah3, al3);
#pragma unroll
                        for (int nt = 0; nt < KT; ++nt) {
                            if (nt >= nkt) break;
                            // the cross terms in their own accumulator: two independent chains
                            mma_tf32(acx[mi][nt], al0, al1, al2, al3, bh[nt][0], bh[nt][1]);
                            mma_tf32(acx[mi][nt], ah0, ah1, ah2, ah3, bl[nt][0], bl[nt][1]);
                            mma_tf32(acc[mi][nt], ah0, ah1, ah2, ah3, bh[nt][0], bh[nt][1]);
                        }
                    }
                }
                __syncthreads();
                if (nst == 1 && t + 1 < ntl) issue(t + 1);
            }
            cp_async_wait<0>();
            __syncthreads();
            float* Rs = cks;
            const int ldr = kwp + 1;
            const int i0 = mt0 * 16, i1 = min(n, (mt0 + 8 * NTW) * 16);
#pragma unroll
            for (int mi = 0; mi < NTW; ++mi) {
                const int mt = mt0 + warp + 8 * mi;
                if (mt >= nmt) break;
#pragma unroll
                for (int nt = 0; nt < KT; ++nt) {
                    if (nt >= nkt) break;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = mt * 16 + g + ((e >> 1) ? 8 : 0), j = nt * 8 + 2 * t4 + (e & 1);
                        if (i >= n) continue;
                        if (nparts > 1) Rpart[(size_t)i * kwp + j] = acc[mi][nt][e] + acx[mi][nt][e];
                        else Rs[(i - i0) * ldr + j] = acc[mi][nt][e] + acx[mi][nt][e];
                    }
                }
            }
            __syncthreads();
            if (nparts == 1) rho_block(i0, i1);
        }
        if (nparts > 1) {
            // publish this part; the CTA that brings the item's last part sums
            // all parts in part order and applies the test
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(sc.cplan + src.count() + 1 + item, 1) == nparts - 1;
            __syncthreads();
            if (!s_last) continue;
            __threadfence();
            const float* Ritem = sc.G + (size_t)item * n * n;
            for (int mt0 = 0; mt0 < nmt; mt0 += 8 * NTW) {
                const int i0 = mt0 * 16, i1 = min(n, (mt0 + 8 * NTW) * 16);
                float* Rs = cks;
                const int ldr = kwp + 1;
                __syncthreads();
                for (int e = tid; e < (i1 - i0) * kwp; e += blockDim.x) {
                    const int i = i0 + e / kwp, j = e - (e / kwp) * kwp;
                    float r = 0.f;
                    for (int q = 0; q < nparts; ++q) r += __ldcg(Ritem + (size_t)q * n * kwp + (size_t)i * kwp + j);
                    Rs[(i - i0) * ldr + j] = r;
                }
                __syncthreads();
                rho_block(i0, i1);
            }
        }
        __syncthreads();
        if (tid == 0) {
            for (int j = 0; j < kw; ++j) s_rho[j] = sqrtf(s_rho[j]);
            const float sm = sqrtf(fmaxf(sc.thm[(size_t)item * m + m - 1], 0.f));
            int kt = kc;
            if (sc.kxi) {              // only the pairs the energy rule keeps are tested
                const int ki = xi_rank_of(s_sig, kw, sc.energy[item], sc.xi);
                sc.kxi[item] = ki;
                kt = min(kc, ki);
            }
            if (!cert_pass(s_sig, s_rho, kt, sm)) {
                const int p = atomicAdd(sc.list, 1);
                sc.list[2 + p] = item;
            }
        }
    }
}

// Above the refinement's size limit every listed item counts as not converged.
static __global__ void k_count_listed(const int* list, int* noconv) {
    if (threadIdx.x == 0 && noconv && list[0] > 0) atomicAdd(noconv, list[0]);
}

// ---------------------------------------------------------------------------
// k_refine: NTW 16-row tiles of W (n x kRefineM) per warp (n <= 256 NTW).
// ---------------------------------------------------------------------------
template <class Src, typename Tin, int NTW>
__global__ void __launch_bounds__(kRefineThreads, 1) k_refine(Src src, TcScratch sc, int n, int kw) {
    constexpr int MR = kRefineM, NT = MR / 8, LH = MR + 1;
    extern __shared__ __align__(16) float rfs[];
    __shared__ JacobiScratch<float> js;
    __shared__ float red[32], coef[MR], s_th[MR], s_rho[MR], s_sig[MR], s_sgn[MR];
    __shared__ int perm[MR];
    __shared__ int s_done;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int ldq = rf_ldq(), ldx = ck_ldx(n), ncp = (n + 31) / 32 * 32, n8 = (n + 7) / 8 * 8;
    const int nmt = (n + 15) / 16;
    const int m = sc.m;
    const int kwp = (kw + 7) / 8 * 8, nkt = kwp / 8;
    float* Qs = rfs;                                  // ncp x ldq
    float* Xs = rfs + (size_t)ncp * ldq;              // TR x ldx   (pass)
    float* Ys = Xs + (size_t)kRefineTR * ldx;         // TR x ldq   (pass)
    float* Hs = Xs;                                   // MR x LH    (Rayleigh-Ritz)
    float* Zs = Hs + MR * LH;                         // MR x LH
    const int nlist = sc.list[0];
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const int item = sc.list[2 + li];
        const int rows = src.rows(item), kc = src.kcap(item, kw);
        const auto cx = src.ctx(item, sizeof(Tin));
        const bool vec = rows_vec16<Src, Tin>(src, item, n);
        float* Wg = sc.G + (size_t)item * n * n;      // n x MR (n >= MR on the tensor path)
        float* vt_o = src.vt_out(item, kw);
        __syncthreads();
        // starting basis: the sketch's Q~ (m columns), random signs in the rest
        {
            const float* Qf = sc.Qf + (size_t)item * n * m;
            for (int e = tid; e < ncp * MR; e += nthr) {
                const int l = e / MR, c = e - (e / MR) * MR;
                float v = 0.f;
                if (l < n) v = c < m ? Qf[(size_t)l * m + c] : (((omega_row_bits((uint32_t)l) >> c) & 1) ? 1.f : -1.f);
                Qs[l * ldq + c] = v;
            }
            __syncthreads();
            mgs_orth<float>(Qs, ldq, n, MR, red, coef);
        }
        int pass = 0;
        for (;;) {
            ++pass;
            // ---- one pass over the rows: Y = X Q, W = X^T Y, H = Y^T Y
            float wacc[NTW][NT][4];
            float hacc[2][4];
#pragma unroll
            for (int a = 0; a < NTW; ++a)
#pragma unroll
                for (int b = 0; b < NT; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) wacc[a][b][c] = 0.f;
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) hacc[b][c] = 0.f;
            for (int r0 = 0; r0 < rows; r0 += kRefineTR) {
                ld_xtile<Src, Tin>(src, cx, r0, kRefineTR, rows, n, ncp, Xs, ldx, vec);
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
                // Y tile (TR x MR): warp -> 16-row tile (warp & 1), 8-column tile (warp >> 1)
                {
                    const int mt = warp & 1, nt = warp >> 1;
                    float y[4] = {0.f, 0.f, 0.f, 0.f};
                    const float* xa = Xs + (mt * 16 + g) * ldx + t4;
                    const float* qb = Qs + t4 * ldq + nt * 8 + g;
                    for (int k0 = 0; k0 < n8; k0 += 8) {
                        uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3, bh0, bl0, bh1, bl1;
                        tf32_split_trunc(xa[k0], ah0, al0);
                        tf32_split_trunc(xa[8 * ldx + k0], ah1, al1);
                        tf32_split_trunc(xa[k0 + 4], ah2, al2);
                        tf32_split_trunc(xa[8 * ldx + k0 + 4], ah3, al3);
                        tf32_split(qb[k0 * ldq], bh0, bl0);
                        tf32_split(qb[(k0 + 4) * ldq], bh1, bl1);
                        mma_tf32(y, al0, al1, al2, al3, bh0, bh1);
                        mma_tf32(y, ah0, ah1, ah2, ah3, bl0, bl1);
                        mma_tf32(y, ah0, ah1, ah2, ah3, bh0, bh1);
                    }
                    float* yp = Ys + (mt * 16 + g) * ldq + nt * 8 + 2 * t4;
                    yp[0] = y[0];
                    yp[1] = y[1];
                    yp[8 * ldq] = y[2];
                    yp[8 * ldq + 1] = y[3];
                }
                __syncthreads();
                // W += X^T Y: warp -> 16-row tiles warp, warp + 16 of W, all MR columns
                for (int k0 = 0; k0 < kRefineTR; k0 += 8) {
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        uint32_t bh[NT / 2][2], bl[NT / 2][2];
#pragma unroll
                        for (int u = 0; u < NT / 2; ++u) {
                            const int nt = half * (NT / 2) + u;
                            tf32_split(Ys[(k0 + t4) * ldq + nt * 8 + g], bh[u][0], bl[u][0]);
                            tf32_split(Ys[(k0 + t4 + 4) * ldq + nt * 8 + g], bh[u][1], bl[u][1]);
                        }
#pragma unroll
                        for (int mi = 0; mi < NTW; ++mi) {
                            const int mt = warp + 16 * mi;
                            if (mt >= nmt) break;
                            const float* xa = Xs + (k0 + t4) * ldx + mt * 16 + g;
                            uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
                            tf32_split_trunc(xa[0], ah0, al0);
                            tf32_split_trunc(xa[8], ah1, al1);
                            tf32_split_trunc(xa[4 * ldx], ah2, al2);
                            tf32_split_trunc(xa[4 * ldx + 8], ah3, al3);
#pragma unroll
                            for (int u = 0; u < NT / 2; ++u) {
                                float* c = wacc[mi][half * (NT / 2) + u];
                                mma_tf32(c, al0, al1, al2, al3, bh[u][0], bh[u][1]);
                                mma_tf32(c, ah0, ah1, ah2, ah3, bl[u][0], bl[u][1]);
                                mma_tf32(c, ah0, ah1, ah2, ah3, bh[u][0], bh[u][1]);
                            }
                        }
                    }
                }
                // H += Y^T Y: warp -> 16-row tile (warp & 3), 8-column tiles (warp >> 2) and (warp >> 2) + 4
                {
                    const int mt = warp & 3, nb = warp >> 2;
                    for (int k0 = 0; k0 < kRefineTR; k0 += 8) {
                        const float* ya = Ys + (k0 + t4) * ldq + mt * 16 + g;
                        uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
                        tf32_split(ya[0], ah0, al0);
                        tf32_split(ya[8], ah1, al1);
                        tf32_split(ya[4 * ldq], ah2, al2);
                        tf32_split(ya[4 * ldq + 8], ah3, al3);
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float* yb = Ys + (k0 + t4) * ldq + (nb + 4 * u) * 8 + g;
                            uint32_t bh0, bl0, bh1, bl1;
                            tf32_split(yb[0], bh0, bl0);
                            tf32_split(yb[4 * ldq], bh1, bl1);
                            mma_tf32(hacc[u], al0, al1, al2, al3, bh0, bh1);
                            mma_tf32(hacc[u], ah0, ah1, ah2, ah3, bl0, bl1);
                            mma_tf32(hacc[u], ah0, ah1, ah2, ah3, bh0, bh1);
                        }
                    }
                }
                __syncthreads();                          // Xs, Ys are rewritten by the next tile
            }
            // W to global scratch (n x MR), H to shared memory
#pragma unroll
            for (int mi = 0; mi < NTW; ++mi) {
                const int mt = warp + 16 * mi;
                if (mt >= nmt) break;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = mt * 16 + g + ((e >> 1) ? 8 : 0), j = nt * 8 + 2 * t4 + (e & 1);
                        if (i < n) Wg[(size_t)i * MR + j] = wacc[mi][nt][e];
                    }
            }
            {
                const int mt = warp & 3, nb = warp >> 2;
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = mt * 16 + g + ((e >> 1) ? 8 : 0), j = (nb + 4 * u) * 8 + 2 * t4 + (e & 1);
                        Hs[i * LH + j] = hacc[u][e];
                    }
            }
            __syncthreads();
            for (int e = tid; e < MR * MR; e += nthr) {
                const int i = e / MR, j = e - (e / MR) * MR;
                if (i < j) {
                    const float v = 0.5f * (Hs[i * LH + j] + Hs[j * LH + i]);
                    Hs[i * LH + j] = v;
                    Hs[j * LH + i] = v;
                }
            }
            __syncthreads();
            // ---- Rayleigh-Ritz on span(Q) (Q orthonormal): H = Z Theta Z^T
            // relative convergence test only (floor 1e-14 lambda_1, below the
            // rank tolerance): the small Ritz values keep their relative accuracy
            jacobi_eig<float>(Hs, LH, Zs, LH, MR, js, 40, true, 1e-7f);
            sort_desc<float>(Hs, LH, MR, perm);
            if (tid < MR) s_th[tid] = fmaxf(Hs[perm[tid] * LH + perm[tid]], 0.f);
            __syncthreads();
            // ---- residuals r_j = W z_j - theta_j v_j with v_j = Q z_j (v_j into the V^T output row j)
            for (int j = warp; j < kw; j += kRefineThreads / 32) {
                const int pj = perm[j];
                float ss = 0.f;
                for (int l = lane; l < n; l += 32) {
                    float v = 0.f, wz = 0.f;
                    for (int c = 0; c < MR; ++c) {
                        const float z = Zs[c * LH + pj];
                        v = fmaf(Qs[l * ldq + c], z, v);
                        wz = fmaf(Wg[(size_t)l * MR + c], z, wz);
                    }
                    const float d = wz - s_th[j] * v;
                    ss = fmaf(d, d, ss);
                    vt_o[(size_t)j * n + l] = v;
                }
                ss = warp_sum(ss);
                if (lane == 0) s_rho[j] = sqrtf(ss) / fmaxf(sqrtf(s_th[j]), 1e-30f);
            }
            const float s0 = sqrtf(s_th[0]);
            if (tid < kw) {
                float sv = sqrtf(s_th[tid]);
                if (!(tid < kc && sv > kRankTolF32 * s0)) sv = 0.f;
                s_sig[tid] = sv;
            }
            __syncthreads();
            if (tid == 0) {
                int kt = kc;
                if (sc.kxi) {          // the energy rule's rank from the refined values
                    const int ki = xi_rank_of(s_sig, kw, sc.energy[item], sc.xi);
                    sc.kxi[item] = ki;
                    kt = min(kc, ki);
                }
                const bool ok = cert_pass(s_sig, s_rho, kt, sqrtf(s_th[MR - 1]));
                s_done = ok ? 1 : (pass >= kRefineMaxPasses ? 2 : 0);
            }
            __syncthreads();
            if (s_done) break;
            // ---- next basis: Q = orth(W)
            for (int e = tid; e < n * MR; e += nthr) {
                const int l = e / MR, c = e - (e / MR) * MR;
                Qs[l * ldq + c] = Wg[e];
            }
            __syncthreads();
            mgs_orth<float>(Qs, ldq, n, MR, red, coef);
        }
        if (tid == 0 && s_done == 2 && sc.noconv) atomicAdd(sc.noconv, 1);
        if (tid == 0 && sc.refined) atomicAdd(sc.refined, 1);
        // ---- outputs from the last iterate: signs (largest-|.| entry of v_j
        // positive, lowest index on ties), V^T, sigma and the forms that go with them
        for (int j = warp; j < kw; j += kRefineThreads / 32) {
            const float* vo = vt_o + (size_t)j * n;
            float best = -1.f;
            int bi = 0x7fffffff;
            for (int l = lane; l < n; l += 32) {
                const float av = fabsf(vo[l]);
                if (av > best || (av == best && l < bi)) { best = av; bi = l; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) s_sgn[j] = (bi < n && vo[bi] < 0.f) ? -1.f : 1.f;
        }
        __syncthreads();
        float* w_o = src.w_out(item, kw);
        for (int e = tid; e < kw * n; e += nthr) {
            const int j = e / n;
            const float vv = s_sig[j] > 0.f ? s_sgn[j] * vt_o[e] : 0.f;
            vt_o[e] = vv;
            if (w_o) w_o[e] = s_sig[j] * vv;
        }
        if (tid < kw) src.sig_out(item, kw)[tid] = s_sig[tid];
        __syncthreads();
        if constexpr (std::is_same<Src, SrcQuery>::value) {
            const QPlan& P = src.a.plans[item];
            const int kout = src.a.kout;
            for (int c = tid; c < kout; c += nthr) ((float*)P.S_out)[c] = c < kw ? s_sig[c] : 0.f;
            if (tid == 0 && P.rank) {
                int r = 0;
                for (int c = 0; c < kw; ++c) r += s_sig[c] > 0.f;
                *P.rank = r;
            }
            for (int e = tid; e < n * kout; e += nthr) {
                const int l = e / kout, c = e - (e / kout) * kout;
                ((float*)P.V_out)[(size_t)l * P.ldv + c] = c < kw ? vt_o[(size_t)c * n + l] : 0.f;
            }
        }
        // ---- U = X V Sigma^-1 (signs folded in): one more pass over the rows
        for (int e = tid; e < ncp * kwp; e += nthr) {
            const int l = e / kwp, c = e - (e / kwp) * kwp;
            Qs[l * ldq + c] = (l < n && c < kw && s_sig[c] > 0.f) ? vt_o[(size_t)c * n + l] / s_sig[c] : 0.f;
        }
        float* u_o = src.u_out(item, kw);
        for (int r0 = 0; r0 < rows; r0 += kRefineTR) {
            __syncthreads();
            ld_xtile<Src, Tin>(src, cx, r0, kRefineTR, rows, n, ncp, Xs, ldx, vec);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            const int mt = warp & 1, nt = warp >> 1;
            if (nt < nkt) {
                float y[4] = {0.f, 0.f, 0.f, 0.f};
                const float* xa = Xs + (mt * 16 + g) * ldx + t4;
                const float* qb = Qs + t4 * ldq + nt * 8 + g;
                for (int k0 = 0; k0 < n8; k0 += 8) {
                    uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3, bh0, bl0, bh1, bl1;
                    tf32_split_trunc(xa[k0], ah0, al0);
                    tf32_split_trunc(xa[8 * ldx + k0], ah1, al1);
                    tf32_split_trunc(xa[k0 + 4], ah2, al2);
                    tf32_split_trunc(xa[8 * ldx + k0 + 4], ah3, al3);
                    tf32_split(qb[k0 * ldq], bh0, bl0);
                    tf32_split(qb[(k0 + 4) * ldq], bh1, bl1);
                    mma_tf32(y, al0, al1, al2, al3, bh0, bh1);
                    mma_tf32(y, ah0, ah1, ah2, ah3, bl0, bl1);
                    mma_tf32(y, ah0, ah1, ah2, ah3, bh0, bh1);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = r0 + mt * 16 + g + ((e >> 1) ? 8 : 0), c = nt * 8 + 2 * t4 + (e & 1);
                    if (r < rows && c < kw) u_o[(size_t)r * kw + c] = y[e];
                }
            }
        }
    }
}

}  // namespace zs
