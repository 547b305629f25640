// zs_rowappend.cu - Algorithm 1 as printed: every arriving row updates its
// block's rank-k SVD by Eq. 2-3 and the result is truncated back to rank k
// (Section 3.2, Section 2.2; the cost of Theorem 1, O(k^2 (rows + n)) per
// row).  Used for every block of a store created with ZS_FLAG_ROW_APPEND.
//
// One CTA per block folds the block's new rows in order.  The state of a
// block is K = diag(sigma) V^T (k rows of n, rows orthogonal) and U (rows x k).
// For each arriving row a:
//   1. projection on the current right basis B = diag(1/sigma) K (the rows of
//      V^T): p = B a, a' = a - B^T p, done twice (classical Gram-Schmidt with
//      one reorthogonalisation), r = |a'|, q = a' / r.  Then the stacked
//      matrix of Eq. 2 is [K; a] = M [B; q^T] with the (k+1) x (k+1) matrix
//      M = [diag(sigma) 0; p^T r];
//   2. one-sided Jacobi (Hestenes) on M's rows: rotations J with M = J M' and
//      the rows of M' orthogonal; P sorts them by norm.  As [B; q^T] has
//      orthonormal rows, [K; a] = (J P) (P^T M' [B; q^T]) is its SVD;
//   3. truncation to rank k: K <- the k longest rows of M' [B; q^T], and
//      U <- blockdiag(U, 1) (J P)(:, 0:k) (Eq. 3).
// U is updated lazily: U = [U_old C; U_pend], with the k x k product C of the
// updates since the last flush and up to kRaPend recent rows U_pend in shared
// memory; U_old in global memory is multiplied by C once every kRaPend rows
// and at the end of the call.
// At the end sigma_c = |K_c|, V_c^T = K_c / sigma_c, with the sign rule R6 on
// each pair.  Everything is in the store's factor type (FP32 or FP64).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "zs_internal.h"
#include "zs_linalg.cuh"

namespace zs {

template <typename T>
__device__ __forceinline__ T ra_load(const void* p, int64_t i, int kind) {
    if (kind == IN_F64) return (T)((const double*)p)[i];
    if (kind == IN_F32) return (T)((const float*)p)[i];
    return (T)__bfloat162float(((const __nv_bfloat16*)p)[i]);
}

// Convergence of the one-sided Jacobi: a pair counts as orthogonal once
// |x.y| <= 2 sqrt(n) eps |x||y|, the rounding level of the computed dot
// product itself (a smaller threshold is never met and every sweep runs).
template <typename T>
__device__ __forceinline__ T ra_eps();
template <> __device__ __forceinline__ float ra_eps<float>() { return 1.1920929e-7f; }
template <> __device__ __forceinline__ double ra_eps<double>() { return 2.220446049250313e-16; }

constexpr int kRaPend = 64;                          // U rows kept in shared memory between flushes

// Shared-memory layout (offsets in elements of the factor type; the integer
// arrays - sort permutation and pair schedule - follow).
struct RaLayout {
    size_t K0, K1, arow, M, J, W, Mpp, C, C2, P, P2, sg, pv, cf, nrm, sgn, end;
};
__host__ __device__ __forceinline__ RaLayout ra_layout(int n, int k) {
    const size_t m = (size_t)k + 1, kk = (size_t)k, F = kRaPend;
    RaLayout L;
    size_t o = 0;
    L.K0 = o;   o += kk * n;
    L.K1 = o;   o += kk * n;
    L.arow = o; o += (size_t)n;
    L.M = o;    o += m * m;
    L.J = o;    o += m * m;
    L.W = o;    o += m * kk;
    L.Mpp = o;  o += kk * m;
    L.C = o;    o += kk * kk;
    L.C2 = o;   o += kk * kk;
    L.P = o;    o += F * kk;
    L.P2 = o;   o += F * kk;
    L.sg = o;   o += 66;
    L.pv = o;   o += 66;
    L.cf = o;   o += 66;
    L.nrm = o;  o += 66;
    L.sgn = o;  o += 66;
    L.end = o + (o & 1);
    return L;
}
__host__ __device__ __forceinline__ size_t row_append_smem(int n, int k, size_t tsz) {
    return tsz * ra_layout(n, k).end + 4 * 66 + 4 * 66 * 33 + 64;
}

// The Jacobi rounds give each pair of M's rows g lanes - a whole warp, or 16
// lanes when ceil((k+1)/2) warps would pass 1024 threads (k = 63, 64): all
// pairs of a round run at once on jt threads (whole warps).  A round is one
// dependent chain (dot products, their reduction, the rotation, the update),
// so fewer lanes per pair (more elements per lane) measured slower.  The
// rest of the kernel runs on max(256, jt) threads.
__host__ __device__ __forceinline__ int ra_group(int k) {
    const int m = k + 1, npair = (m + (m & 1)) / 2;
    return 32 * npair <= 1024 ? 32 : 16;
}
__host__ __device__ __forceinline__ int ra_jacobi_threads(int k) {
    const int m = k + 1, npair = (m + (m & 1)) / 2;
    return (npair * ra_group(k) + 31) / 32 * 32;
}
__host__ __device__ __forceinline__ int row_append_threads(int k) {
    const int t = ra_jacobi_threads(k);
    return t < 256 ? 256 : t;
}

// The rotation that makes rows x, y orthogonal (Hestenes): with
// zeta = (|y|^2 - |x|^2) / (2 x.y), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t, tau = s / (1 + c).  In Rutishauser's form
// the effective cosine is 1 - s tau, so an error e in c changes c^2 + s^2 by
// O(t^2 e) only: FP32 takes the hardware reciprocal and reciprocal square
// root here (a few ulp), FP64 the correctly rounded operations.
__device__ __forceinline__ void rotation(float app, float aqq, float apq, float& s, float& tau) {
    const float zeta = (aqq - app) * __frcp_rn(2.f * apq);
    const float t = copysignf(__frcp_rn(fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))), zeta);
    const float c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
    tau = s * __frcp_rn(1.f + c);
}
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double& s, double& tau) {
    const double zeta = (aqq - app) / (2.0 * apq);
    const double t = copysign(1.0 / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0))), zeta);
    const double c = 1.0 / sqrt(fma(t, t, 1.0));
    s = c * t;
    tau = s / (1.0 + c);
}

template <typename T>
__device__ __forceinline__ void warp_sum2(T& a, T& b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
}

// p_i = K_i . x / sigma_i and cf_i = K_i . x / sigma_i^2 for every row of K
// (one warp per row); with norms, also sigma_i = |K_i|.
template <typename T>
__device__ __forceinline__ void ra_project(const T* K, const T* x, int k, int n, bool norms, T* sg, T* pv, T* cf,
                                           int warp, int lane, int nw) {
    for (int p = warp; p < k; p += nw) {
        T ss = 0, pa = 0;
        for (int l = lane; l < n; l += 32) {
            const T v = K[(size_t)p * n + l];
            ss += v * v;
            pa += v * x[l];
        }
        warp_sum2(ss, pa);
        if (lane == 0) {
            if (norms) sg[p] = zsqrt(ss);
            const T s2 = sg[p] * sg[p];
            const bool live = sg[p] > T(0);
            pv[p] = live ? pa / sg[p] : T(0);
            cf[p] = live ? pa / s2 : T(0);
        }
    }
}

// U rows [0, r_old) <- U C diag(g) and rows [r_old, r_old + r_p) <- P diag(g)
// (g = 1 when sg == nullptr): one warp per 4 rows, the rows' entries
// broadcast by shuffles.
template <typename T>
__device__ void ra_flush(T* U, int k, int r_old, const T* C, const T* P, int r_p, const T* g, int warp, int lane,
                         int nw, int tid, int nt) {
    const T g0 = (g && lane < k) ? g[lane] : T(1);
    const T g1 = (g && lane + 32 < k) ? g[lane + 32] : T(1);
    for (int r = 4 * warp; r < r_old; r += 4 * nw) {
        T u0[4], u1[4], o0[4], o1[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const bool in = r + h < r_old;
            const T* ur = U + (size_t)(r + h) * k;
            u0[h] = (in && lane < k) ? ur[lane] : T(0);
            u1[h] = (in && lane + 32 < k) ? ur[lane + 32] : T(0);
            o0[h] = T(0);
            o1[h] = T(0);
        }
        for (int l = 0; l < k; ++l) {
            const T c0 = lane < k ? C[(size_t)l * k + lane] : T(0);
            const T c1 = lane + 32 < k ? C[(size_t)l * k + lane + 32] : T(0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const T ul = __shfl_sync(0xffffffffu, l < 32 ? u0[h] : u1[h], l & 31);
                o0[h] += ul * c0;
                o1[h] += ul * c1;
            }
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            if (r + h >= r_old) break;
            T* ur = U + (size_t)(r + h) * k;
            if (lane < k) ur[lane] = o0[h] * g0;
            if (lane + 32 < k) ur[lane + 32] = o1[h] * g1;
        }
    }
    for (int e = tid; e < r_p * k; e += nt) {
        const int c = e % k;
        U[(size_t)r_old * k + e] = P[e] * (g ? g[c] : T(1));
    }
}

// One-sided Jacobi on the rows of M (m <= MR <= 32) by one warp in
// registers: lane i holds row i of M and column i of J; in each round a lane
// fetches its partner's row and column by shuffles, both lanes of a pair form
// the same dot products (same values, same order) and so the same rotation,
// and each updates its own row and column.  No barrier: rounds are ordered
// by the warp itself.  prt[r * 32 + i] is lane i's partner in round r (i
// itself, or an index >= m, when it has none).
template <typename T, int MR>
__device__ void ra_jacobi_warp(T* M, T* J, int m, int mm, const int* prt, T tol2, int lane) {
    T x[MR], jc[MR];
#pragma unroll
    for (int c = 0; c < MR; ++c) {
        x[c] = (lane < m && c < m) ? M[lane * m + c] : T(0);
        jc[c] = (lane < m && c < m) ? J[c * m + lane] : T(0);
    }
    for (int sweep = 0; sweep < 40; ++sweep) {
        bool any = false;
        for (int r = 0; r < mm - 1; ++r) {
            const int j = prt[r * 32 + lane];
            const int js = j < 32 ? j : lane;                 // shuffle source (no partner: itself)
            T y[MR];
            T app = 0, aqq = 0, apq = 0;
#pragma unroll
            for (int c = 0; c < MR; ++c) {
                y[c] = __shfl_sync(0xffffffffu, x[c], js);
                app += x[c] * x[c];
                aqq += y[c] * y[c];
                apq += x[c] * y[c];
            }
            const bool isp = lane < j;
            const T a_pp = isp ? app : aqq, a_qq = isp ? aqq : app;
            T s = 0, tau = 0;
            if (lane < m && j < m && j != lane && apq != T(0) && apq * apq > tol2 * (a_pp * a_qq)) {
                rotation(a_pp, a_qq, apq, s, tau);
                any = true;
            }
            // Rutishauser's form: p' = p - s (q + tau p), q' = q + s (p - tau q),
            // i.e. own' = own + sg (other + rho own)
            const T sg = isp ? -s : s, rho = isp ? tau : -tau;
#pragma unroll
            for (int c = 0; c < MR; ++c) {
                const T yj = __shfl_sync(0xffffffffu, jc[c], js);
                x[c] += sg * (y[c] + rho * x[c]);
                jc[c] += sg * (yj + rho * jc[c]);
            }
        }
        if (!__any_sync(0xffffffffu, any)) break;
    }
    if (lane < m) {
#pragma unroll
        for (int c = 0; c < MR; ++c) {
            if (c < m) {
                M[lane * m + c] = x[c];
                J[c * m + lane] = jc[c];
            }
        }
    }
}

template <typename T, int MR>
__global__ void __launch_bounds__(MR > 0 ? 256 : 1024) k_row_append(RowAppendArgs a) {
    extern __shared__ __align__(16) unsigned char ras[];
    const int j = blockIdx.x;
    if (j >= a.nblk) return;
    const int n = a.n, k = a.k, b = a.b, m = k + 1;
    const int mm = m + (m & 1), npair = mm / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x, nw = nt >> 5;
    const RaLayout L = ra_layout(n, k);
    T* sm = (T*)ras;
    T* K = sm + L.K0;
    T* Kn = sm + L.K1;
    T* arow = sm + L.arow;
    T* M = sm + L.M;
    T* J = sm + L.J;
    T* W = sm + L.W;
    T* Mpp = sm + L.Mpp;
    T* C = sm + L.C;
    T* C2 = sm + L.C2;
    T* P = sm + L.P;
    T* P2 = sm + L.P2;
    T* sg = sm + L.sg;
    T* pv = sm + L.pv;
    T* cf = sm + L.cf;
    T* nrm = sm + L.nrm;
    T* sgn = sm + L.sgn;
    int* perm = (int*)(sm + L.end);
    int* pairs = perm + 66;                          // round-robin schedule, (mm - 1) x npair
    __shared__ T s_r;
    const int64_t slot = (int64_t)a.slot0 + j;
    T* U = (T*)a.U + slot * b * k;
    T* sig = (T*)a.sig + slot * k;
    T* Vt = (T*)a.vt + slot * k * n;
    // this block's new rows: block 0 starts at row r0 of its block
    const int r0 = j == 0 ? a.r0 : 0;
    const int64_t first = j == 0 ? 0 : (int64_t)b * j - a.r0;
    const int nr = (int)min((int64_t)(b - r0), a.rows_total - first);
    // a pair of M's rows counts as orthogonal once |x.y| <= 2 sqrt(k+1) eps |x||y|,
    // the rounding level of the computed dot product itself (a smaller
    // threshold is never met and every sweep runs)
    const T tol = T(2) * zsqrt(T(m)) * ra_eps<T>();
    const T tol2 = tol * tol;
    const int g = ra_group(k), jt = ra_jacobi_threads(k);
    if constexpr (MR > 0) {
        // each lane's partner per round (itself where it has none)
        for (int e = tid; e < (mm - 1) * 32; e += nt) pairs[e] = e & 31;
        __syncthreads();
        for (int e = tid; e < (mm - 1) * npair; e += nt) {
            int p, q;
            const int r = e / npair;
            rr_pair(mm, r, e % npair, p, q);
            pairs[r * 32 + p] = q;
            if (q < 32) pairs[r * 32 + q] = p;
        }
    } else {
        for (int e = tid; e < (mm - 1) * npair; e += nt) {
            int p, q;
            rr_pair(mm, e / npair, e % npair, p, q);
            pairs[e] = p | (q << 16);
        }
    }
    // the state: K = diag(sigma) V^T of the rows so far (empty for a new block)
    for (int e = tid; e < k * n; e += nt) K[e] = r0 > 0 ? sig[e / n] * Vt[e] : T(0);
    for (int e = tid; e < k * k; e += nt) C[e] = (e / k == e % k) ? T(1) : T(0);
    if (r0 == 0)
        for (int64_t e = tid; e < (int64_t)b * k; e += nt) U[e] = T(0);
    int r_old = r0, r_p = 0;
    __syncthreads();
    for (int i = 0; i < nr; ++i) {
        for (int c = tid; c < n; c += nt) arow[c] = ra_load<T>(a.A, (first + i) * a.lda + c, a.in_kind);
        __syncthreads();
        // ---- 1. p = B a, a' = a - B^T p, twice; r = |a'|, q = a' / r
        ra_project(K, arow, k, n, true, sg, pv, cf, warp, lane, nw);
        __syncthreads();
        for (int l = tid; l < n; l += nt) {
            T x = arow[l];
            for (int c = 0; c < k; ++c) x -= cf[c] * K[(size_t)c * n + l];
            arow[l] = x;
        }
        __syncthreads();
        ra_project(K, arow, k, n, false, sg, nrm, cf, warp, lane, nw);
        __syncthreads();
        for (int l = tid; l < n; l += nt) {
            T x = arow[l];
            for (int c = 0; c < k; ++c) x -= cf[c] * K[(size_t)c * n + l];
            arow[l] = x;
        }
        for (int c = tid; c < k; c += nt) pv[c] += nrm[c];
        __syncthreads();
        if (warp == 0) {
            T ss = 0, dummy = 0;
            for (int l = lane; l < n; l += 32) ss += arow[l] * arow[l];
            warp_sum2(ss, dummy);
            if (lane == 0) s_r = zsqrt(ss);
        }
        __syncthreads();
        const T r = s_r;
        const T rinv = r > T(0) ? T(1) / r : T(0);
        for (int l = tid; l < n; l += nt) arow[l] *= rinv;
        // ---- 2. M = [diag(sigma) 0; p^T r], J = I; one-sided Jacobi on M's rows
        for (int e = tid; e < m * m; e += nt) {
            const int row = e / m, col = e - row * m;
            M[e] = row < k ? (row == col ? sg[row] : T(0)) : (col < k ? pv[col] : r);
            J[e] = row == col ? T(1) : T(0);
        }
        __syncthreads();
        if constexpr (MR > 0) {
            // m <= 32: one warp in registers (the other warps wait at the barrier)
            if (warp == 0) ra_jacobi_warp<T, MR>(M, J, m, mm, pairs, tol2, lane);
        } else if (tid < jt) {
            // g lanes per pair, all pairs of a round at once; only the first jt
            // threads (whole warps) take part and synchronise on barrier 1
            const int pi = tid / g, sl = tid - pi * g;
            for (int sweep = 0; sweep < 40; ++sweep) {
                int any = 0;
                for (int rd = 0; rd < mm - 1; ++rd) {
                    int p = 0, q = m;
                    if (pi < npair) {
                        const int pq = pairs[rd * npair + pi];
                        p = pq & 0xffff;
                        q = pq >> 16;
                    }
                    const bool real = q < m;
                    T* xp = M + (size_t)p * m;
                    T* yq = M + (size_t)(real ? q : p) * m;
                    T app = 0, aqq = 0, apq = 0;
                    if (real)
                        for (int l = sl; l < m; l += g) {
                            const T x = xp[l], y = yq[l];
                            app += x * x;
                            aqq += y * y;
                            apq += x * y;
                        }
                    for (int o = g >> 1; o > 0; o >>= 1) {
                        app += __shfl_xor_sync(0xffffffffu, app, o);
                        aqq += __shfl_xor_sync(0xffffffffu, aqq, o);
                        apq += __shfl_xor_sync(0xffffffffu, apq, o);
                    }
                    if (real && apq != T(0) && apq * apq > tol2 * (app * aqq)) {
                        T s, tau;
                        rotation(app, aqq, apq, s, tau);
                        any = 1;
                        // Rutishauser's form of the rotation, x' = x - s (y + tau x),
                        // y' = y + s (x - tau y): c = 1 - s tau is never rounded on
                        // its own, so small rotations do not add the t^2 of energy
                        // per step that c rounded to 1 would
                        for (int l = sl; l < m; l += g) {
                            const T x = xp[l], y = yq[l];
                            xp[l] = x - s * (y + tau * x);
                            yq[l] = y + s * (x - tau * y);
                            const T u = J[(size_t)l * m + p], v = J[(size_t)l * m + q];
                            J[(size_t)l * m + p] = u - s * (v + tau * u);
                            J[(size_t)l * m + q] = v + s * (u - tau * v);
                        }
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(jt) : "memory");
                }
                int more;
                asm volatile(
                    "{\n\t.reg .pred pa, pr;\n\t"
                    "setp.ne.s32 pa, %1, 0;\n\t"
                    "bar.red.or.pred pr, 1, %2, pa;\n\t"
                    "selp.s32 %0, 1, 0, pr;\n\t}"
                    : "=r"(more)
                    : "r"(any), "r"(jt)
                    : "memory");
                if (!more) break;
            }
        }
        __syncthreads();
        // ---- the rows' norms and their order (descending, lower index on ties)
        for (int p = tid; p < m; p += nt) {
            T ss = 0;
            for (int l = 0; l < m; ++l) ss += M[(size_t)p * m + l] * M[(size_t)p * m + l];
            nrm[p] = ss;
        }
        __syncthreads();
        for (int p = tid; p < m; p += nt) {
            int rk = 0;
            for (int q = 0; q < m; ++q) rk += (nrm[q] > nrm[p]) || (nrm[q] == nrm[p] && q < p);
            perm[rk] = p;
        }
        __syncthreads();
        // ---- 3. W = (J P)(:, 0:k); Mpp = the kept rows of M' over [K; q] (the
        // 1/sigma of B folded in)
        for (int e = tid; e < m * k; e += nt) {
            const int l = e / k, c = e - l * k;
            W[e] = J[(size_t)l * m + perm[c]];
        }
        for (int e = tid; e < k * m; e += nt) {
            const int c = e / m, l = e - c * m;
            const T v = M[(size_t)perm[c] * m + l];
            Mpp[e] = l == k ? v : (sg[l] > T(0) ? v / sg[l] : T(0));
        }
        __syncthreads();
        // K <- Mpp [K; q^T]
        for (int c = 0; c < k; ++c) {
            const T* mr = Mpp + (size_t)c * m;
            for (int l = tid; l < n; l += nt) {
                T x = mr[k] * arow[l];
                for (int jj = 0; jj < k; ++jj) x += mr[jj] * K[(size_t)jj * n + l];
                Kn[(size_t)c * n + l] = x;
            }
        }
        // U = [U_old C; P]: C <- C W_top, P <- [P W_top; W(k, :)]
        for (int e = tid; e < k * k + (r_p + 1) * k; e += nt) {
            if (e < k * k) {
                const int row = e / k, c = e - row * k;
                T x = 0;
                for (int l = 0; l < k; ++l) x += C[(size_t)row * k + l] * W[(size_t)l * k + c];
                C2[e] = x;
            } else {
                const int f = e - k * k, row = f / k, c = f - row * k;
                T x = 0;
                if (row < r_p)
                    for (int l = 0; l < k; ++l) x += P[(size_t)row * k + l] * W[(size_t)l * k + c];
                else
                    x = W[(size_t)k * k + c];
                P2[f] = x;
            }
        }
        __syncthreads();
        T* t = K;
        K = Kn;
        Kn = t;
        t = C;
        C = C2;
        C2 = t;
        t = P;
        P = P2;
        P2 = t;
        ++r_p;
        if (r_p == kRaPend) {
            ra_flush<T>(U, k, r_old, C, P, r_p, nullptr, warp, lane, nw, tid, nt);
            r_old += r_p;
            r_p = 0;
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) C[e] = (e / k == e % k) ? T(1) : T(0);
            __syncthreads();
        }
    }
    // ---- outputs: sigma, V^T, Sigma V^T, with R5 (zero below the rank
    // tolerance) and R6 (largest-|.| entry of v_c positive, U flipped with it)
    for (int c = warp; c < k; c += nw) {
        T ss = 0, dummy = 0;
        for (int l = lane; l < n; l += 32) ss += K[(size_t)c * n + l] * K[(size_t)c * n + l];
        warp_sum2(ss, dummy);
        if (lane == 0) nrm[c] = zsqrt(ss);
    }
    __syncthreads();
    const T tolr = sizeof(T) == 8 ? T(kRankTolF64) : T(kRankTolF32);
    for (int c = warp; c < k; c += nw) {
        const T sv = nrm[c];
        const bool live = sv > tolr * nrm[0] && sv > T(0);
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int l = lane; l < n; l += 32) {
            const T v = zabs(K[(size_t)c * n + l]);
            if (v > best || (v == best && l < bi)) { best = v; bi = l; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const T sg_ = (bi < n && K[(size_t)c * n + bi] < T(0)) ? T(-1) : T(1);
        if (lane == 0) {
            sig[c] = live ? sv : T(0);
            sgn[c] = live ? sg_ : T(0);              // the column's factor for U
        }
        for (int l = lane; l < n; l += 32) {
            const T v = live ? sg_ * K[(size_t)c * n + l] / sv : T(0);
            Vt[(size_t)c * n + l] = v;
            if (a.w) ((T*)a.w)[slot * k * n + (size_t)c * n + l] = live ? sv * v : T(0);
        }
    }
    __syncthreads();
    ra_flush<T>(U, k, r_old, C, P, r_p, sgn, warp, lane, nw, tid, nt);
}

size_t row_append_smem_bytes(int n, int k, bool fp64) { return row_append_smem(n, k, fp64 ? 8 : 4); }

// FP32 with m = k + 1 <= 32: the register Jacobi (MR = m rounded up to 8),
// 256 threads (measured 54 -> 40 us per row at n = 256, k = 16); larger k, and
// FP64, whose one-warp chains wait on the SM's narrow FP64 pipe (151 -> 279 us
// per row at k = 8): the block-wide Jacobi
template <typename T, int MR>
static cudaError_t row_append_go(const RowAppendArgs& a, size_t sm, cudaStream_t st) {
    cudaError_t e;
    if (sm > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_row_append<T, MR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
        return e;
    k_row_append<T, MR><<<a.nblk, MR > 0 ? 256 : row_append_threads(a.k), sm, st>>>(a);
    return cudaSuccess;
}
template <typename T>
static cudaError_t row_append_dispatch(const RowAppendArgs& a, size_t sm, cudaStream_t st) {
    const int m = a.k + 1;
    if constexpr (sizeof(T) == 8) {
        return row_append_go<T, 0>(a, sm, st);
    } else {
        if (m <= 8) return row_append_go<T, 8>(a, sm, st);
        if (m <= 16) return row_append_go<T, 16>(a, sm, st);
        if (m <= 24) return row_append_go<T, 24>(a, sm, st);
        if (m <= 32) return row_append_go<T, 32>(a, sm, st);
        return row_append_go<T, 0>(a, sm, st);
    }
}

cudaError_t launch_row_append(const RowAppendArgs& a, bool fp64, cudaStream_t st) {
    if (a.nblk < 1) return cudaSuccess;
    const size_t sm = row_append_smem(a.n, a.k, fp64 ? 8 : 4);
    cudaError_t e = fp64 ? row_append_dispatch<double>(a, sm, st) : row_append_dispatch<float>(a, sm, st);
    if (e != cudaSuccess) return e;
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace zs
