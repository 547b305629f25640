// zs_rowappend.cu - Algorithm 1 as printed: every arriving row updates its
// block's rank-k SVD by Eq. 2-3 and the result is truncated back to rank k
// (Section 3.2, Section 2.2; the cost of Theorem 1, O(k^2 (rows + n)) per
// row).  Used for every block of a store created with ZS_FLAG_ROW_APPEND.
//
// One CTA per block folds the block's new rows in order.  The state of a
// block is its stored factors: K = diag(sigma) V^T (k rows of n) and U
// (rows x k).  For each arriving row a:
//   1. K <- [K; a]  ((k+1) x n, the stacked matrix of Eq. 2);
//   2. one-sided Jacobi on K's rows: rotations J make the rows orthogonal,
//      K = J K', so that K = (J P) (P^T K') is its SVD once P sorts the rows
//      of K' by norm (Hestenes' method on K^T);
//   3. U <- blockdiag(U, 1) J P, keeping the first k columns (Eq. 3), and
//      K <- the k longest rows of K' (truncation to rank k).
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

// Shared memory: two K buffers ((k+1) x n each), J ((k+1) x (k+1)), the
// pairs' rotations, norms and the sort permutation.
__host__ __device__ __forceinline__ size_t row_append_smem(int n, int k, size_t tsz) {
    const size_t m = (size_t)k + 1;
    return tsz * (2 * m * n + m * m + 4 * 66) + 4 * 66 + 64;
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_append(RowAppendArgs a) {
    extern __shared__ __align__(16) unsigned char ras[];
    const int j = blockIdx.x;
    if (j >= a.nblk) return;
    const int n = a.n, k = a.k, b = a.b, m = k + 1;
    const int mm = m + (m & 1), npair = mm / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    T* K0 = (T*)ras;
    T* K1 = K0 + (size_t)m * n;
    T* J = K1 + (size_t)m * n;
    T* rot = J + (size_t)m * m;                      // c, s per pair (2 * 33)
    T* nrm = rot + 2 * 66;                           // row norms^2 (m)
    int* perm = (int*)(nrm + 2 * 66);
    __shared__ int s_flag;
    const int64_t slot = (int64_t)a.slot0 + j;
    T* U = (T*)a.U + slot * b * k;
    T* sig = (T*)a.sig + slot * k;
    T* Vt = (T*)a.vt + slot * k * n;
    // this block's new rows: block 0 starts at row r0 of its block
    const int r0 = j == 0 ? a.r0 : 0;
    const T tol = T(2) * zsqrt(T(n)) * ra_eps<T>();
    const int64_t first = j == 0 ? 0 : (int64_t)b * j - a.r0;
    const int nr = (int)min((int64_t)(b - r0), a.rows_total - first);
    T* K = K0;
    T* Kn = K1;
    // the state: K = diag(sigma) V^T of the rows so far (empty for a new block)
    for (int e = tid; e < k * n; e += blockDim.x) {
        const int c = e / n;
        K[e] = r0 > 0 ? sig[c] * Vt[e] : T(0);
    }
    if (r0 == 0)
        for (int64_t e = tid; e < (int64_t)b * k; e += blockDim.x) U[e] = T(0);
    __syncthreads();
    for (int i = 0; i < nr; ++i) {
        const int rt = r0 + i;                       // the new row's index in the block
        for (int c = tid; c < n; c += blockDim.x) K[(size_t)k * n + c] = ra_load<T>(a.A, (first + i) * a.lda + c, a.in_kind);
        for (int e = tid; e < m * m; e += blockDim.x) J[e] = (e / m == e % m) ? T(1) : T(0);
        __syncthreads();
        // ---- one-sided Jacobi on K's rows (round-robin pairs, one warp each)
        for (int sweep = 0; sweep < 40; ++sweep) {
            if (tid == 0) s_flag = 0;
            __syncthreads();
            for (int r = 0; r < mm - 1; ++r) {
                for (int pi = warp; pi < npair; pi += nw) {
                    int p, q;
                    rr_pair(mm, r, pi, p, q);
                    T s = T(0);
                    if (q < m) {
                        T app = 0, aqq = 0, apq = 0;
                        for (int l = lane; l < n; l += 32) {
                            const T x = K[(size_t)p * n + l], y = K[(size_t)q * n + l];
                            app += x * x;
                            aqq += y * y;
                            apq += x * y;
                        }
                        app = warp_sum(app);
                        aqq = warp_sum(aqq);
                        apq = warp_sum(apq);
                        T tau = T(0);
                        if (apq != T(0) && zabs(apq) > tol * zsqrt(app * aqq)) {
                            const T zeta = (aqq - app) / (T(2) * apq);
                            const T t = (zeta >= T(0) ? T(1) : T(-1)) / (zabs(zeta) + zsqrt(T(1) + zeta * zeta));
                            const T c = T(1) / zsqrt(T(1) + t * t);
                            s = c * t;
                            tau = s / (T(1) + c);
                            if (lane == 0) s_flag = 1;
                        }
                        // Rutishauser's form of the rotation, x' = x - s (y + tau x),
                        // y' = y + s (x - tau y), tau = s / (1 + c): c = 1 - s tau is
                        // never rounded on its own, so small rotations do not add the
                        // t^2 of energy per step that c rounded to 1 would
                        if (s != T(0)) {
                            for (int l = lane; l < n; l += 32) {
                                const T x = K[(size_t)p * n + l], y = K[(size_t)q * n + l];
                                K[(size_t)p * n + l] = x - s * (y + tau * x);
                                K[(size_t)q * n + l] = y + s * (x - tau * y);
                            }
                            for (int l = lane; l < m; l += 32) {
                                const T x = J[(size_t)l * m + p], y = J[(size_t)l * m + q];
                                J[(size_t)l * m + p] = x - s * (y + tau * x);
                                J[(size_t)l * m + q] = y + s * (x - tau * y);
                            }
                        }
                    }
                }
                __syncthreads();
            }
            const int f = s_flag;
            __syncthreads();
            if (!f) break;
        }
        // ---- the rows' norms and their order (descending, lower index on ties)
        for (int p = warp; p < m; p += nw) {
            T ss = 0;
            for (int l = lane; l < n; l += 32) ss += K[(size_t)p * n + l] * K[(size_t)p * n + l];
            ss = warp_sum(ss);
            if (lane == 0) nrm[p] = ss;
        }
        __syncthreads();
        for (int p = tid; p < m; p += blockDim.x) {
            int rk = 0;
            for (int q = 0; q < m; ++q) rk += (nrm[q] > nrm[p]) || (nrm[q] == nrm[p] && q < p);
            perm[rk] = p;
        }
        __syncthreads();
        // ---- U <- blockdiag(U, 1) J P (first k columns), one row per thread
        for (int row = tid; row <= rt; row += blockDim.x) {
            T out[64];
            if (row < rt) {
                T old[64];
#pragma unroll 4
                for (int c = 0; c < k; ++c) old[c] = U[(size_t)row * k + c];
                for (int c = 0; c < k; ++c) {
                    const int pc = perm[c];
                    T acc = 0;
                    for (int l = 0; l < k; ++l) acc += old[l] * J[(size_t)l * m + pc];
                    out[c] = acc;
                }
            } else {
                for (int c = 0; c < k; ++c) out[c] = J[(size_t)k * m + perm[c]];
            }
            for (int c = 0; c < k; ++c) U[(size_t)row * k + c] = out[c];
        }
        // ---- K <- the k longest rows of K' (truncation to rank k)
        for (int e = tid; e < k * n; e += blockDim.x) {
            const int c = e / n, l = e - c * n;
            Kn[e] = K[(size_t)perm[c] * n + l];
        }
        __syncthreads();
        T* t = K;
        K = Kn;
        Kn = t;
    }
    // ---- outputs: sigma, V^T, Sigma V^T, with R5 (zero below the rank
    // tolerance) and R6 (largest-|.| entry of v_c positive, U flipped with it)
    for (int c = warp; c < k; c += nw) {
        T ss = 0;
        for (int l = lane; l < n; l += 32) ss += K[(size_t)c * n + l] * K[(size_t)c * n + l];
        ss = warp_sum(ss);
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
        const T sg = (bi < n && K[(size_t)c * n + bi] < T(0)) ? T(-1) : T(1);
        if (lane == 0) {
            sig[c] = live ? sv : T(0);
            rot[c] = live ? sg : T(0);               // the column's factor for U
        }
        for (int l = lane; l < n; l += 32) {
            const T v = live ? sg * K[(size_t)c * n + l] / sv : T(0);
            Vt[(size_t)c * n + l] = v;
            if (a.w) ((T*)a.w)[slot * k * n + (size_t)c * n + l] = live ? sv * v : T(0);
        }
    }
    __syncthreads();
    const int rows = r0 + nr;
    for (int64_t e = tid; e < (int64_t)rows * k; e += blockDim.x) U[e] *= rot[e % k];
}

size_t row_append_smem_bytes(int n, int k, bool fp64) { return row_append_smem(n, k, fp64 ? 8 : 4); }

cudaError_t launch_row_append(const RowAppendArgs& a, bool fp64, cudaStream_t st) {
    if (a.nblk < 1) return cudaSuccess;
    const size_t sm = row_append_smem(a.n, a.k, fp64 ? 8 : 4);
    cudaError_t e;
    if (fp64) {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_row_append<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
                cudaSuccess)
            return e;
        k_row_append<double><<<a.nblk, 256, sm, st>>>(a);
    } else {
        if (sm > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_row_append<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
                cudaSuccess)
            return e;
        k_row_append<float><<<a.nblk, 256, sm, st>>>(a);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace zs
