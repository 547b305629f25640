// zs_linalg.cuh - CTA-wide dense linear algebra used by the range-SVD kernels.
//
// Every routine here is called by all threads of one CTA with the operands in
// shared memory (or, for the n x n Gram matrix, in L2-resident global memory)
// and contains its own __syncthreads().  Nothing spins: every loop has a fixed
// upper bound.
//
//  * jacobi_eig   cyclic two-sided Jacobi eigensolver for a symmetric m x m
//                 matrix (m <= ZS_MAXM), round-robin ("circle") ordering so the
//                 m/2 rotations of one step are disjoint and applied in
//                 parallel.  Two-sided Jacobi on X^T X performs the rotations
//                 of one-sided (Hestenes) Jacobi on X, so this is the
//                 "small-core Jacobi SVD" of every Gram-form core below.
//  * mgs_orth     modified Gram-Schmidt (two passes) of an n x m column block
//                 with replacement of numerically dependent columns.
//  * sort_desc    permutation that orders eigenvalues descending.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#ifndef ZS_MAXM
#define ZS_MAXM 64
#endif

namespace zs {

// Energy rule (Eq. 1): the smallest rank whose leading singular values
// (sig, descending, k of them) hold a fraction >= xi of the energy e; k if
// they never do, 0 for an empty block.  FP64 sums in a fixed order.
template <typename T>
__device__ __forceinline__ int xi_rank_of(const T* sig, int k, double e, double xi) {
    if (!(e > 0.0)) return 0;
    const double goal = xi * e;
    double cum = 0.0;
    for (int l = 0; l < k; ++l) {
        cum += (double)sig[l] * (double)sig[l];
        if (cum >= goal) return l + 1;
    }
    return k;
}

template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }
template <> __device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }

__device__ __forceinline__ float zsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double zsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float zabs(float x) { return fabsf(x); }
__device__ __forceinline__ double zabs(double x) { return fabs(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA-wide sum; `red` is shared scratch of >= 32 elements.  Result returned to
// every thread.
template <typename T>
__device__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T r = 0;
    for (int i = 0; i < nw; ++i) r += red[i];
    return r;
}

// Pair (p, q), p < q, of slot i in step r of the round-robin schedule over mm
// (even) indices: index 0 stays, the others rotate.  Over mm - 1 steps every
// pair meets exactly once.
__device__ __forceinline__ void rr_pair(int mm, int r, int i, int& p, int& q) {
    const int a = (i == 0) ? 0 : ((i - 1 + r) % (mm - 1)) + 1;
    const int b = ((mm - 2 - i + r) % (mm - 1)) + 1;
    p = a < b ? a : b;
    q = a < b ? b : a;
}

// Shared scratch the Jacobi routine needs (static size).
template <typename T>
struct JacobiScratch {
    T cs[ZS_MAXM];        // c, s per pair
    int pq[ZS_MAXM];      // p, q per pair
    int flag;
    T scale;
};

// Symmetric eigen-decomposition A = Z diag(lambda) Z^T, in place: on return the
// diagonal of A holds the eigenvalues (unsorted) and the columns of Z the
// eigenvectors.  If init_z, Z starts as the identity, else the rotations are
// accumulated into the Z given (warm start / refinement).  Returns sweeps used.
// The CTA needs at least m/2 + 1 threads (all callers run 128 or more, m <= 64).
template <typename T>
__device__ int jacobi_eig(T* A, int lda, T* Z, int ldz, int m, JacobiScratch<T>& js,
                          int max_sweeps, bool init_z, T floor_mult = T(64)) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (init_z)
        for (int e = tid; e < m * m; e += nt) Z[(e / m) * ldz + (e % m)] = (e / m == e % m) ? T(1) : T(0);
    // FP32: the upper triangle defines A, and the 2 x 2 block updates below
    // keep both halves equal
    constexpr bool kBlock = std::is_same<T, float>::value;
    if (kBlock)
        for (int e = tid; e < m * m; e += nt) {
            const int p = e / m, q = e - (e / m) * m;
            if (q < p) A[p * lda + q] = A[q * lda + p];
        }
    if (tid == 0) {
        T mx = 0;
        for (int i = 0; i < m; ++i) mx = fmax(mx, zabs(A[i * lda + i]));
        js.scale = mx;
    }
    __syncthreads();
    if (m < 2) return 0;
    const int mm = m + (m & 1), np = mm >> 1;
    // a pair counts as converged once |a_pq| <= 64 eps sqrt(a_pp a_qq): the
    // rounding noise of the parallel updates sits near eps |A|, so a tighter
    // threshold only burns sweeps; the eigenvalue error left is O(tol^2).
    const T tol = T(64) * eps_of<T>();
    // absolute floor: in FP32 the updates leave noise ~eps * max|a_ii| in every
    // entry, so pairs between small eigenvalues would otherwise rotate forever
    // (floor_mult lowers it where small eigenvalues must keep their relative
    // accuracy: the off-diagonals of an accurately formed graded matrix shrink
    // with its diagonal, and the relative test alone converges)
    const T floor_ = (sizeof(T) == 4 ? floor_mult : T(1)) * eps_of<T>() * js.scale;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // a sweep starts only if some pair is still above the thresholds (a
        // sweep without rotations would leave A as it is)
        if (tid == 0) js.flag = 0;
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int p = e / m, q = e - (e / m) * m;
            if (q <= p) continue;
            const T aa = zabs(A[p * lda + q]);
            if (aa > floor_ && aa > tol * zsqrt(zabs(A[p * lda + p] * A[q * lda + q]))) js.flag = 1;
        }
        __syncthreads();
        if (!js.flag) break;
        for (int r = 0; r < mm - 1; ++r) {
            for (int i = tid; i < np; i += nt) {
                int p, q;
                rr_pair(mm, r, i, p, q);
                T c = 1, s = 0;
                if (q < m) {
                    const T apq = A[p * lda + q], app = A[p * lda + p], aqq = A[q * lda + q];
                    const T aa = zabs(apq);
                    if (aa > floor_ && aa > tol * zsqrt(zabs(app * aqq))) {
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (zabs(tau) + zsqrt(T(1) + tau * tau));
                        c = T(1) / zsqrt(T(1) + t * t);
                        s = t * c;
                    }
                }
                js.pq[2 * i] = p;
                js.pq[2 * i + 1] = q;
                js.cs[2 * i] = c;
                js.cs[2 * i + 1] = s;
            }
            __syncthreads();
            if (!kBlock) {
                // FP64: rows A <- J^T A, then columns A <- A J and Z <- Z J
                for (int e = tid; e < np * m; e += nt) {
                    const int i = e / m, j = e - (e / m) * m;
                    const T s = js.cs[2 * i + 1];
                    if (s == T(0)) continue;
                    const T c = js.cs[2 * i];
                    const int p = js.pq[2 * i], q = js.pq[2 * i + 1];
                    const T ap = A[p * lda + j], aq = A[q * lda + j];
                    A[p * lda + j] = c * ap - s * aq;
                    A[q * lda + j] = s * ap + c * aq;
                }
                __syncthreads();
                for (int e = tid; e < np * m; e += nt) {
                    const int i = e / m, row = e - (e / m) * m;
                    const T s = js.cs[2 * i + 1];
                    if (s == T(0)) continue;
                    const T c = js.cs[2 * i];
                    const int p = js.pq[2 * i], q = js.pq[2 * i + 1];
                    const T ap = A[row * lda + p], aq = A[row * lda + q];
                    A[row * lda + p] = c * ap - s * aq;
                    A[row * lda + q] = s * ap + c * aq;
                    const T zp = Z[row * ldz + p], zq = Z[row * ldz + q];
                    Z[row * ldz + p] = c * zp - s * zq;
                    Z[row * ldz + q] = s * zp + c * zq;
                }
                __syncthreads();
                continue;
            }
            // FP32: A <- J^T A J one 2 x 2 block at a time: block (i, j) of the pairs
            // (rows p_i, q_i; columns p_j, q_j) becomes R_i B R_j^T, written
            // with its mirror (j, i), so A stays exactly symmetric.  The blocks
            // partition A, so the updates are independent and run in place.
            // Thread t takes column pair j = t mod np and row pairs i = t / np,
            // t / np + ng, ... (i <= j); then rows of Z for pair j likewise.
            const int ng = nt / np;
            if (tid < ng * np) {
                const int j = tid % np, g = tid / np;
                const T sj = js.cs[2 * j + 1], cj = js.cs[2 * j];
                const int u = js.pq[2 * j], v = js.pq[2 * j + 1];
                const bool hv = v < m;
                for (int i = g; i <= j; i += ng) {
                    const T si = js.cs[2 * i + 1];
                    if (si == T(0) && sj == T(0)) continue;
                    const T ci = js.cs[2 * i];
                    const int p = js.pq[2 * i], q = js.pq[2 * i + 1];
                    const bool hq = q < m;
                    const T a00 = A[p * lda + u];
                    const T a01 = hv ? A[p * lda + v] : T(0);
                    const T a10 = hq ? A[q * lda + u] : T(0);
                    const T a11 = (hq && hv) ? A[q * lda + v] : T(0);
                    const T b00 = ci * a00 - si * a10, b01 = ci * a01 - si * a11;
                    const T b10 = si * a00 + ci * a10, b11 = si * a01 + ci * a11;
                    const T d00 = cj * b00 - sj * b01, d01 = sj * b00 + cj * b01;
                    const T d10 = cj * b10 - sj * b11, d11 = sj * b10 + cj * b11;
                    A[p * lda + u] = d00;
                    if (hv) A[p * lda + v] = d01;
                    if (hq) A[q * lda + u] = d10;
                    if (hq && hv) A[q * lda + v] = d11;
                    if (i != j) {
                        A[u * lda + p] = d00;
                        if (hv) A[v * lda + p] = d01;
                        if (hq) A[u * lda + q] = d10;
                        if (hq && hv) A[v * lda + q] = d11;
                    }
                }
                // Z <- Z J for pair j, four rows' loads issued together
                if (sj != T(0))
                    for (int r0 = g; r0 < m; r0 += 4 * ng) {
                        T zp[4], zq[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int row = r0 + h * ng;
                            zp[h] = row < m ? Z[row * ldz + u] : T(0);
                            zq[h] = row < m ? Z[row * ldz + v] : T(0);
                        }
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const int row = r0 + h * ng;
                            if (row < m) {
                                Z[row * ldz + u] = cj * zp[h] - sj * zq[h];
                                Z[row * ldz + v] = sj * zp[h] + cj * zq[h];
                            }
                        }
                    }
            }
            __syncthreads();
        }
    }
    return sweep;
}

// perm[r] = index of the r-th largest diagonal entry of A (stable on ties).
template <typename T>
__device__ void sort_desc(const T* A, int lda, int m, int* perm) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const T v = A[i * lda + i];
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const T w = A[j * lda + j];
            rk += (w > v) || (w == v && j < i);
        }
        perm[rk] = i;
    }
    __syncthreads();
}

// Orthonormalise the m columns of Q (n x m, row stride ldq, best odd) in
// place by classical Gram-Schmidt with a second projection pass (CGS2).  A
// column whose norm collapses below 1e3*eps of its starting norm (rank
// deficiency) is replaced by a coordinate vector and re-projected.  `red` is
// shared scratch (>= 32), `coef` shared scratch (>= m).
template <typename T>
__device__ void mgs_orth(T* Q, int ldq, int n, int m, T* red, T* coef) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    for (int c = 0; c < m; ++c) {
        T ss = 0;
        for (int i = tid; i < n; i += nt) ss += Q[i * ldq + c] * Q[i * ldq + c];
        const T nrm0 = zsqrt(block_sum(ss, red));
        T nrm = 0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt == 1) {
                __syncthreads();
                for (int i = tid; i < n; i += nt) Q[i * ldq + c] = T(0);
                __syncthreads();
                if (tid == 0) Q[((c * 7919 + 13) % n) * ldq + c] = T(1);
                __syncthreads();
            }
            for (int pass = 0; pass < 2 && c > 0; ++pass) {
                for (int d = wid; d < c; d += nw) {
                    T dot = 0;
                    for (int i = lane; i < n; i += 32) dot += Q[i * ldq + d] * Q[i * ldq + c];
                    dot = warp_sum(dot);
                    if (lane == 0) coef[d] = dot;
                }
                __syncthreads();
                for (int i = tid; i < n; i += nt) {
                    T acc = Q[i * ldq + c];
                    for (int d = 0; d < c; ++d) acc -= coef[d] * Q[i * ldq + d];
                    Q[i * ldq + c] = acc;
                }
                __syncthreads();
            }
            ss = 0;
            for (int i = tid; i < n; i += nt) ss += Q[i * ldq + c] * Q[i * ldq + c];
            nrm = zsqrt(block_sum(ss, red));
            const T base = attempt == 0 ? nrm0 : T(1);
            if (nrm > T(1e3) * eps_of<T>() * base && nrm > T(0)) break;
        }
        const T inv = nrm > T(0) ? T(1) / nrm : T(0);
        for (int i = tid; i < n; i += nt) Q[i * ldq + c] *= inv;
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// Warp-level variants: one warp owns one small problem in its own shared
// memory slice and synchronises with __syncwarp only, so the warps of a CTA
// work on different problems without CTA barriers.
// ---------------------------------------------------------------------------
template <typename T>
struct WarpRot {
    int p[ZS_MAXM / 2], q[ZS_MAXM / 2];
    T c[ZS_MAXM / 2], s[ZS_MAXM / 2];
};

// Cyclic Jacobi for one warp: lanes < m/2 compute the rotations of a
// round-robin step and publish them in `wr` (shared memory); then every lane
// applies all of them to its own column (row phase) and to its own row of A
// and Z (column phase).  The pair updates are independent, so they pipeline.
template <typename T>
__device__ int warp_jacobi(T* A, int lda, T* Z, int ldz, int m, int max_sweeps, bool init_z, WarpRot<T>& wr) {
    const int lane = threadIdx.x & 31;
    if (init_z)
        for (int e = lane; e < m * m; e += 32) Z[(e / m) * ldz + (e % m)] = (e / m == e % m) ? T(1) : T(0);
    __syncwarp();
    if (m < 2) return 0;
    T mx = 0;
    for (int i = lane; i < m; i += 32) mx = fmax(mx, zabs(A[i * lda + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int mm = m + (m & 1), np = mm >> 1;
    const T tol = T(64) * eps_of<T>();
    const T floor_ = (sizeof(T) == 4 ? T(64) : T(1)) * eps_of<T>() * mx;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < mm - 1; ++r) {
            T c = 1, sn = 0;
            if (lane < np) {
                int p, q;
                rr_pair(mm, r, lane, p, q);
                if (q < m) {
                    const T apq = A[p * lda + q], app = A[p * lda + p], aqq = A[q * lda + q];
                    const T aa = zabs(apq);
                    if (aa > floor_ && aa > tol * zsqrt(zabs(app * aqq))) {
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (zabs(tau) + zsqrt(T(1) + tau * tau));
                        c = T(1) / zsqrt(T(1) + t * t);
                        sn = t * c;
                    }
                } else {
                    q = p;      // dummy index of an odd m: never rotated
                }
                wr.p[lane] = p;
                wr.q[lane] = q;
                wr.c[lane] = c;
                wr.s[lane] = sn;
            }
            rotated |= __any_sync(0xffffffffu, sn != T(0));
            __syncwarp();
            // rows: A <- J^T A, lane owns column j
            for (int j = lane; j < m; j += 32) {
#pragma unroll 4
                for (int i = 0; i < np; ++i) {
                    const T si = wr.s[i];
                    if (si == T(0)) continue;
                    const T ci = wr.c[i];
                    const int pi = wr.p[i], qi = wr.q[i];
                    const T ap = A[pi * lda + j], aq = A[qi * lda + j];
                    A[pi * lda + j] = ci * ap - si * aq;
                    A[qi * lda + j] = si * ap + ci * aq;
                }
            }
            __syncwarp();
            // columns: A <- A J and Z <- Z J, lane owns row `row`
            for (int row = lane; row < m; row += 32) {
#pragma unroll 4
                for (int i = 0; i < np; ++i) {
                    const T si = wr.s[i];
                    if (si == T(0)) continue;
                    const T ci = wr.c[i];
                    const int pi = wr.p[i], qi = wr.q[i];
                    const T ap = A[row * lda + pi], aq = A[row * lda + qi];
                    A[row * lda + pi] = ci * ap - si * aq;
                    A[row * lda + qi] = si * ap + ci * aq;
                    const T zp = Z[row * ldz + pi], zq = Z[row * ldz + qi];
                    Z[row * ldz + pi] = ci * zp - si * zq;
                    Z[row * ldz + qi] = si * zp + ci * zq;
                }
            }
            __syncwarp();
        }
        if (!rotated) break;
    }
    return sweep;
}

// perm[r] = index of the r-th largest diagonal entry (warp-level, stable).
template <typename T>
__device__ void warp_sort_desc(const T* A, int lda, int m, int* perm) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < m; i += 32) {
        const T v = A[i * lda + i];
        int rk = 0;
        for (int j = 0; j < m; ++j) {
            const T w = A[j * lda + j];
            rk += (w > v) || (w == v && j < i);
        }
        perm[rk] = i;
    }
    __syncwarp();
}

// One refinement sweep in closed form for a nearly diagonal symmetric B (the
// FP64 Rayleigh quotient Z^T A Z of FP32 eigenvectors Z): the rotations of a
// Jacobi sweep over such a B have angles B_ij / (B_jj - B_ii) to first order,
// so W = I + E with E_ij = B_ij / (B_jj - B_ii) (i != j), and the eigenvalues
// to second order are B_jj + sum_i B_ij E_ij.  E is skew-symmetric, so W is
// orthogonal up to E^2: only pairs with |E_ij| <= 1e-3 are corrected, which
// keeps the columns orthonormal to ~1e-6; the others (gaps within 1e3 |B_ij|,
// where the FP32 rotations leave an eigenvalue error below B_ij^2 / gap) and
// pairs whose gap is at the rounding level of B are left alone.  The
// refined eigenvalues replace B's diagonal.  Called by all threads of a warp
// (sync = __syncwarp) or a CTA (sync = __syncthreads); thread t0 of tn.
template <typename T, typename Sync>
__device__ void refine_sweep(T* B, int ldb, T* W, int ldw, int m, int t0, int tn, T* theta, Sync sync) {
    for (int j = t0; j < m; j += tn) {
        const T bjj = B[j * ldb + j];
        T corr = 0;
        for (int i = 0; i < m; ++i) {
            T e = 0;
            if (i != j) {
                const T bij = B[i * ldb + j], bii = B[i * ldb + i];
                const T gap = bjj - bii;
                if (zabs(gap) > T(1e-9) * (zabs(bii) + zabs(bjj)) && zabs(bij) <= T(1e-3) * zabs(gap)) {
                    e = bij / gap;
                    corr += bij * e;
                }
            }
            W[i * ldw + j] = (i == j) ? T(1) : e;
        }
        theta[j] = bjj + corr;
    }
    sync();
    for (int j = t0; j < m; j += tn) B[j * ldb + j] = theta[j];
    sync();
}

// ---------------------------------------------------------------------------
// Register-resident warp routines for one 32 x 32 problem per warp: lane l
// holds column l.  Pairing is the round-robin schedule of rr_pair (index 0
// fixed, 1..31 rotating) in closed form, so each lane finds its partner
// without a table.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rr_partner32(int x, int r) {
    if (x == 0) return (r + 30) % 31 + 1;
    int v = (2 * r - 2 - (x - 1)) % 31;
    if (v < 0) v += 31;
    const int y = v + 1;
    return y == x ? 0 : y;
}

// The loops below run over the pivot index without unrolling (the code stays
// small); the lane's vector is shifted down one register per step so that
// the pivot element is always register 0 and every index stays static.

// Cholesky A = L L^T of the warp's symmetric 32 x 32 matrix held as column
// `lane` in a[].  L goes to the per-warp tile T (row-major, stride 33); on
// return a[] holds column `lane` of L.  A pivot <= 0 gives a zero column.
__device__ __forceinline__ void warp_chol32(float (&a)[32], float* T, int lane) {
    for (int j = 0; j < 32; ++j) {
        // a[0..31-j] hold rows j.. of column `lane`
        const float piv = __shfl_sync(0xffffffffu, a[0], j);
        const float d = piv > 0.f ? sqrtf(piv) : 0.f;
        const float inv = d > 0.f ? 1.f / d : 0.f;
        const float slj = a[0] * inv;                       // L[lane][j] for lane > j
        if (lane == j) T[j * 33 + j] = d;
#pragma unroll
        for (int i = 1; i < 32; ++i) {
            const float lij = __shfl_sync(0xffffffffu, a[i], j) * inv;   // L[j+i][j]
            if (lane == j && j + i < 32) T[(j + i) * 33 + j] = lij;
            if (lane > j) a[i] = fmaf(-lij, slj, a[i]);
        }
#pragma unroll
        for (int i = 0; i < 31; ++i) a[i] = a[i + 1];
        a[31] = 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = i >= lane ? T[i * 33 + lane] : 0.f;
    __syncwarp();
}

// x = L^-1 h for every lane's own vector h (L row-major in T, stride 33).
// The solution is also left in W as W[i][lane] (row-major, stride 33).
__device__ __forceinline__ void warp_fsub32(const float* T, float (&h)[32], float (&x)[32], float* W, int lane) {
    for (int p = 0; p < 32; ++p) {
        const float dpp = T[p * 33 + p];
        const float xp = dpp > 0.f ? h[0] / dpp : 0.f;
        W[p * 33 + lane] = xp;
#pragma unroll
        for (int i = 1; i < 32; ++i)
            if (p + i < 32) h[i] = fmaf(-T[(p + i) * 33 + p], xp, h[i]);
#pragma unroll
        for (int i = 0; i < 31; ++i) h[i] = h[i + 1];
        h[31] = 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = W[i * 33 + lane];
}

// z = L^-T w for every lane's own vector w (L row-major in T); W as above.
__device__ __forceinline__ void warp_bsub32(const float* T, float (&w)[32], float (&z)[32], float* W, int lane) {
    for (int i = 31; i >= 0; --i) {
        // w[31 - q] holds w_{i - q}
        const float dii = T[i * 33 + i];
        const float zi = dii > 0.f ? w[31] / dii : 0.f;
        W[i * 33 + lane] = zi;
#pragma unroll
        for (int q = 1; q < 32; ++q)
            if (q <= i) w[31 - q] = fmaf(-T[i * 33 + (i - q)], zi, w[31 - q]);
#pragma unroll
        for (int q = 31; q > 0; --q) w[q] = w[q - 1];
        w[0] = 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = W[i * 33 + lane];
}

// One-sided (Hestenes) Jacobi on the warp's 32 x 32 matrix G (column `lane`
// in x[]; v[] is scratch): orthogonalises the columns of G by plane
// rotations over the round-robin pairing.  On return x[] holds the unit
// vector of column `lane` and the result is its squared norm: for G = R^T
// with R^T R = A these are the eigenvectors and eigenvalues of A.
__device__ __forceinline__ float warp_hestenes32(float (&x)[32], float (&v)[32], int lane) {
    // one-sided Jacobi on the columns of G
    float al = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) al = fmaf(x[i], x[i], al);
    // converged when every pair is orthogonal to 1e-5: safely above the
    // rounding level of a 32-term fp32 dot product, which a tighter test
    // could keep rotating at
    const float tol = 1e-5f;
    for (int sweep = 0; sweep < 15; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < 31; ++r) {
            const int pr = rr_partner32(lane, r);
            const bool isp = lane < pr;
            float g4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                v[i] = __shfl_sync(0xffffffffu, x[i], pr);
                g4[i & 3] = fmaf(x[i], v[i], g4[i & 3]);
            }
            const float g = (g4[0] + g4[1]) + (g4[2] + g4[3]);
            const float ao = __shfl_sync(0xffffffffu, al, pr);
            const float app = isp ? al : ao, aqq = isp ? ao : al;
            float c = 1.f, s = 0.f;
            if (g * g > (tol * tol) * (app * aqq) && g != 0.f) {
                // zeta and t need only be near the optimum (the sweep
                // repeats); c gets a Newton step so that c^2 + s^2 = 1 to
                // rounding and the column norms do not drift
                const float zeta = __fdividef(aqq - app, 2.f * g);
                const float r1 = fmaf(zeta, zeta, 1.f);
                const float t = __fdividef(copysignf(1.f, zeta), fabsf(zeta) + r1 * rsqrtf(r1));
                const float u = fmaf(t, t, 1.f);
                float cc = rsqrtf(u);
                cc = cc * fmaf(-0.5f * u * cc, cc, 1.5f);
                c = cc;
                s = cc * t;
                al = isp ? app - t * g : aqq + t * g;
                rotated = 1;
            }
            // p: c x_p - s x_q; q: s x_p + c x_q (branch-free across the pair)
            const float sv = isp ? -s : s;
#pragma unroll
            for (int i = 0; i < 32; ++i) x[i] = fmaf(sv, v[i], c * x[i]);
        }
        if (!__any_sync(0xffffffffu, rotated)) break;
        al = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) al = fmaf(x[i], x[i], al);
    }
    al = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) al = fmaf(x[i], x[i], al);
    const float sg = sqrtf(al);
    const float inv = sg > 0.f ? 1.f / sg : 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] *= inv;
    return al;
}

}  // namespace zs
