// zs_kernels_dev.cuh - sm_103a device kernels of the range-SVD hot path.
//
// Storage phase (Section 3.2, Algorithm 1; one launch set per chunk of blocks):
//   k_gram_compress   G_i = A_i^T A_i for every block (symmetric tiles)
//   k_eig_compress    top-k eigenpairs of G_i -> sigma_i, V_i (Section 2.1)
//   k_form_u          U_i = A_i V_i Sigma_i^{-1}
// Query phase (Section 3.3; persistent work-list kernels over a batch):
//   k_partial         Partial-SVD of the boundary blocks (Algorithm 3, Eq. 5-6)
//   k_stack           stack Sigma_i V_i^T of the interior blocks (Algorithm 2)
//   k_gram_query      M^T M of the stacked matrix
//   k_eig_query       top-k_q eigenpairs -> Sigma_r, V_r (Algorithm 2)
//   k_ur              U_r = M V_r Sigma_r^{-1} and the per-slab lift
//                     coefficients (Partial-SVD slabs folded with their Sigma V~ Sigma~^-1)
// The tensor-core kernels of the float path are in zs_tc_kernels.cuh (included
// at the end).  Every launcher translation unit includes this header and
// instantiates only the kernels it launches.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "zs_internal.h"
#include "zs_linalg.cuh"

namespace zs {

__device__ __forceinline__ double ld_in(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_in(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_in(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16*>(p)));
}

template <typename T, bool REF> struct Prec { using TR = T; };
template <> struct Prec<float, true> { using TR = double; };

// ---------------------------------------------------------------------------
// Gram tiles: G[I0:I0+64, J0:J0+64] (and its mirror) of rows x n matrix A.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_pair(int p, int ntile, int& ti, int& tj) {
    ti = 0;
    while (p >= ntile - ti) { p -= ntile - ti; ++ti; }
    tj = ti + p;
}

template <typename Tin, typename T>
__device__ void gram_tile(const Tin* __restrict__ A, int64_t lda, int rows, int n,
                          T* __restrict__ G, int ti, int tj, T (*As)[64], T (*Bs)[64]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int I0 = ti * 64, J0 = tj * 64;
    const bool diag = (ti == tj);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int r0 = 0; r0 < rows; r0 += 32) {
        for (int e = tid; e < 32 * 64; e += 256) {
            const int r = e >> 6, c = e & 63, gr = r0 + r;
            const bool rv = gr < rows;
            As[r][c] = (rv && I0 + c < n) ? T(ld_in(A + (int64_t)gr * lda + I0 + c)) : T(0);
            if (!diag) Bs[r][c] = (rv && J0 + c < n) ? T(ld_in(A + (int64_t)gr * lda + J0 + c)) : T(0);
        }
        __syncthreads();
        const T(*Bp)[64] = diag ? As : Bs;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            T a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[r][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bp[r][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = I0 + ty + 16 * i, col = J0 + tx + 16 * j;
            if (row < n && col < n) {
                G[(int64_t)row * n + col] = acc[i][j];
                if (!diag) G[(int64_t)col * n + row] = acc[i][j];
            }
        }
}

template <typename Tin, typename T>
__global__ void __launch_bounds__(256) k_gram_compress(CompressChunk c) {
    __shared__ __align__(16) T As[32][64];
    __shared__ __align__(16) T Bs[32][64];
    const int ntile = (c.n + 63) / 64;
    int ti, tj;
    tile_pair(blockIdx.x, ntile, ti, tj);
    for (int j = blockIdx.y; j < c.nblk; j += gridDim.y) {
        const int64_t r0 = (int64_t)j * c.b;
        const int rows = (int)min((int64_t)c.b, c.rows_total - r0);
        gram_tile<Tin, T>((const Tin*)c.A + r0 * c.lda, c.lda, rows, c.n,
                          (T*)c.G + (int64_t)j * c.n * c.n, ti, tj, As, Bs);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram_query(QueryArgs a) {
    __shared__ __align__(16) T As[32][64];
    __shared__ __align__(16) T Bs[32][64];
    const int ntile = (a.n + 63) / 64;
    int ti, tj;
    tile_pair(blockIdx.x, ntile, ti, tj);
    const int nq = a.hdr->nq;
    for (int q = blockIdx.y; q < nq; q += gridDim.y) {
        const QPlan& P = a.plans[q];
        gram_tile<T, T>((const T*)a.M + P.slab0 * a.k * a.n, a.n, P.nslab * a.k, a.n,
                        (T*)a.G + (int64_t)q * a.n * a.n, ti, tj, As, Bs);
    }
}

// ---------------------------------------------------------------------------
// Small symmetric eigenproblem with optional FP64 refinement.
//   in : A_T (m x m, ld) in T; when REF also A_R (same matrix, double, ld)
//   out: theta[c] descending (TR) and eigenvector c = column perm[c] of Zo
// ---------------------------------------------------------------------------
template <typename T, bool REF>
struct SmallEig {
    using TR = typename Prec<T, REF>::TR;
    T* A_T;
    T* Z_T;
    double* A_R;   // REF only
    double* X;     // REF only
    double* W;     // REF only
    int ld;
};

template <typename T, bool REF>
__device__ void small_eig(SmallEig<T, REF>& s, int m, JacobiScratch<T>& js, JacobiScratch<double>& jd,
                          typename Prec<T, REF>::TR* theta, int* perm, typename Prec<T, REF>::TR*& Zo) {
    using TR = typename Prec<T, REF>::TR;
    const int tid = threadIdx.x, nt = blockDim.x, ld = s.ld;
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (m <= 32) {
            // one warp, in registers: Cholesky A = G G^T, then one-sided
            // Jacobi on G's columns gives the eigenpairs (written sorted)
            __shared__ float tile[32 * 33];
            __syncthreads();
            if (tid < 32) {
                const int lane = tid;
                float x[32], v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] = (i < m && lane < m) ? s.A_T[i * ld + lane] : 0.f;
                warp_chol32(x, tile, lane);
                const float th = warp_hestenes32(x, v, lane);
                int rk = 0;
#pragma unroll
                for (int o = 0; o < 32; ++o) {
                    const float ot = __shfl_sync(0xffffffffu, th, o);
                    rk += (ot > th) || (ot == th && o < lane);
                }
                if (rk < m) {
                    if (!REF) theta[rk] = th;
                    perm[rk] = rk;
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < m) s.Z_T[i * ld + rk] = x[i];
                }
            }
            __syncthreads();
            if constexpr (!REF) {
                Zo = reinterpret_cast<TR*>(s.Z_T);
                return;
            }
            done = true;
        }
    }
    const int sweeps = std::is_same<T, double>::value ? 40 : 30;
    if (!done) jacobi_eig<T>(s.A_T, ld, s.Z_T, ld, m, js, sweeps, true);
    if constexpr (REF) {
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            double acc = 0;
            for (int l = 0; l < m; ++l) acc += s.A_R[i * ld + l] * (double)s.Z_T[l * ld + c];
            s.X[i * ld + c] = acc;
        }
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int a = e / m, c = e - (e / m) * m;
            double acc = 0;
            for (int i = 0; i < m; ++i) acc += (double)s.Z_T[i * ld + a] * s.X[i * ld + c];
            s.A_R[a * ld + c] = acc;
        }
        __syncthreads();
        // one FP64 refinement sweep (closed form: A_R is diagonal to FP32 rounding)
        refine_sweep<double>(s.A_R, ld, s.W, ld, m, tid, nt, reinterpret_cast<double*>(theta),
                             [] { __syncthreads(); });
        for (int e = tid; e < m * m; e += nt) {
            const int i = e / m, c = e - (e / m) * m;
            double acc = 0;
            for (int a = 0; a < m; ++a) acc += (double)s.Z_T[i * ld + a] * s.W[a * ld + c];
            s.X[i * ld + c] = acc;
        }
        __syncthreads();
        sort_desc<double>(s.A_R, ld, m, perm);
        for (int c = tid; c < m; c += nt) theta[c] = s.A_R[perm[c] * ld + perm[c]];
        Zo = reinterpret_cast<TR*>(s.X);
    } else {
        sort_desc<T>(s.A_T, ld, m, perm);
        for (int c = tid; c < m; c += nt) theta[c] = s.A_T[perm[c] * ld + perm[c]];
        Zo = reinterpret_cast<TR*>(s.Z_T);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Top-kw eigenpairs of the symmetric PSD n x n matrix G (global, row-major).
// Dense Jacobi when m == n (n <= 64); otherwise subspace iteration with
// Rayleigh-Ritz on m columns started from the m columns of G with the largest
// diagonal.  Output: theta[c] (c < kw) descending and the eigenvectors as
// columns of V (n x kw, row stride ldv) in shared memory.
// ---------------------------------------------------------------------------
template <typename T, bool REF>
struct EigWork {
    T* Q;       // n x ldq, shared memory
    T* Y;       // n x ldq, shared memory or (yglob) this CTA's global workspace
    int ldq;
    bool yglob;
    SmallEig<T, REF> se;
};

template <typename T, bool REF>
__device__ __forceinline__ size_t eig_carve(char* base, int n, int m, bool yglob, void* ws, EigWork<T, REF>& w) {
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base + off; off += (bytes + 15) & ~size_t(15); return p; };
    const bool dense = (m == n && n <= 64);
    const int ld = m + 1;
    w.ldq = ld;
    w.yglob = yglob && !dense;
    if (dense) {
        w.Q = nullptr;
        w.Y = nullptr;
    } else {
        w.Q = (T*)take(sizeof(T) * (size_t)n * ld);
        w.Y = w.yglob ? (T*)ws + (size_t)blockIdx.x * n * ld : (T*)take(sizeof(T) * (size_t)n * ld);
    }
    w.se.ld = ld;
    w.se.A_T = (T*)take(sizeof(T) * (size_t)m * ld);
    w.se.Z_T = (T*)take(sizeof(T) * (size_t)m * ld);
    if (REF) {
        w.se.A_R = (double*)take(sizeof(double) * (size_t)m * ld);
        w.se.X = (double*)take(sizeof(double) * (size_t)m * ld);
        w.se.W = (double*)take(sizeof(double) * (size_t)m * ld);
    } else {
        w.se.A_R = w.se.X = w.se.W = nullptr;
    }
    return off;
}

struct EigStatic {
    int perm[ZS_MAXM];
    double theta[ZS_MAXM];
    double resid[ZS_MAXM];
    double red[32];
    double coef[ZS_MAXM];
    int flag;
};

template <typename T, bool REF, int MB>
__device__ void eig_solve(const T* __restrict__ G, int n, int m, int kw, EigWork<T, REF>& w,
                          JacobiScratch<T>& js, JacobiScratch<double>& jd, EigStatic& es,
                          T*& V, int& ldv) {
    using TR = typename Prec<T, REF>::TR;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = (nt + 31) >> 5;
    TR* theta = reinterpret_cast<TR*>(es.theta);
    T* red = reinterpret_cast<T*>(es.red);
    T* coef = reinterpret_cast<T*>(es.coef);
    const int ld = w.se.ld;
    TR* Zo;
    if (m == n && n <= 64) {
        // dense Jacobi on G itself
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e - (e / n) * n;
            const T g = G[(int64_t)i * n + j];
            w.se.A_T[i * ld + j] = g;
            if (REF) w.se.A_R[i * ld + j] = (double)g;
        }
        __syncthreads();
        small_eig<T, REF>(w.se, n, js, jd, theta, es.perm, Zo);
        // selected eigenvectors -> columns of A_T (no longer needed)
        for (int e = tid; e < n * kw; e += nt) {
            const int i = e / kw, c = e - (e / kw) * kw;
            w.se.A_T[i * ld + c] = (T)Zo[i * ld + es.perm[c]];
        }
        __syncthreads();
        V = w.se.A_T;
        ldv = ld;
        return;
    }
    T* Q = w.Q;
    T* Y = w.Y;
    const int ldq = w.ldq;
    // pivots: the m largest diagonal entries of G (stable on ties); diag in Y[0..n)
    for (int i = tid; i < n; i += nt) Y[i] = G[(int64_t)i * n + i];
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const T v = Y[i];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const T u = Y[j];
            rk += (u > v) || (u == v && j < i);
        }
        if (rk < m) es.perm[rk] = i;
    }
    __syncthreads();
    for (int e = tid; e < n * m; e += nt) {
        const int c = e / n, i = e - (e / n) * n;
        Q[i * ldq + c] = G[(int64_t)es.perm[c] * n + i];     // column perm[c] of G (symmetric)
    }
    __syncthreads();
    mgs_orth<T>(Q, ldq, n, m, red, coef);
    const T tol_r = T(8) * eps_of<T>() * zsqrt(T(n));
    const int maxit = std::is_same<T, double>::value ? 60 : 30;
    for (int it = 0; it < maxit; ++it) {
        // Y = G Q
        for (int i = tid; i < n; i += nt) {
            T acc[MB];
#pragma unroll
            for (int c = 0; c < MB; ++c) acc[c] = T(0);
            for (int l0 = 0; l0 < n; l0 += 8) {
                T g[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) g[u] = (l0 + u < n) ? G[(int64_t)(l0 + u) * n + i] : T(0);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (l0 + u >= n) break;
                    const T* qr = Q + (l0 + u) * ldq;
#pragma unroll
                    for (int c = 0; c < MB; ++c)
                        if (c < m) acc[c] += g[u] * qr[c];
                }
            }
#pragma unroll
            for (int c = 0; c < MB; ++c)
                if (c < m) Y[i * ldq + c] = acc[c];
        }
        __syncthreads();
        // Rayleigh quotient  Q^T Y  (FP64-accumulated when REF)
        for (int e = tid; e < m * m; e += nt) {
            const int a = e / m, c = e - (e / m) * m;
            if (c < a) continue;
            TR acc = 0;
            for (int i = 0; i < n; ++i) acc += (TR)Q[i * ldq + a] * (TR)Y[i * ldq + c];
            w.se.A_T[a * ld + c] = (T)acc;
            w.se.A_T[c * ld + a] = (T)acc;
            if (REF) {
                w.se.A_R[a * ld + c] = (double)acc;
                w.se.A_R[c * ld + a] = (double)acc;
            }
        }
        __syncthreads();
        small_eig<T, REF>(w.se, m, js, jd, theta, es.perm, Zo);
        // Ritz vectors in place: Q <- Q Z(:, perm), Y <- Y Z(:, perm)
        for (int i = tid; i < n; i += nt) {
            T row[MB];
#pragma unroll
            for (int a = 0; a < MB; ++a) row[a] = (a < m) ? Q[i * ldq + a] : T(0);
            for (int c = 0; c < m; ++c) {
                const TR* zc = Zo + es.perm[c];
                TR acc = 0;
#pragma unroll
                for (int a = 0; a < MB; ++a)
                    if (a < m) acc += (TR)row[a] * zc[a * ld];
                Q[i * ldq + c] = (T)acc;
            }
#pragma unroll
            for (int a = 0; a < MB; ++a) row[a] = (a < m) ? Y[i * ldq + a] : T(0);
            for (int c = 0; c < m; ++c) {
                const TR* zc = Zo + es.perm[c];
                TR acc = 0;
#pragma unroll
                for (int a = 0; a < MB; ++a)
                    if (a < m) acc += (TR)row[a] * zc[a * ld];
                Y[i * ldq + c] = (T)acc;
            }
        }
        __syncthreads();
        // residuals of the wanted pairs
        for (int c = wid; c < kw; c += nw) {
            const T th = (T)theta[c];
            T ss = 0;
            for (int i = lane; i < n; i += 32) {
                const T d = Y[i * ldq + c] - th * Q[i * ldq + c];
                ss += d * d;
            }
            ss = warp_sum(ss);
            if (lane == 0) es.resid[c] = (double)zsqrt(ss);
        }
        __syncthreads();
        if (tid == 0) {
            double mx = 0;
            for (int c = 0; c < kw; ++c) mx = fmax(mx, es.resid[c]);
            const double th0 = (double)theta[0];
            es.flag = (th0 <= 0.0) || (mx <= (double)tol_r * th0);
        }
        __syncthreads();
        const int done = es.flag;
        __syncthreads();
        if (done || it == maxit - 1) break;
        // next block: orthonormalised Ritz-rotated G Q
        if (w.yglob) {
            for (int e = tid; e < n * m; e += nt) {
                const int i = e / m, c = e - (e / m) * m;
                Q[i * ldq + c] = Y[i * ldq + c];
            }
            __syncthreads();
        } else {
            T* t = Q;
            Q = Y;
            Y = t;
        }
        mgs_orth<T>(Q, ldq, n, m, red, coef);
    }
    V = Q;
    ldv = ldq;
}

// Make the largest-|.| entry of each column positive (lowest index on ties).
template <typename T>
__device__ void canon_signs(T* V, int ldv, int n, int kw, int* sgn) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
    for (int c = wid; c < kw; c += nw) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const T v = zabs(V[i * ldv + c]);
            if (v > best || (v == best && i < bi)) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) sgn[c] = (bi < n && V[bi * ldv + c] < T(0)) ? -1 : 1;
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T rank_tol();
template <> __device__ __forceinline__ float rank_tol<float>() { return kRankTolF32; }
template <> __device__ __forceinline__ double rank_tol<double>() { return kRankTolF64; }

// ---------------------------------------------------------------------------
// Storage phase: eigen-core per block, then U = A V Sigma^-1.
// ---------------------------------------------------------------------------
template <typename T, bool REF, int MB>
__global__ void __launch_bounds__(256) k_eig_compress(CompressChunk c, int m, int yglob, void* ws) {
    extern __shared__ __align__(16) char dsm[];
    __shared__ JacobiScratch<T> js;
    __shared__ JacobiScratch<double> jd;
    __shared__ EigStatic es;
    __shared__ int sgn[ZS_MAXM];
    EigWork<T, REF> w;
    eig_carve<T, REF>(dsm, c.n, m, yglob != 0, ws, w);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = blockIdx.x; j < c.nblk; j += gridDim.x) {
        const int64_t r0 = (int64_t)j * c.b;
        const int rows = (int)min((int64_t)c.b, c.rows_total - r0);
        const int kcap = min(c.k, min(rows, c.n));
        T* V;
        int ldv;
        eig_solve<T, REF, MB>((const T*)c.G + (int64_t)j * c.n * c.n, c.n, m, c.k, w, js, jd, es, V, ldv);
        canon_signs<T>(V, ldv, c.n, c.k, sgn);
        using TR = typename Prec<T, REF>::TR;
        const TR* theta = reinterpret_cast<const TR*>(es.theta);
        const T s0 = zsqrt((T)fmax((double)theta[0], 0.0));
        const int slot = c.slot0 + j;
        T* sig = (T*)c.sig + (int64_t)slot * c.k;
        T* vt = (T*)c.vt + (int64_t)slot * c.k * c.n;
        for (int e = tid; e < c.k; e += nt) {
            const T s = zsqrt((T)fmax((double)theta[e], 0.0));
            sig[e] = (e < kcap && s > rank_tol<T>() * s0) ? s : T(0);
        }
        for (int e = tid; e < c.k * c.n; e += nt) {
            const int cc = e / c.n, i = e - (e / c.n) * c.n;
            const T s = zsqrt((T)fmax((double)theta[cc], 0.0));
            const bool live = (cc < kcap && s > rank_tol<T>() * s0);
            vt[e] = live ? (T)sgn[cc] * V[i * ldv + cc] : T(0);
        }
        __syncthreads();
    }
}

template <typename Tin, typename T>
__global__ void __launch_bounds__(256) k_form_u(CompressChunk c) {
    extern __shared__ __align__(16) char dsm[];
    const int n = c.n, k = c.k, ldn = n + 1;
    T* Vs = (T*)dsm;                         // k x (n+1)
    T* As = Vs + (size_t)k * ldn;            // 32 x (n+1)
    T* sg = As + (size_t)32 * ldn;           // k
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = blockIdx.y; j < c.nblk; j += gridDim.y) {
        const int64_t r0 = (int64_t)j * c.b;
        const int rows = (int)min((int64_t)c.b, c.rows_total - r0);
        const int slot = c.slot0 + j;
        const T* vt = (const T*)c.vt + (int64_t)slot * k * n;
        const T* sig = (const T*)c.sig + (int64_t)slot * k;
        T* U = (T*)c.U + (int64_t)slot * c.b * k;
        const Tin* A = (const Tin*)c.A + r0 * c.lda;
        for (int e = tid; e < k * n; e += nt) Vs[(e / n) * ldn + (e % n)] = vt[e];
        for (int e = tid; e < k; e += nt) sg[e] = sig[e];
        __syncthreads();
        for (int t0 = blockIdx.x * 32; t0 < c.b; t0 += gridDim.x * 32) {
            for (int e = tid; e < 32 * n; e += nt) {
                const int r = e / n, l = e - (e / n) * n;
                As[r * ldn + l] = (t0 + r < rows) ? T(ld_in(A + (int64_t)(t0 + r) * c.lda + l)) : T(0);
            }
            __syncthreads();
            for (int e = tid; e < 32 * k; e += nt) {
                const int r = e / k, cc = e - (e / k) * k;
                if (t0 + r >= c.b) continue;
                T acc = 0;
                const T* ar = As + r * ldn;
                const T* vr = Vs + cc * ldn;
                for (int l = 0; l < n; ++l) acc += ar[l] * vr[l];
                const T s = sg[cc];
                U[(int64_t)(t0 + r) * k + cc] = (t0 + r < rows && s > T(0)) ? acc / s : T(0);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Query phase.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_query(const int64_t* prefix, int nq, int64_t s) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct BlockRange { int blk, lo, hi, rows_i; };

// Rows [lo, hi) of block S + t that slab t of query P covers.
__device__ __forceinline__ BlockRange slab_rows(const QPlan& P, int t, int b, int64_t Trows) {
    BlockRange r;
    r.blk = P.S + t;
    const int64_t row0 = (int64_t)r.blk * b;
    r.rows_i = (int)min((int64_t)b, Trows - row0);
    r.lo = (t == 0) ? (int)(P.ts - row0) : 0;
    r.hi = (t == P.nslab - 1) ? (int)(P.te - row0 + 1) : r.rows_i;
    return r;
}

// Partial-SVD (Algorithm 3) of boundary slab `side` of each query:
//   H = Sigma (X U)^T (X U) Sigma  ->  V~, Sigma~^2   (SVD of X U Sigma, Eq. 5)
//   slab rows  Sigma~ V~^T V^T   (= Sigma' V'^T, Eq. 6) into M
//   lift coefficient  Sigma V~ Sigma~^{-1}  (U' = X U Sigma V~ Sigma~^{-1})
template <typename T, bool REF>
__global__ void __launch_bounds__(256) k_partial(QueryArgs a) {
    using TR = typename Prec<T, REF>::TR;
    extern __shared__ __align__(16) char dsm[];
    __shared__ JacobiScratch<T> js;
    __shared__ JacobiScratch<double> jd;
    __shared__ EigStatic es;
    __shared__ T sgs[ZS_MAXM];
    __shared__ T st[ZS_MAXM];
    const int k = a.k, n = a.n, ld = k + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    SmallEig<T, REF> se;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = dsm + off; off += (bytes + 15) & ~size_t(15); return p; };
    se.ld = ld;
    se.A_T = (T*)take(sizeof(T) * k * ld);
    se.Z_T = (T*)take(sizeof(T) * k * ld);
    if (REF) {
        se.A_R = (double*)take(sizeof(double) * k * ld);
        se.X = (double*)take(sizeof(double) * k * ld);
        se.W = (double*)take(sizeof(double) * k * ld);
    }
    T* Us = (T*)take(sizeof(T) * 64 * ld);   // 64 staged rows of U
    const int nq = a.hdr->nq;
    const int64_t Trows = a.hdr->T;
    const int npair_max = (ZS_MAXM * (ZS_MAXM + 1) / 2 + 255) / 256;
    for (int p = blockIdx.x; p < 2 * nq; p += gridDim.x) {
        const int q = p >> 1, side = p & 1;
        const QPlan& P = a.plans[q];
        if (side == 1 && P.nslab == 1) continue;
        const int t = side ? P.nslab - 1 : 0;
        const BlockRange br = slab_rows(P, t, a.b, Trows);
        const int ki = min(k, min(br.rows_i, n));
        const T* U = (const T*)a.U + (int64_t)br.blk * a.b * k;
        const T* sg = (const T*)a.sig + (int64_t)br.blk * k;
        const T* vt = (const T*)a.vt + (int64_t)br.blk * k * n;
        for (int e = tid; e < k; e += nt) sgs[e] = sg[e];
        // H (upper triangle pairs over ki), FP64-accumulated when REF
        const int np = ki * (ki + 1) / 2;
        TR acc[npair_max];
        int pa[npair_max], pc[npair_max];
#pragma unroll
        for (int s = 0; s < npair_max; ++s) {
            acc[s] = 0;
            int e = tid + s * nt, aa = 0;
            while (e >= ki - aa && aa < ki) { e -= ki - aa; ++aa; }
            pa[s] = aa;
            pc[s] = aa + e;
        }
        for (int r0 = br.lo; r0 < br.hi; r0 += 64) {
            const int nr = min(64, br.hi - r0);
            __syncthreads();
            for (int e = tid; e < nr * k; e += nt) {
                const int r = e / k, c = e - (e / k) * k;
                Us[r * ld + c] = U[(int64_t)(r0 + r) * k + c];
            }
            __syncthreads();
#pragma unroll
            for (int s = 0; s < npair_max; ++s) {
                if (tid + s * nt < np) {
                    if constexpr (REF && std::is_same<T, float>::value) {
                        // FP64-grade sum from FP32 operations (GB300 issues FP64
                        // at 1/64 of the FP32 rate): each product split exactly
                        // into p + e by an FMA, the running sum kept as hi + lo
                        // with Knuth's TwoSum, so the chunk's sum carries about
                        // 48 significant bits before it joins acc in FP64
                        float hi = 0.f, lo = 0.f;
                        for (int r = 0; r < nr; ++r) {
                            const float x = Us[r * ld + pa[s]], y = Us[r * ld + pc[s]];
                            const float pr = x * y, pe = fmaf(x, y, -pr);
                            const float sm = hi + pr, bb = sm - hi;
                            lo += ((hi - (sm - bb)) + (pr - bb)) + pe;
                            hi = sm;
                        }
                        acc[s] += (TR)hi + (TR)lo;
                    } else {
                        TR sacc = 0;
                        for (int r = 0; r < nr; ++r) sacc += (TR)Us[r * ld + pa[s]] * (TR)Us[r * ld + pc[s]];
                        acc[s] += sacc;
                    }
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < k * ld; e += nt) se.A_T[e] = T(0);
        __syncthreads();
#pragma unroll
        for (int s = 0; s < npair_max; ++s) {
            if (tid + s * nt < np) {
                const TR h = acc[s] * (TR)sgs[pa[s]] * (TR)sgs[pc[s]];
                se.A_T[pa[s] * ld + pc[s]] = (T)h;
                se.A_T[pc[s] * ld + pa[s]] = (T)h;
                if (REF) {
                    se.A_R[pa[s] * ld + pc[s]] = (double)h;
                    se.A_R[pc[s] * ld + pa[s]] = (double)h;
                }
            }
        }
        __syncthreads();
        TR* Zo;
        TR* theta = reinterpret_cast<TR*>(es.theta);
        small_eig<T, REF>(se, ki, js, jd, theta, es.perm, Zo);
        // keep r = min(rows, ki) pairs (the rank of X U Sigma)
        const int r = min(br.hi - br.lo, ki);
        for (int j = tid; j < k; j += nt) {
            const T s = (j < r) ? zsqrt((T)fmax((double)theta[j], 0.0)) : T(0);
            st[j] = s;
        }
        __syncthreads();
        const T s0 = st[0];
        for (int j = tid; j < k; j += nt)
            if (!(st[j] > rank_tol<T>() * s0)) st[j] = T(0);
        __syncthreads();
        // slab rows of M
        T* Ms = (T*)a.M + (P.slab0 + t) * k * n;
        if constexpr (REF && std::is_same<T, float>::value) {
            // The FP64 eigenvectors split into two floats each (z = zh + zl to
            // ~2^-48 relative), columns in sorted order, in the FP32 tiles that
            // the eigensolver no longer needs; each dot product then runs at
            // the FP32 rate with the exact-product / TwoSum sum used for H above
            float* Zh = se.A_T;
            float* Zl = se.Z_T;
            for (int e = tid; e < ki * ki; e += nt) {
                const int aa = e / ki, j = e - (e / ki) * ki;
                const double z = Zo[aa * ld + es.perm[j]];
                const float h = (float)z;
                Zh[aa * ld + j] = h;
                Zl[aa * ld + j] = (float)(z - (double)h);
            }
            __syncthreads();
            for (int e = tid; e < k * n; e += nt) {
                const int j = e / n, l = e - (e / n) * n;
                float v = 0.f;
                if (st[j] > 0.f) {
                    float hi = 0.f, lo = 0.f;
                    for (int aa = 0; aa < ki; ++aa) {
                        const float x = vt[(int64_t)aa * n + l], zh = Zh[aa * ld + j];
                        const float pr = zh * x, pe = fmaf(zh, x, -pr);
                        const float sm = hi + pr, bb = sm - hi;
                        lo += ((hi - (sm - bb)) + (pr - bb)) + fmaf(Zl[aa * ld + j], x, pe);
                        hi = sm;
                    }
                    v = st[j] * (hi + lo);
                }
                Ms[e] = v;
            }
        } else {
            for (int e = tid; e < k * n; e += nt) {
                const int j = e / n, l = e - (e / n) * n;
                T v = T(0);
                if (st[j] > T(0)) {
                    TR accv = 0;
                    const int pj = es.perm[j];
                    for (int aa = 0; aa < ki; ++aa) accv += Zo[aa * ld + pj] * (TR)vt[(int64_t)aa * n + l];
                    v = st[j] * (T)accv;
                }
                Ms[e] = v;
            }
        }
        // lift coefficients Sigma V~ Sigma~^{-1}  (k x k)
        T* tc = (T*)a.tco + (int64_t)p * k * k;
        for (int e = tid; e < k * k; e += nt) {
            const int aa = e / k, j = e - (e / k) * k;
            T v = T(0);
            if (aa < ki && st[j] > T(0)) v = (T)((TR)sgs[aa] * Zo[aa * ld + es.perm[j]] / (TR)st[j]);
            tc[e] = v;
        }
        __syncthreads();
    }
}

// Stacked Sigma_i V_i^T of the interior blocks (Algorithm 2, stack step).
template <typename T>
__global__ void __launch_bounds__(256) k_stack(QueryArgs a) {
    const int nq = a.hdr->nq;
    const int64_t total = a.hdr->nslab_total;
    const int k = a.k, n = a.n;
    for (int64_t s = blockIdx.x; s < total; s += gridDim.x) {
        const int q = find_query(a.slab_prefix, nq, s);
        const QPlan& P = a.plans[q];
        const int t = (int)(s - P.slab0);
        if (t == 0 || t == P.nslab - 1) continue;
        const int blk = P.S + t;
        const T* sg = (const T*)a.sig + (int64_t)blk * k;
        const T* vt = (const T*)a.vt + (int64_t)blk * k * n;
        T* Ms = (T*)a.M + s * k * n;
        if constexpr (std::is_same<T, float>::value) {
            if ((n & 3) == 0) {
                // rows of n/4 float4 groups: row j scaled by sigma_j
                const int n4 = n >> 2;
                const float4* v4 = reinterpret_cast<const float4*>(vt);
                float4* m4 = reinterpret_cast<float4*>(Ms);
                const int tot = k * n4, stride = blockDim.x;
                // four loads in flight per thread before the stores
                for (int e0 = threadIdx.x; e0 < tot; e0 += 4 * stride) {
                    float4 v[4];
                    float sj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * stride;
                        if (e < tot) {
                            v[u] = __ldg(v4 + e);
                            sj[u] = __ldg(sg + e / n4);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * stride;
                        if (e < tot) m4[e] = make_float4(v[u].x * sj[u], v[u].y * sj[u], v[u].z * sj[u], v[u].w * sj[u]);
                    }
                }
                continue;
            }
        }
        for (int e = threadIdx.x; e < k * n; e += blockDim.x) Ms[e] = sg[e / n] * vt[e];
    }
}

// Stitched core: top-k_q eigenpairs of M^T M -> Sigma_r, V_r; results S, V.
template <typename T, bool REF, int MB>
__global__ void __launch_bounds__(256) k_eig_query(QueryArgs a, int m, int yglob, void* ws) {
    extern __shared__ __align__(16) char dsm[];
    __shared__ JacobiScratch<T> js;
    __shared__ JacobiScratch<double> jd;
    __shared__ EigStatic es;
    __shared__ int sgn[ZS_MAXM];
    __shared__ int s_rank;
    EigWork<T, REF> w;
    eig_carve<T, REF>(dsm, a.n, m, yglob != 0, ws, w);
    const int tid = threadIdx.x, nt = blockDim.x, n = a.n, kq = a.kq, kout = a.kout;
    const int nq = a.hdr->nq;
    using TR = typename Prec<T, REF>::TR;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const QPlan& P = a.plans[q];
        T* V;
        int ldv;
        eig_solve<T, REF, MB>((const T*)a.G + (int64_t)q * n * n, n, m, kq, w, js, jd, es, V, ldv);
        canon_signs<T>(V, ldv, n, kq, sgn);
        const TR* theta = reinterpret_cast<const TR*>(es.theta);
        const T s0 = zsqrt((T)fmax((double)theta[0], 0.0));
        T* sr = (T*)a.sr + (int64_t)q * kq;
        T* vr = (T*)a.vr + (int64_t)q * kq * n;
        if (tid == 0) s_rank = 0;
        __syncthreads();
        for (int c = tid; c < kout; c += nt) {
            T s = T(0);
            if (c < kq) {
                s = zsqrt((T)fmax((double)theta[c], 0.0));
                if (!(c < P.kcap && s > rank_tol<T>() * s0)) s = T(0);
                sr[c] = s;
            }
            ((T*)P.S_out)[c] = s;
            if (s > T(0)) atomicAdd(&s_rank, 1);
        }
        __syncthreads();
        for (int e = tid; e < n * kout; e += nt) {
            const int i = e / kout, c = e - (e / kout) * kout;
            T v = T(0);
            if (c < kq) {
                const T s = sr[c];
                v = (s > T(0)) ? (T)sgn[c] * V[i * ldv + c] : T(0);
                vr[(int64_t)c * n + i] = v;
            }
            ((T*)P.V_out)[(int64_t)i * P.ldv + c] = v;
        }
        if (tid == 0 && P.rank) *P.rank = s_rank;
        __syncthreads();
    }
}

// U_r = M V_r Sigma_r^{-1} per slab; boundary slabs are pre-multiplied by their
// Partial-SVD coefficient so that the lift is U_i(rows) C for every slab.
template <typename T>
__global__ void __launch_bounds__(256) k_ur(QueryArgs a) {
    extern __shared__ __align__(16) char dsm[];
    const int k = a.k, n = a.n, kq = a.kq, ldn = n + 1;
    T* Vr = (T*)dsm;                          // kq x (n+1)
    T* Ms = Vr + (size_t)kq * ldn;            // k x (n+1)
    T* Us = Ms + (size_t)k * ldn;             // k x kq
    T* Tc = Us + (size_t)k * kq;              // k x k
    __shared__ T srs[ZS_MAXM];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nq = a.hdr->nq;
    for (int q = blockIdx.x; q < nq; q += gridDim.x) {
        const QPlan& P = a.plans[q];
        const T* vr = (const T*)a.vr + (int64_t)q * kq * n;
        for (int e = tid; e < kq * n; e += nt) Vr[(e / n) * ldn + (e % n)] = vr[e];
        for (int e = tid; e < kq; e += nt) srs[e] = ((const T*)a.sr)[(int64_t)q * kq + e];
        __syncthreads();
        for (int t = 0; t < P.nslab; ++t) {
            const int64_t s = P.slab0 + t;
            const T* Mg = (const T*)a.M + s * k * n;
            for (int e = tid; e < k * n; e += nt) Ms[(e / n) * ldn + (e % n)] = Mg[e];
            const bool bnd = (t == 0) || (t == P.nslab - 1);
            if (bnd) {
                const int p = 2 * q + ((t == 0) ? 0 : 1);
                const T* tg = (const T*)a.tco + (int64_t)p * k * k;
                for (int e = tid; e < k * k; e += nt) Tc[e] = tg[e];
            }
            __syncthreads();
            for (int e = tid; e < k * kq; e += nt) {
                const int j = e / kq, c = e - (e / kq) * kq;
                T acc = 0;
                const T* mr = Ms + j * ldn;
                const T* vc = Vr + c * ldn;
                for (int l = 0; l < n; ++l) acc += mr[l] * vc[l];
                Us[e] = (srs[c] > T(0)) ? acc / srs[c] : T(0);
            }
            __syncthreads();
            T* Cg = (T*)a.C + s * k * kq;
            if (bnd) {
                for (int e = tid; e < k * kq; e += nt) {
                    const int aa = e / kq, c = e - (e / kq) * kq;
                    T acc = 0;
                    for (int j = 0; j < k; ++j) acc += Tc[aa * k + j] * Us[j * kq + c];
                    Cg[e] = acc;
                }
            } else {
                for (int e = tid; e < k * kq; e += nt) Cg[e] = Us[e];
            }
            __syncthreads();
        }
    }
}

// Lift (Eq. 9): output rows of each slab = U_i(rows) C_slab, zero past k_q.
// One warp per slab, one output row per lane: the warp keeps C_slab in its own
// shared-memory slice (read as warp-wide broadcasts), each lane reads its row
// of U_i (contiguous, vector loads) and writes its contiguous output row; RU
// rows per lane are in flight at once.  No CTA barrier: while one warp loads
// its next slab's coefficients the others stream rows.
template <typename T, int KMAX, int QMAX>
__global__ void __launch_bounds__(256) k_lift(QueryArgs a) {
    extern __shared__ __align__(16) char dsm[];
    const int k = a.k, kq = a.kq, kout = a.kout;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    T* Cs = (T*)dsm + (size_t)warp * KMAX * QMAX;
    const int nq = a.hdr->nq;
    const int64_t total = a.hdr->nslab_total, Trows = a.hdr->T;
    constexpr int RU = KMAX >= 64 ? 1 : (KMAX >= 32 ? 2 : 4);   // register budget
    for (int64_t s = (int64_t)blockIdx.x * wpc + warp; s < total; s += (int64_t)gridDim.x * wpc) {
        const int q = find_query(a.slab_prefix, nq, s);
        const QPlan& P = a.plans[q];
        const int t = (int)(s - P.slab0);
        const BlockRange br = slab_rows(P, t, a.b, Trows);
        const T* U = (const T*)a.U + (int64_t)br.blk * a.b * k;
        const T* Cg = (const T*)a.C + s * k * kq;
        __syncwarp();
        for (int e = lane; e < KMAX * QMAX; e += 32) {
            const int aa = e / QMAX, c = e % QMAX;
            Cs[e] = (aa < k && c < kq) ? Cg[aa * kq + c] : T(0);
        }
        __syncwarp();
        T* out = (T*)P.U;
        const int64_t o0 = (int64_t)br.blk * a.b - P.ts;
        const bool vec = (sizeof(T) == 4) && (k % 4 == 0) && (kout % 4 == 0) && (P.ldu % 4 == 0) &&
                         ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
        for (int r0 = br.lo + lane; r0 < br.hi; r0 += RU * 32) {
            T u[RU][KMAX];
#pragma unroll
            for (int x = 0; x < RU; ++x) {
                const int r = r0 + x * 32;
                const T* ur = U + (int64_t)r * k;
                if (vec) {
#pragma unroll
                    for (int j = 0; j < KMAX; j += 4) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (j < k && r < br.hi) v = __ldg(reinterpret_cast<const float4*>(ur + j));
                        u[x][j] = v.x; u[x][j + 1] = v.y; u[x][j + 2] = v.z; u[x][j + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < KMAX; ++j) u[x][j] = (j < k && r < br.hi) ? ur[j] : T(0);
                }
            }
#pragma unroll
            for (int x = 0; x < RU; ++x) {
                const int r = r0 + x * 32;
                if (r >= br.hi) break;
                T acc[QMAX];
#pragma unroll
                for (int c = 0; c < QMAX; ++c) acc[c] = T(0);
#pragma unroll
                for (int j = 0; j < KMAX; ++j) {
                    if (j >= k) break;
                    const T uj = u[x][j];
#pragma unroll
                    for (int c = 0; c < QMAX; ++c) acc[c] += uj * Cs[j * QMAX + c];
                }
                T* orow = out + (o0 + r) * P.ldu;
                if (vec) {
#pragma unroll
                    for (int c = 0; c < QMAX; c += 4) {
                        if (c >= kout) break;
                        *reinterpret_cast<float4*>(orow + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < QMAX; ++c)
                        if (c < kout) orow[c] = acc[c];
                }
            }
        }
    }
}

}  // namespace zs

#include "zs_tc_kernels.cuh"
#include "zs_certify.cuh"
