// zs_internal.h - structures shared by the kernels (zs_kernels_dev.cuh) and the host
// runtime (zs_api.cu, zs_serve.cpp).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

namespace zs {

enum InKind { IN_F64 = 0, IN_F32 = 1, IN_BF16 = 2 };

// Singular values at or below this fraction of sigma_1 are reported as zero
// (their U/V columns are zero and rank_out excludes them).
constexpr double kRankTolF64 = 1e-13;
constexpr float kRankTolF32 = 1e-7f;

// One storage-phase launch covers `nblk` consecutive blocks of b rows that start
// at row 0 of `A` (row stride lda, element type in_kind); the last of them may
// be short (rows_total - (nblk-1)*b rows).  Their factors go to store slots
// slot0 .. slot0+nblk-1.  G is scratch for nblk n x n Gram matrices.
struct CompressChunk {
    const void* A;
    int64_t lda;
    int64_t rows_total;
    int32_t nblk;
    int32_t slot0;
    int32_t b;
    int32_t n;
    int32_t k;
    int32_t in_kind;
    void* G;          // nblk * n * n accumulator type
    void* U;          // store: slot-major, b * k per slot
    void* sig;        // store: k per slot
    void* vt;         // store: k * n per slot
    void* w;          // store (tensor path, optional): Sigma V^T, k * n per slot
    void* ews;        // eigen-core workspace (ews_ctas CTAs x n x 65 elements)
    int32_t ews_ctas;
    void* qb;         // tensor path: nblk x n x m subspace bases (fp32 holding tf32 values)
    void* ys;         // tensor path: nblk x b x 64 floats (Y = X Q~)
    void* aux;        // tensor path: tc_aux_bytes(nblk, nblk*ceil(b/128), m, k)
    int* fault;       // device word set to 1 when a bounded wait gives up (or null)
    int* noconv;      // device count of blocks whose refinement stopped at its pass cap (or null)
    int* refined;     // device count of blocks that needed refinement (or null)
    double xi;        // > 0: energy rule of Eq. 1 per block (rank k_i <= k), else fixed k
    double* energy;   // xi > 0: nblk doubles of scratch (each block's squared Frobenius norm)
    int* kxi;         // xi > 0: nblk ints, each block's rank k_i as the accuracy test decided it
};

// Row-by-row storage (Algorithm 1 as printed, zs_rowappend.cu): blocks
// slot0 .. slot0 + nblk - 1 receive the rows_total rows at A (row stride lda,
// element type in_kind) in order; block slot0 already holds r0 rows (its
// factors are the state), the others start empty.  nblk > 1 needs r0 == 0.
struct RowAppendArgs {
    const void* A;
    int64_t lda;
    int64_t rows_total;
    int32_t nblk;
    int32_t slot0;
    int32_t r0;
    int32_t in_kind;
    int32_t b, n, k;
    void* U;          // store: slot-major, b * k per slot (factor type)
    void* sig;        // store: k per slot
    void* vt;         // store: k * n per slot
    void* w;          // store (tensor path, optional): Sigma V^T, k * n per slot
};
cudaError_t launch_row_append(const RowAppendArgs& a, bool fp64, cudaStream_t st);
size_t row_append_smem_bytes(int n, int k, bool fp64);

// Per-query plan of a batch (host-computed, then copied to the device).
// Reading R1: rows are 0-based, ranges inclusive; S = t_s / b, E = t_e / b.
struct QPlan {
    int64_t ts, te;
    int32_t S, E;
    int32_t nslab;        // E - S + 1 slabs of k rows in the stacked matrix M
    int32_t kcap;         // min(kq, structural rank of M)
    int64_t slab0;        // global index of this query's first slab
    // (pad0 below: first 128-row tile of this query's stacked matrix, tensor path)
    void* U;              // result buffers (caller device memory)
    int64_t ldu;
    void* S_out;
    void* V_out;
    int64_t ldv;
    int32_t* rank;
    int32_t pad0, pad1;
};

// Header of a query batch, read by the kernels from device memory so that one
// set of persistent launches (and one captured graph) serves any batch shape
// up to the executor's capacity.
struct BatchHdr {
    int32_t nq;
    int32_t pad;
    int64_t nslab_total;
    int64_t T;            // rows in the store when the batch was planned
    int64_t ntiles_total; // 128-row tiles of all stacked matrices (tensor path)
};

// Grid sizes of a query launch set: the actual batch (eager launches) or the
// executor's capacity (launches captured once into a CUDA graph and replayed).
struct QueryGrid {
    int nq;
    int64_t slabs;
    int64_t tiles;
    int max_rows;
};

// Device pointers of a store and its query scratch, passed by value.
struct QueryArgs {
    const BatchHdr* hdr;
    const QPlan* plans;
    const int64_t* slab_prefix;   // nq + 1 entries: plans[q].slab0, then total
    // store
    const void* U;
    const void* sig;
    const void* vt;
    const void* wst;  // tensor path: store Sigma V^T (interior slabs read from it), or null
    int64_t w_rows;   // rows allocated behind wst (capacity blocks x k)
    int32_t b, n, k;
    int32_t kq;                   // eigenpairs computed per query (= min(k_out, n))
    int32_t kout;
    int32_t fp64_refine;
    int32_t lift;     // 1: materialise U (the lift); 0: leave U factored as the per-slab coefficients C
    // scratch
    void* M;          // nslab_total * k * n     stacked Sigma_i V_i^T
    int64_t m_rows;   // rows allocated behind M (slab capacity x k)
    void* G;          // nq * n * n              Gram of M
    void* sr;         // nq * kq                 stitched singular values
    void* vr;         // nq * kq * n             stitched right vectors (transposed)
    void* tco;        // 2 * nq * k * k          Partial-SVD lift coefficients
    void* C;          // nslab_total * k * kq    lift coefficients per slab
    void* ews;        // eigen-core workspace (ews_ctas CTAs x n x 65 elements)
    int32_t ews_ctas;
    void* qb;         // tensor path: nq x n x m subspace bases (fp32 holding tf32 values)
    void* ys;         // tensor path: nslab_total x k x 64 floats (Y = M Q~)
    void* aux;        // tensor path: tc_aux_bytes(nq, aux_tiles, m, kq)
    int64_t aux_tiles;
    int* fault;       // device word set to 1 when a bounded wait gives up (or null)
    int* noconv;      // device count of queries whose refinement stopped at its pass cap (or null)
    int* refined;     // device count of queries that needed refinement (or null)
    // ragged stacks (energy-rule stores on the tensor path; else null): interior
    // slabs contribute only their live rows; kpre (blocks + 1) is the prefix of
    // the stored blocks' live ranks, formed at the start of each batch; rowmap
    // maps each stacked row to its source (>= 0: row of the store's Sigma V^T,
    // < 0: -1 - row of M), and the stitched U_r lands compact in Cc before it
    // is spread to C
    int64_t* kpre;
    int* rowmap;      // slab capacity x k ints, at slab0 * k per query
    void* Cc;         // slab capacity x k x kq
};

// Launch configuration chosen by the autotuner (or defaults).
struct Tuning {
    int gram_threads = 256;
    int lift_rows = 64;          // rows staged per lift tile
    int slab_ctas_per_sm = 4;    // persistent grid for slab work lists
    int eig_m_extra = 16;        // subspace oversampling p (m = kq + p)
    int power_its = 1;           // tensor path: power steps on the bf16 Gram
    int project_ctas_per_sm = 8; // persistent grid of the projection kernel
    int fused_sketch = 1;        // tensor path: sketch kernel (else the bf16 Gram) where it fits
    int pipe_sub_blocks = 0;     // tensor path: blocks per sub-chunk of the two-stream append pipeline (0: off)
    int tc5_project = 1;         // tensor path: projection on tcgen05 (TMEM accumulator) where it applies
};

// The tensor-core path (bf16 Gram for the subspace, split-bf16 projection and
// Rayleigh-Ritz for accuracy) serves float factor stores with n >= 64 (the
// subspace width m <= 64 must not exceed n) unless the store asks for the
// exact FP32 Gram.
inline bool use_tc_path(bool fp64, int n, int flags) { return !fp64 && n >= 64 && !(flags & 2); }
// Subspace width m = kq + p rounded up to 8: the oversampling p is `extra`,
// reduced (not below 8) where that keeps m <= 32, the width of the register
// Rayleigh-Ritz core.
inline int tc_width(int kq, int extra) {
    int p = extra;
    if (kq + p > 32) p = std::max(8, std::min(extra, 32 - kq));
    int m = ((kq + p) + 7) / 8 * 8;
    return m > 64 ? 64 : m;
}
// Floats of subspace-basis scratch per item on the tensor path: Q~ (n x m)
// followed, for the tcgen05 projection, by Q~^T as 32-column chunks in the
// canonical K-major layout (round16(m) x n).
inline size_t tc_qb_floats(int m, int n) { return (size_t)(m + (m + 15) / 16 * 16) * n; }

// Launchers (zs_launch_common.cu).  All enqueue on `st` and return cudaError_t of the
// launch.  `fp64` selects the double-precision instantiation (F64 store).
cudaError_t launch_compress(const CompressChunk& c, bool fp64, int flags, const Tuning& tu,
                            int num_sms, cudaStream_t st);
cudaError_t launch_query(const QueryArgs& a, bool fp64, const QueryGrid& g, int flags, const Tuning& tu,
                         int num_sms, cudaStream_t st);
struct EigPlan {
    int m = 0;          // subspace width (n for the dense path)
    bool yglob = false; // Y block in global workspace
    size_t smem = 0;    // dynamic shared memory bytes
    bool ok = false;
};
EigPlan eig_plan(int n, int kq, int extra, bool fp64, bool refine);
size_t eig_smem_bytes(int n, int m, bool fp64, bool refine, bool yglob);
size_t eig_ws_bytes(int n, bool fp64, int ctas);
size_t tc_aux_bytes(int64_t items, int64_t tiles, int m, int kw);
// the tensor path takes the sketch kernels (no shared per-CTA workspace) for
// this n and subspace width m
bool tc_sketch_path(int n, int m, int fused_sketch);
void note_launches(int64_t n);
void profile_enable(int on);
void profile_reset();
int profile_count();
bool profile_get(int i, const char** name, int64_t* launches, double* ms);
bool profiling_on();

}  // namespace zs
