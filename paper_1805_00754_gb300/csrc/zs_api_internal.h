// zs_api_internal.h - host-side store and executor types shared by zs_api.cu
// and zs_serve.cpp.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "zoomsvd.h"
#include "zs_internal.h"

namespace zs {

// Scratch and pinned plan staging for one stream of query batches.
struct QueryExec {
    int cap_nq = 0;
    int64_t cap_slabs = 0;
    int cap_kq = 0;
    void* d_blob = nullptr;       // BatchHdr | QPlan[] | prefix[]
    void* h_blob = nullptr;       // pinned mirror
    size_t blob_bytes = 0;
    void *M = nullptr, *G = nullptr, *sr = nullptr, *vr = nullptr, *tco = nullptr, *C = nullptr;
    void* ews = nullptr;
    int ews_ctas = 1;
    void* qb = nullptr;
    void* ys = nullptr;
    void* aux = nullptr;
    int64_t aux_tiles = 0;
    void* rowmap = nullptr;       // ragged stacks (energy-rule stores): cap_slabs x k ints
    void* Cc = nullptr;           // ragged stacks: compact U_r, cap_slabs x k x cap_kq
    void* kpre = nullptr;         // ragged stacks: prefix of the blocks' live ranks (store capacity + 1)
    cudaEvent_t done = nullptr;   // last batch that used this scratch
    // one captured launch set (plan upload + all query kernels) for this
    // executor's capacity, replayed for every batch that fits it
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int g_kq = -1, g_kout = -1, g_lift = -1, g_ragged = -1;
    int w_kq = -1, w_kout = -1, w_lift = -1;   // shape of the last eager batch
    int64_t g_launches = 0;
    ~QueryExec();
    void release();
    zs_status reserve(const zs_store& st, int nq, int64_t nslab, int kq);
    static size_t bytes_for(const zs_store& st, int nq, int64_t nslab, int kq);
};

zs_status fail(zs_status s, const char* fmt, ...);
zs_status cuda_fail(cudaError_t e, const char* what);
zs_status plan_queries(const zs_store& st, int64_t Trows, const int64_t* ts, const int64_t* te, int nq, int kq,
                       std::vector<QPlan>& plans, std::vector<int64_t>& prefix);
// coef != null: U stays factored; the batch's per-slab coefficients (nslab
// * k rows of kout) are copied to coef (device, factor type) from row coef_row0
zs_status run_batch(zs_store& st, QueryExec& x, int64_t Trows, std::vector<QPlan>& plans,
                    std::vector<int64_t>& prefix, int kq, int kout, cudaStream_t stream, void* coef = nullptr,
                    int64_t coef_row0 = 0);
zs_status query_batch_locked(zs_store* st, QueryExec& x, const int64_t* ts, const int64_t* te, int nq, int kout,
                             const zs_result* res, cudaStream_t stream, int64_t Trows, void* coef = nullptr,
                             int64_t coef_rows = 0);

}  // namespace zs

struct zs_store {
    zs_store_config cfg;
    bool fp64 = false;
    int tsize = 4;                 // factor element bytes
    int insize = 4;                // input element bytes
    int num_sms = 1;
    int64_t T = 0;                 // rows appended (published)
    int64_t cap_blocks = 0;
    void* U = nullptr;             // cap_blocks x b x k
    void* sig = nullptr;           // cap_blocks x k
    void* vt = nullptr;            // cap_blocks x k x n
    void* w = nullptr;             // tensor path: cap_blocks x k x n, Sigma V^T (the stack-ready slabs)
    int* d_fault = nullptr;        // device fault word (bounded waits that gave up)
    double xi = 0.0;               // > 0: energy rule (Eq. 1) picks each block's rank <= k
    double* d_energy = nullptr;    // xi > 0: per slot ||X_i||_F^2 (cap_blocks doubles)
    int* d_rank = nullptr;         // xi > 0: per slot rank k_i as the accuracy test decided it
    void* tail = nullptr;          // b x n raw rows of the open block
    void* gscr = nullptr;          // gchunk x n x n Gram scratch
    void* ews = nullptr;           // eigen-core workspace
    int ews_ctas = 1;
    void* qb = nullptr;            // tensor path: subspace bases (gchunk x n x m, tf32 values)
    void* ys = nullptr;            // tensor path: projections (gchunk x b x m float)
    void* aux = nullptr;           // tensor path: Rayleigh-Ritz scratch
    int gchunk = 1;
    size_t gram_budget = (size_t)512 << 20;    // per-chunk scratch: Gram + bases + projections
    void* stage[2] = {nullptr, nullptr};
    int stage_blocks = 1;
    size_t stage_budget = (size_t)256 << 20;
    size_t query_budget = (size_t)8 << 30;
    bool use_graphs = true;        // replay query batches as one captured CUDA graph
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    cudaEvent_t stage_full[2] = {nullptr, nullptr};
    cudaEvent_t append_done = nullptr;
    cudaEvent_t entry = nullptr;
    // appends whose device work may still run: (first row of the first block
    // they (re)write, completion event).  A query waits only for those whose
    // blocks it reads.
    std::vector<std::pair<int64_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> event_pool;
    // append pipeline: a short append of whole blocks is staged block by block
    // into one of kPipe slots, each compressed on its own stream with its own
    // one-block scratch, so consecutive small appends overlap on the device
    static constexpr int kPipe = 4;
    struct PipeSlot {
        cudaStream_t stream = nullptr;
        cudaEvent_t staged = nullptr;     // rows copied into stage
        cudaEvent_t free = nullptr;       // compression of the slot finished
        void* stage = nullptr;            // b x n input rows
        void *G = nullptr, *qb = nullptr, *ys = nullptr, *aux = nullptr, *ews = nullptr;
    } pipe[kPipe];
    int pipe_next = 0;
    // chunk pipeline of large device appends on the tensor path: sub-chunks of
    // `sub_blocks` blocks alternate between two streams, each with its own half
    // of the chunk scratch, so that one sub-chunk's latency-bound kernels
    // overlap the next one's streaming passes
    cudaStream_t cstream[2] = {nullptr, nullptr};
    cudaEvent_t cfork = nullptr;
    cudaEvent_t cjoin[2] = {nullptr, nullptr};
    int sub_blocks = 0;             // 0: no chunk pipeline
    size_t aux_region = 0;          // bytes of Rayleigh-Ritz scratch per half
    std::mutex mu;
    zs::Tuning tune;
    zs::QueryExec qx;
};
