// zs_api.cu - host runtime behind the C ABI in include/zoomsvd.h: the device
// store (Def. 2), the storage-phase driver (Algorithm 1 block by block, with
// double-buffered host->device staging), query planning (Algorithm 3's index
// arithmetic) and the batch executor that runs the query kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zoomsvd.h"
#include "zs_api_internal.h"
#include "zs_internal.h"

namespace zs {
int64_t launch_count_total();
void tune_cache_load(zs_store* st);
void prune_pending(zs_store* st);

thread_local std::string g_last_error;

zs_status fail(zs_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

zs_status cuda_fail(cudaError_t e, const char* what) {
    return fail(ZS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ZS_CU(call, what)                                     \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev_) cudaSetDevice(prev_);
    }

   private:
    int prev_ = 0;
};

static size_t in_size(int dt) { return dt == ZS_F64 ? 8 : (dt == ZS_F32 ? 4 : 2); }

// ---------------------------------------------------------------------------
// Query executor: scratch + pinned staging for one stream of batches.
// ---------------------------------------------------------------------------
QueryExec::~QueryExec() { release(); }

void QueryExec::release() {
    auto f = [](void*& p) { if (p) cudaFree(p); p = nullptr; };
    auto fh = [](void*& p) { if (p) cudaFreeHost(p); p = nullptr; };
    if (done) { cudaEventSynchronize(done); cudaEventDestroy(done); done = nullptr; }
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    if (cap_stream) { cudaStreamDestroy(cap_stream); cap_stream = nullptr; }
    g_kq = g_kout = -1;
    g_ragged = -1;
    w_kq = w_kout = -1;
    f(d_blob); f(M); f(G); f(sr); f(vr); f(tco); f(C); f(ews); f(qb); f(ys); f(aux); f(rowmap); f(Cc); f(kpre);
    fh(h_blob);
    cap_nq = 0;
    cap_slabs = 0;
}

zs_status QueryExec::reserve(const zs_store& st, int nq, int64_t nslab, int kq) {
    const size_t ts = st.tsize;
    const int64_t n = st.cfg.n, k = st.cfg.k;
    if (nq <= cap_nq && nslab <= cap_slabs && kq <= cap_kq) return ZS_OK;
    // grow geometrically
    const int want_nq = std::max(nq, std::max(cap_nq * 3 / 2, 16));
    const int64_t want_sl = std::max(nslab, std::max(cap_slabs * 3 / 2, (int64_t)64));
    const int want_kq = std::max(kq, cap_kq);
    if (done) cudaEventSynchronize(done);
    release();
    ZS_CU(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "event");
    ZS_CU(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking), "capture stream");
    const size_t blob = ((sizeof(BatchHdr) + 15) & ~size_t(15)) + sizeof(QPlan) * want_nq +
                        sizeof(int64_t) * (want_nq + 1) + 256;
    ZS_CU(cudaMalloc(&d_blob, blob), "query plan buffer");
    ZS_CU(cudaMallocHost(&h_blob, blob), "pinned plan buffer");
    blob_bytes = blob;
    auto al = [](void** p, size_t bytes, const char* what) -> zs_status {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(ZS_ENOMEM, "query scratch (%s): %s", what, cudaGetErrorString(e)); }
        return ZS_OK;
    };
    zs_status s;
    if ((s = al(&M, ts * want_sl * k * n, "stack")) != ZS_OK) return s;
    if ((s = al(&G, ts * (size_t)want_nq * n * n, "gram")) != ZS_OK) return s;
    if ((s = al(&sr, ts * (size_t)want_nq * want_kq, "sigma")) != ZS_OK) return s;
    if ((s = al(&vr, ts * (size_t)want_nq * want_kq * n, "v")) != ZS_OK) return s;
    if ((s = al(&tco, ts * (size_t)2 * want_nq * k * k, "partial")) != ZS_OK) return s;
    if ((s = al(&C, ts * want_sl * k * want_kq, "lift coeff")) != ZS_OK) return s;
    ews_ctas = std::max(1, st.num_sms) * (st.fp64 ? 1 : 2);   // float: two subspace CTAs per SM
    aux_tiles = (int64_t)want_sl * k / 128 + want_nq;
    if ((s = al(&ews, eig_ws_bytes((int)n, st.fp64, ews_ctas), "eigen workspace")) != ZS_OK) return s;
    if (use_tc_path(st.fp64, (int)n, st.cfg.flags)) {
        const size_t m = tc_width(want_kq, st.tune.eig_m_extra);
        if ((s = al(&qb, 4 * tc_qb_floats((int)m, (int)n) * want_nq, "subspace bases")) != ZS_OK) return s;
        if ((s = al(&ys, 4 * m * (size_t)want_sl * k, "projections")) != ZS_OK) return s;
        aux_tiles = (int64_t)want_sl * k / 128 + want_nq;
        if ((s = al(&aux, tc_aux_bytes(want_nq, aux_tiles, (int)m, want_kq), "Rayleigh-Ritz scratch")) != ZS_OK)
            return s;
    }
    cap_nq = want_nq;
    cap_slabs = want_sl;
    cap_kq = want_kq;
    return ZS_OK;
}

size_t QueryExec::bytes_for(const zs_store& st, int nq, int64_t nslab, int kq) {
    const size_t ts = st.tsize;
    const size_t n = st.cfg.n, k = st.cfg.k;
    const size_t m = 64;
    return tc_aux_bytes(nq, (int64_t)nslab * k / 128 + nq, 64, kq) + ts * (nslab * k * n + (size_t)nq * n * n + (size_t)nq * kq * (n + 1) + 2 * (size_t)nq * k * k +
                 nslab * k * kq + nslab * k * m + (size_t)nq * n * m) + sizeof(QPlan) * nq;
}

// Drop the appends that have finished on the device.
void prune_pending(zs_store* st) {
    size_t keep = 0;
    for (size_t i = 0; i < st->pending.size(); ++i) {
        const cudaError_t q = cudaEventQuery(st->pending[i].second);
        if (q == cudaSuccess) {
            st->event_pool.push_back(st->pending[i].second);
            continue;
        }
        if (q != cudaErrorNotReady) cudaGetLastError();
        st->pending[keep++] = st->pending[i];
    }
    st->pending.resize(keep);
}

// ---------------------------------------------------------------------------
// Planning (Algorithm 3, first steps; reading R1: 0-based inclusive ranges).
// ---------------------------------------------------------------------------
zs_status plan_queries(const zs_store& st, int64_t Trows, const int64_t* ts, const int64_t* te, int nq,
                       int kq, std::vector<QPlan>& plans, std::vector<int64_t>& prefix) {
    const int64_t b = st.cfg.b, n = st.cfg.n, k = st.cfg.k;
    plans.resize(nq);
    prefix.resize(nq + 1);
    int64_t slab = 0;
    for (int q = 0; q < nq; ++q) {
        if (ts[q] < 0 || ts[q] > te[q] || te[q] >= Trows)
            return fail(ZS_ERANGE, "query %d: range [%lld, %lld] outside [0, %lld)", q, (long long)ts[q],
                        (long long)te[q], (long long)Trows);
        QPlan& P = plans[q];
        memset(&P, 0, sizeof P);
        P.ts = ts[q];
        P.te = te[q];
        P.S = (int32_t)(ts[q] / b);
        P.E = (int32_t)(te[q] / b);
        P.nslab = P.E - P.S + 1;
        P.slab0 = slab;
        prefix[q] = slab;
        slab += P.nslab;
        // structural rank of the stacked matrix: sum of slab ranks
        auto rows_of = [&](int64_t i) { return std::min<int64_t>(b, Trows - i * b); };
        auto ki = [&](int64_t i) { return std::min<int64_t>(k, std::min<int64_t>(rows_of(i), n)); };
        int64_t reff;
        if (P.nslab == 1) {
            reff = std::min<int64_t>(te[q] - ts[q] + 1, ki(P.S));
        } else {
            const int64_t rS = rows_of(P.S) - (ts[q] - (int64_t)P.S * b);
            const int64_t rE = te[q] - (int64_t)P.E * b + 1;
            reff = std::min(rS, ki(P.S)) + std::min(rE, ki(P.E)) + (int64_t)(P.nslab - 2) * ki(P.S + 1);
        }
        P.kcap = (int32_t)std::min<int64_t>(kq, reff);
    }
    prefix[nq] = slab;
    return ZS_OK;
}

// Run one planned batch on `stream` with executor `x`.  Results go to the
// buffers recorded in plans.
zs_status run_batch(zs_store& st, QueryExec& x, int64_t Trows, std::vector<QPlan>& plans,
                    std::vector<int64_t>& prefix, int kq, int kout, cudaStream_t stream, void* coef,
                    int64_t coef_row0) {
    const int lift = coef ? 0 : 1;
    const int nq = (int)plans.size();
    const int64_t nslab = prefix[nq];
    zs_status s = x.reserve(st, nq, nslab, kq);
    if (s != ZS_OK) return s;
    // the pinned plan buffer may still be read by the previous batch's copy
    ZS_CU(cudaEventSynchronize(x.done), "plan buffer wait");
    char* hb = (char*)x.h_blob;
    BatchHdr* hh = (BatchHdr*)hb;
    hh->nq = nq;
    hh->pad = 0;
    hh->nslab_total = nslab;
    hh->T = Trows;
    int64_t ntiles = 0;   // first 128-row tile of each query's stacked matrix
    for (QPlan& P : plans) {
        P.pad0 = (int32_t)ntiles;
        ntiles += ((int64_t)P.nslab * st.cfg.k + 127) / 128;
    }
    hh->ntiles_total = ntiles;
    // fixed offsets (by capacity): a captured graph bakes these pointers in
    const size_t o_plans = (sizeof(BatchHdr) + 15) & ~size_t(15);
    const size_t o_pref = o_plans + sizeof(QPlan) * x.cap_nq;
    memcpy(hb + o_plans, plans.data(), sizeof(QPlan) * nq);
    memcpy(hb + o_pref, prefix.data(), sizeof(int64_t) * (nq + 1));
    const size_t bytes = o_pref + sizeof(int64_t) * (nq + 1);
    QueryArgs a;
    memset(&a, 0, sizeof a);
    char* db = (char*)x.d_blob;
    a.hdr = (const BatchHdr*)db;
    a.plans = (const QPlan*)(db + o_plans);
    a.slab_prefix = (const int64_t*)(db + o_pref);
    a.U = st.U;
    a.sig = st.sig;
    a.vt = st.vt;
    a.wst = st.w;
    a.w_rows = st.cap_blocks * st.cfg.k;
    a.fault = st.d_fault;
    a.noconv = st.d_fault + 2;
    a.refined = st.d_fault + 4;
    a.b = (int32_t)st.cfg.b;
    a.n = (int32_t)st.cfg.n;
    a.k = st.cfg.k;
    a.kq = kq;
    a.kout = kout;
    a.fp64_refine = (st.cfg.flags & ZS_FLAG_FP64_REFINE) ? 1 : 0;
    a.lift = lift;
    a.M = x.M;
    a.m_rows = x.cap_slabs * st.cfg.k;
    a.G = x.G;
    a.sr = x.sr;
    a.vr = x.vr;
    a.tco = x.tco;
    a.C = x.C;
    a.ews = x.ews;
    a.ews_ctas = x.ews_ctas;
    a.qb = x.qb;
    a.ys = x.ys;
    a.aux = x.aux;
    a.aux_tiles = x.aux_tiles;
    // ragged stacks on energy-rule stores of the tensor path (interior slabs
    // contribute their live rows only)
    const int ragged = (st.xi > 0.0 && st.w && use_tc_path(st.fp64, (int)st.cfg.n, st.cfg.flags)) ? 1 : 0;
    if (ragged && !x.rowmap) {
        const size_t rows = (size_t)x.cap_slabs * st.cfg.k;
        cudaError_t e = cudaMalloc(&x.rowmap, std::max<size_t>(4 * rows, 256));
        if (e == cudaSuccess) e = cudaMalloc(&x.Cc, std::max<size_t>(st.tsize * rows * x.cap_kq, 256));
        if (e == cudaSuccess) e = cudaMalloc(&x.kpre, sizeof(int64_t) * (size_t)(st.cap_blocks + 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (x.rowmap) cudaFree(x.rowmap);
            if (x.Cc) cudaFree(x.Cc);
            x.rowmap = x.Cc = nullptr;
            return fail(ZS_ENOMEM, "query scratch (ragged stack row map)");
        }
    }
    if (ragged) {
        a.kpre = (int64_t*)x.kpre;
        a.rowmap = (int*)x.rowmap;
        a.Cc = x.Cc;
    }
    int max_rows = 0;
    for (const QPlan& P : plans) max_rows = std::max(max_rows, P.nslab * (int)st.cfg.k);
    // the first batch of a (k_q, k_out) shape runs eagerly (it also sets the
    // kernels' attributes); later ones replay a captured graph
    const bool warm = (x.w_kq == kq && x.w_kout == kout && x.w_lift == lift && x.g_ragged == ragged);
    if (profiling_on() || !st.use_graphs || !warm) {
        x.w_kq = kq;
        x.w_kout = kout;
        x.w_lift = lift;
        if (x.g_ragged != ragged && x.gexec) { cudaGraphExecDestroy(x.gexec); x.gexec = nullptr; }
        x.g_ragged = ragged;
        // eager: grids sized to this batch (the profiler brackets each launch)
        ZS_CU(cudaMemcpyAsync(x.d_blob, x.h_blob, bytes, cudaMemcpyHostToDevice, stream), "plan upload");
        QueryGrid g{nq, nslab, ntiles, max_rows};
        cudaError_t e = launch_query(a, st.fp64, g, st.cfg.flags, st.tune, st.num_sms, stream);
        if (e != cudaSuccess) return cuda_fail(e, "query kernels");
    } else {
        if (!x.gexec || x.g_kq != kq || x.g_kout != kout || x.g_lift != lift) {
            if (x.gexec) { cudaGraphExecDestroy(x.gexec); x.gexec = nullptr; }
            // capture the plan upload (whole buffer) and the kernels, with
            // grids sized to the executor's capacity
            const int64_t l0 = launch_count_total();
            ZS_CU(cudaStreamBeginCapture(x.cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t e = cudaMemcpyAsync(x.d_blob, x.h_blob, x.blob_bytes, cudaMemcpyHostToDevice, x.cap_stream);
            QueryGrid g{x.cap_nq, x.cap_slabs, x.aux_tiles, 0};
            if (e == cudaSuccess) e = launch_query(a, st.fp64, g, st.cfg.flags, st.tune, st.num_sms, x.cap_stream);
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(x.cap_stream, &graph);
            if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "query kernels (capture)"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
            e = cudaGraphInstantiate(&x.gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { x.gexec = nullptr; return cuda_fail(e, "graph instantiate"); }
            x.g_kq = kq;
            x.g_kout = kout;
            x.g_lift = lift;
            x.g_launches = launch_count_total() - l0;
            note_launches(-x.g_launches);   // counted when replayed
        }
        ZS_CU(cudaGraphLaunch(x.gexec, stream), "graph launch");
        note_launches(x.g_launches);
    }
    if (coef) {
        // the factored U: every slab's coefficients (stored U rows x C = the
        // answer's rows in that block), k rows per slab, kout columns
        const size_t ts = st.tsize;
        char* dst = (char*)coef + ts * (size_t)coef_row0 * kout;
        const int64_t rows = nslab * st.cfg.k;
        ZS_CU(cudaMemcpy2DAsync(dst, ts * kout, x.C, ts * kq, ts * kq, rows, cudaMemcpyDeviceToDevice, stream),
              "coefficient copy");
        if (kout > kq)
            ZS_CU(cudaMemset2DAsync(dst + ts * kq, ts * kout, 0, ts * (kout - kq), rows, stream), "coefficient pad");
    }
    ZS_CU(cudaEventRecord(x.done, stream), "event record");
    return ZS_OK;
}

}  // namespace zs

using namespace zs;

// ---------------------------------------------------------------------------
// Store lifetime.
// ---------------------------------------------------------------------------
static zs_status store_alloc(zs_store* st) {
    const zs_store_config& c = st->cfg;
    const size_t ts = st->tsize;
    st->cap_blocks = (c.capacity_rows + c.b - 1) / c.b;
    const size_t nb = (size_t)std::max<int64_t>(st->cap_blocks, 1);
    auto al = [&](void** p, size_t bytes, const char* what) -> zs_status {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(ZS_ENOMEM, "%s (%zu bytes): %s", what, bytes, cudaGetErrorString(e)); }
        return ZS_OK;
    };
    zs_status s;
    if ((s = al(&st->U, ts * nb * c.b * c.k, "store U")) != ZS_OK) return s;
    if ((s = al(&st->sig, ts * nb * c.k, "store sigma")) != ZS_OK) return s;
    if ((s = al(&st->vt, ts * nb * c.k * c.n, "store V")) != ZS_OK) return s;
    if (use_tc_path(st->fp64, (int)c.n, c.flags))
        if ((s = al(&st->w, ts * nb * c.k * c.n, "store Sigma V^T")) != ZS_OK) return s;
    // status words: [0] fault (a bounded wait gave up), [1] blocks and [2]
    // queries whose refinement stopped at its pass cap, [3] blocks and [4]
    // queries that needed refinement
    if ((s = al((void**)&st->d_fault, 8 * sizeof(int), "status words")) != ZS_OK) return s;
    ZS_CU(cudaMemset(st->d_fault, 0, 8 * sizeof(int)), "memset");
    if ((s = al(&st->tail, st->insize * (size_t)c.b * c.n, "open-block rows")) != ZS_OK) return s;
    // Gram scratch: chunk of blocks whose n x n Grams stay L2-sized
    const size_t gper = ts * (size_t)c.n * c.n;
    const size_t mtc = use_tc_path(st->fp64, (int)c.n, c.flags) ? tc_width(c.k, st->tune.eig_m_extra) : 0;
    const size_t per_block = gper + (mtc ? 4 * tc_qb_floats((int)mtc, (int)c.n) : 0) + 4 * mtc * c.b +
                             (mtc ? 4 * mtc * mtc * ((c.b + 127) / 128 + 1) + 4 * mtc * c.k + 4 * c.k : 0);
    st->gchunk = (int)std::max<size_t>(1, std::min<size_t>(st->gram_budget / per_block, 65535));
    if ((s = al(&st->gscr, gper * st->gchunk, "gram scratch")) != ZS_OK) return s;
    if (use_tc_path(st->fp64, (int)c.n, c.flags)) {
        const size_t m = tc_width(c.k, st->tune.eig_m_extra);
        if ((s = al(&st->qb, 4 * tc_qb_floats((int)m, (int)c.n) * st->gchunk, "subspace bases")) != ZS_OK)
            return s;
        if ((s = al(&st->ys, 4 * m * (size_t)c.b * st->gchunk, "projections")) != ZS_OK) return s;
        if ((s = al(&st->aux, tc_aux_bytes(st->gchunk, (int64_t)st->gchunk * ((c.b + 127) / 128), (int)m, c.k),
                    "Rayleigh-Ritz scratch")) != ZS_OK)
            return s;
    }
    st->ews_ctas = std::max(1, st->num_sms) * (st->fp64 ? 1 : 2);   // float: two subspace CTAs per SM
    if ((s = al(&st->ews, eig_ws_bytes((int)c.n, st->fp64, st->ews_ctas), "eigen workspace")) != ZS_OK) return s;
    // host staging: two device buffers of whole blocks
    const size_t blk_bytes = st->insize * (size_t)c.b * c.n;
    st->stage_blocks = (int)std::max<size_t>(1, std::min<size_t>(st->stage_budget / blk_bytes, st->gchunk));
    for (int i = 0; i < 2; ++i)
        if ((s = al(&st->stage[i], blk_bytes * st->stage_blocks, "host staging")) != ZS_OK) return s;
    // append pipeline slots: one block of staging and scratch each
    {
        const size_t mt = use_tc_path(st->fp64, (int)c.n, c.flags) ? tc_width(c.k, st->tune.eig_m_extra) : 0;
        for (int i = 0; i < zs_store::kPipe; ++i) {
            auto& ps = st->pipe[i];
            if ((s = al(&ps.stage, blk_bytes, "append pipeline staging")) != ZS_OK) return s;
            if ((s = al(&ps.G, gper, "append pipeline gram")) != ZS_OK) return s;
            if ((s = al(&ps.ews, eig_ws_bytes((int)c.n, st->fp64, 1), "append pipeline workspace")) != ZS_OK) return s;
            if (mt) {
                if ((s = al(&ps.qb, 4 * tc_qb_floats((int)mt, (int)c.n), "append pipeline bases")) != ZS_OK)
                    return s;
                if ((s = al(&ps.ys, 4 * mt * (size_t)c.b, "append pipeline projections")) != ZS_OK) return s;
                if ((s = al(&ps.aux, tc_aux_bytes(1, (c.b + 127) / 128, (int)mt, c.k), "append pipeline RR")) != ZS_OK)
                    return s;
            }
            ZS_CU(cudaStreamCreateWithFlags(&ps.stream, cudaStreamNonBlocking), "stream");
            ZS_CU(cudaEventCreateWithFlags(&ps.staged, cudaEventDisableTiming), "event");
            ZS_CU(cudaEventCreateWithFlags(&ps.free, cudaEventDisableTiming), "event");
            ZS_CU(cudaEventRecord(ps.free, ps.stream), "event");
        }
    }
    ZS_CU(cudaMemset(st->U, 0, ts * nb * c.b * c.k), "memset");
    ZS_CU(cudaMemset(st->sig, 0, ts * nb * c.k), "memset");
    ZS_CU(cudaMemset(st->vt, 0, ts * nb * c.k * c.n), "memset");
    if (st->w) ZS_CU(cudaMemset(st->w, 0, ts * nb * c.k * c.n), "memset");
    ZS_CU(cudaStreamCreateWithFlags(&st->copy_stream, cudaStreamNonBlocking), "stream");
    // chunk pipeline (tensor path with the sketch kernel: no shared per-CTA workspace)
    if (use_tc_path(st->fp64, (int)c.n, c.flags) &&
        tc_sketch_path((int)c.n, tc_width(c.k, st->tune.eig_m_extra), st->tune.fused_sketch) && st->gchunk >= 2 &&
        st->tune.pipe_sub_blocks > 0) {
        const int m = tc_width(c.k, st->tune.eig_m_extra);
        const int sub = std::min(st->gchunk / 2, st->tune.pipe_sub_blocks);
        const int64_t tpb = (c.b + 127) / 128;
        const size_t region = (tc_aux_bytes(sub, (int64_t)sub * tpb, m, c.k) + 255) & ~(size_t)255;
        if (2 * region <= tc_aux_bytes(st->gchunk, (int64_t)st->gchunk * tpb, m, c.k)) {
            st->sub_blocks = sub;
            st->aux_region = region;
            for (int i = 0; i < 2; ++i) {
                ZS_CU(cudaStreamCreateWithFlags(&st->cstream[i], cudaStreamNonBlocking), "stream");
                ZS_CU(cudaEventCreateWithFlags(&st->cjoin[i], cudaEventDisableTiming), "event");
            }
            ZS_CU(cudaEventCreateWithFlags(&st->cfork, cudaEventDisableTiming), "event");
        }
    }
    for (int i = 0; i < 2; ++i) {
        ZS_CU(cudaEventCreateWithFlags(&st->stage_free[i], cudaEventDisableTiming), "event");
        ZS_CU(cudaEventCreateWithFlags(&st->stage_full[i], cudaEventDisableTiming), "event");
        ZS_CU(cudaEventRecord(st->stage_free[i], st->copy_stream), "event");
    }
    ZS_CU(cudaEventCreateWithFlags(&st->append_done, cudaEventDisableTiming), "event");
    ZS_CU(cudaEventCreateWithFlags(&st->entry, cudaEventDisableTiming), "event");
    ZS_CU(cudaEventRecord(st->append_done, st->copy_stream), "event");
    ZS_CU(cudaDeviceSynchronize(), "store init");
    return ZS_OK;
}

extern "C" zs_status zs_store_create(const zs_store_config* cfg, zs_store** out) {
    if (!cfg || !out) return fail(ZS_EINVAL, "null argument");
    *out = nullptr;
    const zs_store_config& c = *cfg;
    if (c.in_dtype != ZS_F64 && c.in_dtype != ZS_F32 && c.in_dtype != ZS_BF16)
        return fail(ZS_EDTYPE, "unknown in_dtype %d", c.in_dtype);
    if (c.n < 1 || c.n > 1024 || c.b < 1 || c.k < 1 || c.k > 64 || c.k > c.n || c.capacity_rows < 1 ||
        c.b > (int64_t)1 << 24)
        return fail(ZS_EINVAL, "bad store config (n=%lld b=%lld k=%d capacity=%lld)", (long long)c.n,
                    (long long)c.b, c.k, (long long)c.capacity_rows);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return fail(ZS_ECUDA, "device %d not available", c.device);
    }
    const bool fp64 = (c.in_dtype == ZS_F64);
    const bool ref = (c.flags & ZS_FLAG_FP64_REFINE) && !fp64;
    if (!eig_plan((int)c.n, c.k, 16, fp64, ref).ok)
        return fail(ZS_EINVAL, "n=%lld with k=%d does not fit the eigen core's shared memory", (long long)c.n, c.k);
    if ((c.flags & ZS_FLAG_ROW_APPEND) && row_append_smem_bytes((int)c.n, c.k, fp64) > 227 * 1024)
        return fail(ZS_EINVAL, "row-by-row storage needs %zu bytes of shared memory for n=%lld, k=%d (227 KB at most)",
                    row_append_smem_bytes((int)c.n, c.k, fp64), (long long)c.n, c.k);
    DeviceGuard g(c.device);
    zs_store* st = new zs_store();
    st->cfg = c;
    st->fp64 = fp64;
    st->tsize = fp64 ? 8 : 4;
    st->insize = in_size(c.in_dtype);
    cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, c.device);
    tune_cache_load(st);
    zs_status s = store_alloc(st);
    if (s != ZS_OK) {
        zs_store_destroy(st);
        return s;
    }
    *out = st;
    return ZS_OK;
}

extern "C" void zs_store_destroy(zs_store* st) {
    if (!st) return;
    DeviceGuard g(st->cfg.device);
    if (st->copy_stream) cudaStreamSynchronize(st->copy_stream);
    for (int i = 0; i < 2; ++i)
        if (st->cstream[i]) cudaStreamSynchronize(st->cstream[i]);
    cudaDeviceSynchronize();
    st->qx.release();
    auto f = [](void*& p) { if (p) cudaFree(p); p = nullptr; };
    f(st->U); f(st->sig); f(st->vt); f(st->w); if (st->d_fault) cudaFree(st->d_fault); f(st->tail); f(st->gscr); f(st->stage[0]); f(st->stage[1]); f(st->ews);
    f(st->qb); f(st->ys); f(st->aux);
    if (st->d_energy) cudaFree(st->d_energy);
    if (st->d_rank) cudaFree(st->d_rank);
    for (int i = 0; i < 2; ++i) {
        if (st->stage_free[i]) cudaEventDestroy(st->stage_free[i]);
        if (st->stage_full[i]) cudaEventDestroy(st->stage_full[i]);
    }
    for (auto& ps : st->pipe) {
        if (ps.stream) cudaStreamSynchronize(ps.stream);
        f(ps.stage); f(ps.G); f(ps.qb); f(ps.ys); f(ps.aux); f(ps.ews);
        if (ps.staged) cudaEventDestroy(ps.staged);
        if (ps.free) cudaEventDestroy(ps.free);
        if (ps.stream) cudaStreamDestroy(ps.stream);
    }
    for (auto& pe : st->pending) cudaEventDestroy(pe.second);
    for (auto e : st->event_pool) cudaEventDestroy(e);
    if (st->append_done) cudaEventDestroy(st->append_done);
    if (st->entry) cudaEventDestroy(st->entry);
    if (st->copy_stream) cudaStreamDestroy(st->copy_stream);
    for (int i = 0; i < 2; ++i) {
        if (st->cstream[i]) cudaStreamDestroy(st->cstream[i]);
        if (st->cjoin[i]) cudaEventDestroy(st->cjoin[i]);
    }
    if (st->cfork) cudaEventDestroy(st->cfork);
    delete st;
}

// ---------------------------------------------------------------------------
// Storage phase.
// ---------------------------------------------------------------------------
// Compress blocks slot0 .. slot0 + nblk - 1 from the rows at A (row 0 of block
// slot0 first).  The first block's rows [0, r0) were compressed before: the
// batched path recompresses the block as it stands, the row-by-row path
// (ZS_FLAG_ROW_APPEND) folds in only rows r0 .. onto the stored state.
static zs_status compress_blocks(zs_store* st, const void* A, int64_t lda, int64_t rows_total, int nblk,
                                 int64_t slot0, cudaStream_t stream, const zs_store::PipeSlot* ps = nullptr,
                                 int64_t r0 = 0) {
    const zs_store_config& c = st->cfg;
    if (c.flags & ZS_FLAG_ROW_APPEND) {
        RowAppendArgs ra;
        memset(&ra, 0, sizeof ra);
        ra.A = (const char*)A + (size_t)r0 * lda * st->insize;
        ra.lda = lda;
        ra.rows_total = rows_total - r0;
        ra.nblk = nblk;
        ra.slot0 = (int32_t)slot0;
        ra.r0 = (int32_t)r0;
        ra.in_kind = c.in_dtype;
        ra.b = (int32_t)c.b;
        ra.n = (int32_t)c.n;
        ra.k = c.k;
        ra.U = st->U;
        ra.sig = st->sig;
        ra.vt = st->vt;
        ra.w = st->w;
        cudaError_t e = launch_row_append(ra, st->fp64, stream);
        if (e != cudaSuccess) return cuda_fail(e, "row-by-row storage");
        return ZS_OK;
    }
    if (!ps && st->sub_blocks > 0 && nblk > st->sub_blocks) {
        // two-stream chunk pipeline: sub-chunk i runs on stream i % 2 with half
        // i % 2 of the scratch; both streams join back into `stream`
        const int sub = st->sub_blocks;
        const int m = tc_width(c.k, st->tune.eig_m_extra);
        ZS_CU(cudaEventRecord(st->cfork, stream), "event");
        for (int i = 0; i < 2; ++i) ZS_CU(cudaStreamWaitEvent(st->cstream[i], st->cfork, 0), "wait");
        int i = 0;
        for (int j0 = 0; j0 < nblk; j0 += sub, ++i) {
            const int r = i & 1;
            const int nb = std::min(sub, nblk - j0);
            CompressChunk ch;
            memset(&ch, 0, sizeof ch);
            ch.A = (const char*)A + (size_t)j0 * c.b * lda * st->insize;
            ch.lda = lda;
            ch.rows_total = std::min<int64_t>(rows_total - (int64_t)j0 * c.b, (int64_t)nb * c.b);
            ch.nblk = nb;
            ch.slot0 = (int32_t)(slot0 + j0);
            ch.b = (int32_t)c.b;
            ch.n = (int32_t)c.n;
            ch.k = c.k;
            ch.in_kind = c.in_dtype;
            ch.G = (char*)st->gscr + (size_t)r * sub * st->tsize * c.n * c.n;
            ch.U = st->U;
            ch.sig = st->sig;
            ch.vt = st->vt;
            ch.w = st->w;
            ch.fault = st->d_fault;
            ch.noconv = st->d_fault + 1;
            ch.refined = st->d_fault + 3;
            ch.xi = st->xi;
            ch.energy = st->d_energy ? st->d_energy + ch.slot0 : nullptr;
            ch.kxi = st->d_rank ? st->d_rank + ch.slot0 : nullptr;
            ch.ews = st->ews;
            ch.ews_ctas = st->ews_ctas;
            ch.qb = (char*)st->qb + (size_t)r * sub * 4 * tc_qb_floats((int)m, (int)c.n);
            ch.ys = (char*)st->ys + (size_t)r * sub * 4 * m * c.b;
            ch.aux = (char*)st->aux + (size_t)r * st->aux_region;
            cudaError_t e = launch_compress(ch, st->fp64, c.flags, st->tune, st->num_sms, st->cstream[r]);
            if (e != cudaSuccess) return cuda_fail(e, "compression kernels");
        }
        for (int q = 0; q < 2; ++q) {
            ZS_CU(cudaEventRecord(st->cjoin[q], st->cstream[q]), "event");
            ZS_CU(cudaStreamWaitEvent(stream, st->cjoin[q], 0), "wait");
        }
        return ZS_OK;
    }
    const int chunk = ps ? 1 : st->gchunk;
    for (int j0 = 0; j0 < nblk; j0 += chunk) {
        const int nb = std::min(chunk, nblk - j0);
        CompressChunk ch;
        memset(&ch, 0, sizeof ch);
        ch.A = (const char*)A + (size_t)j0 * c.b * lda * st->insize;
        ch.lda = lda;
        ch.rows_total = std::min<int64_t>(rows_total - (int64_t)j0 * c.b, (int64_t)nb * c.b);
        ch.nblk = nb;
        ch.slot0 = (int32_t)(slot0 + j0);
        ch.b = (int32_t)c.b;
        ch.n = (int32_t)c.n;
        ch.k = c.k;
        ch.in_kind = c.in_dtype;
        ch.G = st->gscr;
        ch.U = st->U;
        ch.sig = st->sig;
        ch.vt = st->vt;
        ch.w = st->w;
        ch.fault = st->d_fault;
        ch.noconv = st->d_fault + 1;
        ch.refined = st->d_fault + 3;
        ch.xi = st->xi;
        ch.energy = st->d_energy ? st->d_energy + ch.slot0 : nullptr;
        ch.kxi = st->d_rank ? st->d_rank + ch.slot0 : nullptr;
        ch.ews = st->ews;
        ch.ews_ctas = st->ews_ctas;
        ch.qb = st->qb;
        ch.ys = st->ys;
        ch.aux = st->aux;
        if (ps) {
            ch.G = ps->G;
            ch.qb = ps->qb;
            ch.ys = ps->ys;
            ch.aux = ps->aux;
            ch.ews = ps->ews;
            ch.ews_ctas = 1;
        }
        cudaError_t e = launch_compress(ch, st->fp64, c.flags, st->tune, st->num_sms, stream);
        if (e != cudaSuccess) return cuda_fail(e, "compression kernels");
    }
    return ZS_OK;
}

// copy `rows` rows (stride ld elements) from src to dst (stride n), either side
static zs_status copy_rows(zs_store* st, void* dst, const void* src, int64_t rows, int64_t ld, bool src_dev,
                           cudaStream_t s) {
    if (rows <= 0) return ZS_OK;
    const size_t es = st->insize;
    const size_t w = es * st->cfg.n;
    ZS_CU(cudaMemcpy2DAsync(dst, w, src, es * ld, w, rows, src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
          "row copy");
    return ZS_OK;
}

extern "C" zs_status zs_store_append(zs_store* st, const void* rows, int64_t nrows, int64_t ld,
                                     int32_t rows_on_device, void* stream_) {
    if (!st) return fail(ZS_EINVAL, "null store");
    if (nrows == 0) return ZS_OK;
    if (!rows || nrows < 0 || ld < st->cfg.n) return fail(ZS_EINVAL, "bad rows/nrows/ld");
    std::lock_guard<std::mutex> lk(st->mu);
    const zs_store_config& c = st->cfg;
    if (st->T + nrows > st->cap_blocks * c.b)
        return fail(ZS_ENOMEM, "append of %lld rows exceeds capacity %lld", (long long)nrows,
                    (long long)(st->cap_blocks * c.b));
    DeviceGuard g(c.device);
    cudaStream_t stream = (cudaStream_t)stream_;
    const bool dev = rows_on_device != 0;
    const size_t es = st->insize;
    const int64_t b = c.b;
    int64_t pos = 0;
    int64_t T = st->T;
    zs_status s;
    prune_pending(st);
    // device rows may still be being written on the caller's stream
    ZS_CU(cudaEventRecord(st->entry, stream), "event");
    ZS_CU(cudaStreamWaitEvent(st->copy_stream, st->entry, 0), "wait");
    // short appends of whole blocks with no open block: pipeline them
    if (T % b == 0 && nrows % b == 0 && nrows / b <= zs_store::kPipe) {
        for (int64_t j = 0; j < nrows / b; ++j) {
            auto& ps = st->pipe[st->pipe_next];
            st->pipe_next = (st->pipe_next + 1) % zs_store::kPipe;
            // the caller's stream copies the block into the slot once the slot's
            // previous compression is done; compression then runs on the slot's stream
            ZS_CU(cudaStreamWaitEvent(stream, ps.free, 0), "wait");
            ZS_CU(cudaMemcpy2DAsync(ps.stage, es * c.n, (const char*)rows + es * j * b * ld, es * ld, es * c.n, b,
                                    dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream),
                  "row copy");
            ZS_CU(cudaEventRecord(ps.staged, stream), "event");
            ZS_CU(cudaStreamWaitEvent(ps.stream, ps.staged, 0), "wait");
            if ((s = compress_blocks(st, ps.stage, c.n, b, 1, T / b, ps.stream, &ps)) != ZS_OK) return s;
            ZS_CU(cudaEventRecord(ps.free, ps.stream), "event");
            cudaEvent_t ev = nullptr;
            if (!st->event_pool.empty()) {
                ev = st->event_pool.back();
                st->event_pool.pop_back();
            } else {
                ZS_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
            }
            ZS_CU(cudaEventRecord(ev, ps.stream), "event");
            st->pending.emplace_back(T, ev);
            ZS_CU(cudaEventRecord(st->append_done, ps.stream), "event");
            T += b;
        }
        if (!dev) ZS_CU(cudaStreamSynchronize(stream), "host copy");
        st->T = T;
        return ZS_OK;
    }
    // (1) extend the open block
    const int64_t tail_rows = T % b;
    if (tail_rows > 0) {
        const int64_t f = std::min(b - tail_rows, nrows);
        ZS_CU(cudaStreamWaitEvent(st->copy_stream, st->append_done, 0), "wait");
        if ((s = copy_rows(st, (char*)st->tail + es * tail_rows * c.n, rows, f, ld, dev, st->copy_stream)) != ZS_OK)
            return s;
        ZS_CU(cudaEventRecord(st->stage_full[0], st->copy_stream), "event");
        ZS_CU(cudaStreamWaitEvent(stream, st->stage_full[0], 0), "wait");
        if ((s = compress_blocks(st, st->tail, c.n, tail_rows + f, 1, T / b, stream, nullptr, tail_rows)) != ZS_OK)
            return s;
        pos = f;
        T += f;
    }
    // (2) whole blocks
    const int64_t full = (nrows - pos) / b;
    if (full > 0) {
        const char* src = (const char*)rows + es * pos * ld;
        if (dev) {
            if ((s = compress_blocks(st, src, ld, full * b, (int)full, T / b, stream)) != ZS_OK) return s;
        } else {
            int which = 0;
            for (int64_t j = 0; j < full; j += st->stage_blocks, which ^= 1) {
                const int64_t nb = std::min<int64_t>(st->stage_blocks, full - j);
                ZS_CU(cudaStreamWaitEvent(st->copy_stream, st->stage_free[which], 0), "wait");
                if ((s = copy_rows(st, st->stage[which], src + es * j * b * ld, nb * b, ld, false, st->copy_stream)) != ZS_OK)
                    return s;
                ZS_CU(cudaEventRecord(st->stage_full[which], st->copy_stream), "event");
                ZS_CU(cudaStreamWaitEvent(stream, st->stage_full[which], 0), "wait");
                if ((s = compress_blocks(st, st->stage[which], c.n, nb * b, (int)nb, (T + j * b) / b, stream)) != ZS_OK)
                    return s;
                ZS_CU(cudaEventRecord(st->stage_free[which], stream), "event");
            }
        }
        pos += full * b;
        T += full * b;
    }
    // (3) rows of a new open block
    const int64_t rem = nrows - pos;
    if (rem > 0) {
        ZS_CU(cudaEventRecord(st->append_done, stream), "event");   // tail no longer read
        ZS_CU(cudaStreamWaitEvent(st->copy_stream, st->append_done, 0), "wait");
        if ((s = copy_rows(st, st->tail, (const char*)rows + es * pos * ld, rem, ld, dev, st->copy_stream)) != ZS_OK)
            return s;
        ZS_CU(cudaEventRecord(st->stage_full[0], st->copy_stream), "event");
        ZS_CU(cudaStreamWaitEvent(stream, st->stage_full[0], 0), "wait");
        if ((s = compress_blocks(st, st->tail, c.n, rem, 1, T / b, stream)) != ZS_OK) return s;
        T += rem;
    }
    ZS_CU(cudaEventRecord(st->append_done, stream), "event");
    {
        cudaEvent_t ev = nullptr;
        if (!st->event_pool.empty()) {
            ev = st->event_pool.back();
            st->event_pool.pop_back();
        } else {
            ZS_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        }
        ZS_CU(cudaEventRecord(ev, stream), "event");
        st->pending.emplace_back((st->T / b) * b, ev);
    }
    // host rows are free to reuse once the copies have run
    if (!dev) ZS_CU(cudaStreamSynchronize(st->copy_stream), "host copy");
    st->T = T;
    return ZS_OK;
}

extern "C" zs_status zs_store_reset(zs_store* st) {
    if (!st) return fail(ZS_EINVAL, "null store");
    std::lock_guard<std::mutex> lk(st->mu);
    DeviceGuard g(st->cfg.device);
    ZS_CU(cudaEventSynchronize(st->append_done), "reset wait");
    if (st->qx.done) ZS_CU(cudaEventSynchronize(st->qx.done), "reset wait");
    for (auto& pe : st->pending) {
        cudaEventSynchronize(pe.second);
        st->event_pool.push_back(pe.second);
    }
    st->pending.clear();
    st->T = 0;
    return ZS_OK;
}

extern "C" zs_status zs_store_set_xi(zs_store* st, double xi) {
    if (!st) return fail(ZS_EINVAL, "null store");
    if (!(xi >= 0.0 && xi <= 1.0)) return fail(ZS_EINVAL, "xi %g not in [0, 1]", xi);
    if (xi > 0.0 && (st->cfg.flags & ZS_FLAG_ROW_APPEND))
        return fail(ZS_EINVAL, "the energy rule is not combined with row-by-row storage");
    std::lock_guard<std::mutex> lk(st->mu);
    DeviceGuard g(st->cfg.device);
    if (xi > 0.0 && !st->d_energy) {
        const size_t nb = (size_t)std::max<int64_t>(st->cap_blocks, 1);
        if (cudaMalloc((void**)&st->d_energy, sizeof(double) * nb) != cudaSuccess ||
            cudaMalloc((void**)&st->d_rank, sizeof(int) * nb) != cudaSuccess) {
            cudaGetLastError();
            if (st->d_energy) cudaFree(st->d_energy);
            st->d_energy = nullptr;
            st->d_rank = nullptr;
            return fail(ZS_ENOMEM, "block energies and ranks (%zu bytes)", 12 * nb);
        }
    }
    st->xi = xi;
    return ZS_OK;
}

extern "C" zs_status zs_store_fault(const zs_store* st, int32_t* flag) {
    if (!st || !flag) return fail(ZS_EINVAL, "null argument");
    DeviceGuard g(st->cfg.device);
    int v = 0;
    ZS_CU(cudaMemcpy(&v, st->d_fault, sizeof(int), cudaMemcpyDeviceToHost), "fault word");
    *flag = v;
    return ZS_OK;
}

extern "C" zs_status zs_store_status(const zs_store* st, int64_t* unconverged_blocks, int64_t* unconverged_queries,
                                     int64_t* refined_blocks, int64_t* refined_queries) {
    if (!st) return fail(ZS_EINVAL, "null store");
    DeviceGuard g(st->cfg.device);
    ZS_CU(cudaDeviceSynchronize(), "status wait");
    int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    ZS_CU(cudaMemcpy(v, st->d_fault, sizeof v, cudaMemcpyDeviceToHost), "status words");
    if (unconverged_blocks) *unconverged_blocks = v[1];
    if (unconverged_queries) *unconverged_queries = v[2];
    if (refined_blocks) *refined_blocks = v[3];
    if (refined_queries) *refined_queries = v[4];
    if (v[0]) return fail(ZS_ETIMEDOUT, "a bounded wait of a tensor-core kernel gave up; results are undefined");
    if (v[1] || v[2])
        return fail(ZS_ENOCONV, "%d block(s) and %d query result(s) did not pass the accuracy test within the pass cap",
                    v[1], v[2]);
    return ZS_OK;
}

extern "C" zs_status zs_store_block_stats(const zs_store* st_, int64_t nblocks, int32_t* ranks, double* kept,
                                         double* energy) {
    zs_store* st = const_cast<zs_store*>(st_);
    if (!st || nblocks < 0) return fail(ZS_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(st->mu);
    const int64_t T = st->T, b = st->cfg.b, n = st->cfg.n, k = st->cfg.k;
    const int64_t nb = (T + b - 1) / b;
    if (nblocks > nb) return fail(ZS_ENOTFOUND, "%lld blocks asked for, the store holds %lld", (long long)nblocks,
                                  (long long)nb);
    if (nblocks == 0) return ZS_OK;
    DeviceGuard g(st->cfg.device);
    ZS_CU(cudaDeviceSynchronize(), "stats wait");
    std::vector<double> sig((size_t)nblocks * k);
    if (st->fp64) {
        ZS_CU(cudaMemcpy(sig.data(), st->sig, 8 * sig.size(), cudaMemcpyDeviceToHost), "sigma copy");
    } else {
        std::vector<float> f(sig.size());
        ZS_CU(cudaMemcpy(f.data(), st->sig, 4 * f.size(), cudaMemcpyDeviceToHost), "sigma copy");
        for (size_t i = 0; i < f.size(); ++i) sig[i] = f[i];
    }
    std::vector<double> en;
    if (energy && st->xi > 0.0 && st->d_energy) {
        en.resize(nblocks);
        ZS_CU(cudaMemcpy(en.data(), st->d_energy, 8 * nblocks, cudaMemcpyDeviceToHost), "energy copy");
    }
    for (int64_t i = 0; i < nblocks; ++i) {
        const int64_t rows = std::min(b, T - i * b);
        const int64_t cap = std::min(k, std::min(rows, n));
        int32_t ki = (int32_t)cap;
        double kk = 0.0;
        if (st->xi > 0.0) {      // the energy rule's rank: the columns it kept are the nonzero ones
            ki = 0;
            for (int64_t j = 0; j < cap; ++j) ki += sig[i * k + j] > 0.0;
        }
        for (int64_t j = 0; j < cap; ++j) kk += sig[i * k + j] * sig[i * k + j];
        if (ranks) ranks[i] = ki;
        if (kept) kept[i] = kk;
        if (energy) energy[i] = en.empty() ? -1.0 : en[i];
    }
    return ZS_OK;
}

extern "C" zs_status zs_store_info(const zs_store* st, int64_t* rows, int64_t* nblocks, int64_t* bytes) {
    if (!st) return fail(ZS_EINVAL, "null store");
    const int64_t T = st->T, b = st->cfg.b;
    const int64_t nb = (T + b - 1) / b;
    if (rows) *rows = T;
    if (nblocks) *nblocks = nb;
    if (bytes) *bytes = nb * (b * st->cfg.k + st->cfg.k + st->cfg.k * st->cfg.n) * st->tsize;
    return ZS_OK;
}

extern "C" zs_status zs_store_export_block(const zs_store* st_, int64_t i, void* U, void* sigma, void* Vt,
                                           int32_t* rows_i, int32_t* k_i, void* stream_) {
    zs_store* st = const_cast<zs_store*>(st_);
    if (!st) return fail(ZS_EINVAL, "null store");
    std::lock_guard<std::mutex> lk(st->mu);
    const int64_t T = st->T, b = st->cfg.b, n = st->cfg.n, k = st->cfg.k;
    const int64_t nb = (T + b - 1) / b;
    if (i < 0 || i >= nb) return fail(ZS_ENOTFOUND, "block %lld not in [0, %lld)", (long long)i, (long long)nb);
    DeviceGuard g(st->cfg.device);
    cudaStream_t s = (cudaStream_t)stream_;
    ZS_CU(cudaStreamWaitEvent(s, st->append_done, 0), "wait");
    for (auto& pe : st->pending) ZS_CU(cudaStreamWaitEvent(s, pe.second, 0), "wait");
    const int64_t r = std::min(b, T - i * b);
    const size_t ts = st->tsize;
    if (U) ZS_CU(cudaMemcpyAsync(U, (char*)st->U + ts * i * b * k, ts * r * k, cudaMemcpyDeviceToDevice, s), "copy");
    if (sigma) ZS_CU(cudaMemcpyAsync(sigma, (char*)st->sig + ts * i * k, ts * k, cudaMemcpyDeviceToDevice, s), "copy");
    if (Vt) ZS_CU(cudaMemcpyAsync(Vt, (char*)st->vt + ts * i * k * n, ts * k * n, cudaMemcpyDeviceToDevice, s), "copy");
    if (rows_i) *rows_i = (int32_t)r;
    if (k_i) *k_i = (int32_t)std::min<int64_t>(k, std::min<int64_t>(r, n));
    return ZS_OK;
}

// ---------------------------------------------------------------------------
// Query phase.
// ---------------------------------------------------------------------------
namespace zs {
zs_status query_batch_locked(zs_store* st, QueryExec& x, const int64_t* ts, const int64_t* te, int nq, int kout,
                             const zs_result* res, cudaStream_t stream, int64_t Trows, void* coef,
                             int64_t coef_rows) {
    const int kq = std::min<int>(kout, (int)st->cfg.n);
    const bool ref = (st->cfg.flags & ZS_FLAG_FP64_REFINE) && !st->fp64;
    if (!eig_plan((int)st->cfg.n, kq, st->tune.eig_m_extra, st->fp64, ref).ok)
        return fail(ZS_EINVAL, "k_out=%d with n=%lld does not fit the eigen core's shared memory", kout,
                    (long long)st->cfg.n);
    std::vector<QPlan> plans;
    std::vector<int64_t> prefix;
    zs_status s = plan_queries(*st, Trows, ts, te, nq, kq, plans, prefix);
    if (s != ZS_OK) return s;
    if (coef && prefix[nq] * st->cfg.k > coef_rows)
        return fail(ZS_EINVAL, "coefficient buffer holds %lld rows; the batch needs %lld", (long long)coef_rows,
                    (long long)(prefix[nq] * st->cfg.k));
    for (int q = 0; q < nq; ++q) {
        const zs_result& r = res[q];
        if ((!coef && (!r.U || r.ldu < kout)) || !r.S || !r.V || r.ldv < kout)
            return fail(ZS_EINVAL, "query %d: bad result buffers", q);
        plans[q].U = r.U;
        plans[q].ldu = r.ldu;
        plans[q].S_out = r.S;
        plans[q].V_out = r.V;
        plans[q].ldv = r.ldv;
        plans[q].rank = r.rank;
    }
    // wait only for appends still running that rewrite blocks this batch reads
    // (short appends run on several pipeline streams, so every such append's
    // event is waited for; the list holds only appends not yet finished)
    {
        int64_t max_te = -1;
        for (int q = 0; q < nq; ++q) max_te = std::max(max_te, te[q]);
        prune_pending(st);
        for (auto& pe : st->pending)
            if (pe.first <= max_te) ZS_CU(cudaStreamWaitEvent(stream, pe.second, 0), "wait for appends");
    }
    // the executor's scratch may still be in use by a batch on another stream
    if (x.done) ZS_CU(cudaStreamWaitEvent(stream, x.done, 0), "wait for previous batch");
    // split batches whose scratch would exceed the budget
    int q0 = 0;
    while (q0 < nq) {
        int q1 = q0;
        int64_t sl = 0;
        while (q1 < nq) {
            const int64_t add = plans[q1].nslab;
            if (q1 > q0 && QueryExec::bytes_for(*st, q1 - q0 + 1, sl + add, kq) > st->query_budget) break;
            sl += add;
            ++q1;
        }
        std::vector<QPlan> sub(plans.begin() + q0, plans.begin() + q1);
        std::vector<int64_t> pre(q1 - q0 + 1);
        int64_t base = sub[0].slab0;
        for (int q = 0; q < q1 - q0; ++q) {
            sub[q].slab0 -= base;
            pre[q] = sub[q].slab0;
        }
        pre[q1 - q0] = sl;
        if ((s = run_batch(*st, x, Trows, sub, pre, kq, kout, stream, coef, base * st->cfg.k)) != ZS_OK) return s;
        q0 = q1;
    }
    return ZS_OK;
}
}  // namespace zs

extern "C" zs_status zs_query_batch(zs_store* st, const int64_t* ts, const int64_t* te, int32_t nq, int32_t k_out,
                                    const zs_result* results, void* stream) {
    if (!st || !ts || !te || !results || nq < 0) return fail(ZS_EINVAL, "null argument");
    if (nq == 0) return ZS_OK;
    if (k_out < 1 || k_out > 64) return fail(ZS_EINVAL, "k_out %d not in 1..64", k_out);
    std::lock_guard<std::mutex> lk(st->mu);
    DeviceGuard g(st->cfg.device);
    return query_batch_locked(st, st->qx, ts, te, nq, k_out, results, (cudaStream_t)stream, st->T);
}

extern "C" zs_status zs_query_batch_factored(zs_store* st, const int64_t* ts, const int64_t* te, int32_t nq,
                                             int32_t k_out, const zs_result* results, void* coef, int64_t coef_rows,
                                             void* stream) {
    if (!st || !ts || !te || !results || !coef || nq < 0 || coef_rows < 0) return fail(ZS_EINVAL, "null argument");
    if (nq == 0) return ZS_OK;
    if (k_out < 1 || k_out > 64) return fail(ZS_EINVAL, "k_out %d not in 1..64", k_out);
    std::lock_guard<std::mutex> lk(st->mu);
    DeviceGuard g(st->cfg.device);
    return query_batch_locked(st, st->qx, ts, te, nq, k_out, results, (cudaStream_t)stream, st->T, coef, coef_rows);
}

// ---------------------------------------------------------------------------
// Autotuner: time the query launch set under candidate grid shapes on this
// device and keep the fastest (results do not depend on the choice).
// ---------------------------------------------------------------------------
static std::string tune_key(const zs_store* st) {
    char b[160];
    snprintf(b, sizeof b, "n=%lld,b=%lld,k=%d,dtype=%d,flags=%d,sms=%d", (long long)st->cfg.n, (long long)st->cfg.b,
             st->cfg.k, st->cfg.in_dtype, st->cfg.flags, st->num_sms);
    return b;
}

static void tune_cache_store(const zs_store* st) {
    const char* path = getenv("ZS_TUNE_CACHE");
    if (!path || !*path) return;
    std::string key = tune_key(st);
    std::vector<std::string> lines;
    if (FILE* f = fopen(path, "r")) {
        char buf[512];
        while (fgets(buf, sizeof buf, f)) {
            std::string l(buf);
            if (l.compare(0, key.size() + 1, key + " ") != 0) lines.push_back(l);
        }
        fclose(f);
    }
    char v[128];
    snprintf(v, sizeof v, " %d %d\n", st->tune.slab_ctas_per_sm, st->tune.project_ctas_per_sm);
    lines.push_back(key + v);
    if (FILE* f = fopen(path, "w")) {
        for (auto& l : lines) fputs(l.c_str(), f);
        fclose(f);
    }
}

void zs::tune_cache_load(zs_store* st) {
    const char* path = getenv("ZS_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    const std::string key = tune_key(st);
    char buf[512];
    while (fgets(buf, sizeof buf, f)) {
        std::string l(buf);
        if (l.compare(0, key.size() + 1, key + " ") == 0) {
            int a = 0, c = 0;
            if (sscanf(l.c_str() + key.size() + 1, "%d %d", &a, &c) == 2 && a > 0 && c > 0) {
                st->tune.slab_ctas_per_sm = a;
                st->tune.project_ctas_per_sm = c;
            }
        }
    }
    fclose(f);
}

extern "C" zs_status zs_store_autotune(zs_store* st, int32_t nq, void* stream_) {
    if (!st || nq < 1) return fail(ZS_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(st->mu);
    DeviceGuard g(st->cfg.device);
    const int64_t T = st->T, b = st->cfg.b;
    if (T < 1) return fail(ZS_EINVAL, "autotune needs appended rows");
    cudaStream_t stream = (cudaStream_t)stream_;
    const int k = st->cfg.k, kq = std::min<int>(k, (int)st->cfg.n);
    // nq ranges of up to 16 blocks, spread over the store (deterministic)
    std::vector<int64_t> ts(nq), te(nq);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    int64_t rows_total = 0;
    for (int q = 0; q < nq; ++q) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        const int64_t len = std::max<int64_t>(1, std::min<int64_t>(T, (int64_t)(x % (16 * b)) + 1));
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        ts[q] = (int64_t)(x % (uint64_t)(T - len + 1));
        te[q] = ts[q] + len - 1;
        rows_total += len;
    }
    const size_t ts_ = st->tsize;
    void *U = nullptr, *S = nullptr, *V = nullptr;
    auto fre = [&]() { if (U) cudaFree(U); if (S) cudaFree(S); if (V) cudaFree(V); };
    if (cudaMalloc(&U, ts_ * rows_total * k) != cudaSuccess || cudaMalloc(&S, ts_ * (size_t)nq * k) != cudaSuccess ||
        cudaMalloc(&V, ts_ * (size_t)nq * st->cfg.n * k) != cudaSuccess) {
        cudaGetLastError();
        fre();
        return fail(ZS_ENOMEM, "autotune buffers");
    }
    std::vector<zs_result> res(nq);
    int64_t off = 0;
    for (int q = 0; q < nq; ++q) {
        res[q].U = (char*)U + ts_ * off * k;
        res[q].ldu = k;
        res[q].S = (char*)S + ts_ * (size_t)q * k;
        res[q].V = (char*)V + ts_ * (size_t)q * st->cfg.n * k;
        res[q].ldv = k;
        res[q].rank = nullptr;
        off += te[q] - ts[q] + 1;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool graphs = st->use_graphs;
    st->use_graphs = false;          // time the eager launch set of each candidate
    const Tuning keep = st->tune;
    Tuning best = keep;
    float best_ms = 1e30f;
    zs_status s = ZS_OK;
    for (int slab : {2, 4, 8, 16}) {
        for (int proj : {4, 8, 16}) {
            st->tune = keep;
            st->tune.slab_ctas_per_sm = slab;
            st->tune.project_ctas_per_sm = proj;
            float tot = 0;
            for (int rep = 0; rep < 3 && s == ZS_OK; ++rep) {
                cudaEventRecord(e0, stream);
                s = query_batch_locked(st, st->qx, ts.data(), te.data(), nq, kq, res.data(), stream, T);
                cudaEventRecord(e1, stream);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;          // first run warms caches and attributes
            }
            if (s != ZS_OK) break;
            if (tot < best_ms) { best_ms = tot; best = st->tune; }
        }
        if (s != ZS_OK) break;
    }
    st->tune = (s == ZS_OK) ? best : keep;
    st->use_graphs = graphs;
    st->qx.release();                  // captured graphs used the old launch shapes
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(stream);
    fre();
    if (s == ZS_OK) tune_cache_store(st);
    return s;
}

extern "C" zs_status zs_query(zs_store* st, int64_t t_s, int64_t t_e, int32_t k_out, const zs_result* res,
                              void* stream) {
    if (!res) return fail(ZS_EINVAL, "null result");
    return zs_query_batch(st, &t_s, &t_e, 1, k_out, res, stream);
}

extern "C" const char* zs_status_str(zs_status s) {
    switch (s) {
        case ZS_OK: return "ok";
        case ZS_EINVAL: return "invalid argument";
        case ZS_ERANGE: return "range out of bounds";
        case ZS_ENOMEM: return "out of memory";
        case ZS_EBUSY: return "busy";
        case ZS_ETIMEDOUT: return "timed out";
        case ZS_EDTYPE: return "unsupported dtype";
        case ZS_ECUDA: return "CUDA error";
        case ZS_EINTERNAL: return "internal error";
        case ZS_ENOTFOUND: return "not found";
        case ZS_ENOCONV: return "not converged";
    }
    return "unknown status";
}

extern "C" const char* zs_last_error(void) { return g_last_error.c_str(); }

extern "C" int64_t zs_launch_count(void) { return launch_count_total(); }

extern "C" void zs_profile_enable(int32_t on) { profile_enable(on); }
extern "C" void zs_profile_reset(void) { profile_reset(); }
extern "C" int32_t zs_profile_count(void) { return profile_count(); }
extern "C" zs_status zs_profile_get(int32_t i, const char** name, int64_t* launches, double* total_ms) {
    if (!profile_get(i, name, launches, total_ms)) return fail(ZS_ENOTFOUND, "no profile entry %d", i);
    return ZS_OK;
}
