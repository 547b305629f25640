// zs_serve.cpp - continuous-batching server for range-SVD queries.
//
// One host thread owns a set of execution slots (a CUDA stream plus its own
// query scratch each).  Requests queue as they arrive; whenever a slot is free
// the thread takes the oldest requests that share a width k_out, as many as
// max_batch and the device-memory budget allow, plans them against the rows
// published at that moment and launches the batch kernels on that slot's
// stream.  Requests that arrive while batches run join the next batch; up to
// max_inflight batches overlap on the device.  Completion is detected by
// polling each batch's CUDA event; latency is submit -> event complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "zoomsvd.h"
#include "zs_api_internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket = 0;
    int64_t ts = 0, te = 0;
    int32_t kout = 0;
    zs_result dst{};
    Clock::time_point t_submit;
    int32_t status = ZS_OK;
    bool done = false;
    size_t bytes = 0;
};

struct Slot {
    zs::QueryExec x;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    bool launching = false;
    size_t bytes = 0;
    std::vector<Request*> reqs;
};

}  // namespace

struct zs_server {
    zs_store* st = nullptr;
    zs_serve_config cfg{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Slot>> slots;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::atomic<bool> thread_error{false};
    size_t bytes_inflight = 0;
    // stats
    int64_t completed = 0, rejected = 0, batches = 0, batched_reqs = 0;
    std::vector<double> lat_ms;
    Clock::time_point t_start;
};

static size_t request_bytes(const zs_store& st, int64_t ts, int64_t te, int kout) {
    const int64_t nslab = te / st.cfg.b - ts / st.cfg.b + 1;
    const int kq = std::min<int>(kout, (int)st.cfg.n);
    return zs::QueryExec::bytes_for(st, 1, nslab, kq);
}

static void finish_slot(zs_server* sv, Slot& s, int32_t status) {
    const auto now = Clock::now();
    for (Request* r : s.reqs) {
        r->status = status;
        r->done = true;
        sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
        ++sv->completed;
    }
    s.reqs.clear();
    sv->bytes_inflight -= s.bytes;
    s.bytes = 0;
    s.busy = false;
}

static void serve_loop(zs_server* sv) {
    cudaSetDevice(sv->st->cfg.device);
    std::vector<int64_t> ts, te;
    std::vector<zs_result> res;
    for (;;) {
        bool idle = true;
        Slot* launch_slot = nullptr;
        int kout = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // completions
            for (auto& sp : sv->slots) {
                Slot& s = *sp;
                if (!s.busy || s.launching) continue;
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaErrorNotReady) continue;
                finish_slot(sv, s, q == cudaSuccess ? ZS_OK : ZS_ECUDA);
                idle = false;
                sv->cv_done.notify_all();
            }
            // admission into one free slot: the oldest requests sharing a k_out,
            // up to max_batch and the memory budget
            for (auto& sp : sv->slots) {
                Slot& s = *sp;
                if (s.busy || sv->queue.empty()) continue;
                kout = sv->queue.front()->kout;
                size_t bytes = 0;
                s.reqs.clear();
                for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)s.reqs.size() < sv->cfg.max_batch;) {
                    Request* r = *it;
                    if (r->kout != kout) { ++it; continue; }
                    const bool alone = s.reqs.empty() && sv->bytes_inflight == 0;
                    if (!alone && sv->bytes_inflight + bytes + r->bytes > (size_t)sv->cfg.memory_budget) break;
                    s.reqs.push_back(r);
                    bytes += r->bytes;
                    it = sv->queue.erase(it);
                }
                if (s.reqs.empty()) break;   // memory budget full: wait for completions
                s.bytes = bytes;
                s.busy = true;
                s.launching = true;
                sv->bytes_inflight += bytes;
                ++sv->batches;
                sv->batched_reqs += (int64_t)s.reqs.size();
                launch_slot = &s;
                break;
            }
            bool any_busy = false;
            for (auto& sp : sv->slots) any_busy |= sp->busy;
            if (!launch_slot && sv->stopping && sv->queue.empty() && !any_busy) break;
        }
        if (launch_slot) {
            // plan and launch without holding the server lock (submitters keep going)
            Slot& s = *launch_slot;
            const size_t nb = s.reqs.size();
            ts.resize(nb);
            te.resize(nb);
            res.resize(nb);
            for (size_t i = 0; i < nb; ++i) {
                ts[i] = s.reqs[i]->ts;
                te[i] = s.reqs[i]->te;
                res[i] = s.reqs[i]->dst;
            }
            zs_status st;
            {
                std::lock_guard<std::mutex> sl(sv->st->mu);
                st = zs::query_batch_locked(sv->st, s.x, ts.data(), te.data(), (int)nb, kout, res.data(),
                                            s.stream, sv->st->T);
            }
            const bool ok = (st == ZS_OK) && cudaEventRecord(s.ev, s.stream) == cudaSuccess;
            std::unique_lock<std::mutex> lk(sv->mu);
            s.launching = false;
            if (!ok) {
                cudaStreamSynchronize(s.stream);
                finish_slot(sv, s, st != ZS_OK ? st : ZS_ECUDA);
                sv->cv_done.notify_all();
            }
            idle = false;
        }
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" zs_status zs_serve_start(zs_store* st, const zs_serve_config* cfg, zs_server** out) {
    if (!st || !cfg || !out) return zs::fail(ZS_EINVAL, "null argument");
    if (cfg->max_batch < 1 || cfg->max_inflight < 1 || cfg->queue_capacity < 1 || cfg->memory_budget < 1)
        return zs::fail(ZS_EINVAL, "bad serve config");
    *out = nullptr;
    cudaSetDevice(st->cfg.device);
    auto sv = new zs_server();
    sv->st = st;
    sv->cfg = *cfg;
    for (int i = 0; i < cfg->max_inflight; ++i) {
        auto s = std::make_unique<Slot>();
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
            delete sv;
            return zs::fail(ZS_ECUDA, "serve stream/event creation failed");
        }
        sv->slots.push_back(std::move(s));
    }
    sv->t_start = Clock::now();
    sv->th = std::thread(serve_loop, sv);
    *out = sv;
    return ZS_OK;
}

extern "C" zs_status zs_serve_submit(zs_server* sv, int64_t t_s, int64_t t_e, int32_t k_out, const zs_result* dst,
                                     uint64_t* ticket) {
    if (!sv || !dst || !ticket) return zs::fail(ZS_EINVAL, "null argument");
    if (k_out < 1 || k_out > 64) return zs::fail(ZS_EINVAL, "k_out %d not in 1..64", k_out);
    int64_t T;
    {
        std::lock_guard<std::mutex> sl(sv->st->mu);
        T = sv->st->T;
    }
    if (t_s < 0 || t_s > t_e || t_e >= T) return zs::fail(ZS_ERANGE, "range [%lld, %lld] outside [0, %lld)",
                                                          (long long)t_s, (long long)t_e, (long long)T);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return zs::fail(ZS_EINVAL, "server is stopping");
    if ((int)sv->queue.size() >= sv->cfg.queue_capacity) {
        ++sv->rejected;
        return zs::fail(ZS_EBUSY, "queue full (%d)", sv->cfg.queue_capacity);
    }
    auto r = std::make_unique<Request>();
    r->ticket = sv->next_ticket++;
    r->ts = t_s;
    r->te = t_e;
    r->kout = k_out;
    r->dst = *dst;
    r->t_submit = Clock::now();
    r->bytes = request_bytes(*sv->st, t_s, t_e, k_out);
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->reqs.emplace(r->ticket, std::move(r));
    return ZS_OK;
}

extern "C" zs_status zs_serve_poll(zs_server* sv, uint64_t ticket, int32_t* done, int32_t* req_status) {
    if (!sv || !done) return zs::fail(ZS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return zs::fail(ZS_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->done ? 1 : 0;
    if (it->second->done) {
        if (req_status) *req_status = it->second->status;
        sv->reqs.erase(it);
    }
    return ZS_OK;
}

extern "C" zs_status zs_serve_wait(zs_server* sv, uint64_t ticket, int64_t timeout_ms, int32_t* req_status) {
    if (!sv) return zs::fail(ZS_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return zs::fail(ZS_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second.get();
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    if (!ok) return zs::fail(ZS_ETIMEDOUT, "ticket %llu not done after %lld ms", (unsigned long long)ticket,
                             (long long)timeout_ms);
    if (req_status) *req_status = r->status;
    sv->reqs.erase(it);
    return ZS_OK;
}

extern "C" zs_status zs_serve_stop(zs_server* sv, zs_serve_stats* stats) {
    if (!sv) return zs::fail(ZS_EINVAL, "null server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    if (sv->th.joinable()) sv->th.join();
    const double wall = std::chrono::duration<double>(Clock::now() - sv->t_start).count();
    if (stats) {
        zs_serve_stats s{};
        s.completed = sv->completed;
        s.rejected = sv->rejected;
        s.batches = sv->batches;
        s.wall_s = wall;
        s.queries_per_s = wall > 0 ? sv->completed / wall : 0.0;
        s.mean_batch = sv->batches ? (double)sv->batched_reqs / sv->batches : 0.0;
        std::vector<double> l = sv->lat_ms;
        std::sort(l.begin(), l.end());
        if (!l.empty()) {
            auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
            s.p50_ms = pct(0.50);
            s.p99_ms = pct(0.99);
            s.max_ms = l.back();
            double sum = 0;
            for (double v : l) sum += v;
            s.mean_ms = sum / l.size();
        }
        *stats = s;
    }
    for (auto& sp : sv->slots) {
        if (sp->stream) cudaStreamSynchronize(sp->stream);
        sp->x.release();
        if (sp->ev) cudaEventDestroy(sp->ev);
        if (sp->stream) cudaStreamDestroy(sp->stream);
    }
    delete sv;
    return ZS_OK;
}
