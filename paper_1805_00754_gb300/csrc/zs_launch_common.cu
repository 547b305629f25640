// zs_launch_common.cu - host side shared by every launch: the kernel profiler
// (CUDA events on the launch stream), the launch counter, the eigen-core and
// tensor-path scratch plans, and the dispatch of the storage- and query-phase
// launch sets to their per-precision translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "zs_internal.h"
#include "zs_linalg.cuh"
#include "zs_prof.h"

namespace zs {

static std::atomic<int64_t> g_launches{0};
void note_launches(int64_t n) { g_launches += n; }
int64_t launch_count_total() { return g_launches.load(); }

// ---------------------------------------------------------------------------
// Kernel profiler: CUDA events around each launch, on the launch stream.
// ---------------------------------------------------------------------------
namespace prof {
struct Pending { int id; cudaEvent_t a, b; };
struct Entry { std::string name; int64_t launches = 0; double ms = 0; };
static std::atomic<int> g_on{0};
static std::mutex g_mu;
static std::vector<Pending> g_pending;
static std::vector<Entry> g_table;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t get_event() {
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
static void drain_locked() {
    for (auto& p : g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        g_table[p.id].launches += 1;
        g_table[p.id].ms += ms;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace prof

prof::Scope::Scope(const char* name, cudaStream_t s) : st(s) {
    using namespace prof;
    if (!g_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_table.size(); ++i)
        if (g_table[i].name == name) { id = (int)i; break; }
    if (id < 0) { g_table.push_back(Entry{name}); id = (int)g_table.size() - 1; }
    a = get_event();
    b = get_event();
    cudaEventRecord(a, st);
}

prof::Scope::~Scope() {
    using namespace prof;
    if (id < 0) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(Pending{id, a, b});
    if (g_pending.size() > 4096) drain_locked();
}

void profile_enable(int on) { prof::g_on.store(on); }
void profile_reset() {
    std::lock_guard<std::mutex> lk(prof::g_mu);
    prof::drain_locked();
    prof::g_table.clear();
}
int profile_count() {
    std::lock_guard<std::mutex> lk(prof::g_mu);
    prof::drain_locked();
    return (int)prof::g_table.size();
}
bool profile_get(int i, const char** name, int64_t* launches, double* ms) {
    std::lock_guard<std::mutex> lk(prof::g_mu);
    prof::drain_locked();
    if (i < 0 || i >= (int)prof::g_table.size()) return false;
    if (name) *name = prof::g_table[i].name.c_str();
    if (launches) *launches = prof::g_table[i].launches;
    if (ms) *ms = prof::g_table[i].ms;
    return true;
}

size_t eig_smem_bytes(int n, int m, bool fp64, bool refine, bool yglob) {
    const size_t ts = fp64 ? 8 : 4;
    const bool dense = (m == n && n <= 64);
    const size_t ld = m + 1;
    auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    size_t s = 0;
    if (!dense) s += (yglob ? 1 : 2) * r16(ts * n * ld);
    s += 2 * r16(ts * m * ld);
    if (refine && !fp64) s += 3 * r16(8 * m * ld);
    return s;
}

// Subspace width m = kq + p (p = extra, at most 64 columns); the Y block moves
// to global memory when shared memory cannot hold both n x m blocks.
EigPlan eig_plan(int n, int kq, int extra, bool fp64, bool refine) {
    EigPlan p;
    const bool ref = refine && !fp64;
    const size_t cap = 200 * 1024;
    if (n <= 64) {
        p.m = n;
        p.yglob = false;
        p.smem = eig_smem_bytes(n, n, fp64, ref, false);
        p.ok = p.smem <= cap;
        return p;
    }
    int m = std::min(std::min(n, kq + extra), ZS_MAXM);
    if (eig_smem_bytes(n, m, fp64, ref, false) <= cap) {
        p.m = m;
        p.yglob = false;
    } else {
        while (m > kq + 2 && eig_smem_bytes(n, m, fp64, ref, true) > cap) --m;
        p.m = m;
        p.yglob = true;
    }
    p.smem = eig_smem_bytes(n, p.m, fp64, ref, p.yglob);
    p.ok = p.smem <= cap && p.m >= kq;
    return p;
}

size_t eig_ws_bytes(int n, bool fp64, int ctas) {
    return (size_t)(fp64 ? 8 : 4) * n * (ZS_MAXM + 1) * std::max(ctas, 1);
}

// Opt in to the dynamic shared memory a launch needs (static + dynamic may not
size_t tc_aux_bytes(int64_t items, int64_t tiles, int m, int kw) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    return r(4 * (size_t)tiles * m * m) + r(4 * (size_t)items * m * m) + r(4 * (size_t)items * m * kw) +
           r(4 * (size_t)items * kw);
}

cudaError_t launch_compress_simt(const CompressChunk& c, bool fp64, int flags, const Tuning& tu, int num_sms,
                                 cudaStream_t st);
cudaError_t launch_compress_tc(const CompressChunk& c, int flags, const Tuning& tu, int num_sms, cudaStream_t st);
cudaError_t launch_query_f64(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st);
cudaError_t launch_query_f32(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st);
cudaError_t launch_query_f32_refine(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu,
                                    int num_sms, cudaStream_t st);

cudaError_t launch_compress(const CompressChunk& c, bool fp64, int flags, const Tuning& tu, int num_sms,
                            cudaStream_t st) {
    if (use_tc_path(fp64, c.n, flags)) return launch_compress_tc(c, flags, tu, num_sms, st);
    return launch_compress_simt(c, fp64, flags, tu, num_sms, st);
}

cudaError_t launch_query(const QueryArgs& a, bool fp64, const QueryGrid& g, int flags, const Tuning& tu,
                         int num_sms, cudaStream_t st) {
    if (fp64) return launch_query_f64(a, g, flags, tu, num_sms, st);
    return a.fp64_refine ? launch_query_f32_refine(a, g, flags, tu, num_sms, st)
                         : launch_query_f32(a, g, flags, tu, num_sms, st);
}

bool profiling_on() { return prof::g_on.load() != 0; }

}  // namespace zs
