// zs_launch_common.cu - host side shared by every launch: the kernel profiler
// (CUDA events on the launch stream), the launch counter, the eigen-core and
// tensor-path scratch plans, and the dispatch of the storage- and query-phase
// launch sets to their per-precision translation units.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
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
           r(4 * (size_t)items * kw) + r(4 * (size_t)items * m) + r(4 * (size_t)(items + 2)) +
           r(4 * (size_t)(2 * items + 1));
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

// ---------------------------------------------------------------------------
// Energy rule (Eq. 1) per block: k_i = the smallest rank whose leading
// singular values hold a fraction >= xi of the block's energy ||X_i||_F^2
// (the sum of all its sigma_j^2), capped at the stored k.  Applied after the
// block's rank-k factors are formed: columns k_i.. of U, sigma, V^T (and the
// stored Sigma V^T) become zero, which the query phase treats as rank
// deficiency.
// ---------------------------------------------------------------------------
// ||X_i||_F^2 of each block of the chunk, FP64 sums in a fixed order
template <typename Tin>
__global__ void __launch_bounds__(256) k_block_energy(CompressChunk c) {
    __shared__ double red[8];
    const int j = blockIdx.x;
    if (j >= c.nblk) return;
    const int rows = (int)min((int64_t)c.b, c.rows_total - (int64_t)j * c.b);
    const Tin* X = (const Tin*)c.A + (size_t)j * c.b * c.lda;
    double e = 0.0;
    for (int64_t f = threadIdx.x; f < (int64_t)rows * c.n; f += 256) {
        const int64_t r = f / c.n, col = f - (f / c.n) * c.n;
        double x;
        if constexpr (std::is_same<Tin, __nv_bfloat16>::value) x = (double)__bfloat162float(X[r * c.lda + col]);
        else x = (double)X[r * c.lda + col];
        e = fma(x, x, e);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        c.energy[j] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_xi_truncate(CompressChunk c) {
    __shared__ int ki_s;
    const int j = blockIdx.x;
    if (j >= c.nblk) return;
    const int64_t slot = (int64_t)c.slot0 + j;
    const int k = c.k, n = c.n;
    T* sig = (T*)c.sig + slot * k;
    if (threadIdx.x == 0) ki_s = c.kxi ? c.kxi[j] : xi_rank_of(sig, k, c.energy[j], c.xi);
    __syncthreads();
    const int ki = ki_s;
    if (ki >= k) return;
    const int rows = (int)min((int64_t)c.b, c.rows_total - (int64_t)j * c.b);
    T* U = (T*)c.U + slot * c.b * k;
    T* Vt = (T*)c.vt + slot * k * n;
    T* W = c.w ? (T*)c.w + slot * k * n : nullptr;
    const int dk = k - ki;
    for (int l = threadIdx.x; l < dk; l += 256) sig[ki + l] = T(0);
    for (int64_t f = threadIdx.x; f < (int64_t)rows * dk; f += 256) {
        const int64_t r = f / dk;
        U[r * k + ki + (f - r * dk)] = T(0);
    }
    for (int64_t f = threadIdx.x; f < (int64_t)dk * n; f += 256) {
        Vt[(int64_t)ki * n + f] = T(0);
        if (W) W[(int64_t)ki * n + f] = T(0);
    }
}

cudaError_t launch_compress(const CompressChunk& c, bool fp64, int flags, const Tuning& tu, int num_sms,
                            cudaStream_t st) {
    const bool xi = c.xi > 0.0 && c.energy && c.nblk >= 1;
    const bool tc = use_tc_path(fp64, c.n, flags);
    cudaError_t e;
    if (xi) {
        // the blocks' energies first: the tensor path's accuracy test applies
        // the energy rule and tests only the ranks it keeps
        prof::Scope ps("xi_energy", st);
        if (c.in_kind == IN_F64) k_block_energy<double><<<c.nblk, 256, 0, st>>>(c);
        else if (c.in_kind == IN_BF16) k_block_energy<__nv_bfloat16><<<c.nblk, 256, 0, st>>>(c);
        else k_block_energy<float><<<c.nblk, 256, 0, st>>>(c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    e = tc ? launch_compress_tc(c, flags, tu, num_sms, st) : launch_compress_simt(c, fp64, flags, tu, num_sms, st);
    if (e != cudaSuccess || !xi) return e;
    // the tensor path recorded each block's rank k_i; the CUDA-core path decides it here
    CompressChunk ct = c;
    if (!tc || !c.kxi) ct.kxi = nullptr;
    prof::Scope ps("xi_truncate", st);
    if (fp64) k_xi_truncate<double><<<c.nblk, 256, 0, st>>>(ct);
    else k_xi_truncate<float><<<c.nblk, 256, 0, st>>>(ct);
    return cudaGetLastError();
}

cudaError_t launch_query(const QueryArgs& a, bool fp64, const QueryGrid& g, int flags, const Tuning& tu,
                         int num_sms, cudaStream_t st) {
    if (fp64) return launch_query_f64(a, g, flags, tu, num_sms, st);
    return a.fp64_refine ? launch_query_f32_refine(a, g, flags, tu, num_sms, st)
                         : launch_query_f32(a, g, flags, tu, num_sms, st);
}

bool profiling_on() { return prof::g_on.load() != 0; }

}  // namespace zs
