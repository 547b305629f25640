// zs_noalloc.cu - storage-phase compression that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, plug-ins living inside a host application that owns every
// device allocation through its own pool, or latency-critical loops that must
// never enter the driver's allocator.  For them zs_compress_noalloc runs the
// same storage-phase kernels as zs_store_append, but their scratch (the n x n
// Gram matrix of each block and, for large n, the eigen core's subspace block)
// lives in one file-scope device array of fixed size instead of memory the
// library allocates.  The caller supplies the input rows and the output
// factor buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "zoomsvd.h"
#include "zs_api_internal.h"
#include "zs_internal.h"

namespace {

// Fixed scratch, resident on every device that loads this library until the
// process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
// Status words of the last call: [0] a bounded wait of a tensor-core kernel
// gave up (results undefined), [1] blocks whose accuracy refinement stopped at
// its pass cap.  Cleared at the start of every call.
__device__ __align__(16) int g_noalloc_status[4];

// Device addresses of the two arrays, looked up once per device with that
// device current (host code may not use the symbols themselves as device
// pointers).  They stay valid for the life of the device's primary context:
// after cudaDeviceReset the module is loaded again at new addresses, so a
// process that resets a device must not call zs_compress_noalloc on it again.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};
int* g_stat[kMaxDevices] = {nullptr};

zs_status scratch_address(int dev, void** out, int** stat) {
    if (dev < 0 || dev >= kMaxDevices) return zs::fail(ZS_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return zs::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        e = cudaGetSymbolAddress(&q, g_noalloc_status);
        if (e != cudaSuccess) return zs::cuda_fail(e, "cudaGetSymbolAddress(no-alloc status)");
        g_addr[dev] = p;
        g_stat[dev] = (int*)q;
    }
    *out = g_addr[dev];
    if (stat) *stat = g_stat[dev];
    return ZS_OK;
}

}  // namespace

extern "C" zs_status zs_compress_noalloc(const void* rows, int64_t nrows, int64_t ld, int32_t in_dtype, int64_t n,
                                         int64_t b, int32_t k, int32_t flags, void* U, void* sigma, void* Vt,
                                         void* stream) {
    if (in_dtype != ZS_F64 && in_dtype != ZS_F32 && in_dtype != ZS_BF16)
        return zs::fail(ZS_EDTYPE, "unknown in_dtype %d", in_dtype);
    if (n < 1 || n > 1024 || b < 1 || b > ((int64_t)1 << 24) || k < 1 || k > 64 || k > n || nrows < 0 || ld < n)
        return zs::fail(ZS_EINVAL, "bad sizes (n=%lld b=%lld k=%d nrows=%lld ld=%lld)", (long long)n, (long long)b,
                        k, (long long)nrows, (long long)ld);
    if (nrows == 0) return ZS_OK;
    if (!rows || !U || !sigma || !Vt) return zs::fail(ZS_EINVAL, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "cudaGetDevice");
    void* scratch = nullptr;
    int* stat = nullptr;
    zs_status s = scratch_address(dev, &scratch, &stat);
    if (s != ZS_OK) return s;
    int num_sms = 1;
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "cudaDeviceGetAttribute");

    const bool fp64 = (in_dtype == ZS_F64);
    const bool ref = (flags & ZS_FLAG_FP64_REFINE) && !fp64;
    const zs::Tuning tune;
    const zs::EigPlan ep = zs::eig_plan((int)n, k, tune.eig_m_extra, fp64, ref);
    if (!ep.ok) return zs::fail(ZS_EINVAL, "n=%lld with k=%d does not fit the eigen core", (long long)n, k);
    const size_t ts = fp64 ? 8 : 4;
    const size_t insize = in_dtype == ZS_F64 ? 8 : (in_dtype == ZS_F32 ? 4 : 2);
    // carve: [eigen workspace | Gram matrices of one chunk of blocks]
    int ews_ctas = 0;
    size_t ews_bytes = 0;
    if (ep.yglob) {
        ews_ctas = std::max(1, num_sms);
        while (ews_ctas > 1 && zs::eig_ws_bytes((int)n, fp64, ews_ctas) > kNoAllocScratchBytes / 2) ews_ctas /= 2;
        ews_bytes = (zs::eig_ws_bytes((int)n, fp64, ews_ctas) + 255) & ~(size_t)255;
    }
    // per block: its Gram matrix (or subspace sketch) and, on the tensor path,
    // its tf32 subspace basis and projection block
    const bool tc = zs::use_tc_path(fp64, (int)n, flags);
    const size_t mt = tc ? (size_t)zs::tc_width(k, tune.eig_m_extra) : 0;
    if (tc && ews_bytes == 0) {
        ews_ctas = std::max(1, num_sms);
        while (ews_ctas > 1 && zs::eig_ws_bytes((int)n, fp64, ews_ctas) > kNoAllocScratchBytes / 4) ews_ctas /= 2;
        ews_bytes = (zs::eig_ws_bytes((int)n, fp64, ews_ctas) + 255) & ~(size_t)255;
    }
    auto r256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t qper = tc ? r256(4 * zs::tc_qb_floats((int)mt, (int)n)) : 0;
    const size_t proj = r256(4 * mt * (size_t)b);
    // Rayleigh-Ritz scratch of one block (tile partials, Q~^T Q~, Ritz data,
    // the accuracy test's list) with slack for the alignment of its sections
    const size_t auxp = tc ? r256(4 * mt * mt * ((b + 127) / 128 + 1) + 4 * mt * k + 4 * k + 4 * mt + 4 + 2048) : 0;
    const size_t yper = proj + auxp;
    const size_t gper = ((ts * (size_t)n * n) + 255) & ~(size_t)255;
    if (ews_bytes + gper + qper + yper > kNoAllocScratchBytes)
        return zs::fail(ZS_EINVAL,
                        "n=%lld, b=%lld, k=%d need %zu scratch bytes per block (n x n Gram, and on the float tensor "
                        "path a basis of n x %zu and b x %zu projections); the no-alloc scratch holds %zu",
                        (long long)n, (long long)b, k, ews_bytes + gper + qper + yper, mt, mt, kNoAllocScratchBytes);
    const int chunk = (int)std::min<size_t>((kNoAllocScratchBytes - ews_bytes) / (gper + qper + yper), 65535);
    const int64_t nblk = (nrows + b - 1) / b;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(stat, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return zs::cuda_fail(e, "status clear");
    for (int64_t j0 = 0; j0 < nblk; j0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, nblk - j0);
        zs::CompressChunk ch;
        memset(&ch, 0, sizeof ch);
        ch.A = (const char*)rows + (size_t)j0 * b * ld * insize;
        ch.lda = ld;
        ch.rows_total = std::min<int64_t>(nrows - j0 * b, (int64_t)nb * b);
        ch.nblk = nb;
        ch.slot0 = 0;
        ch.b = (int32_t)b;
        ch.n = (int32_t)n;
        ch.k = k;
        ch.in_kind = in_dtype;
        ch.G = (char*)scratch + ews_bytes;
        ch.qb = tc ? (char*)scratch + ews_bytes + gper * chunk : nullptr;
        ch.ys = tc ? (char*)scratch + ews_bytes + (gper + qper) * chunk : nullptr;
        // the Rayleigh-Ritz scratch follows the projections of the chunk
        ch.aux = tc ? (char*)ch.ys + proj * chunk : nullptr;
        ch.ews = (ep.yglob || tc) ? scratch : nullptr;
        ch.ews_ctas = ews_ctas;
        ch.U = (char*)U + ts * (size_t)j0 * b * k;
        ch.sig = (char*)sigma + ts * (size_t)j0 * k;
        ch.vt = (char*)Vt + ts * (size_t)j0 * k * n;
        ch.fault = stat;
        ch.noconv = stat + 1;
        e = zs::launch_compress(ch, fp64, flags, tune, num_sms, st);
        if (e != cudaSuccess) return zs::cuda_fail(e, "compression kernels");
    }
    return ZS_OK;
}

extern "C" zs_status zs_noalloc_status(int32_t* fault, int32_t* unconverged_blocks) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return zs::cuda_fail(e, "cudaGetDevice");
    void* scratch = nullptr;
    int* stat = nullptr;
    zs_status s = scratch_address(dev, &scratch, &stat);
    if (s != ZS_OK) return s;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return zs::cuda_fail(e, "status wait");
    int v[4] = {0, 0, 0, 0};
    e = cudaMemcpy(v, stat, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return zs::cuda_fail(e, "status read");
    if (fault) *fault = v[0];
    if (unconverged_blocks) *unconverged_blocks = v[1];
    if (v[0]) return zs::fail(ZS_ETIMEDOUT, "a bounded wait of a tensor-core kernel gave up; results are undefined");
    if (v[1]) return zs::fail(ZS_ENOCONV, "%d block(s) did not pass the accuracy test within the pass cap", v[1]);
    return ZS_OK;
}
