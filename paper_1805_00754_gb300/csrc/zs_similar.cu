// zs_similar.cu - similar-range search (Section 6, case study) over the
// batched query phase.
//
// The base range [t_s, t_e] (length L) is answered with k_out = 1, then every
// window of length L that starts at t_s - j * stride >= 0 (j = 1, 2, ...) is
// answered through zs_query_batch in chunks of windows.  Each window is
// scored by the cosine of its first left singular vector with the base's
// (Section 6 compares the temporal patterns u_1 of equally long ranges),
// computed on the device with a fixed reduction order.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "zoomsvd.h"
#include "zs_api_internal.h"
#include "zs_internal.h"

namespace zs {

// One CTA per window: <u1, u_w>, |u1|^2 and |u_w|^2 over the L rows (thread
// partials in row order, then a fixed warp-shuffle and cross-warp tree), then
// cos = <u1, u_w> / sqrt(|u1|^2 |u_w|^2), or 0 when a vector is zero.
template <typename T>
__global__ void __launch_bounds__(256) k_window_cos(const T* __restrict__ u1, const T* __restrict__ U, int64_t L,
                                                    int nwin, double* __restrict__ cos_out) {
    __shared__ double red[3][8];
    const int w = blockIdx.x;
    if (w >= nwin) return;
    const T* u = U + (size_t)w * L;
    double d = 0.0, a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < L; i += 256) {
        const double x = (double)u1[i], y = (double)u[i];
        d = fma(x, y, d);
        a = fma(x, x, a);
        b = fma(y, y, b);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, off);
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = d;
        red[1][warp] = a;
        red[2][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sd = 0.0, sa = 0.0, sb = 0.0;
        for (int i = 0; i < 8; ++i) {
            sd += red[0][i];
            sa += red[1][i];
            sb += red[2][i];
        }
        const double nn = sa * sb;
        cos_out[w] = nn > 0.0 ? sd / sqrt(nn) : 0.0;
    }
}

}  // namespace zs

using zs::fail;

extern "C" zs_status zs_similar_ranges(zs_store* st, int64_t base_ts, int64_t base_te, int64_t stride,
                                       int32_t max_windows, int64_t* starts, double* cos, int32_t* nwin,
                                       void* stream_) {
    if (!st || !starts || !cos || !nwin) return fail(ZS_EINVAL, "null argument");
    if (stride < 1 || max_windows < 0) return fail(ZS_EINVAL, "stride %lld or max_windows %d out of range",
                                                   (long long)stride, max_windows);
    int64_t T = 0;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        T = st->T;
    }
    if (base_ts < 0 || base_ts > base_te || base_te >= T)
        return fail(ZS_ERANGE, "base range [%lld, %lld] outside [0, %lld)", (long long)base_ts, (long long)base_te,
                    (long long)T);
    const int64_t L = base_te - base_ts + 1;
    const int nw = (int)std::min<int64_t>(max_windows, base_ts / stride);
    *nwin = nw;
    for (int j = 0; j < nw; ++j) starts[j] = base_ts - (int64_t)(j + 1) * stride;
    if (nw == 0) return ZS_OK;
    cudaStream_t stream = (cudaStream_t)stream_;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != st->cfg.device) cudaSetDevice(st->cfg.device);
    const size_t ts = st->tsize, n = (size_t)st->cfg.n;
    // windows per zs_query_batch: their first left vectors in <= 256 MiB
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)nw, 4096,
                                                                    ((int64_t)256 << 20) / (L * (int64_t)ts)}));
    void *u1 = nullptr, *s1 = nullptr, *v1 = nullptr, *Uw = nullptr, *Sw = nullptr, *Vw = nullptr;
    double* dcos = nullptr;
    zs_status s = ZS_OK;
    auto al = [&](void** p, size_t bytes) {
        if (s != ZS_OK) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(ZS_ENOMEM, "similar-range scratch (%zu bytes)", bytes);
        }
    };
    al(&u1, ts * L);
    al(&s1, ts);
    al(&v1, ts * n);
    al(&Uw, ts * L * chunk);
    al(&Sw, ts * chunk);
    al(&Vw, ts * n * chunk);
    al((void**)&dcos, sizeof(double) * nw);
    if (s == ZS_OK) {
        zs_result rb{u1, 1, s1, v1, 1, nullptr};
        s = zs_query(st, base_ts, base_te, 1, &rb, stream);
    }
    std::vector<int64_t> wts, wte;
    std::vector<zs_result> res;
    for (int j0 = 0; s == ZS_OK && j0 < nw; j0 += chunk) {
        const int c = std::min(chunk, nw - j0);
        wts.resize(c);
        wte.resize(c);
        res.resize(c);
        for (int j = 0; j < c; ++j) {
            wts[j] = starts[j0 + j];
            wte[j] = starts[j0 + j] + L - 1;
            res[j] = zs_result{(char*)Uw + ts * L * j, 1, (char*)Sw + ts * j, (char*)Vw + ts * n * j, 1, nullptr};
        }
        s = zs_query_batch(st, wts.data(), wte.data(), c, 1, res.data(), stream);
        if (s != ZS_OK) break;
        if (st->fp64)
            zs::k_window_cos<double><<<c, 256, 0, stream>>>((const double*)u1, (const double*)Uw, L, c, dcos + j0);
        else
            zs::k_window_cos<float><<<c, 256, 0, stream>>>((const float*)u1, (const float*)Uw, L, c, dcos + j0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = zs::cuda_fail(e, "window cosine kernel");
        // the next chunk's queries reuse the window buffers after this
        // kernel in stream order
    }
    if (s == ZS_OK) {
        cudaError_t e = cudaMemcpyAsync(cos, dcos, sizeof(double) * nw, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) s = zs::cuda_fail(e, "copy cosines");
    } else {
        cudaStreamSynchronize(stream);      // nothing in flight uses the scratch when it is freed
    }
    for (void* p : {u1, s1, v1, Uw, Sw, Vw, (void*)dcos})
        if (p) cudaFree(p);
    if (prev != st->cfg.device) cudaSetDevice(prev);
    return s;
}
