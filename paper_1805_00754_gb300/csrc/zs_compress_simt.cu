// zs_compress_simt.cu - storage-phase launch set of the CUDA-core path (FP64
// stores, n < 64, or the exact FP32 Gram): Gram, eigen core, U = A V Sigma^-1
// over every block of a chunk (Section 3.2).
#include "zs_launch.cuh"

namespace zs {

template <typename Tin, typename T, bool REF>
static cudaError_t compress_impl(const CompressChunk& c, const Tuning& tu, int num_sms, cudaStream_t st) {
    const int ntile = (c.n + 63) / 64;
    const int npairs = ntile * (ntile + 1) / 2;
    dim3 gg(npairs, std::min(c.nblk, 65535));
    {
        prof::Scope ps("gram_compress", st);
        k_gram_compress<Tin, T><<<gg, 256, 0, st>>>(c);
    }
    ZS_TRY(cudaGetLastError());
    const bool fp64 = std::is_same<T, double>::value;
    const EigPlan ep = eig_plan(c.n, c.k, tu.eig_m_extra, fp64, REF);
    if (!ep.ok) return cudaErrorInvalidValue;
    const int grid_e = std::min(c.nblk, ep.yglob ? c.ews_ctas : 65535);
    if (ep.m <= 32) {
        ZS_TRY(set_smem(k_eig_compress<T, REF, 32>, ep.smem));
        prof::Scope ps("eig_compress", st);
        k_eig_compress<T, REF, 32><<<grid_e, 256, ep.smem, st>>>(c, ep.m, ep.yglob, c.ews);
    } else {
        ZS_TRY(set_smem(k_eig_compress<T, REF, 64>, ep.smem));
        prof::Scope ps("eig_compress", st);
        k_eig_compress<T, REF, 64><<<grid_e, 256, ep.smem, st>>>(c, ep.m, ep.yglob, c.ews);
    }
    ZS_TRY(cudaGetLastError());
    const size_t smu = sizeof(T) * ((size_t)c.k * (c.n + 1) + 32 * (size_t)(c.n + 1) + c.k) + 64;
    ZS_TRY(set_smem(k_form_u<Tin, T>, smu));
    dim3 gu(std::min((c.b + 31) / 32, 8), std::min(c.nblk, 65535));
    {
        prof::Scope ps("form_u", st);
        k_form_u<Tin, T><<<gu, 256, smu, st>>>(c);
    }
    ZS_TRY(cudaGetLastError());
    note_launches(3);
    (void)num_sms;
    return cudaSuccess;
}

cudaError_t launch_compress_simt(const CompressChunk& c, bool fp64, int flags, const Tuning& tu, int num_sms,
                                 cudaStream_t st) {
    const bool ref = (flags & 1) != 0;
    if (fp64) return compress_impl<double, double, false>(c, tu, num_sms, st);
    if (c.in_kind == IN_BF16)
        return ref ? compress_impl<__nv_bfloat16, float, true>(c, tu, num_sms, st)
                   : compress_impl<__nv_bfloat16, float, false>(c, tu, num_sms, st);
    return ref ? compress_impl<float, float, true>(c, tu, num_sms, st)
               : compress_impl<float, float, false>(c, tu, num_sms, st);
}

}  // namespace zs
