// zs_compress_tc.cu - storage-phase launch set of the tensor-core path (float
// factor stores, n >= 64): bf16 Gram, subspace, split-bf16 projection,
// Rayleigh-Ritz core and outputs over every block of a chunk (Section 3.2).
#include "zs_launch.cuh"

namespace zs {

template <typename Tin, bool REF>
static cudaError_t compress_tc(const CompressChunk& c, const Tuning& tu, int num_sms, cudaStream_t st) {
    TcScratch sc;
    sc.G = (float*)c.G;
    sc.Qf = (float*)c.qb;
    sc.Y = (float*)c.ys;
    sc.ews = c.ews;
    sc.ews_ctas = std::max(1, c.ews_ctas);
    sc.m = tc_width(c.k, tu.eig_m_extra);
    sc.power_its = tu.power_its;
    tc_aux_carve(c.aux, c.nblk, (int64_t)c.nblk * ((c.b + 127) / 128), sc.m, c.k, sc);
    sc.fault = c.fault;
    sc.noconv = c.noconv;
    sc.refined = c.refined;
    sc.xi = c.xi;
    sc.energy = c.energy;
    sc.kxi = (c.xi > 0.0 && c.energy) ? c.kxi : nullptr;
    SrcCompress src{c};
    const bool aligned = (reinterpret_cast<uintptr_t>(c.A) % 16 == 0) && (c.lda % 4 == 0);
    return tc_core<SrcCompress, Tin, REF, false>(src, sc, c.n, c.k, c.nblk,
                                                 (int64_t)c.nblk * ((c.b + 127) / 128), sc.ews_ctas, num_sms,
                                                 tu, st, aligned);
}

bool tc_sketch_path(int n, int m, int fused_sketch) { return fused_sketch && sketch_fits(n, m); }

cudaError_t launch_compress_tc(const CompressChunk& c, int flags, const Tuning& tu, int num_sms, cudaStream_t st) {
    const bool ref = (flags & 1) != 0;
    if (c.in_kind == IN_BF16)
        return ref ? compress_tc<__nv_bfloat16, true>(c, tu, num_sms, st)
                   : compress_tc<__nv_bfloat16, false>(c, tu, num_sms, st);
    return ref ? compress_tc<float, true>(c, tu, num_sms, st) : compress_tc<float, false>(c, tu, num_sms, st);
}

}  // namespace zs
