// zs_query_f32r.cu - query-phase launch set (Section 3.3: Partial-SVD, stack,
// Stitched-SVD, lift) for float factor stores with the FP64 refinement of the cores.
#include "zs_launch.cuh"

namespace zs {

cudaError_t launch_query_f32_refine(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                                    cudaStream_t st) {
    return query_impl<float, true>(a, g, flags, tu, num_sms, st);
}

}  // namespace zs
