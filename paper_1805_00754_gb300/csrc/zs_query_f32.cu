// zs_query_f32.cu - query-phase launch set (Section 3.3: Partial-SVD, stack,
// Stitched-SVD, lift) for float factor stores (FP32 cores).
#include "zs_launch.cuh"

namespace zs {

cudaError_t launch_query_f32(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st) {
    return query_impl<float, false>(a, g, flags, tu, num_sms, st);
}

}  // namespace zs
