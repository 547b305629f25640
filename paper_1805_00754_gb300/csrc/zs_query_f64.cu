// zs_query_f64.cu - query-phase launch set (Section 3.3: Partial-SVD, stack,
// Stitched-SVD, lift) for FP64 stores.
#include "zs_launch.cuh"

namespace zs {

cudaError_t launch_query_f64(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st) {
    return query_impl<double, false>(a, g, flags, tu, num_sms, st);
}

}  // namespace zs
