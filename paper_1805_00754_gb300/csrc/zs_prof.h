// zs_prof.h - the library's per-kernel profiler scope (host only).
#pragma once

#include <cuda_runtime.h>

namespace zs {

// CUDA events around one launch on its stream, recorded only while the
// library's profiler is on (zs_profile_enable); defined in zs_launch_common.cu.
namespace prof {
struct Scope {
    int id = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st;
    Scope(const char* name, cudaStream_t s);
    ~Scope();
};
}  // namespace prof

}  // namespace zs
