// Step kernels instantiated for __nv_bfloat16 storage (see lbm_step.cuh).
#include "lbm_step.cuh"

namespace lbm {

cudaError_t launch_step_bf16(int kind, const void *src, void *dst, const Geo &g, const CollBoth &c, LaunchShape s,
                             cudaStream_t stream)
{
    return step_any<__nv_bfloat16>(kind, const_cast<void *>(src), dst, g, c, s, stream);
}

}  // namespace lbm
