// Dispatch of the stream + collide step to the per-precision instantiations
// (kernels in lbm_step.cuh, one translation unit per storage precision so that
// they compile in parallel).
#include "lbm_launch.h"

namespace lbm {

cudaError_t launch_step_f64(int, const void *, void *, const Geo &, const CollBoth &, LaunchShape, cudaStream_t);
cudaError_t launch_step_f32(int, const void *, void *, const Geo &, const CollBoth &, LaunchShape, cudaStream_t);
cudaError_t launch_step_f16(int, const void *, void *, const Geo &, const CollBoth &, LaunchShape, cudaStream_t);
cudaError_t launch_step_bf16(int, const void *, void *, const Geo &, const CollBoth &, LaunchShape, cudaStream_t);

cudaError_t launch_step(int prec, int kind, const void *src, void *dst, const Geo &g, const CollBoth &c,
                        LaunchShape s, cudaStream_t stream)
{
    switch (prec) {
    case P_F64: return launch_step_f64(kind, src, dst, g, c, s, stream);
    case P_F32: return launch_step_f32(kind, src, dst, g, c, s, stream);
    case P_F16: return launch_step_f16(kind, src, dst, g, c, s, stream);
    case P_BF16: return launch_step_bf16(kind, src, dst, g, c, s, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
