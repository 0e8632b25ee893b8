// mergepath_f32c.cu -- warp-per-pair merge-path instantiations, F32C precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f32c(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<float, kF32C>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
