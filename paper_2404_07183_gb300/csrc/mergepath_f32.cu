// mergepath_f32.cu -- warp-per-pair merge-path instantiations, F32 precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f32(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<float, kF32>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
