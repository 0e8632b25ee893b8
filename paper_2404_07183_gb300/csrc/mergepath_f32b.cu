// mergepath_f32b.cu -- warp-per-pair merge-path instantiations, F32B precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f32b(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<float, kF32B>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
