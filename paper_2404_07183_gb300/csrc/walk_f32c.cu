// walk_f32c.cu -- instantiations of the tile walk for the F32C precision.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f32c(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_t<float, kF32C>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
