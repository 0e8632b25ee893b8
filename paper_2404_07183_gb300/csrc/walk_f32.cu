// walk_f32.cu -- instantiations of the tile walk for the F32 precision.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f32(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_t<float, kF32>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
