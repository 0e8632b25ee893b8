// walk_f64.cu -- instantiations of the tile walk for the F64 precision.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f64(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_t<double, kF64>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
