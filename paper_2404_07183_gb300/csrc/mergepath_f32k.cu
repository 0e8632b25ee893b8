// mergepath_f32k.cu -- keyed warp-per-pair merge-path instantiations (float64 input), F32 precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f32k(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<float, kF32, true>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
