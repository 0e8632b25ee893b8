// mergepath_f32bk.cu -- keyed warp-per-pair merge-path instantiations (float64 input), F32B precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f32bk(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<float, kF32B, true>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
