// walk_f32k_t512x3.cu -- keyed tile walk (float64 input, exact order keys): F32 precision, 512-thread CTAs, 3 per SM.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f32k_t512x3(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_tt<float, kF32, 512, 3, 0, true>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
