// walk_f32bk_t512.cu -- keyed tile walk (float64 input, exact order keys): F32B precision, 512-thread CTAs.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f32bk_t512(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_tt<float, kF32B, 512, 2, 0, true>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
