// walk_f32bk_t1024w.cu -- keyed tile walk with exp(-lambda t) weights: F32B precision, 1024-thread CTAs.
#include "walk.cuh"

namespace pcfgb {
cudaError_t launch_walk_f32bk_t1024w(int combo, const WalkArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_walk_tt<float, kF32B, 1024, 1, 1, true>(combo, a, grid, smem, s);
}
}  // namespace pcfgb
