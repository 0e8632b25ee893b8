// mergepath_f64.cu -- warp-per-pair merge-path instantiations, F64 precision.
#include "mergepath.cuh"

namespace pcfgb {
cudaError_t launch_mergepath_f64(int combo, const WalkArgs& a, int64_t npairs, int grid, cudaStream_t s)
{
    return launch_mergepath_t<double, kF64>(combo, a, npairs, grid, s);
}
}  // namespace pcfgb
