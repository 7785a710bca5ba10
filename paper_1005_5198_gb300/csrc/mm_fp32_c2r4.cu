// mm_fp32_c2r4.cu -- FP32 shooting kernel instantiated for thread layout 1: 2 lattice
// column(s) x 4 rows per thread, float-float sums in registers,
// registers sized for 2 CTA(s) per SM (see mm_fp32.cuh).
#include "mm_fp32.cuh"

namespace mm {
cudaError_t launch_fp32_layout1(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s)
{
    return dev::launch_fp32_layout<2, 4, true, 2>(args, grid, dump, split, s);
}
}  // namespace mm
