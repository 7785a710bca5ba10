// mm_fp32_c1r8.cu -- FP32 shooting kernel instantiated for thread layout 0: 1 lattice
// column(s) x 8 rows per thread, float-float sums in registers,
// registers sized for 2 CTA(s) per SM (see mm_fp32.cuh).
#include "mm_fp32.cuh"

namespace mm {
cudaError_t launch_fp32_layout0(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s)
{
    return dev::launch_fp32_layout<1, 8, true, 2>(args, grid, dump, split, s);
}
}  // namespace mm
