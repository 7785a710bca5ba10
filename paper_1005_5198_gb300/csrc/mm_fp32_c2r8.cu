// mm_fp32_c2r8.cu -- FP32 shooting kernel instantiated for thread layout 2: 2 lattice
// column(s) x 8 rows per thread, float-float sums in shared memory,
// registers sized for 2 CTA(s) per SM (see mm_fp32.cuh).
#include "mm_fp32.cuh"

namespace mm {
cudaError_t launch_fp32_layout2(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s)
{
    return dev::launch_fp32_layout<2, 8, false, 2>(args, grid, dump, split, s);
}
}  // namespace mm
