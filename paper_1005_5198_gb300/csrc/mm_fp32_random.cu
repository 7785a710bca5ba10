// mm_fp32_random.cu -- FP32 shooting kernel for maps of random rays (mm_params.ray_mode
// MM_RAYS_RANDOM), instantiated for thread layout 3: 2 lattice columns x 4 rows per thread,
// float-float sums in registers, registers sized for 1 CTA per SM (the per-ray offsets need more
// registers than 2 CTAs leave; see mm_fp32.cuh).
#include "mm_fp32.cuh"

namespace mm {
cudaError_t launch_shoot_fp32_random(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s)
{
    static_assert(kRandomLayout == 3, "the random-ray kernel is instantiated for layout 3");
    return dev::launch_fp32_layout<2, 4, true, 1, true>(args, grid, dump, split, s);
}
}  // namespace mm
