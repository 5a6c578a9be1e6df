// rollout_mb2.cu -- the rollout kernel built for two resident blocks per SM
// (a larger register budget), in its own translation unit so that the two
// variants compile in parallel.
#include "rollout_kernel.cuh"

namespace mrs {

int rollout_occupancy_mb2(size_t smem) { return rollout_occupancy_t<2>(smem); }

cudaError_t rollout_configure_mb2(size_t smem) { return rollout_configure_t<2, kAllSizes>(smem); }

cudaError_t rollout_launch_mb2(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                               cudaStream_t s, bool pdl)
{
    return rollout_launch_t<2, kAllSizes>(P, D, L, iter, s, pdl);
}

}  // namespace mrs
