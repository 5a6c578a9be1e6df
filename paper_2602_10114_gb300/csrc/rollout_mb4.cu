// rollout_mb4.cu -- the rollout kernel built for four resident blocks per SM
// (64 registers per thread), in its own translation unit so that the
// variants compile in parallel.
#include "rollout_kernel.cuh"

namespace mrs {

int rollout_occupancy_mb4(size_t smem) { return rollout_occupancy_t<4>(smem); }

cudaError_t rollout_configure_mb4(size_t smem) { return rollout_configure_t<4, kAllSizes>(smem); }

cudaError_t rollout_launch_mb4(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                               cudaStream_t s, bool pdl)
{
    return rollout_launch_t<4, kAllSizes>(P, D, L, iter, s, pdl);
}

}  // namespace mrs
