// rollout_spg4.cu -- the rollout kernel built for arms of 4 spheres per
// sphere group (the routines of those sizes only), for each
// register budget; a translation unit of its own so that the builds compile
// in parallel.
#include "rollout_kernel.cuh"

namespace mrs {

cudaError_t rollout_configure_spg4(size_t smem)
{
    cudaError_t e = rollout_configure_t<2, kSizes4>(smem);
    if (e == cudaSuccess) e = rollout_configure_t<3, kSizes4>(smem);
    return e != cudaSuccess ? e : rollout_configure_t<4, kSizes4>(smem);
}

cudaError_t rollout_launch_spg4(int variant, const Params &P, const Dev &D, const LaunchPlan &L,
                                int iter, cudaStream_t s, bool pdl)
{
    if (variant == 2) return rollout_launch_t<2, kSizes4>(P, D, L, iter, s, pdl);
    if (variant == 4) return rollout_launch_t<4, kSizes4>(P, D, L, iter, s, pdl);
    return rollout_launch_t<3, kSizes4>(P, D, L, iter, s, pdl);
}

}  // namespace mrs
