// rollout_spg57.cu -- the rollout kernel built for arms of 5 and 7 spheres
// per sphere group (the routines of those sizes only), for each
// register budget; a translation unit of its own so that the builds compile
// in parallel.
#include "rollout_kernel.cuh"

namespace mrs {

cudaError_t rollout_configure_spg57(size_t smem)
{
    cudaError_t e = rollout_configure_t<2, kSizes57>(smem);
    if (e == cudaSuccess) e = rollout_configure_t<3, kSizes57>(smem);
    return e != cudaSuccess ? e : rollout_configure_t<4, kSizes57>(smem);
}

cudaError_t rollout_launch_spg57(int variant, const Params &P, const Dev &D, const LaunchPlan &L,
                                int iter, cudaStream_t s, bool pdl)
{
    if (variant == 2) return rollout_launch_t<2, kSizes57>(P, D, L, iter, s, pdl);
    if (variant == 4) return rollout_launch_t<4, kSizes57>(P, D, L, iter, s, pdl);
    return rollout_launch_t<3, kSizes57>(P, D, L, iter, s, pdl);
}

}  // namespace mrs
