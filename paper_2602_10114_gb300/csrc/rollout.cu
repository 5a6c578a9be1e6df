// rollout.cu -- host side of the rollout kernel (rollout_kernel.cuh):
// shared-memory size, attributes, resident blocks, launch; instantiates the
// three-blocks-per-SM variant.
#include "rollout_kernel.cuh"

namespace mrs {

size_t rollout_smem_bytes(const Params &P, int n_arms)
{
    // the layout of k_rollout's dynamic shared memory, in its order
    auto a16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t n_other = (size_t)rollout_other_cap(P, n_arms);
    const size_t n_cl = (size_t)rollout_cluster_cap(P, n_arms);
    return a16(sizeof(float4) * n_other) + a16(sizeof(float4) * 2 * P.aabb_cap) +
           a16(sizeof(float4) * P.max_ns) + a16(sizeof(float4) * P.max_ns * 32) +
           a16(sizeof(float4) * 2 * n_cl) + a16(sizeof(float4) * 2 * P.max_ns) +
           a16(sizeof(int) * P.max_ns) + a16(sizeof(int2) * P.max_pairs) +
           a16(sizeof(int) * n_cl) + a16(sizeof(int) * (MRS_MAX_ARMS + 1)) +
           a16(sizeof(int) * MRS_MAX_ARMS) + a16(sizeof(float) * 2 * MRS_MAX_ARMS) +
           a16(sizeof(int) * MRS_MAX_ARMS) + a16(sizeof(float2) * 2 * kMaxDof * 32) +
           a16(sizeof(float4) * kMaxDof) + a16(sizeof(float2) * kMaxDof) +
           2 * a16(sizeof(float) * 12) + a16(n_other) +
           a16(sizeof(unsigned short) * kGroups * (size_t)rollout_cand_cap(P, n_arms)) +
           a16(sizeof(int2) * kObstaclePairCap) + sizeof(int) * 2 * (2 + (size_t)n_arms) * 32;
}

cudaError_t configure_rollout(const LaunchPlan &L)
{
    cudaError_t e = rollout_configure_t<3, kAllSizes>(L.smem_rollout);
    if (e == cudaSuccess) e = rollout_configure_mb2(L.smem_rollout);
    if (e == cudaSuccess) e = rollout_configure_mb4(L.smem_rollout);
    if (e == cudaSuccess) e = rollout_configure_spg4(L.smem_rollout);
    if (e == cudaSuccess) e = rollout_configure_spg5(L.smem_rollout);
    return e != cudaSuccess ? e : rollout_configure_spg57(L.smem_rollout);
}

// Resident blocks per SM: the largest of the variants' (the four-block
// variant's, unless its shared memory does not fit)
int rollout_blocks_per_sm(size_t smem)
{
    return std::max(std::max(rollout_occupancy_t<3>(smem), rollout_occupancy_mb2(smem)),
                    std::min(4, rollout_occupancy_mb4(smem)));
}

cudaError_t launch_rollout(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                           cudaStream_t s, bool pdl)
{
    // the smallest build that holds the size of every arm that rolls out
    const unsigned m = L.rollout_sizes;
    if (m == kSizes5) return rollout_launch_spg5(L.rollout_variant, P, D, L, iter, s, pdl);
    if (m == kSizes4) return rollout_launch_spg4(L.rollout_variant, P, D, L, iter, s, pdl);
    if (m && (m & ~kSizes57) == 0)
        return rollout_launch_spg57(L.rollout_variant, P, D, L, iter, s, pdl);
    if (L.rollout_variant == 2) return rollout_launch_mb2(P, D, L, iter, s, pdl);
    if (L.rollout_variant == 4) return rollout_launch_mb4(P, D, L, iter, s, pdl);
    return rollout_launch_t<3, kAllSizes>(P, D, L, iter, s, pdl);
}

}  // namespace mrs
