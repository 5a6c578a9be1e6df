// kernels.cuh -- launch wrappers of the control-cycle kernels (host side).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "mlp_fused.cuh"
#include "mrs_device.cuh"

struct mrs_mlp;

namespace mrs {

// One arm whose self clearance comes from a surrogate network.
struct SurrogateSlot {
    int arm, rows;          // rows = K * H rollout steps
    int K, dof;
    long long off_kh;       // the arm's offset in Dev::dhat
    long long off_khd;      // the arm's offset in Dev::traj
    mrs_mlp *net;
};

// arms that share one surrogate network: one fused inference launch
struct SurrogateGroup {
    mrs_mlp *net;
    fused::TrajSegs segs;
};

// (arm, neighbour) pairs that share one arm-pair network: one launch
struct PairGroup {
    mrs_mlp *net;
    fused::PairSegs segs;
};

struct LaunchPlan {
    int n_arms;
    int n_sample_tiles, n_rollout_tiles, n_cost_tiles, n_update_tiles;
    const SampleTile *sample_tiles;
    const RolloutTile *rollout_tiles;
    const CostTile *cost_tiles;
    const UpdateTile *update_tiles;
    size_t smem_prep, smem_sample, smem_rollout, smem_toplan;
    int sample_tile;    // samples per sampling block: 16 (every arm of at most 1024 samples) or 32
    bool merge_prep;    // Sense + Shift inside the first sample launch (every arm of at most
                        // 1024 samples) instead of a kernel of their own
    int rollout_grid;   // persistent rollout blocks (resident blocks per SM x SMs)
    int rollout_variant;   // register budget of the rollout kernel: 2, 3 or 4 blocks per SM
    unsigned rollout_sizes;   // sphere-group sizes of the arms that roll out (bit s for size s)
    int *done_counter;  // last-block-done counter of k_toplan
    int n_surrogates;
    SurrogateSlot surrogates[MRS_MAX_ARMS];
    int n_groups;
    SurrogateGroup groups[MRS_MAX_ARMS];
    int n_pair_groups;
    PairGroup *pair_groups;   // host array owned by the context
    size_t board_bytes;       // plan spheres of the board (copied for evaluation)
    int total_kh;             // rollout steps of all arms, sum K * H
};

// surrogate network (mlp.cu): input width, and the fused forward pass over
// the sin/cos features of every rollout step of a set of arms into their
// slices of dhat, on stream s
int mlp_in_dim(const mrs_mlp *m);
cudaError_t mlp_infer_trajs(mrs_mlp *m, const float *traj, const fused::TrajSegs &segs,
                            float *dhat, int *err, cudaStream_t s);
cudaError_t mlp_infer_pairs(mrs_mlp *m, const float *traj, const float *plan,
                            const fused::PairSegs &segs, float *rhohat, int *err, cudaStream_t s);
// surrogate.cu
cudaError_t enqueue_self_dataset(const Dev &D, int arm, int n, unsigned long long seed, float *x,
                                 float *t, float *q, cudaStream_t s);
cudaError_t enqueue_self_clearance_rows(const Dev &D, int arm, int n, const float *q, float *out,
                                        cudaStream_t s);
cudaError_t enqueue_self_clearance_traj(const Dev &D, int arm, int rows, float *out, cudaStream_t s);
cudaError_t enqueue_self_surrogate(const Dev &D, const SurrogateGroup &g, cudaStream_t s);
cudaError_t enqueue_pair_surrogate(const Dev &D, const PairGroup &g, cudaStream_t s);
// arm-pair training data: rows of (q_a, q_b, pose) with q uniform within the
// limits and the pose one of poses[n_pose][7] (arm b's base in arm a's frame)
// jittered by +-jit_t per axis and +-jit_yaw about z; features x [n][2 d_a +
// 2 d_b + 7], exact clearance t [n], joints qa [n][d_a], qb [n][d_b] and the
// jittered poses [n][7] (the last three may be null)
cudaError_t enqueue_pair_dataset(const Dev &D, int a, int b, int n, unsigned long long seed,
                                 const float *poses, int n_pose, float jit_t, float jit_yaw,
                                 float *x, float *t, float *qa, float *qb, float *pose_out,
                                 cudaStream_t s);
// exact clearance of every rollout step of arm a to arm b's published plan at
// the same step: out [H_a][K_a]
cudaError_t enqueue_pair_clearance_traj(const Dev &D, int a, int b, int rows, float *out,
                                        cudaStream_t s);

// Launch of kernel k on stream s, with programmatic stream serialisation
// when pdl is set (the kernel then calls pdl_wait() before it reads what its
// predecessor writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                     bool pdl, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}

// A kernel's dynamic shared-memory limit belongs to the process (on the
// current device), not to a context: contexts of different sizes launch the
// same kernels with different amounts.  Raise the limit of `kernel` to at
// least `bytes`, never lower it (serialised over threads).
cudaError_t raise_smem_limit(const void *kernel, size_t bytes);

// The rollout kernel (rollout.cu): shared-memory size for the given
// capacities, attribute set-up and launch.
size_t rollout_smem_bytes(const Params &P, int n_arms);
cudaError_t configure_rollout(const LaunchPlan &L);
int rollout_blocks_per_sm(size_t smem);
cudaError_t launch_rollout(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                           cudaStream_t s, bool pdl = false);

// Everything one control cycle enqueues on `s` (Algorithm 1 for all arms).
// With `events` non-null, events[0] is recorded before the first kernel and
// events[i + 1] after stage i (3 + 5 * iterations events: prep, per iteration
// sample, surrogate, rollout, costs, update, then toplan); `capturing` makes
// them external event nodes of the graph being captured.
cudaError_t enqueue_cycle(const Params &P, const Dev &D, const LaunchPlan &L, cudaStream_t s,
                          cudaEvent_t *events = nullptr, bool capturing = false);
cudaError_t configure_kernels(const LaunchPlan &L);
// Fill the derived per-arm constants and reset the controller state.
cudaError_t enqueue_init(const Params &P, const Dev &D, int n_arms, int total_hdd, int total_hd,
                         cudaStream_t s);
// Cholesky factors of the state's covariances in the buffers of the given
// parity (after an initialisation or a state load)
// the rollout's copy of the world in spatial order (one block), at the
// current world time
cudaError_t enqueue_world_order(const Params &P, const Dev &D, cudaStream_t s);
cudaError_t enqueue_state_factors(const Dev &D, const LaunchPlan &L, int parity, cudaStream_t s);
cudaError_t enqueue_fk(const Dev &D, int arm, int n, const float *q, float *ee, float *spheres,
                       cudaStream_t s);
cudaError_t enqueue_debug_spheres(const Dev &D, int n_req, const int *anh, float *out,
                                  cudaStream_t s);
cudaError_t enqueue_philox(int n, const uint4 *ctr, uint2 key, uint4 *out, cudaStream_t s);
// Forward kinematics staged in the library's static device scratch of
// `device` (mrs_fk_static.cu); no device memory is allocated.
cudaError_t fk_static(const Dev &D, int device, int arm, int dof, int ns, int n,
                      const float *q_host, float *ee_host, float *spheres_host, cudaStream_t s,
                      std::string &why, bool &too_large);
size_t fk_static_capacity_floats();

}  // namespace mrs
