/*
 * mrs.h -- C ABI of the GB300 (sm_103a) MR-STORM control-cycle library.
 *
 * The library runs, for several robot arms at once, the per-control-cycle
 * MPPI update of MR-STORM (arxiv 2602.10114): each arm samples K joint-
 * acceleration sequences around its Gaussian control distribution, rolls
 * them out over its horizon H, scores every step (goal pose, stopping
 * velocity, joint limits, world and self clearance, and clearance against
 * the other arms' published plans weighted by the dynamic priority rule),
 * and updates the distribution from the exponentiated costs.  All stages
 * run in the library's own CUDA kernels on the context's stream.
 *
 * Conventions common to every call
 *  - Every call returns an mrs_status; no exception or abort crosses the
 *    ABI.  On failure, mrs_last_error(ctx) gives a one-line reason.
 *  - Host pointers are read or written only during the call; the caller
 *    owns all memory it passes.  Device pointers (the *_device calls) are
 *    used in stream order on the context's stream.
 *  - Per-arm arrays are concatenated in arm order.  With d_a, H_a, K_a and
 *    NS_a the DoF, horizon, samples and spheres of arm a:
 *      "hd"  = sum_a H_a*d_a          "hs" = sum_a H_a*NS_a*4
 *      "d"   = sum_a d_a              "k"  = sum_a K_a
 *  - Floats are IEEE binary32.  Lengths are metres, angles radians, time
 *    seconds.  Non-finite inputs are rejected with MRS_EINVAL.
 *  - One context per host thread; calls on one context are not reentrant.
 *  - A context belongs to the device of its stream.  Every call on a
 *    context makes that device current for the call's duration and gives
 *    the caller's current device back before it returns.
 */
#ifndef MRS_H
#define MRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrs_ctx mrs_ctx;

typedef enum {
    MRS_OK = 0,
    MRS_EINVAL = 1,        /* bad argument: null, out of range, non-finite */
    MRS_ENOMEM = 2,        /* device or pinned host allocation failed */
    MRS_ECUDA = 3,         /* a CUDA runtime call failed */
    MRS_ETIMEOUT = 4,      /* a bounded wait (host or device) gave up */
    MRS_ESTATE = 5,        /* call not valid in the context's state */
    MRS_EUNSUPPORTED = 6   /* valid request the build does not support */
} mrs_status;

/* Limits of this build. */
#define MRS_MAX_ARMS 32
#define MRS_MAX_DOF 9
#define MRS_MAX_SPHERES 64
#define MRS_MAX_HORIZON 128
#define MRS_MAX_SAMPLES 8192
#define MRS_MAX_WORLD_SPHERES 1024
#define MRS_MAX_AABBS 64

/* One arm (Sec. IV-A: an arm is a DH chain whose collision geometry is N_S
 * spheres at constant transforms from its links).  Copied at create.
 *  dh          [dof][4]   a, d, alpha, theta_offset of the standard DH
 *                         convention  T_i = T_{i-1} Rz(q_i + theta_i) Tz(d_i)
 *                         Tx(a_i) Rx(alpha_i),  T_0 = base pose.
 *  q_lo, q_hi  [dof]      joint limits of the soft joint-limit cost.
 *  qd_max      [dof]      velocity limit of the safe-stopping cost.
 *  sphere_body [NS]       body of each sphere, 1..dof for link i, dof+1 for
 *                         the tool (carried by frame dof); non-decreasing.
 *                         The self-collision term (C_self of Eq. 5) runs
 *                         over the sphere pairs on bodies at least three
 *                         apart whose clearance with every joint at zero
 *                         (the rest pose) is at least B_self: pairs that
 *                         touch, or lie in the safety band, at rest belong
 *                         to the arm's build and are ignored.
 *  sphere_xyzr [NS][4]    centre in the body's frame and radius.
 *  base_pose   [7]        base position and unit quaternion (w, x, y, z).
 *  K, H                   samples per iteration and horizon.
 *  external               0: this context optimises the arm; 1: the arm is
 *                         controlled elsewhere (another process, Sec. IV-C:
 *                         each arm runs its own Algorithm 1) and only its
 *                         published plan, given through mrs_share_plans,
 *                         is used here.  Its outputs are left untouched.  */
typedef struct {
    int dof, n_spheres, K, H;
    const float *dh;
    const float *q_lo, *q_hi, *qd_max;
    const int *sphere_body;
    const float *sphere_xyzr;
    float base_pose[7];
    int external;
} mrs_arm_desc;

/* Controller parameters.
 *  dt           control period and rollout step.
 *  lambda       temperature of the MPPI weights (Eq. 2).
 *  gamma        discount of Eq. 1.
 *  alpha_mu, alpha_sigma   EMA steps of Eq. 4.
 *  sigma_init   initial standard deviation of every control (Sigma = s^2 I),
 *               also the covariance given to the new last step at a shift.
 *  w_*          weights of Eq. 5 (w_coll world, w_self self collision) and
 *               w_dyn of the coordination term (Sec. IV-A/B).
 *  B            coordination safety buffer; B_world, B_self the ramps of
 *               the world and self clearance terms.
 *  tau          priority trust exponent (Sec. IV-B).
 *  q_margin     soft-limit margin of the joint cost.
 *  iterations   optimisation iterations per cycle (the paper's K).
 *  seed         Philox key of the sampling.
 *  reserved     must be 0.  (Exact or learned clearance terms are chosen
 *               per arm after create: mrs_set_self_surrogate and
 *               mrs_set_pair_surrogate; without them every term is exact.)
 *  max_plan_age a board entry older than this many cycles counts as not
 *               published and is ignored (Sec. IV-C); 0 = no limit.
 *  w_manip      weight of C_manip of Eq. 5 (singularity avoidance, Sec.
 *               III-B): max(0, 1 - w / manip_w0) of the end-effector
 *               Jacobian's manipulability w = sqrt(det(J J^T)) (J^T J below
 *               6 DoF); 0 = term off.
 *  manip_w0     manipulability below which C_manip is positive (> 0 when
 *               w_manip > 0; ignored otherwise).                         */
typedef struct {
    int n_arms;
    const mrs_arm_desc *arms;
    float dt, lambda, gamma, alpha_mu, alpha_sigma, sigma_init;
    float w_pose, w_rot, w_stop, w_joint, w_coll, w_self, w_dyn;
    float B, B_world, B_self, tau, q_margin;
    int iterations;
    unsigned long long seed;
    int reserved;
    int max_plan_age;
    float w_manip, manip_w0;
} mrs_config;

/* Sensed state of one arm for one cycle (Alg. 1, Sense): host pointers.
 *  q, qd [dof]; goal_p [3]; goal_R [9] row-major rotation of the goal. */
typedef struct {
    const float *q, *qd, *goal_p, *goal_R;
} mrs_arm_state;

/* Results of one cycle, caller-allocated host buffers (any may be NULL).
 *  mean_plan    "hd"   mu after the update (the mean plan).
 *  plan_spheres "hs"   ToPlan(mu): the anticipated plan of Sec. IV-A,
 *                      time-major [h][sphere][x, y, z, r], h = 1..H.
 *  plan_q       "hd"   joint positions of that plan.
 *  u_star       "d"    U_* (Sec. III-A Act): first step of the cheapest
 *                      sampled sequence of the last iteration.
 *  dist_to_goal [A]    ||ee_p - g_p|| at Sense (published with the plan).
 *  min_cost     [A]    cheapest total rollout cost of the last iteration. */
typedef struct {
    float *mean_plan;
    float *plan_spheres;
    float *plan_q;
    float *u_star;
    float *dist_to_goal;
    float *min_cost;
} mrs_step_out;

/* Sizes of the concatenated arrays, for allocation by the caller. */
typedef struct {
    size_t n_arms, hd, hs, d, k, hdd;
    size_t input_floats;   /* packed device input of mrs_step_device */
    size_t output_floats;  /* packed device output (see mrs_output_device) */
    size_t state_bytes;    /* blob of mrs_save_state / mrs_load_state */
    size_t workspace_bytes;
} mrs_sizes;

/* Create a context for cfg on `stream` (a cudaStream_t, or NULL for a
 * stream the library creates).  Validates and copies cfg; allocates pinned
 * host staging; device memory comes from mrs_bind_workspace or, if that is
 * never called, is allocated at the first call that needs it.
 * Errors: MRS_EINVAL (bad cfg or limits exceeded), MRS_ENOMEM, MRS_ECUDA. */
mrs_status mrs_create(const mrs_config *cfg, void *stream, mrs_ctx **out);

/* Release everything the context allocated (not a bound workspace). */
void mrs_destroy(mrs_ctx *ctx);

/* One-line reason of the last failure on ctx ("" if none); with ctx NULL,
 * the reason of the last failed mrs_create on this thread.  mrs_create
 * returns MRS_EUNSUPPORTED when the rollout's shared-memory staging (world
 * spheres + n_arms x the largest sphere count, their clusters and candidate
 * lists) exceeds the device's per-block limit, and mrs_set_world when a
 * larger world would; within this header's limits the staging needs at most
 * about 180 KB, so on a device with 227 KB per block neither happens. */
const char *mrs_last_error(const mrs_ctx *ctx);

mrs_status mrs_query_sizes(const mrs_ctx *ctx, mrs_sizes *out);

/* Device workspace: bytes needed, and binding caller-owned device memory
 * (at least that many bytes, 256-byte aligned) that must outlive the
 * context.  Binding resets the controller to its initial state.
 * Errors: MRS_EINVAL (null, too small, misaligned). */
mrs_status mrs_workspace_size(const mrs_ctx *ctx, size_t *bytes);
mrs_status mrs_bind_workspace(mrs_ctx *ctx, void *dev_ptr, size_t bytes);

/* World obstacles (Sec. III-A Sense: the obstacle representation; treated
 * as static over the horizon unless velocities are given, in which case a
 * sphere is predicted at constant velocity: centre + vel * (t + h dt), t
 * being the time since this call; the rollout reads a copy of the spheres
 * in a spatial order, refreshed every cycle, which changes no result).
 * Host pointers:
 *  spheres [n][4] centre + radius; vel [n][3] or NULL; aabbs [m][6] centre
 *  and half extents.  n <= MRS_MAX_WORLD_SPHERES, m <= MRS_MAX_AABBS. */
mrs_status mrs_set_world(mrs_ctx *ctx, const float *spheres, const float *vel, int n_spheres,
                         const float *aabbs, int n_aabbs);

/* Publish (Alg. 1, Publish; Sec. IV-A plan communication): overwrite arm
 * `arm`'s entry of the plan board that the next mrs_step reads, with an
 * anticipated plan received from elsewhere.  plan_spheres [H_arm][NS][4]
 * time-major, plan_q [H_arm][dof] (may be NULL: then the entry carries no
 * joints and an arm-pair surrogate takes the exact pass for it), dist_to_goal >= 0 its
 * published distance-to-goal, `cycle` its publication stamp.  A negative
 * dist_to_goal withdraws the entry (the arm is then ignored, Sec. IV-C). */
mrs_status mrs_share_plans(mrs_ctx *ctx, int arm, const float *plan_spheres, const float *plan_q,
                           float dist_to_goal, long long cycle);

/* One control cycle for every arm (Algorithm 1: Sense, Shift, `iterations`
 * x {SampleControls, Rollout, UpdateDistribution}, ToPlan, Publish to the
 * board for the next cycle, PickBest).  `states` [n_arms] host pointers.
 * Blocks until the results are in `out` or until a bounded wait gives up
 * (MRS_ETIMEOUT).  After a host-side timeout (the cycle did not finish within
 * 10 s) the context must be destroyed; after a device-side one (see
 * mrs_set_wait_limit) the outputs and the state are not valid until a state
 * is loaded. */
mrs_status mrs_step(mrs_ctx *ctx, const mrs_arm_state *states, mrs_step_out *out);

/* Same cycle with device-resident inputs, enqueued on the context stream
 * without waiting.  d_input: input_floats floats, per arm in arm order
 * [q(d), qd(d), goal_p(3), goal_R(9)].  Results stay in device memory
 * (mrs_output_device). */
mrs_status mrs_step_device(mrs_ctx *ctx, const float *d_input);

/* Device pointers of the packed result buffer written by every step:
 * mean_plan(hd), plan_spheres(hs), plan_q(hd), u_star(d), dist_to_goal(A),
 * min_cost(A), each starting at a 16-byte boundary; out->* receive device
 * pointers into it. */
mrs_status mrs_output_device(mrs_ctx *ctx, mrs_step_out *out);

/* Host pointers into the context's pinned copy of that result buffer (the
 * same layout, output_floats floats), which mrs_step refreshes on every call,
 * also when its out argument is NULL.  out->* receive pointers into it, valid
 * until the context is destroyed; they hold the results of the last
 * mrs_step and are overwritten by the next one.  A caller that copies the
 * results anyway can pass out = NULL to mrs_step and copy the block from
 * here once, instead of having mrs_step copy each result into its own
 * buffer first. */
mrs_status mrs_output_host(mrs_ctx *ctx, mrs_step_out *out);

/* Wait (bounded by timeout_s seconds) for the work enqueued on the context
 * stream; MRS_ETIMEOUT if it does not finish in time. */
mrs_status mrs_sync(mrs_ctx *ctx, double timeout_s);

/* Capture the cycle in a CUDA graph (on = 1, the default) or launch the
 * kernels one by one (on = 0). */
mrs_status mrs_use_graph(mrs_ctx *ctx, int on);

/* Checkpoint / resume of the controller: state_bytes bytes holding the cycle
 * index, the world clock, mu, Sigma and the plan board.  Layout (little
 * endian): u32 magic 0x3152534d, u32 version 1, u32 n_arms, u32 pad,
 * i64 cycle, f32 world_t, f32 pad, then per arm mu[H][d], Sigma[H][d][d]
 * (f32), then per arm {i32 valid, i32 pad, i64 stamp, f32 dist, f32 pad,
 * plan_spheres[H][NS][4], plan_q[H][d]}.  Loading checks sizes and finiteness
 * and recomputes what derives from the state (the Cholesky factors of Sigma
 * that the next cycle's Shift moves), so a loaded state continues bit for
 * bit as the saved one would have. */
mrs_status mrs_save_state(mrs_ctx *ctx, void *blob, size_t bytes);
mrs_status mrs_load_state(mrs_ctx *ctx, const void *blob, size_t bytes);

/* Forward kinematics of arm `arm` for n joint vectors q [n][dof] (host):
 * ee [n][12] = rotation row-major then position of frame dof; spheres
 * [n][NS][4] world centres + radii (may be NULL).  Uses the same device code
 * as the rollout. */
mrs_status mrs_fk(mrs_ctx *ctx, int arm, int n, const float *q, float *ee, float *spheres);

/* Forward kinematics like mrs_fk, for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a library service).  A
 * control loop with a hard period cannot afford cudaMalloc/cudaFree, which may
 * block and synchronise the device, and a process whose device memory belongs
 * to another allocator may not call them at all; mrs_fk does both on every
 * call.  This call stages q and its results in one file-scope static device
 * array of 2^20 floats (4 MiB) that every GPU loading the library holds until
 * the process exits, and calls no allocating routine.
 *  - Limit: round_up(n * dof, 4) + 12 n + 4 n N_S <= 1048576 floats; larger
 *    requests fail with MRS_EINVAL before any device work.
 *  - The context must have a bound workspace (MRS_ESTATE otherwise: binding
 *    on demand would allocate).
 *  - The first call on each device (the context's device) looks up the
 *    array's device address on that device; make that first call before any
 *    stream capture.
 *  - All calls in the process share the one array and it keeps the last
 *    call's contents (nothing in it needs to start at zero: every value
 *    returned is written by the call).  Calls that overlap on the GPU, from
 *    several threads or contexts, race on it: serialise them.
 * Blocks until ee [n][12] and spheres [n][NS][4] (may be NULL) are written. */
mrs_status mrs_fk_static(mrs_ctx *ctx, int arm, int n, const float *q, float *ee, float *spheres);

/* Inspection of the last completed cycle (host outputs):
 * mrs_debug_costs   : C_n of the last iteration, [K_arm].
 * mrs_debug_spheres : sphere centres of sampled rollouts at (arm, n, h)
 *                     triples anh[n_req][3] (h 0-based), [n_req][64][4],
 *                     recomputed by the rollout's own kinematics from the
 *                     stored joint trajectory.
 * mrs_debug_alpha   : priority weights [A][A] used by the last cycle. */
mrs_status mrs_debug_costs(mrs_ctx *ctx, int arm, float *costs);
mrs_status mrs_debug_spheres(mrs_ctx *ctx, int n_req, const int *anh, float *out);
mrs_status mrs_debug_alpha(mrs_ctx *ctx, float *alpha);

/* Test hook of the device-side bounded waits: the number of polls the
 * rollout's wait for its staged plan copies may take before it gives up
 * (polls < 0: the default, 2^22; 0: give up at once).  A wait that gives up
 * sets the context's error word, waits with the default limit for its copies
 * still in flight, and ends its block; mrs_step then returns MRS_ETIMEOUT.
 * After MRS_ETIMEOUT from a device-side wait the cycle's outputs and the
 * controller state are not valid: mrs_load_state (which also clears the
 * error word) or mrs_bind_workspace makes the context usable again.  Errors:
 * MRS_EINVAL for polls above the default. */
mrs_status mrs_set_wait_limit(mrs_ctx *ctx, long long polls);

/* Debug switch: zero_noise = 1 samples eps = 0 (every rollout is the mean). */
mrs_status mrs_set_zero_noise(mrs_ctx *ctx, int zero_noise);

/* Per-stage timing of the cycle: with on = 1 every following cycle records
 * CUDA events on the context stream between its stages (also inside the
 * captured graph).  mrs_kernel_times writes the durations (ms) of the last
 * cycle's stages, in launch order: prep, then per iteration sample,
 * surrogate (zero without a surrogate), rollout, costs, update, then toplan
 * (2 + 5 * iterations values); prep is zero when Sense + Shift run inside the
 * first sample launch (every arm with at most 32 blocks of 32 samples).  *n
 * gives the capacity of ms on entry and the count on return.  Waits for the
 * cycle. */
mrs_status mrs_enable_timing(mrs_ctx *ctx, int on);
mrs_status mrs_kernel_times(mrs_ctx *ctx, float *ms, int *n);

/* Launch shape of the rollout (the kernel that runs FK, the collision passes
 * and the stage cost of every sampled step; the paper fixes no GPU mapping):
 *   tile_samples   samples per work unit, a multiple of 32 in [32, 1024]: the
 *                  unit's inputs (world at the step's time, neighbour plans
 *                  at the step) are staged once, the samples pass through
 *                  in groups of 32;
 *   blocks_per_sm  resident blocks of the persistent grid per SM, 1 ..
 *                  max_blocks_per_sm (0 = the maximum, at most 4, set by
 *                  the rollout's shared memory); up to two use the kernel
 *                  built with the largest register budget, three and four
 *                  the ones built for three and four resident blocks;
 *   order          0 step-major work list (all arms' units of step h, then
 *                  h + 1: concurrent blocks share the step's plans), 1
 *                  arm-major, 2 step-major from the last step (the later
 *                  steps' wider spread of samples tends to cost more: the
 *                  costlier units first leave a shorter tail).
 * Results do not depend on the shape (each sample's cost is reduced by its
 * own lane in every shape); only the time does.  mrs_set_rollout_shape
 * returns MRS_EINVAL for a shape out of range. */
typedef struct {
    int tile_samples, blocks_per_sm, order;
    float cycle_ms;            /* mrs_autotune: median control-cycle time of the shape */
} mrs_rollout_shape;
mrs_status mrs_set_rollout_shape(mrs_ctx *ctx, const mrs_rollout_shape *shape);
mrs_status mrs_get_rollout_shape(mrs_ctx *ctx, mrs_rollout_shape *shape, int *max_blocks_per_sm);

/* Autotuner: times every shape of the grid {32, 64, 128, 256, 512, 1024}
 * samples x 1 .. max resident blocks per SM x orders {0, 1, 2} over
 * `reps` whole control cycles each (the cycle as mrs_step_device runs it:
 * CUDA graph without per-stage timing, so programmatic launch overlaps the
 * stages; CUDA events around each cycle on the context's stream, median) on
 * the context's current inputs, every shape from the same saved state,
 * and keeps the fastest.  Each trial cycle
 * starts from a cold L2: a temporary device buffer of twice the L2 size is
 * written before it (without room for the buffer, the trials start warm).  The controller state
 * is saved before and restored after the trials, so the next cycle is
 * unaffected; per-stage timing is switched back on if it was on.  Needs one
 * earlier mrs_step / mrs_step_device (the inputs the trials use);
 * otherwise MRS_ESTATE.  `table` (host, capacity `cap`, may be null)
 * receives every shape tried with its time, *n_tried their count; `best`
 * (may be null) the one kept.  If a trial fails, the earlier shape, timing
 * switch and state are put back as far as the device allows and the
 * trial's error is returned. */
mrs_status mrs_autotune(mrs_ctx *ctx, int reps, mrs_rollout_shape *table, int cap, int *n_tried,
                        mrs_rollout_shape *best);

/* Philox4x32-10 self-test (Salmon et al., SC'11): out[n][4] = Philox of
 * ctr[n][4] under key[2], computed by the device generator the sampling
 * uses.  Host arrays; allocates a temporary device buffer. */
mrs_status mrs_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

/* ------------------------------------------------------------------------
 * Learned clearance surrogate (not in the paper: a small MLP that stands in
 * for the exact self-collision distance of Eq. 5, with exact fallback near
 * contact).  in_dim inputs (joint sin/cos features; zero-padded to a multiple
 * of 16), `layers` hidden layers of `width` units (multiple of 16, <= 256)
 * with SiLU, one linear output.  BF16 weights and activations, FP32
 * accumulation on the tensor cores, FP32 master weights trained with Adam.
 * Parameter order (mrs_mlp_get_params / set_params, FP32): per hidden layer
 * W [width][in] row-major then b [width]; then w_out [width], b_out [1].
 * Device pointers are used on the network's stream; batch sizes passed to
 * mrs_mlp_grads / mrs_mlp_train_step must be multiples of 8. */
typedef struct mrs_mlp mrs_mlp;
mrs_status mrs_mlp_create(int in_dim, int width, int layers, unsigned long long seed,
                          void *stream, mrs_mlp **out);
void mrs_mlp_destroy(mrs_mlp *m);
const char *mrs_mlp_last_error(const mrs_mlp *m);
mrs_status mrs_mlp_param_count(const mrs_mlp *m, size_t *n);
/* Training loss: squared error against targets clipped to [-0.1, 0.3] m, an
 * over-prediction (output above the clipped target: a clearance claimed
 * larger than it is, the error that can skip a colliding step) weighted by
 * over_weight >= 1 (1, the default: plain MSE). */
mrs_status mrs_mlp_set_loss(mrs_mlp *m, float over_weight);
/* Launch shape of the fused inference kernel (features, every layer and the
 * output of 128 rows per CTA; weights streamed through a ring of shared
 * memory slots): info[0] resident CTAs per SM for plain rows
 * (mrs_mlp_forward), info[1] for rollout trajectories (inside the control
 * cycle), info[2] ring slots, info[3] dynamic shared memory bytes per CTA,
 * info[4] SMs.  `n` >= 5 entries, host memory. */
mrs_status mrs_mlp_launch_info(const mrs_mlp *m, int *info, int n);
mrs_status mrs_mlp_get_params(mrs_mlp *m, float *host, size_t n);
mrs_status mrs_mlp_set_params(mrs_mlp *m, const float *host, size_t n);
/* y [n] = network(x [n][in_dim]), device pointers. */
mrs_status mrs_mlp_forward(mrs_mlp *m, const float *d_x, int n, float *d_y);
/* Gradients of the mean squared error against targets t [n] clipped to
 * [-0.1, 0.3] m (host output in parameter order, and the loss). */
mrs_status mrs_mlp_grads(mrs_mlp *m, const float *d_x, const float *d_t, int n, float *host_grads,
                         float *host_loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that loss. */
mrs_status mrs_mlp_train_step(mrs_mlp *m, const float *d_x, const float *d_t, int n, float lr,
                              float *host_loss);

/* Use a surrogate for arm `arm`'s self-collision clearance in the cycle
 * (net = NULL: back to exact).  Every rollout step's clearance is predicted
 * from the sin/cos of its joint angles (net input = 2 * dof); steps whose
 * prediction is at least B_self + margin get a zero self term, the others the
 * exact computation.  The network must outlive its use by the context. */
mrs_status mrs_set_self_surrogate(mrs_ctx *ctx, int arm, mrs_mlp *net, float margin);
/* Training data for an arm's surrogate, on the device: n joint vectors
 * uniform within the joint limits (Philox, `seed`), their features d_x
 * [n][2 dof] (sin, cos per joint) and exact self-collision clearance d_t [n]
 * (the minimum over the arm's self-collision pairs, see mrs_arm_desc, of
 * centre distance minus radii); d_q [n][dof] receives the joint vectors (may
 * be NULL). */
mrs_status mrs_self_dataset(mrs_ctx *ctx, int arm, int n, unsigned long long seed, float *d_x,
                            float *d_t, float *d_q);
/* Exact self-collision clearance of joint vectors d_q [n][dof] -> d_out [n]. */
mrs_status mrs_self_distance(mrs_ctx *ctx, int arm, int n, const float *d_q, float *d_out);
/* Of the last cycle, every rollout step [H][K] of an arm: the surrogate's
 * predicted clearance and (recomputed) the exact one; either may be NULL. */
mrs_status mrs_debug_self(mrs_ctx *ctx, int arm, float *dhat, float *exact);

/* Learned arm-to-arm clearance (not in the paper): a network (mrs_mlp with
 * input 2 d_a + 2 d_b + 7: sin, cos of arm a's joints at the sampled step,
 * sin, cos of arm b's published plan joints at the same step, arm b's base
 * pose in arm a's base frame as xyz + quaternion w x y z) that predicts the
 * clearance between arm a's spheres and arm b's plan spheres (the set
 * distance of Eq. 6, unclamped).  With a network set for (a, b) (b = -1:
 * every other arm), every rollout step of arm a is predicted before the
 * rollout, and a step whose prediction is at least B + margin skips the exact
 * pass against b's plan (its coordination term with b is zero); the others,
 * and plans published without joints, take the exact pass.  net = NULL
 * removes it.  The first call allocates the prediction buffer (sum_a K_a H_a
 * x n_arms floats, owned by the context).  The network must outlive its use
 * by the context. */
mrs_status mrs_set_pair_surrogate(mrs_ctx *ctx, int a, int b, mrs_mlp *net, float margin);
/* Arm b's base pose in arm a's base frame, pose[7] = xyz, quaternion w x y z
 * (host): the pose inputs of the arm-pair network. */
mrs_status mrs_relative_pose(mrs_ctx *ctx, int a, int b, float *pose);
/* Arm-pair training data, on the device: n rows of joint vectors of arms a
 * and b uniform within their limits (Philox, `seed`) and a relative pose, one
 * of poses [n_pose][7] (host; NULL: b's actual pose in a's frame) drawn
 * uniformly and jittered by +-jit_t per axis and +-jit_yaw (radians) about
 * its z axis; features d_x [n][2 d_a + 2 d_b + 7], exact clearance d_t [n]
 * (arm a at its base frame, arm b at the pose: minimum over all sphere pairs
 * of centre distance minus radii); d_qa [n][d_a], d_qb [n][d_b] and d_pose
 * [n][7] receive the joints and poses (each may be NULL). */
mrs_status mrs_pair_dataset(mrs_ctx *ctx, int a, int b, int n, unsigned long long seed,
                            const float *poses, int n_pose, float jit_t, float jit_yaw, float *d_x,
                            float *d_t, float *d_qa, float *d_qb, float *d_pose);
/* Of the last cycle, every rollout step [H_a][K_a] of arm a: the arm-pair
 * surrogate's predicted clearance to arm b's plan and (recomputed) the exact
 * one against b's plan spheres at step min(h, H_b - 1) as that cycle read
 * them (with an arm-pair surrogate set, the cycle keeps a copy: the board
 * holds the new plans after it); either may be NULL (host). */
mrs_status mrs_debug_pair(mrs_ctx *ctx, int a, int b, float *rhohat, float *exact);

/* Tensor-core GEMM self-test: C [M][N] (FP32) = A [M][K] B [N][K]^T with A, B
 * BF16 bit patterns (host arrays); N multiple of 16 up to 256, K multiple of 8. */
mrs_status mrs_selftest_gemm(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *C);

#ifdef __cplusplus
}
#endif
#endif /* MRS_H */
