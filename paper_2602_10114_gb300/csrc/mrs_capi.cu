// mrs_capi.cu -- the C ABI declared in include/mrs.h: context, validation,
// workspace layout, work lists, CUDA-graph capture, bounded waits, state
// checkpointing.  All arithmetic of the method runs in kernels.cu.
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "mrs.h"

using namespace mrs;

struct mrs_ctx {
    int device = 0;            // the device of the context's stream, made current by every call
    Params P{};
    Dev D{};
    LaunchPlan L{};
    int A = 0;
    std::vector<ArmDev> arms;
    mrs_sizes sz{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    bool bound = false;
    float *pin_in = nullptr, *pin_out = nullptr;
    int *pin_err = nullptr;    // the word after the output block in pin_out
    cudaEvent_t done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // mrs_step's graph: the input upload from pin_in, the cycle, and the
    // download of the output block and the error word after it into pin_out
    cudaGraph_t graph_io = nullptr;
    cudaGraphExec_t gexec_io = nullptr;
    bool use_graph = true;
    bool timing = false;
    std::vector<cudaEvent_t> events;
    std::string err;
    // workspace offsets (bytes)
    struct Layout {
        size_t arms, input, world, world_vel, world_s, world_vel_s, aabb, world_n, mu, Sigma, L, board_sph, board_q,
            board_valid, board_stamp, board_dist, traj, eps, stage_lim, stage, costs, alpha,
            e_now, n_star, out, cycle, world_t, done_counter, Lst, sample_tiles, rollout_tiles,
            cost_tiles, update_tiles, self_pairs, self_t2, work, dhat, total;
    } lay{};
    std::vector<SampleTile> sample_tiles;
    std::vector<RolloutTile> rollout_tiles;
    std::vector<CostTile> cost_tiles;
    std::vector<UpdateTile> update_tiles;
    std::vector<int> self_pairs;
    std::vector<float> self_t2;   // (r1 + B_self + r2)^2 of each self pair
    int num_sms = 0;
    // rollout launch shape (mrs_set_rollout_shape / mrs_autotune)
    int tile_samples = 32, blocks_per_sm = 0, tile_order = 0, max_blocks_per_sm = 1;
    bool has_input = false;
    int smem_optin = 0;
    // arm-pair surrogate: (arm, neighbour, network) slots, their launch groups
    // and the prediction buffer ([sum K*H][A] floats, allocated on first use)
    struct PairSlot { int a, b; mrs_mlp *net; };
    std::vector<PairSlot> pair_slots;
    std::vector<PairGroup> pair_groups;
    float *rhohat = nullptr;
    float4 *pair_board = nullptr;
};

static const char *g_noctx = "null context";
// reason of the last failed mrs_create on this thread (mrs_last_error(NULL))
static thread_local std::string g_create_err;

static mrs_status fail(mrs_ctx *c, mrs_status s, const std::string &m)
{
    if (c) c->err = m;
    return s;
}

static mrs_status cuda_fail(mrs_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, MRS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

// Makes the context's device current for one call and gives the caller's
// current device back at its end: a thread may call into a context while
// another device is current, and the context's stream, workspace, graph and
// static scratch all belong to the context's device.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(const mrs_ctx *c)
    {
        int cur = 0;
        if (c && cudaGetDevice(&cur) == cudaSuccess && cur != c->device &&
            cudaSetDevice(c->device) == cudaSuccess)
            prev = cur;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

static bool finite_arr(const float *p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static void build_layout(mrs_ctx *c)
{
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = align_up(o, 256);
        size_t at = o;
        o += bytes;
        return at;
    };
    const int A = c->A;
    size_t khd = 0, kh = 0;
    for (auto &a : c->arms) {
        khd += (size_t)a.K * a.H * a.dof;
        kh += (size_t)a.K * a.H;
    }
    auto &L = c->lay;
    L.arms = take(sizeof(ArmDev) * A);
    L.input = take(sizeof(float) * c->sz.input_floats);
    L.world = take(sizeof(float4) * MRS_MAX_WORLD_SPHERES);
    L.world_vel = take(sizeof(float4) * MRS_MAX_WORLD_SPHERES);
    L.world_s = take(sizeof(float4) * MRS_MAX_WORLD_SPHERES);
    L.world_vel_s = take(sizeof(float4) * MRS_MAX_WORLD_SPHERES);
    L.aabb = take(sizeof(float4) * 2 * MRS_MAX_AABBS);
    L.world_n = take(sizeof(int) * 2);
    L.mu = take(sizeof(float) * 2 * c->sz.hd);       // two buffers (cycle parity)
    L.Sigma = take(sizeof(float) * 2 * c->sz.hdd);
    L.L = take(sizeof(float) * c->sz.hdd);
    L.Lst = take(sizeof(float) * 2 * c->sz.hdd);
    L.board_sph = take(sizeof(float) * c->sz.hs);
    L.board_q = take(sizeof(float) * c->sz.hd);
    L.board_valid = take(sizeof(int) * A);
    L.board_stamp = take(sizeof(long long) * A);
    L.board_dist = take(sizeof(float) * A);
    L.traj = take(sizeof(float) * khd);
    L.eps = take(sizeof(float) * khd);
    L.stage_lim = take(sizeof(float) * kh);
    L.stage = take(sizeof(float) * kh);
    L.costs = take(sizeof(float) * c->sz.k);
    L.alpha = take(sizeof(float) * A * A);
    L.e_now = take(sizeof(float) * A);
    L.n_star = take(sizeof(int) * A);
    // the error word sits right after the output block: one download brings both
    L.out = take(sizeof(float) * (c->sz.output_floats + 4));
    L.cycle = take(sizeof(long long));
    L.world_t = take(sizeof(float));
    L.done_counter = take(sizeof(int));
    L.sample_tiles = take(sizeof(SampleTile) * c->sample_tiles.size());
    L.rollout_tiles = take(sizeof(RolloutTile) * c->rollout_tiles.size());
    L.cost_tiles = take(sizeof(CostTile) * c->cost_tiles.size());
    L.update_tiles = take(sizeof(UpdateTile) * c->update_tiles.size());
    L.self_pairs = take(sizeof(int) * std::max<size_t>(1, c->self_pairs.size()));
    L.self_t2 = take(sizeof(float) * std::max<size_t>(1, c->self_t2.size()));
    L.work = take(sizeof(int) * 64);
    L.dhat = take(sizeof(float) * kh);
    L.total = align_up(o, 256);
    c->sz.workspace_bytes = L.total;
}

// rollout work units of tile_samples samples; step-major order lets the
// concurrently resident blocks share the step's plan slices in L2
static void build_rollout_tiles(mrs_ctx *c)
{
    c->rollout_tiles.clear();
    const int nsub = c->tile_samples / 32;
    int Hmax = 0;
    for (auto &A : c->arms) Hmax = std::max(Hmax, A.H);
    auto push = [&](int a, int h) {
        const ArmDev &A = c->arms[a];
        for (int n0 = 0; n0 < A.K; n0 += 32 * nsub)
            c->rollout_tiles.push_back({a, h, n0, std::min(nsub, (A.K - n0 + 31) / 32)});
    };
    if (c->tile_order == 0) {
        for (int h = 0; h < Hmax; ++h)
            for (int a = 0; a < c->A; ++a)
                if (h < c->arms[a].H && !c->arms[a].external) push(a, h);
    } else if (c->tile_order == 2) {   // step-major from the last step: the later steps'
                                        // wider sample spread tends to cost more, so they go first
        for (int h = Hmax - 1; h >= 0; --h)
            for (int a = 0; a < c->A; ++a)
                if (h < c->arms[a].H && !c->arms[a].external) push(a, h);
    } else {
        for (int a = 0; a < c->A; ++a)
            if (!c->arms[a].external)
                for (int h = 0; h < c->arms[a].H; ++h) push(a, h);
    }
    // The list's last units (as many as the largest persistent grid has
    // blocks) in quarters: the blocks take their last units at different
    // times, and smaller pieces there even out when they finish.  Samples
    // keep their lanes, so no result changes; the list stays shorter than
    // the 32-sample one the workspace holds.
    if (nsub >= 4 && c->num_sms > 0) {
        auto &t = c->rollout_tiles;
        const int tail = std::min((int)t.size(), 4 * c->num_sms);
        std::vector<RolloutTile> out(t.begin(), t.end() - tail);
        out.reserve(t.size() + 3 * (size_t)tail);
        for (auto it = t.end() - tail; it != t.end(); ++it) {
            const int q = (it->nsub + 3) / 4;
            for (int k = 0; k < it->nsub; k += q)
                out.push_back({it->arm, it->h, it->n0 + 32 * k, std::min(q, it->nsub - k)});
        }
        t.swap(out);
    }
}

// persistent rollout grid and kernel variant for the shape's blocks per SM
// (0 = the maximum): up to two blocks the variant with the largest register
// budget, three and four the variants built for them
static void set_rollout_grid(mrs_ctx *c)
{
    const int bps = c->blocks_per_sm > 0 ? std::min(c->blocks_per_sm, c->max_blocks_per_sm)
                                         : c->max_blocks_per_sm;
    c->L.rollout_grid = bps * c->num_sms;
    c->L.rollout_variant = bps >= 4 ? 4 : bps >= 3 ? 3 : 2;
}

// every optimised arm has at most kSmallArmK samples: Sense + Shift inside
// the first sampling launch, and 16 samples per sampling block
static bool small_arms(const mrs_ctx *c)
{
    for (auto &A : c->arms)
        if (!A.external && A.K > kSmallArmK) return false;
    return true;
}

static void build_work_lists(mrs_ctx *c)
{
    c->sample_tiles.clear();
    c->rollout_tiles.clear();
    c->cost_tiles.clear();
    c->update_tiles.clear();
    const int tile = small_arms(c) ? 16 : 32;
    for (int a = 0; a < c->A; ++a) {
        const ArmDev &A = c->arms[a];
        if (A.external) continue;   // optimised elsewhere
        for (int n0 = 0; n0 < A.K; n0 += tile) c->sample_tiles.push_back({a, n0});
        for (int n0 = 0; n0 < A.K; n0 += 256) c->cost_tiles.push_back({a, n0});
        for (int h = 0; h < A.H; ++h) c->update_tiles.push_back({a, h});
    }
    build_rollout_tiles(c);
}

static void fill_dev(mrs_ctx *c, char *base)
{
    auto &L = c->lay;
    Dev &D = c->D;
    D.arms = (ArmDev *)(base + L.arms);
    D.input = (float *)(base + L.input);
    D.world = (float4 *)(base + L.world);
    D.world_vel = (float4 *)(base + L.world_vel);
    D.world_s = (float4 *)(base + L.world_s);
    D.world_vel_s = (float4 *)(base + L.world_vel_s);
    D.aabb = (float4 *)(base + L.aabb);
    D.world_n = (int *)(base + L.world_n);
    D.mu = (float *)(base + L.mu);
    D.Sigma = (float *)(base + L.Sigma);
    D.st_hd = (long long)c->sz.hd;
    D.st_hdd = (long long)c->sz.hdd;
    D.L = (float *)(base + L.L);
    D.Lst = (float *)(base + L.Lst);
    D.board_sph = (float4 *)(base + L.board_sph);
    D.board_q = (float *)(base + L.board_q);
    D.board_valid = (int *)(base + L.board_valid);
    D.board_stamp = (long long *)(base + L.board_stamp);
    D.board_dist = (float *)(base + L.board_dist);
    D.next_sph = nullptr;
    D.next_q = nullptr;
    D.traj = (float *)(base + L.traj);
    D.eps = (float *)(base + L.eps);
    D.stage_lim = (float *)(base + L.stage_lim);
    D.stage = (float *)(base + L.stage);
    D.costs = (float *)(base + L.costs);
    D.alpha = (float *)(base + L.alpha);
    D.e_now = (float *)(base + L.e_now);
    D.n_star = (int *)(base + L.n_star);
    D.out = (float *)(base + L.out);
    D.cycle = (long long *)(base + L.cycle);
    D.world_t = (float *)(base + L.world_t);
    D.err = (int *)(D.out + c->sz.output_floats);
    c->L.done_counter = (int *)(base + L.done_counter);
    c->L.sample_tiles = (const SampleTile *)(base + L.sample_tiles);
    c->L.rollout_tiles = (const RolloutTile *)(base + L.rollout_tiles);
    c->L.cost_tiles = (const CostTile *)(base + L.cost_tiles);
    c->L.update_tiles = (const UpdateTile *)(base + L.update_tiles);
    D.self_pairs = (int *)(base + L.self_pairs);
    D.self_t2 = (float *)(base + L.self_t2);
    D.work = (int *)(base + L.work);
    D.dhat = (float *)(base + L.dhat);
}

static void out_offsets(mrs_ctx *c)
{
    size_t o = 0;
    auto take = [&](size_t n) {
        o = align_up(o, 4);
        size_t at = o;
        o += n;
        return (int)at;
    };
    c->D.out_mean = take(c->sz.hd);
    c->D.out_sph = take(c->sz.hs);
    c->D.out_q = take(c->sz.hd);
    c->D.out_u = take(c->sz.d);
    c->D.out_dist = take(c->A);
    c->D.out_min = take(c->A);
    c->sz.output_floats = align_up(o, 4);
}

static mrs_status validate(const mrs_config *cfg, std::string &why)
{
    if (!cfg || !cfg->arms) return why = "null config or arms", MRS_EINVAL;
    if (cfg->n_arms < 1 || cfg->n_arms > MRS_MAX_ARMS) return why = "n_arms out of range", MRS_EINVAL;
    const float sc[] = {cfg->dt, cfg->lambda, cfg->gamma, cfg->alpha_mu, cfg->alpha_sigma,
                        cfg->sigma_init, cfg->w_pose, cfg->w_rot, cfg->w_stop, cfg->w_joint,
                        cfg->w_coll, cfg->w_self, cfg->w_dyn, cfg->B, cfg->B_world, cfg->B_self,
                        cfg->tau, cfg->q_margin};
    if (!finite_arr(sc, sizeof(sc) / sizeof(float))) return why = "non-finite parameter", MRS_EINVAL;
    if (cfg->dt <= 0 || cfg->lambda <= 0 || cfg->sigma_init <= 0 || cfg->B <= 0 ||
        cfg->B_world <= 0 || cfg->B_self <= 0 || cfg->gamma <= 0 || cfg->gamma > 1)
        return why = "dt, lambda, sigma_init, B, B_world, B_self must be > 0 and gamma in (0,1]",
               MRS_EINVAL;
    if (cfg->alpha_mu < 0 || cfg->alpha_mu > 1 || cfg->alpha_sigma < 0 || cfg->alpha_sigma > 1)
        return why = "EMA steps must be in [0,1]", MRS_EINVAL;
    if (cfg->w_pose < 0 || cfg->w_rot < 0 || cfg->w_stop < 0 || cfg->w_joint < 0 ||
        cfg->w_coll < 0 || cfg->w_self < 0 || cfg->w_dyn < 0 || cfg->tau < 0)
        return why = "cost weights and tau must be >= 0", MRS_EINVAL;
    if (cfg->iterations < 1 || cfg->iterations > 64) return why = "iterations out of range", MRS_EINVAL;
    if (cfg->max_plan_age < 0) return why = "max_plan_age must be >= 0", MRS_EINVAL;
    if (!(cfg->w_manip >= 0.f) || !std::isfinite(cfg->w_manip) ||
        (cfg->w_manip > 0.f && !(cfg->manip_w0 > 0.f && std::isfinite(cfg->manip_w0))))
        return why = "w_manip must be >= 0, and manip_w0 > 0 when w_manip > 0", MRS_EINVAL;
    if (cfg->reserved != 0) return why = "mrs_config.reserved must be 0", MRS_EINVAL;
    for (int a = 0; a < cfg->n_arms; ++a) {
        const mrs_arm_desc &d = cfg->arms[a];
        if (d.dof < 1 || d.dof > MRS_MAX_DOF) return why = "dof out of range", MRS_EINVAL;
        if (d.n_spheres < 1 || d.n_spheres > MRS_MAX_SPHERES)
            return why = "n_spheres out of range", MRS_EINVAL;
        if (d.K < 1 || d.K > MRS_MAX_SAMPLES) return why = "K out of range", MRS_EINVAL;
        if (d.H < 1 || d.H > MRS_MAX_HORIZON) return why = "H out of range", MRS_EINVAL;
        if (!d.dh || !d.q_lo || !d.q_hi || !d.qd_max || !d.sphere_body || !d.sphere_xyzr)
            return why = "null arm array", MRS_EINVAL;
        if (!finite_arr(d.dh, 4 * d.dof) || !finite_arr(d.q_lo, d.dof) ||
            !finite_arr(d.q_hi, d.dof) || !finite_arr(d.qd_max, d.dof) ||
            !finite_arr(d.sphere_xyzr, 4 * d.n_spheres) || !finite_arr(d.base_pose, 7))
            return why = "non-finite arm description", MRS_EINVAL;
        for (int s = 0; s < d.n_spheres; ++s) {
            if (d.sphere_body[s] < 0 || d.sphere_body[s] > d.dof + 1)
                return why = "sphere_body out of range", MRS_EINVAL;
            if (s > 0 && d.sphere_body[s] < d.sphere_body[s - 1])
                return why = "sphere_body must be non-decreasing", MRS_EINVAL;
            if (d.sphere_xyzr[4 * s + 3] < 0) return why = "negative sphere radius", MRS_EINVAL;
        }
        const float *qp = d.base_pose + 3;
        if (qp[0] * qp[0] + qp[1] * qp[1] + qp[2] * qp[2] + qp[3] * qp[3] < 1e-12f)
            return why = "zero base quaternion", MRS_EINVAL;
    }
    return MRS_OK;
}

static void invalidate_graph(mrs_ctx *ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->gexec_io) cudaGraphExecDestroy(ctx->gexec_io);
    if (ctx->graph_io) cudaGraphDestroy(ctx->graph_io);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->gexec_io = nullptr;
    ctx->graph_io = nullptr;
}

// Sphere centres and radii of an arm with every joint at zero (its rest
// pose), in double precision: standard DH frames T_i = T_{i-1} Rz(theta_i)
// Tz(d_i) Tx(a_i) Rx(alpha_i) from the base pose.  Used once at set-up, to
// drop the self-collision pairs that touch or lie inside the B_self band at
// rest: they belong to the arm's build (Eq. 5's C_self is over the others).
static void rest_pose_spheres(const mrs_arm_desc &d, std::vector<double> &out)
{
    const float *b = d.base_pose;
    double w = b[3], x = b[4], y = b[5], z = b[6];
    const double n = std::sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    // rotation R (row-major) and translation t of the current frame
    double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    double t[3] = {b[0], b[1], b[2]};
    std::vector<double> frames((size_t)(d.dof + 1) * 12);
    auto keep = [&](int f) {
        for (int k = 0; k < 9; ++k) frames[12 * f + k] = R[k];
        for (int k = 0; k < 3; ++k) frames[12 * f + 9 + k] = t[k];
    };
    keep(0);
    for (int j = 0; j < d.dof; ++j) {
        const double a = d.dh[4 * j], dd = d.dh[4 * j + 1], al = d.dh[4 * j + 2],
                     th = d.dh[4 * j + 3];
        const double ct = std::cos(th), st = std::sin(th), ca = std::cos(al), sa = std::sin(al);
        // local transform Rz(th) Tz(dd) Tx(a) Rx(al): rotation M, offset (a ct, a st, dd)
        const double M[9] = {ct, -st * ca, st * sa, st, ct * ca, -ct * sa, 0.0, sa, ca};
        const double o[3] = {a * ct, a * st, dd};
        double Rn[9], tn[3];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c)
                Rn[3 * r + c] = R[3 * r] * M[c] + R[3 * r + 1] * M[3 + c] + R[3 * r + 2] * M[6 + c];
            tn[r] = t[r] + R[3 * r] * o[0] + R[3 * r + 1] * o[1] + R[3 * r + 2] * o[2];
        }
        std::memcpy(R, Rn, sizeof R);
        std::memcpy(t, tn, sizeof t);
        keep(j + 1);
    }
    out.assign((size_t)d.n_spheres * 4, 0.0);
    for (int s = 0; s < d.n_spheres; ++s) {
        const int f = std::min(d.sphere_body[s], d.dof);
        const double *F = frames.data() + 12 * f;
        const float *p = d.sphere_xyzr + 4 * s;
        for (int r = 0; r < 3; ++r)
            out[4 * s + r] = F[9 + r] + F[3 * r] * p[0] + F[3 * r + 1] * p[1] + F[3 * r + 2] * p[2];
        out[4 * s + 3] = p[3];
    }
}

static double rest_clearance(const std::vector<double> &S, int s1, int s2)
{
    const double *a = S.data() + 4 * s1, *b = S.data() + 4 * s2;
    const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return std::sqrt(dx * dx + dy * dy + dz * dz) - a[3] - b[3];
}

extern "C" {

mrs_status mrs_create(const mrs_config *cfg, void *stream, mrs_ctx **out)
{
    if (!out) return MRS_EINVAL;
    *out = nullptr;
    std::string why;
    g_create_err.clear();
    mrs_status st = validate(cfg, why);
    if (st != MRS_OK) {
        g_create_err = why;
        return st;
    }
    mrs_ctx *ctx = new (std::nothrow) mrs_ctx();
    if (!ctx) return MRS_ENOMEM;
    ctx->A = cfg->n_arms;
    Params &P = ctx->P;
    P.n_arms = cfg->n_arms;
    P.iterations = cfg->iterations;
    P.zero_noise = 0;
    P.dt = cfg->dt; P.lambda = cfg->lambda; P.gamma = cfg->gamma;
    P.alpha_mu = cfg->alpha_mu; P.alpha_sigma = cfg->alpha_sigma; P.sigma_init = cfg->sigma_init;
    P.w_pose = cfg->w_pose; P.w_rot = cfg->w_rot; P.w_stop = cfg->w_stop; P.w_joint = cfg->w_joint;
    P.w_coll = cfg->w_coll; P.w_self = cfg->w_self; P.w_dyn = cfg->w_dyn;
    P.B = cfg->B; P.B_world = cfg->B_world; P.B_self = cfg->B_self; P.tau = cfg->tau;
    P.q_margin = cfg->q_margin; P.seed = cfg->seed;
    P.max_plan_age = cfg->max_plan_age;
    P.w_manip = cfg->w_manip;
    P.manip_w0 = cfg->manip_w0;
    P.wait_polls = tc::kWaitLimit;

    size_t hd = 0, hdd = 0, hs = 0, dsum = 0, ksum = 0, in = 0;
    long long khd = 0, kh = 0;
    int max_ns = 0, max_pairs = 0;
    ctx->arms.resize(ctx->A);
    for (int a = 0; a < ctx->A; ++a) {
        const mrs_arm_desc &d = cfg->arms[a];
        ArmDev &A = ctx->arms[a];
        std::memset(&A, 0, sizeof(A));
        A.dof = d.dof; A.ns = d.n_spheres; A.K = d.K; A.H = d.H;
        A.off_hd = (int)hd; A.off_hdd = (int)hdd; A.off_hs = (int)hs; A.off_d = (int)dsum;
        A.off_k = (int)ksum; A.off_in = (int)in;
        A.spg = (d.n_spheres + kGroups - 1) / kGroups;
        A.off_khd = khd; A.off_kh = kh;
        A.external = d.external ? 1 : 0;
        for (int j = 0; j < d.dof; ++j) {
            A.dh[j] = make_float4(d.dh[4 * j], d.dh[4 * j + 1], d.dh[4 * j + 2], d.dh[4 * j + 3]);
            A.q_lo[j] = d.q_lo[j]; A.q_hi[j] = d.q_hi[j]; A.qd_max[j] = d.qd_max[j];
        }
        for (int k = 0; k < 7; ++k) A.base_pose[k] = d.base_pose[k];
        for (int s = 0; s < d.n_spheres; ++s) {
            A.sph[s] = make_float4(d.sphere_xyzr[4 * s], d.sphere_xyzr[4 * s + 1],
                                   d.sphere_xyzr[4 * s + 2], d.sphere_xyzr[4 * s + 3]);
            A.body[s] = d.sphere_body[s];
            A.frame[s] = std::min(d.sphere_body[s], d.dof);
        }
        // self-collision pairs: bodies at least three apart and clear of the
        // B_self band with every joint at zero (the rest-pose ignore rule)
        A.self_off = (int)ctx->self_pairs.size();
        std::vector<double> rest;
        rest_pose_spheres(d, rest);
        for (int s1 = 0; s1 < d.n_spheres; ++s1)
            for (int s2 = s1 + 1; s2 < d.n_spheres; ++s2)
                if (std::abs(d.sphere_body[s1] - d.sphere_body[s2]) >= 3 &&
                    rest_clearance(rest, s1, s2) >= (double)cfg->B_self) {
                    ctx->self_pairs.push_back(s1 | (s2 << 8));
                    // binary32 sums in the device's order: (r1 + B_self) + r2, squared
                    const float t = (d.sphere_xyzr[4 * s1 + 3] + cfg->B_self) + d.sphere_xyzr[4 * s2 + 3];
                    ctx->self_t2.push_back(t * t);
                }
        A.n_self = (int)ctx->self_pairs.size() - A.self_off;
        max_pairs = std::max(max_pairs, A.n_self);
        hd += (size_t)d.H * d.dof;
        hdd += (size_t)d.H * d.dof * d.dof;
        hs += (size_t)d.H * d.n_spheres * 4;
        dsum += d.dof;
        ksum += d.K;
        in += 2 * d.dof + 12;
        khd += (long long)d.K * d.H * d.dof;
        kh += (long long)d.K * d.H;
        max_ns = std::max(max_ns, d.n_spheres);
    }
    P.max_ns = max_ns;
    P.max_pairs = std::max(max_pairs, 1);
    P.world_cap = 64;
    P.aabb_cap = 8;
    ctx->sz.n_arms = ctx->A;
    ctx->sz.hd = hd; ctx->sz.hdd = hdd; ctx->sz.hs = hs; ctx->sz.d = dsum; ctx->sz.k = ksum;
    ctx->sz.input_floats = in;
    ctx->sz.state_bytes = 32 + sizeof(float) * (hd + hdd) +
                          (size_t)ctx->A * 24 + sizeof(float) * (hs + hd);
    out_offsets(ctx);
    build_work_lists(ctx);
    build_layout(ctx);

    // launch plan
    LaunchPlan &L = ctx->L;
    L.n_arms = ctx->A;
    L.n_sample_tiles = (int)ctx->sample_tiles.size();
    L.n_rollout_tiles = (int)ctx->rollout_tiles.size();
    L.n_cost_tiles = (int)ctx->cost_tiles.size();
    L.n_update_tiles = (int)ctx->update_tiles.size();
    L.total_kh = (int)kh;
    size_t sp = 0, ss = 0, st2 = 0;
    // the merged Sense + Shift repeats the arm's shift in each of its sample
    // blocks: worth a launch less only for a few blocks per arm
    L.merge_prep = small_arms(ctx);
    L.sample_tile = L.merge_prep ? 16 : 32;
    for (auto &A : ctx->arms) {
        sp = std::max(sp, sizeof(float) * (size_t)A.H * (2 * A.dof * A.dof + A.dof));
        // k_sample: the whole horizon, or chunks of it within 96 KB
        const size_t per_h =
            sizeof(float) * (size_t)(A.dof * A.dof + A.dof + 2 * A.dof * L.sample_tile);
        ss = std::max(ss, std::min((size_t)A.H * per_h, std::max(per_h, (size_t)96 * 1024)));
        st2 = std::max(st2, sizeof(float) * (size_t)A.H * 4 * A.dof);
    }
    L.smem_prep = sp;
    L.smem_sample = ss;
    L.smem_toplan = st2;
    L.smem_rollout = rollout_smem_bytes(P, ctx->A);
    // the sphere-group sizes of the arms that roll out: the launch takes the
    // smallest rollout build that holds them all
    L.rollout_sizes = 0;
    for (const ArmDev &A : ctx->arms)
        if (!A.external) L.rollout_sizes |= 1u << A.spg;

    if (stream) {
        ctx->stream = (cudaStream_t)stream;
        if (cudaStreamGetDevice(ctx->stream, &ctx->device) != cudaSuccess) {
            delete ctx;
            g_create_err = "the stream's device could not be read";
            return MRS_ECUDA;
        }
    } else {
        if (cudaGetDevice(&ctx->device) != cudaSuccess) {
            delete ctx;
            g_create_err = "no CUDA device";
            return MRS_ECUDA;
        }
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return MRS_ECUDA;
        }
        ctx->own_stream = true;
    }
    DeviceScope dev_scope(ctx);
    if (cudaHostAlloc((void **)&ctx->pin_in, sizeof(float) * in, cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc((void **)&ctx->pin_out, sizeof(float) * (ctx->sz.output_floats + 4),
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming) != cudaSuccess) {
        mrs_destroy(ctx);
        return MRS_ENOMEM;
    }
    ctx->pin_err = (int *)(ctx->pin_out + ctx->sz.output_floats);
    int dev = ctx->device, smem_optin = 0;
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
        mrs_destroy(ctx);
        g_create_err = "no CUDA device";
        return MRS_ECUDA;
    }
    // the rollout stages the world and every neighbour's plan slice of a step
    // in shared memory: (world spheres + n_arms x the largest sphere count)
    // must fit one block
    if (L.smem_rollout > (size_t)smem_optin) {
        mrs_destroy(ctx);
        g_create_err = "the rollout's shared memory (" + std::to_string(L.smem_rollout) +
                       " bytes for n_arms x the largest sphere count) exceeds the device's " +
                       std::to_string(smem_optin) + " bytes per block";
        return MRS_EUNSUPPORTED;
    }
    if (configure_kernels(L) != cudaSuccess) {
        mrs_destroy(ctx);
        g_create_err = "kernel configuration failed";
        return MRS_ECUDA;
    }
    ctx->smem_optin = smem_optin;
    ctx->max_blocks_per_sm = rollout_blocks_per_sm(L.smem_rollout);
    set_rollout_grid(ctx);
    *out = ctx;
    return MRS_OK;
}

void mrs_destroy(mrs_ctx *ctx)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->rhohat) cudaFree(ctx->rhohat);
    if (ctx->pair_board) cudaFree(ctx->pair_board);
    invalidate_graph(ctx);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    if (ctx->pin_in) cudaFreeHost(ctx->pin_in);
    if (ctx->pin_out) cudaFreeHost(ctx->pin_out);
    if (ctx->done) cudaEventDestroy(ctx->done);
    for (auto e : ctx->events) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *mrs_last_error(const mrs_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_create_err.empty() ? g_noctx : g_create_err.c_str();
}

mrs_status mrs_query_sizes(const mrs_ctx *ctx, mrs_sizes *out)
{
    if (!ctx || !out) return MRS_EINVAL;
    *out = ctx->sz;
    return MRS_OK;
}

mrs_status mrs_workspace_size(const mrs_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return MRS_EINVAL;
    *bytes = ctx->sz.workspace_bytes;
    return MRS_OK;
}

static mrs_status bind(mrs_ctx *ctx, void *dev, size_t bytes)
{
    invalidate_graph(ctx);
    ctx->ws = dev;
    ctx->ws_bytes = bytes;
    fill_dev(ctx, (char *)dev);
    const auto &L = ctx->lay;
    char *base = (char *)dev;
    CK(cudaMemcpyAsync(base + L.arms, ctx->arms.data(), sizeof(ArmDev) * ctx->A,
                       cudaMemcpyHostToDevice, ctx->stream), "upload arms");
    CK(cudaMemcpyAsync(base + L.sample_tiles, ctx->sample_tiles.data(),
                       sizeof(SampleTile) * ctx->sample_tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "upload tiles");
    CK(cudaMemcpyAsync(base + L.rollout_tiles, ctx->rollout_tiles.data(),
                       sizeof(RolloutTile) * ctx->rollout_tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "upload tiles");
    CK(cudaMemcpyAsync(base + L.cost_tiles, ctx->cost_tiles.data(),
                       sizeof(CostTile) * ctx->cost_tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "upload tiles");
    CK(cudaMemcpyAsync(base + L.update_tiles, ctx->update_tiles.data(),
                       sizeof(UpdateTile) * ctx->update_tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "upload tiles");
    if (!ctx->self_pairs.empty())
        CK(cudaMemcpyAsync(base + L.self_pairs, ctx->self_pairs.data(),
                           sizeof(int) * ctx->self_pairs.size(), cudaMemcpyHostToDevice,
                           ctx->stream), "upload self pairs");
    if (!ctx->self_t2.empty())
        CK(cudaMemcpyAsync(base + L.self_t2, ctx->self_t2.data(),
                           sizeof(float) * ctx->self_t2.size(), cudaMemcpyHostToDevice,
                           ctx->stream), "upload self pairs");
    CK(cudaMemsetAsync(base + L.done_counter, 0, sizeof(int), ctx->stream), "memset");
    CK(cudaMemsetAsync(base + L.work, 0, sizeof(int) * 64, ctx->stream), "memset");
    CK(cudaMemsetAsync(base + L.input, 0, sizeof(float) * ctx->sz.input_floats, ctx->stream),
       "memset");
    CK(cudaMemsetAsync(base + L.out, 0, sizeof(float) * ctx->sz.output_floats, ctx->stream),
       "memset");
    CK(cudaMemsetAsync(base + L.world_vel, 0, sizeof(float4) * MRS_MAX_WORLD_SPHERES, ctx->stream),
       "memset");
    CK(enqueue_init(ctx->P, ctx->D, ctx->A, (int)ctx->sz.hdd, (int)ctx->sz.hd, ctx->stream),
       "init kernels");
    CK(enqueue_state_factors(ctx->D, ctx->L, 0, ctx->stream), "initial factors");
    CK(cudaStreamSynchronize(ctx->stream), "sync after init");
    ctx->bound = true;
    return MRS_OK;
}

mrs_status mrs_bind_workspace(mrs_ctx *ctx, void *dev_ptr, size_t bytes)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (!dev_ptr || bytes < ctx->sz.workspace_bytes || ((uintptr_t)dev_ptr & 255))
        return fail(ctx, MRS_EINVAL, "workspace null, too small or not 256-byte aligned");
    if (ctx->own_ws && ctx->ws) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->ws);
        ctx->own_ws = false;
    }
    return bind(ctx, dev_ptr, bytes);
}

static mrs_status ensure_bound(mrs_ctx *ctx)
{
    if (ctx->bound) return MRS_OK;
    void *p = nullptr;
    CK(cudaMalloc(&p, ctx->sz.workspace_bytes), "workspace allocation");
    ctx->own_ws = true;
    return bind(ctx, p, ctx->sz.workspace_bytes);
}

mrs_status mrs_set_world(mrs_ctx *ctx, const float *spheres, const float *vel, int n_spheres,
                         const float *aabbs, int n_aabbs)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (n_spheres < 0 || n_spheres > MRS_MAX_WORLD_SPHERES || n_aabbs < 0 ||
        n_aabbs > MRS_MAX_AABBS || (n_spheres && !spheres) || (n_aabbs && !aabbs))
        return fail(ctx, MRS_EINVAL, "world sizes out of range or null arrays");
    if ((n_spheres && !finite_arr(spheres, 4 * (size_t)n_spheres)) ||
        (vel && n_spheres && !finite_arr(vel, 3 * (size_t)n_spheres)) ||
        (n_aabbs && !finite_arr(aabbs, 6 * (size_t)n_aabbs)))
        return fail(ctx, MRS_EINVAL, "non-finite world");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    if (n_spheres > ctx->P.world_cap || n_aabbs > ctx->P.aabb_cap) {
        // grow the rollout's shared-memory world capacity (powers of two)
        Params grown = ctx->P;
        while (grown.world_cap < n_spheres) grown.world_cap *= 2;
        while (grown.aabb_cap < n_aabbs) grown.aabb_cap *= 2;
        grown.world_cap = std::min(grown.world_cap, MRS_MAX_WORLD_SPHERES);
        grown.aabb_cap = std::min(grown.aabb_cap, MRS_MAX_AABBS);
        const size_t need = rollout_smem_bytes(grown, ctx->A);
        if (need > (size_t)ctx->smem_optin)
            return fail(ctx, MRS_EUNSUPPORTED,
                        "the world does not fit the rollout's shared memory with this many arms "
                        "and spheres");
        ctx->P.world_cap = grown.world_cap;
        ctx->P.aabb_cap = grown.aabb_cap;
        ctx->L.smem_rollout = need;
        CK(configure_rollout(ctx->L), "rollout shared memory");
        ctx->max_blocks_per_sm = rollout_blocks_per_sm(ctx->L.smem_rollout);
        set_rollout_grid(ctx);
        invalidate_graph(ctx);
    }
    std::vector<float4> w(n_spheres), v(n_spheres), b(2 * n_aabbs);
    for (int i = 0; i < n_spheres; ++i) {
        w[i] = make_float4(spheres[4 * i], spheres[4 * i + 1], spheres[4 * i + 2], spheres[4 * i + 3]);
        v[i] = vel ? make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.f)
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = 0; i < n_aabbs; ++i) {
        b[2 * i] = make_float4(aabbs[6 * i], aabbs[6 * i + 1], aabbs[6 * i + 2], 0.f);
        b[2 * i + 1] = make_float4(aabbs[6 * i + 3], aabbs[6 * i + 4], aabbs[6 * i + 5], 0.f);
    }
    int n[2] = {n_spheres, n_aabbs};
    float zero = 0.f;
    if (n_spheres) {
        CK(cudaMemcpyAsync(ctx->D.world, w.data(), sizeof(float4) * n_spheres,
                           cudaMemcpyHostToDevice, ctx->stream), "set_world");
        CK(cudaMemcpyAsync(ctx->D.world_vel, v.data(), sizeof(float4) * n_spheres,
                           cudaMemcpyHostToDevice, ctx->stream), "set_world");
    }
    if (n_aabbs)
        CK(cudaMemcpyAsync(ctx->D.aabb, b.data(), sizeof(float4) * 2 * n_aabbs,
                           cudaMemcpyHostToDevice, ctx->stream), "set_world");
    CK(cudaMemcpyAsync(ctx->D.world_n, n, sizeof(n), cudaMemcpyHostToDevice, ctx->stream),
       "set_world");
    CK(cudaMemcpyAsync(ctx->D.world_t, &zero, sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
       "set_world");
    CK(enqueue_world_order(ctx->P, ctx->D, ctx->stream), "set_world order");
    CK(cudaStreamSynchronize(ctx->stream), "set_world sync");
    return MRS_OK;
}

mrs_status mrs_share_plans(mrs_ctx *ctx, int arm, const float *plan_spheres, const float *plan_q,
                           float dist_to_goal, long long cycle)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (arm < 0 || arm >= ctx->A) return fail(ctx, MRS_EINVAL, "arm out of range");
    if (!std::isfinite(dist_to_goal)) return fail(ctx, MRS_EINVAL, "non-finite distance");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const ArmDev &A = ctx->arms[arm];
    // 1: plan with joints, 2: spheres only (the arm-pair surrogate, which
    // reads the joints, then falls back to the exact pass for it)
    int valid = dist_to_goal >= 0.f ? (plan_q ? 1 : 2) : 0;
    if (valid) {
        if (!plan_spheres) return fail(ctx, MRS_EINVAL, "null plan");
        const size_t nsph = (size_t)A.H * A.ns * 4;
        if (!finite_arr(plan_spheres, nsph) || (plan_q && !finite_arr(plan_q, (size_t)A.H * A.dof)))
            return fail(ctx, MRS_EINVAL, "non-finite plan");
        CK(cudaMemcpyAsync(ctx->D.board_sph + A.off_hs / 4, plan_spheres, sizeof(float) * nsph,
                           cudaMemcpyHostToDevice, ctx->stream), "share_plans");
        if (plan_q)
            CK(cudaMemcpyAsync(ctx->D.board_q + A.off_hd, plan_q, sizeof(float) * A.H * A.dof,
                               cudaMemcpyHostToDevice, ctx->stream), "share_plans");
        CK(cudaMemcpyAsync(ctx->D.board_dist + arm, &dist_to_goal, sizeof(float),
                           cudaMemcpyHostToDevice, ctx->stream), "share_plans");
        CK(cudaMemcpyAsync(ctx->D.board_stamp + arm, &cycle, sizeof(long long),
                           cudaMemcpyHostToDevice, ctx->stream), "share_plans");
    }
    CK(cudaMemcpyAsync(ctx->D.board_valid + arm, &valid, sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream), "share_plans");
    CK(cudaStreamSynchronize(ctx->stream), "share_plans sync");
    return MRS_OK;
}

static mrs_status launch_cycle(mrs_ctx *ctx)
{
    cudaEvent_t *ev = ctx->timing ? ctx->events.data() : nullptr;
    if (!ctx->use_graph) {
        CK(enqueue_cycle(ctx->P, ctx->D, ctx->L, ctx->stream, ev), "cycle launch");
        return MRS_OK;
    }
    if (!ctx->gexec) {
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
        cudaError_t e = enqueue_cycle(ctx->P, ctx->D, ctx->L, ctx->stream, ev, true);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture launch");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "graph end capture");
        ctx->graph = g;
        CK(cudaGraphInstantiate(&ctx->gexec, g, 0), "graph instantiate");
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream), "graph launch");
    return MRS_OK;
}

// mrs_step's graph (capture on first use): one launch per control cycle
static mrs_status launch_cycle_io(mrs_ctx *ctx)
{
    if (!ctx->gexec_io) {
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
        cudaError_t e = cudaMemcpyAsync(ctx->D.input, ctx->pin_in,
                                        sizeof(float) * ctx->sz.input_floats,
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = enqueue_cycle(ctx->P, ctx->D, ctx->L, ctx->stream, nullptr, true);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->pin_out, ctx->D.out,
                                sizeof(float) * ctx->sz.output_floats + sizeof(int),
                                cudaMemcpyDeviceToHost, ctx->stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ctx, e != cudaSuccess ? e : e2, "graph capture (step)");
        }
        ctx->graph_io = g;
        CK(cudaGraphInstantiate(&ctx->gexec_io, g, 0), "graph instantiate (step)");
    }
    CK(cudaGraphLaunch(ctx->gexec_io, ctx->stream), "graph launch");
    return MRS_OK;
}

// Waits for the work enqueued so far, polling: a tight spin for the first
// 2 ms (a control cycle ends well within it), then yielding the core, and
// giving up after timeout_s.
static mrs_status wait_bounded(mrs_ctx *ctx, double timeout_s)
{
    CK(cudaEventRecord(ctx->done, ctx->stream), "event record");
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ctx->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream wait");
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(ctx, MRS_ETIMEOUT, "bounded wait for the cycle gave up");
        if (el > 2e-3) std::this_thread::yield();
    }
    return MRS_OK;
}

mrs_status mrs_step_device(mrs_ctx *ctx, const float *d_input)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !d_input) return fail(ctx, MRS_EINVAL, "null argument");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    CK(cudaMemcpyAsync(ctx->D.input, d_input, sizeof(float) * ctx->sz.input_floats,
                       cudaMemcpyDeviceToDevice, ctx->stream), "input copy");
    ctx->has_input = true;
    return launch_cycle(ctx);
}

mrs_status mrs_step(mrs_ctx *ctx, const mrs_arm_state *states, mrs_step_out *out)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !states) return fail(ctx, MRS_EINVAL, "null argument");
    float *p = ctx->pin_in;
    for (int a = 0; a < ctx->A; ++a) {
        const ArmDev &A = ctx->arms[a];
        const mrs_arm_state &s = states[a];
        if (!s.q || !s.qd || !s.goal_p || !s.goal_R) return fail(ctx, MRS_EINVAL, "null state array");
        if (!finite_arr(s.q, A.dof) || !finite_arr(s.qd, A.dof) || !finite_arr(s.goal_p, 3) ||
            !finite_arr(s.goal_R, 9))
            return fail(ctx, MRS_EINVAL, "non-finite state");
        std::memcpy(p, s.q, sizeof(float) * A.dof);
        std::memcpy(p + A.dof, s.qd, sizeof(float) * A.dof);
        std::memcpy(p + 2 * A.dof, s.goal_p, sizeof(float) * 3);
        std::memcpy(p + 2 * A.dof + 3, s.goal_R, sizeof(float) * 9);
        p += 2 * A.dof + 12;
    }
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    if (ctx->use_graph && !ctx->timing) {
        // upload, cycle and downloads in one graph launch
        st = launch_cycle_io(ctx);
        if (st != MRS_OK) return st;
    } else {
        CK(cudaMemcpyAsync(ctx->D.input, ctx->pin_in, sizeof(float) * ctx->sz.input_floats,
                           cudaMemcpyHostToDevice, ctx->stream), "input upload");
        st = launch_cycle(ctx);
        if (st != MRS_OK) return st;
        CK(cudaMemcpyAsync(ctx->pin_out, ctx->D.out,
                           sizeof(float) * ctx->sz.output_floats + sizeof(int),
                           cudaMemcpyDeviceToHost, ctx->stream), "output and error word download");
    }
    ctx->has_input = true;
    st = wait_bounded(ctx, 10.0);
    if (st != MRS_OK) return st;
    if (*ctx->pin_err) return fail(ctx, MRS_ETIMEOUT, "a device-side bounded wait gave up");
    if (out) {
        const Dev &D = ctx->D;
        const float *o = ctx->pin_out;
        if (out->mean_plan) std::memcpy(out->mean_plan, o + D.out_mean, sizeof(float) * ctx->sz.hd);
        if (out->plan_spheres) std::memcpy(out->plan_spheres, o + D.out_sph, sizeof(float) * ctx->sz.hs);
        if (out->plan_q) std::memcpy(out->plan_q, o + D.out_q, sizeof(float) * ctx->sz.hd);
        if (out->u_star) std::memcpy(out->u_star, o + D.out_u, sizeof(float) * ctx->sz.d);
        if (out->dist_to_goal) std::memcpy(out->dist_to_goal, o + D.out_dist, sizeof(float) * ctx->A);
        if (out->min_cost) std::memcpy(out->min_cost, o + D.out_min, sizeof(float) * ctx->A);
    }
    return MRS_OK;
}

mrs_status mrs_output_device(mrs_ctx *ctx, mrs_step_out *out)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !out) return MRS_EINVAL;
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const Dev &D = ctx->D;
    out->mean_plan = D.out + D.out_mean;
    out->plan_spheres = D.out + D.out_sph;
    out->plan_q = D.out + D.out_q;
    out->u_star = D.out + D.out_u;
    out->dist_to_goal = D.out + D.out_dist;
    out->min_cost = D.out + D.out_min;
    return MRS_OK;
}

mrs_status mrs_output_host(mrs_ctx *ctx, mrs_step_out *out)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !out) return MRS_EINVAL;
    const Dev &D = ctx->D;
    float *o = ctx->pin_out;
    out->mean_plan = o + D.out_mean;
    out->plan_spheres = o + D.out_sph;
    out->plan_q = o + D.out_q;
    out->u_star = o + D.out_u;
    out->dist_to_goal = o + D.out_dist;
    out->min_cost = o + D.out_min;
    return MRS_OK;
}

mrs_status mrs_sync(mrs_ctx *ctx, double timeout_s)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    return wait_bounded(ctx, timeout_s);
}

mrs_status mrs_use_graph(mrs_ctx *ctx, int on)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    ctx->use_graph = on != 0;
    return MRS_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume

namespace {
struct BlobHeader {
    uint32_t magic, version, n_arms, pad;
    int64_t cycle;
    float world_t, pad2;
};
}

mrs_status mrs_save_state(mrs_ctx *ctx, void *blob, size_t bytes)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !blob) return MRS_EINVAL;
    if (bytes < ctx->sz.state_bytes) return fail(ctx, MRS_EINVAL, "state buffer too small");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const int A = ctx->A;
    std::vector<float> mu2(2 * ctx->sz.hd), Sg2(2 * ctx->sz.hdd), sph(ctx->sz.hs), q(ctx->sz.hd),
        dist(A);
    std::vector<int> valid(A);
    std::vector<long long> stamp(A);
    long long cycle = 0;
    float wt = 0.f;
    const Dev &D = ctx->D;
    CK(cudaMemcpyAsync(mu2.data(), D.mu, sizeof(float) * mu2.size(), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(Sg2.data(), D.Sigma, sizeof(float) * Sg2.size(), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(sph.data(), D.board_sph, sizeof(float) * sph.size(), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(q.data(), D.board_q, sizeof(float) * q.size(), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(dist.data(), D.board_dist, sizeof(float) * A, cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(valid.data(), D.board_valid, sizeof(int) * A, cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(stamp.data(), D.board_stamp, sizeof(long long) * A, cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(&cycle, D.cycle, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaMemcpyAsync(&wt, D.world_t, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "save");
    CK(cudaStreamSynchronize(ctx->stream), "save sync");
    // the current state is the buffer of the cycle's parity
    const float *mu = mu2.data() + (cycle & 1) * ctx->sz.hd;
    const float *Sg = Sg2.data() + (cycle & 1) * ctx->sz.hdd;
    char *p = (char *)blob;
    BlobHeader hdr{0x3152534du, 1u, (uint32_t)A, 0u, cycle, wt, 0.f};
    std::memcpy(p, &hdr, sizeof(hdr));
    p += sizeof(hdr);
    for (int a = 0; a < A; ++a) {
        const ArmDev &Ar = ctx->arms[a];
        std::memcpy(p, mu + Ar.off_hd, sizeof(float) * Ar.H * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof;
        std::memcpy(p, Sg + Ar.off_hdd, sizeof(float) * Ar.H * Ar.dof * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof * Ar.dof;
    }
    for (int a = 0; a < A; ++a) {
        const ArmDev &Ar = ctx->arms[a];
        int32_t v[2] = {valid[a], 0};
        std::memcpy(p, v, 8); p += 8;
        int64_t s = stamp[a];
        std::memcpy(p, &s, 8); p += 8;
        float dd[2] = {dist[a], 0.f};
        std::memcpy(p, dd, 8); p += 8;
        std::memcpy(p, sph.data() + Ar.off_hs, sizeof(float) * Ar.H * Ar.ns * 4);
        p += sizeof(float) * Ar.H * Ar.ns * 4;
        std::memcpy(p, q.data() + Ar.off_hd, sizeof(float) * Ar.H * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof;
    }
    return MRS_OK;
}

mrs_status mrs_load_state(mrs_ctx *ctx, const void *blob, size_t bytes)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !blob) return MRS_EINVAL;
    if (bytes < ctx->sz.state_bytes) return fail(ctx, MRS_EINVAL, "state blob too small");
    const char *p = (const char *)blob;
    BlobHeader hdr;
    std::memcpy(&hdr, p, sizeof(hdr));
    p += sizeof(hdr);
    if (hdr.magic != 0x3152534du || hdr.version != 1u || (int)hdr.n_arms != ctx->A)
        return fail(ctx, MRS_EINVAL, "state blob header mismatch");
    if (!std::isfinite(hdr.world_t) || hdr.cycle < 0) return fail(ctx, MRS_EINVAL, "bad clocks");
    const int A = ctx->A;
    std::vector<float> mu(ctx->sz.hd), Sg(ctx->sz.hdd), sph(ctx->sz.hs), q(ctx->sz.hd), dist(A);
    std::vector<int> valid(A);
    std::vector<long long> stamp(A);
    for (int a = 0; a < A; ++a) {
        const ArmDev &Ar = ctx->arms[a];
        std::memcpy(mu.data() + Ar.off_hd, p, sizeof(float) * Ar.H * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof;
        std::memcpy(Sg.data() + Ar.off_hdd, p, sizeof(float) * Ar.H * Ar.dof * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof * Ar.dof;
    }
    for (int a = 0; a < A; ++a) {
        const ArmDev &Ar = ctx->arms[a];
        int32_t v[2];
        std::memcpy(v, p, 8); p += 8;
        int64_t s;
        std::memcpy(&s, p, 8); p += 8;
        float dd[2];
        std::memcpy(dd, p, 8); p += 8;
        valid[a] = v[0] ? 1 : 0;
        stamp[a] = s;
        dist[a] = dd[0];
        std::memcpy(sph.data() + Ar.off_hs, p, sizeof(float) * Ar.H * Ar.ns * 4);
        p += sizeof(float) * Ar.H * Ar.ns * 4;
        std::memcpy(q.data() + Ar.off_hd, p, sizeof(float) * Ar.H * Ar.dof);
        p += sizeof(float) * Ar.H * Ar.dof;
    }
    if (!finite_arr(mu.data(), mu.size()) || !finite_arr(Sg.data(), Sg.size()) ||
        !finite_arr(sph.data(), sph.size()) || !finite_arr(q.data(), q.size()) ||
        !finite_arr(dist.data(), dist.size()))
        return fail(ctx, MRS_EINVAL, "non-finite state");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const Dev &D = ctx->D;
    long long cycle = hdr.cycle;
    float wt = hdr.world_t;
    // into the buffer of the cycle's parity (the state after cycle - 1)
    CK(cudaMemcpyAsync(D.mu + (cycle & 1) * ctx->sz.hd, mu.data(), sizeof(float) * mu.size(),
                       cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.Sigma + (cycle & 1) * ctx->sz.hdd, Sg.data(), sizeof(float) * Sg.size(),
                       cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemsetAsync(D.work, 0, sizeof(int) * 64, ctx->stream), "load");
    CK(cudaMemsetAsync(D.err, 0, sizeof(int), ctx->stream), "load");   // a loaded state is clean
    CK(cudaMemcpyAsync(D.board_sph, sph.data(), sizeof(float) * sph.size(), cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.board_q, q.data(), sizeof(float) * q.size(), cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.board_dist, dist.data(), sizeof(float) * A, cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.board_valid, valid.data(), sizeof(int) * A, cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.board_stamp, stamp.data(), sizeof(long long) * A, cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.cycle, &cycle, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(cudaMemcpyAsync(D.world_t, &wt, sizeof(float), cudaMemcpyHostToDevice, ctx->stream), "load");
    CK(enqueue_state_factors(D, ctx->L, (int)(cycle & 1), ctx->stream), "load factors");
    CK(enqueue_world_order(ctx->P, D, ctx->stream), "load world order");
    CK(cudaStreamSynchronize(ctx->stream), "load sync");
    return MRS_OK;
}

// ---------------------------------------------------------------------------
// kinematics, inspection, self-test

mrs_status mrs_fk(mrs_ctx *ctx, int arm, int n, const float *q, float *ee, float *spheres)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (arm < 0 || arm >= ctx->A || n < 0 || (n && (!q || !ee)))
        return fail(ctx, MRS_EINVAL, "bad fk arguments");
    if (n == 0) return MRS_OK;
    const ArmDev &A = ctx->arms[arm];
    if (!finite_arr(q, (size_t)n * A.dof)) return fail(ctx, MRS_EINVAL, "non-finite q");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    float *dq = nullptr, *dee = nullptr, *ds = nullptr;
    // sub-buffers start on 16-byte boundaries (the sphere output is float4)
    const size_t nq = (size_t)n * A.dof, ne = (size_t)n * 12, nsph = (size_t)n * A.ns * 4;
    const size_t nq_pad = align_up(nq, 4), ne_pad = align_up(ne, 4);
    CK(cudaMalloc(&dq, sizeof(float) * (nq_pad + ne_pad + (spheres ? nsph : 0))), "fk buffer");
    dee = dq + nq_pad;
    ds = spheres ? dee + ne_pad : nullptr;
    cudaError_t e = cudaMemcpyAsync(dq, q, sizeof(float) * nq, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = enqueue_fk(ctx->D, arm, n, dq, dee, ds, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ee, dee, sizeof(float) * ne, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && spheres)
        e = cudaMemcpyAsync(spheres, ds, sizeof(float) * nsph, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dq);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fk");
    return MRS_OK;
}

mrs_status mrs_fk_static(mrs_ctx *ctx, int arm, int n, const float *q, float *ee, float *spheres)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (arm < 0 || arm >= ctx->A || n < 0 || (n && (!q || !ee)))
        return fail(ctx, MRS_EINVAL, "bad fk arguments");
    if (n == 0) return MRS_OK;
    if (!ctx->bound)
        return fail(ctx, MRS_ESTATE, "bind a workspace first: mrs_fk_static allocates nothing");
    const ArmDev &A = ctx->arms[arm];
    if (!finite_arr(q, (size_t)n * A.dof)) return fail(ctx, MRS_EINVAL, "non-finite q");
    std::string why;
    bool too_large = false;
    cudaError_t e = fk_static(ctx->D, ctx->device, arm, A.dof, A.ns, n, q, ee, spheres,
                              ctx->stream, why, too_large);
    if (too_large) return fail(ctx, MRS_EINVAL, why);
    if (e != cudaSuccess) return cuda_fail(ctx, e, ("mrs_fk_static: " + why).c_str());
    return MRS_OK;
}

mrs_status mrs_set_self_surrogate(mrs_ctx *ctx, int arm, mrs_mlp *net, float margin)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (arm < 0 || arm >= ctx->A) return fail(ctx, MRS_EINVAL, "arm out of range");
    ArmDev &A = ctx->arms[arm];
    if (net && (mlp_in_dim(net) != 2 * A.dof || !std::isfinite(margin) || margin < 0.f))
        return fail(ctx, MRS_EINVAL, "surrogate input must be 2 * dof sin/cos features; margin >= 0");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    A.learned = net ? 1 : 0;
    A.self_margin = net ? margin : 0.f;
    // rebuild the slot list in arm order
    LaunchPlan &L = ctx->L;
    int k = 0;
    SurrogateSlot slots[MRS_MAX_ARMS];
    for (int i = 0; i < L.n_surrogates; ++i)
        if (L.surrogates[i].arm != arm) slots[k++] = L.surrogates[i];
    if (net) slots[k++] = SurrogateSlot{arm, A.K * A.H, A.K, A.dof, A.off_kh, A.off_khd, net};
    std::sort(slots, slots + k, [](const SurrogateSlot &x, const SurrogateSlot &y) { return x.arm < y.arm; });
    L.n_surrogates = k;
    for (int i = 0; i < k; ++i) L.surrogates[i] = slots[i];
    // one inference launch per distinct network, over all of its arms
    L.n_groups = 0;
    for (int i = 0; i < k; ++i) {
        const SurrogateSlot &sl = slots[i];
        int gi = 0;
        while (gi < L.n_groups && L.groups[gi].net != sl.net) ++gi;
        if (gi == L.n_groups) {
            L.groups[gi] = SurrogateGroup{};
            L.groups[gi].net = sl.net;
            L.n_groups += 1;
        }
        fused::TrajSegs &g = L.groups[gi].segs;
        g.K[g.n] = sl.K;
        g.dof[g.n] = sl.dof;
        g.off_khd[g.n] = sl.off_khd;
        g.off_kh[g.n] = sl.off_kh;
        g.row_start[g.n + 1] = g.row_start[g.n] + sl.rows;
        g.n += 1;
    }
    // only the surrogate fields: the device copy also holds constants that the
    // device derived at binding (base rotation, twist sines)
    static_assert(offsetof(ArmDev, self_margin) == offsetof(ArmDev, learned) + sizeof(int),
                  "learned and self_margin are adjacent");
    CK(cudaMemcpyAsync(reinterpret_cast<char *>(ctx->D.arms + arm) + offsetof(ArmDev, learned),
                       &A.learned, sizeof(int) + sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
       "upload arm");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    invalidate_graph(ctx);
    return MRS_OK;
}

mrs_status mrs_self_dataset(mrs_ctx *ctx, int arm, int n, unsigned long long seed, float *d_x,
                            float *d_t, float *d_q)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || arm < 0 || arm >= ctx->A || n < 1 || !d_x || !d_t)
        return fail(ctx, MRS_EINVAL, "bad dataset arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    CK(enqueue_self_dataset(ctx->D, arm, n, seed, d_x, d_t, d_q, ctx->stream), "dataset");
    CK(cudaStreamSynchronize(ctx->stream), "dataset sync");
    return MRS_OK;
}

mrs_status mrs_self_distance(mrs_ctx *ctx, int arm, int n, const float *d_q, float *d_out)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || arm < 0 || arm >= ctx->A || n < 1 || !d_q || !d_out)
        return fail(ctx, MRS_EINVAL, "bad arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    CK(enqueue_self_clearance_rows(ctx->D, arm, n, d_q, d_out, ctx->stream), "self distance");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return MRS_OK;
}

mrs_status mrs_debug_self(mrs_ctx *ctx, int arm, float *dhat, float *exact)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || arm < 0 || arm >= ctx->A) return fail(ctx, MRS_EINVAL, "bad arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const ArmDev &A = ctx->arms[arm];
    const int rows = A.K * A.H;
    if (dhat)
        CK(cudaMemcpyAsync(dhat, ctx->D.dhat + A.off_kh, sizeof(float) * rows,
                           cudaMemcpyDeviceToHost, ctx->stream), "download");
    if (exact) {
        float *d = nullptr;
        CK(cudaMalloc(&d, sizeof(float) * rows), "buffer");
        cudaError_t e = enqueue_self_clearance_traj(ctx->D, arm, rows, d, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(exact, d, sizeof(float) * rows, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(d);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "exact self clearance");
    }
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return MRS_OK;
}

// ---------------------------------------------------------------------------
// learned arm-pair clearance

// pose of arm b's base in arm a's base frame: translation R_a^T (t_b - t_a),
// rotation conj(q_a) q_b, computed in double from the float inputs
static void relative_pose(const ArmDev &A, const ArmDev &B, float out[7])
{
    double qa[4], qb[4];
    for (int k = 0; k < 4; ++k) {
        qa[k] = A.base_pose[3 + k];
        qb[k] = B.base_pose[3 + k];
    }
    auto norm = [](double *q) {
        const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int k = 0; k < 4; ++k) q[k] /= n;
    };
    norm(qa);
    norm(qb);
    const double w = qa[0], x = qa[1], y = qa[2], z = qa[3];
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    const double d[3] = {(double)B.base_pose[0] - A.base_pose[0],
                         (double)B.base_pose[1] - A.base_pose[1],
                         (double)B.base_pose[2] - A.base_pose[2]};
    for (int r = 0; r < 3; ++r) out[r] = (float)(R[r] * d[0] + R[3 + r] * d[1] + R[6 + r] * d[2]);
    // conj(qa) * qb
    const double cw = w, cx = -x, cy = -y, cz = -z;
    const double rw = cw * qb[0] - cx * qb[1] - cy * qb[2] - cz * qb[3];
    const double rx = cw * qb[1] + cx * qb[0] + cy * qb[3] - cz * qb[2];
    const double ry = cw * qb[2] - cx * qb[3] + cy * qb[0] + cz * qb[1];
    const double rz = cw * qb[3] + cx * qb[2] - cy * qb[1] + cz * qb[0];
    out[3] = (float)rw; out[4] = (float)rx; out[5] = (float)ry; out[6] = (float)rz;
}

mrs_status mrs_relative_pose(mrs_ctx *ctx, int a, int b, float *pose)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !pose || a < 0 || a >= ctx->A || b < 0 || b >= ctx->A)
        return fail(ctx, MRS_EINVAL, "bad arguments");
    relative_pose(ctx->arms[a], ctx->arms[b], pose);
    return MRS_OK;
}

static void rebuild_pair_groups(mrs_ctx *ctx)
{
    ctx->pair_groups.clear();
    for (const auto &sl : ctx->pair_slots) {
        PairGroup *g = nullptr;
        for (auto &x : ctx->pair_groups)
            if (x.net == sl.net && x.segs.n < fused::kMaxSegs) g = &x;
        if (!g) {
            ctx->pair_groups.push_back(PairGroup{});
            g = &ctx->pair_groups.back();
            g->net = sl.net;
        }
        const ArmDev &A = ctx->arms[sl.a], &B = ctx->arms[sl.b];
        fused::PairSegs &q = g->segs;
        const int k = q.n;
        q.K[k] = A.K;
        q.Hb[k] = B.H;
        q.da[k] = A.dof;
        q.db[k] = B.dof;
        q.off_khd[k] = A.off_khd;
        q.off_hd[k] = B.off_hd;
        q.off_out[k] = A.off_kh * ctx->A + (long long)sl.b * A.K * A.H;
        relative_pose(A, B, q.pose[k]);
        q.row_start[k + 1] = q.row_start[k] + A.K * A.H;
        q.n = k + 1;
    }
    ctx->L.n_pair_groups = (int)ctx->pair_groups.size();
    ctx->L.pair_groups = ctx->pair_groups.data();
}

mrs_status mrs_set_pair_surrogate(mrs_ctx *ctx, int a, int b, mrs_mlp *net, float margin)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (a < 0 || a >= ctx->A || b < -1 || b >= ctx->A || b == a)
        return fail(ctx, MRS_EINVAL, "arm out of range");
    if (net && (!std::isfinite(margin) || margin < 0.f)) return fail(ctx, MRS_EINVAL, "margin >= 0");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    ArmDev &A = ctx->arms[a];
    for (int i = 0; i < ctx->A; ++i) {
        if (i == a || (b >= 0 && i != b)) continue;
        const ArmDev &B = ctx->arms[i];
        if (net && mlp_in_dim(net) != 2 * A.dof + 2 * B.dof + 7)
            return fail(ctx, MRS_EINVAL, "arm-pair surrogate input must be 2 d_a + 2 d_b + 7");
    }
    if (net && !ctx->rhohat) {
        size_t rows = 0;
        for (const auto &x : ctx->arms) rows += (size_t)x.K * x.H;
        CK(cudaMalloc(&ctx->rhohat, sizeof(float) * rows * ctx->A), "arm-pair prediction buffer");
        ctx->D.rhohat = ctx->rhohat;
        ctx->L.board_bytes = sizeof(float) * ctx->sz.hs;
        CK(cudaMalloc(&ctx->pair_board, ctx->L.board_bytes), "plan snapshot buffer");
        ctx->D.pair_board = ctx->pair_board;
    }
    // replace the slots of (a, b) or (a, every other arm)
    std::vector<mrs_ctx::PairSlot> keep;
    for (const auto &sl : ctx->pair_slots)
        if (!(sl.a == a && (b < 0 || sl.b == b))) keep.push_back(sl);
    if (net)
        for (int i = 0; i < ctx->A; ++i)
            if (i != a && (b < 0 || i == b)) keep.push_back({a, i, net});
    std::sort(keep.begin(), keep.end(), [](const mrs_ctx::PairSlot &x, const mrs_ctx::PairSlot &y) {
        return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    ctx->pair_slots = keep;
    A.pair_mask = 0u;
    for (const auto &sl : ctx->pair_slots)
        if (sl.a == a) A.pair_mask |= 1u << sl.b;
    if (net) A.pair_margin = margin;
    rebuild_pair_groups(ctx);
    static_assert(offsetof(ArmDev, pair_margin) == offsetof(ArmDev, pair_mask) + sizeof(unsigned),
                  "pair_mask and pair_margin are adjacent");
    CK(cudaMemcpyAsync(reinterpret_cast<char *>(ctx->D.arms + a) + offsetof(ArmDev, pair_mask),
                       &A.pair_mask, sizeof(unsigned) + sizeof(float), cudaMemcpyHostToDevice,
                       ctx->stream), "upload arm");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    invalidate_graph(ctx);
    return MRS_OK;
}

mrs_status mrs_pair_dataset(mrs_ctx *ctx, int a, int b, int n, unsigned long long seed,
                            const float *poses, int n_pose, float jit_t, float jit_yaw, float *d_x,
                            float *d_t, float *d_qa, float *d_qb, float *d_pose)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || a < 0 || a >= ctx->A || b < 0 || b >= ctx->A || n < 1 || !d_x || !d_t ||
        (poses && n_pose < 1) || !(jit_t >= 0.f) || !(jit_yaw >= 0.f))
        return fail(ctx, MRS_EINVAL, "bad dataset arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    std::vector<float> p;
    if (poses) {
        if (!finite_arr(poses, 7 * (size_t)n_pose)) return fail(ctx, MRS_EINVAL, "non-finite pose");
        p.assign(poses, poses + 7 * (size_t)n_pose);
    } else {
        p.resize(7);
        relative_pose(ctx->arms[a], ctx->arms[b], p.data());
        n_pose = 1;
    }
    float *dp = nullptr;
    CK(cudaMalloc(&dp, sizeof(float) * p.size()), "pose buffer");
    cudaError_t e = cudaMemcpyAsync(dp, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess)
        e = enqueue_pair_dataset(ctx->D, a, b, n, seed, dp, n_pose, jit_t, jit_yaw, d_x, d_t, d_qa,
                                 d_qb, d_pose, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pair dataset");
    return MRS_OK;
}

mrs_status mrs_debug_pair(mrs_ctx *ctx, int a, int b, float *rhohat, float *exact)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || a < 0 || a >= ctx->A || b < 0 || b >= ctx->A || a == b)
        return fail(ctx, MRS_EINVAL, "bad arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const ArmDev &A = ctx->arms[a];
    const int rows = A.K * A.H;
    if (rhohat) {
        if (!ctx->rhohat) return fail(ctx, MRS_ESTATE, "no arm-pair surrogate was set");
        CK(cudaMemcpyAsync(rhohat, ctx->rhohat + A.off_kh * ctx->A + (long long)b * rows,
                           sizeof(float) * rows, cudaMemcpyDeviceToHost, ctx->stream), "download");
    }
    if (exact) {
        float *d = nullptr;
        CK(cudaMalloc(&d, sizeof(float) * rows), "buffer");
        cudaError_t e = enqueue_pair_clearance_traj(ctx->D, a, b, rows, d, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(exact, d, sizeof(float) * rows, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        cudaFree(d);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "exact pair clearance");
    }
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    return MRS_OK;
}

mrs_status mrs_debug_costs(mrs_ctx *ctx, int arm, float *costs)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !costs || arm < 0 || arm >= ctx->A) return fail(ctx, MRS_EINVAL, "bad arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    const ArmDev &A = ctx->arms[arm];
    CK(cudaMemcpyAsync(costs, ctx->D.costs + A.off_k, sizeof(float) * A.K, cudaMemcpyDeviceToHost,
                       ctx->stream), "debug costs");
    CK(cudaStreamSynchronize(ctx->stream), "debug costs");
    return MRS_OK;
}

mrs_status mrs_debug_alpha(mrs_ctx *ctx, float *alpha)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !alpha) return fail(ctx, MRS_EINVAL, "bad arguments");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    CK(cudaMemcpyAsync(alpha, ctx->D.alpha, sizeof(float) * ctx->A * ctx->A, cudaMemcpyDeviceToHost,
                       ctx->stream), "debug alpha");
    CK(cudaStreamSynchronize(ctx->stream), "debug alpha");
    return MRS_OK;
}

mrs_status mrs_debug_spheres(mrs_ctx *ctx, int n_req, const int *anh, float *out)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || n_req < 0 || (n_req && (!anh || !out))) return fail(ctx, MRS_EINVAL, "bad arguments");
    if (n_req == 0) return MRS_OK;
    for (int r = 0; r < n_req; ++r) {
        const int a = anh[3 * r], n = anh[3 * r + 1], h = anh[3 * r + 2];
        if (a < 0 || a >= ctx->A || n < 0 || n >= ctx->arms[a].K || h < 0 || h >= ctx->arms[a].H)
            return fail(ctx, MRS_EINVAL, "request out of range");
    }
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    int *dreq = nullptr;
    const size_t nout = (size_t)n_req * kMaxSpheres * 4;
    const size_t nreq_pad = align_up((size_t)3 * n_req, 4);   // float4 output after it
    CK(cudaMalloc(&dreq, sizeof(int) * nreq_pad + sizeof(float) * nout), "debug buffer");
    float *dout = (float *)(dreq + nreq_pad);
    cudaError_t e = cudaMemsetAsync(dout, 0, sizeof(float) * nout, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dreq, anh, sizeof(int) * 3 * n_req, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = enqueue_debug_spheres(ctx->D, n_req, dreq, dout, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, dout, sizeof(float) * nout, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dreq);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "debug spheres");
    return MRS_OK;
}

mrs_status mrs_enable_timing(mrs_ctx *ctx, int on)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    const size_t need = 3 + 5 * (size_t)ctx->P.iterations;   // one more than the stages
    if (on && ctx->events.size() < need) {
        while (ctx->events.size() < need) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e), "event create");
            ctx->events.push_back(e);
        }
    }
    if ((on != 0) != ctx->timing) invalidate_graph(ctx);
    ctx->timing = on != 0;
    return MRS_OK;
}

mrs_status mrs_kernel_times(mrs_ctx *ctx, float *ms, int *n)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !ms || !n) return MRS_EINVAL;
    if (!ctx->timing) return fail(ctx, MRS_ESTATE, "timing is not enabled");
    const int cnt = 2 + 5 * ctx->P.iterations;                 // stages of one cycle
    if (*n < cnt) return fail(ctx, MRS_EINVAL, "ms has too few entries");
    CK(cudaEventSynchronize(ctx->events[cnt]), "timing wait");
    for (int i = 0; i < cnt; ++i)
        CK(cudaEventElapsedTime(&ms[i], ctx->events[i], ctx->events[i + 1]), "elapsed time");
    *n = cnt;
    return MRS_OK;
}

// ---------------------------------------------------------------------------
// rollout launch shape and its autotuner

static mrs_status apply_shape(mrs_ctx *ctx, int tile_samples, int blocks_per_sm, int order)
{
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    ctx->tile_samples = tile_samples;
    ctx->blocks_per_sm = blocks_per_sm;
    ctx->tile_order = order;
    build_rollout_tiles(ctx);
    LaunchPlan &L = ctx->L;
    L.n_rollout_tiles = (int)ctx->rollout_tiles.size();
    set_rollout_grid(ctx);
    // the list is never longer than the 32-sample list the workspace holds
    CK(cudaMemcpyAsync(const_cast<RolloutTile *>(L.rollout_tiles), ctx->rollout_tiles.data(),
                       sizeof(RolloutTile) * ctx->rollout_tiles.size(), cudaMemcpyHostToDevice,
                       ctx->stream), "upload rollout tiles");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    invalidate_graph(ctx);
    return MRS_OK;
}

mrs_status mrs_set_rollout_shape(mrs_ctx *ctx, const mrs_rollout_shape *shape)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || !shape) return MRS_EINVAL;
    if (shape->tile_samples < 32 || shape->tile_samples > 1024 || shape->tile_samples % 32 ||
        shape->blocks_per_sm < 0 || shape->blocks_per_sm > ctx->max_blocks_per_sm ||
        shape->order < 0 || shape->order > 2)
        return fail(ctx, MRS_EINVAL, "rollout shape out of range");
    return apply_shape(ctx, shape->tile_samples, shape->blocks_per_sm, shape->order);
}

mrs_status mrs_get_rollout_shape(mrs_ctx *ctx, mrs_rollout_shape *shape, int *max_blocks_per_sm)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (shape) {
        shape->tile_samples = ctx->tile_samples;
        shape->blocks_per_sm = ctx->blocks_per_sm;
        shape->order = ctx->tile_order;
        shape->cycle_ms = 0.f;
    }
    if (max_blocks_per_sm) *max_blocks_per_sm = ctx->max_blocks_per_sm;
    return MRS_OK;
}

mrs_status mrs_autotune(mrs_ctx *ctx, int reps, mrs_rollout_shape *table, int cap, int *n_tried,
                        mrs_rollout_shape *best)
{
    DeviceScope dev_scope(ctx);
    if (!ctx || reps < 1 || reps > 1000 || cap < 0) return fail(ctx, MRS_EINVAL, "bad arguments");
    if (!ctx->has_input) return fail(ctx, MRS_ESTATE, "autotune needs the inputs of an earlier step");
    mrs_status st = ensure_bound(ctx);
    if (st != MRS_OK) return st;
    std::vector<char> blob(ctx->sz.state_bytes);
    if ((st = mrs_save_state(ctx, blob.data(), blob.size())) != MRS_OK) return st;
    // Whole cycles are timed as they run in use: the graph without timing
    // nodes, so that each kernel's prologue overlaps its predecessor's tail
    // (programmatic launch).  A shape's rollout time alone misleads: per-stage
    // timing serialises the stages, and a shape that is fast there can leave
    // the following stages waiting under overlap.
    const bool timing = ctx->timing;
    if ((st = mrs_enable_timing(ctx, 0)) != MRS_OK) return st;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return fail(ctx, MRS_ECUDA, "autotune: event create");
    }
    // Each trial cycle starts from a cold L2 (a write of twice its size just
    // before), as a controller's cycle does when other work shares the GPU
    // between cycles; without room for the buffer the trials start warm.
    int dev = 0, l2 = 0;
    void *evict = nullptr;
    size_t evict_bytes = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0) {
        evict_bytes = 2 * (size_t)l2;
        if (cudaMalloc(&evict, evict_bytes) != cudaSuccess) {
            evict = nullptr;
            cudaGetLastError();   // clear the allocation failure
        }
    }
    std::vector<mrs_rollout_shape> tried;
    const mrs_rollout_shape before{ctx->tile_samples, ctx->blocks_per_sm, ctx->tile_order, 0.f};
    mrs_rollout_shape keep = before;
    float best_ms = INFINITY;
    for (int ts : {32, 64, 128, 256, 512, 1024}) {
        for (int bps = 1; bps <= ctx->max_blocks_per_sm && st == MRS_OK; ++bps) {
            for (int order = 0; order < 3 && st == MRS_OK; ++order) {
                if ((st = apply_shape(ctx, ts, bps, order)) != MRS_OK) break;
                // every shape's trials start from the same state (and draw the same
                // samples): the controller's state drifts over the trials, and with
                // it the work of a cycle
                if ((st = mrs_load_state(ctx, blob.data(), blob.size())) != MRS_OK) break;
                std::vector<float> t;
                for (int r = 0; r <= reps; ++r) {   // the first cycle warms up (and instantiates)
                    cudaError_t e = evict ? cudaMemsetAsync(evict, r & 0xff, evict_bytes, ctx->stream)
                                          : cudaSuccess;
                    if (e == cudaSuccess) e = cudaEventRecord(t0, ctx->stream);
                    if (e == cudaSuccess && (st = launch_cycle(ctx)) != MRS_OK) break;
                    if (e == cudaSuccess) e = cudaEventRecord(t1, ctx->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                    if (e != cudaSuccess) {
                        st = cuda_fail(ctx, e, "autotune: cycle timing");
                        break;
                    }
                    if (r > 0) t.push_back(ms);
                }
                if (st != MRS_OK) break;
                std::sort(t.begin(), t.end());
                const float med = t[t.size() / 2];
                tried.push_back(mrs_rollout_shape{ts, bps, order, med});
                if (med < best_ms) {
                    best_ms = med;
                    keep = tried.back();
                }
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (evict) cudaFree(evict);
    if (st != MRS_OK) {
        // put back the shape, the timing switch and the state as far as the
        // device still allows; the trial's error is the one reported
        const std::string why = ctx->err;
        apply_shape(ctx, before.tile_samples, before.blocks_per_sm, before.order);
        mrs_enable_timing(ctx, timing ? 1 : 0);
        mrs_load_state(ctx, blob.data(), blob.size());
        ctx->err = why;
        return st;
    }
    if ((st = apply_shape(ctx, keep.tile_samples, keep.blocks_per_sm, keep.order)) != MRS_OK) return st;
    if ((st = mrs_enable_timing(ctx, timing ? 1 : 0)) != MRS_OK) return st;
    if ((st = mrs_load_state(ctx, blob.data(), blob.size())) != MRS_OK) return st;
    if (n_tried) *n_tried = (int)tried.size();
    if (table)
        for (int i = 0; i < (int)tried.size() && i < cap; ++i) table[i] = tried[i];
    if (best) *best = keep;
    return MRS_OK;
}

mrs_status mrs_set_wait_limit(mrs_ctx *ctx, long long polls)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    if (polls > (long long)tc::kWaitLimit)
        return fail(ctx, MRS_EINVAL, "wait limit above the default " +
                                         std::to_string(tc::kWaitLimit) + " polls");
    ctx->P.wait_polls = polls < 0 ? tc::kWaitLimit : (unsigned)polls;
    invalidate_graph(ctx);
    return MRS_OK;
}

mrs_status mrs_set_zero_noise(mrs_ctx *ctx, int zero_noise)
{
    DeviceScope dev_scope(ctx);
    if (!ctx) return MRS_EINVAL;
    ctx->P.zero_noise = zero_noise ? 1 : 0;
    invalidate_graph(ctx);
    return MRS_OK;
}

mrs_status mrs_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    if (n < 0 || (n && (!ctr || !key || !out))) return MRS_EINVAL;
    if (n == 0) return MRS_OK;
    uint4 *d = nullptr;
    if (cudaMalloc(&d, sizeof(uint4) * 2 * (size_t)n) != cudaSuccess) return MRS_ENOMEM;
    cudaError_t e = cudaMemcpy(d, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = enqueue_philox(n, d, make_uint2(key[0], key[1]), d + n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + n, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? MRS_OK : MRS_ECUDA;
}

}  // extern "C"
