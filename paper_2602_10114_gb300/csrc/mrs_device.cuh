// mrs_device.cuh -- device data layout and arithmetic shared by the kernels of
// the MR-STORM control cycle.  Every quantity that two kernels compute (the
// DH chain, sphere centres, the integration of a control sequence, the
// normals) is written once here with explicit round-to-nearest intrinsics, so
// that, e.g., the zero-noise rollout and ToPlan produce identical bits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mrs.h"

namespace mrs {

constexpr int kMaxDof = MRS_MAX_DOF;
constexpr int kMaxSpheres = MRS_MAX_SPHERES;
constexpr int kGroups = 8;            // sphere groups (= warps) of a rollout CTA
constexpr int kRolloutThreads = 256;  // kGroups warps of 32 samples
constexpr int kTileSamples = 32;
constexpr float kInf = __builtin_inff();

// One arm, resident in device memory.  The derived fields (base rotation,
// sin/cos of the DH twists) are filled on the device by k_init_arms.
struct __align__(16) ArmDev {
    int dof, ns, K, H;
    int off_hd, off_hdd, off_hs, off_d;   // offsets into concatenated arrays
    int off_k, off_in, spg, self_off;     // spg: spheres per group (ceil(ns/8))
    int n_self, external, learned;        // self-collision pairs at self_off in Dev::self_pairs;
                                          // external: optimised elsewhere, plan from the board;
                                          // learned: self clearance from the surrogate (Dev::dhat)
    float self_margin;                    // exact self pass when dhat < B_self + self_margin
    unsigned pair_mask;                   // bit i: the clearance to arm i's plan comes from
                                          // the arm-pair surrogate (Dev::rhohat)
    float pair_margin;                    // exact pass when rhohat < B + pair_margin
    long long off_khd, off_kh;            // offsets into K*H*d and K*H work arrays
    float4 dh[kMaxDof];                   // a, d, alpha, theta_offset
    float2 twist[kMaxDof];                // sin(alpha), cos(alpha)
    float q_lo[kMaxDof], q_hi[kMaxDof], qd_max[kMaxDof];
    float base_pose[8];                   // xyz, quaternion w x y z
    float base_R[9], base_t[3];
    float4 sph[kMaxSpheres];              // centre in body frame, radius
    int frame[kMaxSpheres];               // frame carrying the sphere: min(body, dof)
    int body[kMaxSpheres];
};

struct Params {
    int n_arms, iterations, zero_noise;
    float dt, lambda, gamma, alpha_mu, alpha_sigma, sigma_init;
    float w_pose, w_rot, w_stop, w_joint, w_coll, w_self, w_dyn;
    float B, B_world, B_self, tau, q_margin;
    unsigned long long seed;
    int max_ns, max_pairs;        // largest sphere and self-pair counts of any arm
    int world_cap, aabb_cap;      // shared-memory capacity of the rollout for the world
    int max_plan_age;             // board entries older than this are ignored (0: no limit)
    float w_manip, manip_w0;      // C_manip weight (0: off) and manipulability threshold
    unsigned wait_polls;          // polls of the rollout's bounded wait for its plan copies
};

// A neighbour's board entry is used when it is published and, with a
// staleness limit, at most that many cycles old (Sec. IV-C missing plans).
__device__ __forceinline__ bool plan_usable(const Params &P, int valid, long long stamp,
                                            long long cycle)
{
    return valid && (P.max_plan_age <= 0 || cycle - stamp <= P.max_plan_age);
}

// Device pointers into the workspace.
struct Dev {
    ArmDev *arms;
    float *input;          // packed per arm: q(d) qd(d) goal_p(3) goal_R(9)
    float4 *world;         // [MRS_MAX_WORLD_SPHERES] centre + radius
    float4 *world_vel;     // [MRS_MAX_WORLD_SPHERES] velocity (w unused)
    float4 *world_s;       // the same spheres in a spatial (Morton) order at the next
    float4 *world_vel_s;   // cycle's mid-horizon time, and their velocities: the rollout's copy
    float4 *aabb;          // [MRS_MAX_AABBS][2] centre, half extents
    int *world_n;          // [2] spheres, boxes
    float *mu, *Sigma, *L; // state: [2][hd], [2][hdd] (by cycle parity), [hdd]
    long long st_hd, st_hdd;   // element offset of the second mu / Sigma buffer
    float *Lst;                // [2][sum H d d]: Cholesky factors of the state's covariances,
                               // by cycle parity like Sigma (taken in ToPlan's launch)
    float4 *board_sph;     // plan board read by the cycle: [hs/4]
    float *board_q;        // [hd]
    int *board_valid;      // [A]
    long long *board_stamp;// [A]
    float *board_dist;     // [A]
    float4 *next_sph;      // plans published by this cycle
    float *next_q;
    float *traj;           // [sum K*H*d]  q of every rollout step, [h][j][n]
    float *eps;            // [sum K*H*d]  sampled noise,            [h][j][n]
    float *stage_lim;      // [sum K*H]    stop + joint-limit terms, [h][n]
    float *stage;          // [sum K*H]    full stage cost,          [h][n]
    float *costs;          // [sum K]      C_n of the last iteration
    float *alpha;          // [A][A]
    float *e_now;          // [A]
    int *n_star;           // [A]
    float *out;            // packed outputs
    long long *cycle;      // completed cycles
    float *world_t;        // seconds since the world was set
    int *err;              // device error word (bounded waits)
    int *self_pairs;       // per arm, packed s1 | s2 << 8: bodies >= 3 apart,
                           // clear of the B_self band at the rest pose
    float *self_t2;        // (r1 + B_self + r2)^2 of each self pair, the sums in this order
    float *dhat;           // [sum K*H] surrogate self clearance of every rollout step, [h][n]
    float *rhohat;         // [sum K*H][A] surrogate clearance of every rollout step to each
                           // neighbour's plan: arm j's block at off_kh * A, [i][h][n]
                           // (null without an arm-pair surrogate)
    float4 *pair_board;    // with an arm-pair surrogate: copy of the plan spheres the
                           // cycle read (the board itself holds the new plans afterwards)
    int *work;             // rollout tile counters, one per iteration
    int out_mean, out_sph, out_q, out_u, out_dist, out_min;  // offsets in out (floats)
};

// Programmatic dependent launch.  A kernel launched with programmatic
// stream serialisation may start before its predecessor in the stream has
// finished; pdl_wait() blocks the calling thread until every prerequisite
// grid has completed and its memory is visible.  pdl_trigger() lets the
// next kernel start early; called only after pdl_wait() (or in a kernel
// launched without the attribute), so that when a kernel starts, every
// kernel before its predecessor has completed: its code before pdl_wait()
// may read what those wrote, never what its predecessor writes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// mu and Sigma are double-buffered by cycle parity: the state after cycle
// c - 1 (*D.cycle == c) is in buffer c & 1; cycle c reads it, writes the
// shifted state into buffer (c + 1) & 1 and updates that one.
__device__ __forceinline__ float *mu_buf(const Dev &D, long long parity)
{
    return D.mu + (parity & 1) * D.st_hd;
}
__device__ __forceinline__ float *sigma_buf(const Dev &D, long long parity)
{
    return D.Sigma + (parity & 1) * D.st_hdd;
}
__device__ __forceinline__ float *lst_buf(const Dev &D, long long parity)
{
    return D.Lst + (parity & 1) * D.st_hdd;
}

// Work items of the launch-grid work lists.
// Samples per sampling block: 16 when every arm has at most 1024 samples
// (a warp's two half-warps take two steps of the block's samples, so the
// short sampling launch spans twice the SMs), else 32 (the larger grid
// already fills the GPU, and fewer blocks re-read each step's factors).
constexpr int kSmallArmK = 1024;
struct SampleTile { int arm, n0; };   // samples n0 .. n0 + tile width - 1
struct RolloutTile { int arm, h, n0, nsub; };   // samples n0 .. n0 + 32 nsub - 1 at step h
struct CostTile { int arm, n0; };
struct UpdateTile { int arm, h; };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Top 23 bits, centred: (m + 1/2) 2^-23 is exact in binary32, inside (0, 1).
__device__ __forceinline__ float uniform23(uint32_t x)
{
    return __fmul_rn(__uint2float_rn(x >> 9) + 0.5f, 1.0f / 8388608.0f);
}

// Standard normals z[0..d) for (arm, cycle, iteration, sample n, step h):
// counter = {n, h | block << 16, cycle, arm | iter << 16}, key = seed; each
// Philox block gives two Box-Muller pairs (joints 4b .. 4b+3).
__device__ __forceinline__ void normals(unsigned long long seed, int arm, long long cycle,
                                        int iter, int n, int h, int d, float *z)
{
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
#pragma unroll
    for (int b = 0; b < (kMaxDof + 3) / 4; ++b) {
        if (4 * b >= d) break;
        const uint4 x = philox4x32_10(
            make_uint4((uint32_t)n, (uint32_t)h | ((uint32_t)b << 16),
                       (uint32_t)(unsigned long long)cycle, (uint32_t)arm | ((uint32_t)iter << 16)),
            key);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float ur = uniform23(w[2 * p]);
            const float ua = uniform23(w[2 * p + 1]);
            const float r = sqrtf(-2.0f * logf(ur));
            float s, c;
            sincospif(2.0f * ua, &s, &c);
            const int j0 = 4 * b + 2 * p;
            if (j0 < d) z[j0] = __fmul_rn(r, c);
            if (j0 + 1 < d) z[j0 + 1] = __fmul_rn(r, s);
        }
    }
}

// ---------------------------------------------------------------------------
// Kinematics.  Frame: rotation (row-major) and translation of T_i in world.
struct Frame {
    float R[9];
    float t[3];
};

// rotation of a quaternion (w, x, y, z), normalised first
__device__ __forceinline__ void quat_to_R(float w, float x, float y, float z, float *R)
{
    const float n = sqrtf(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void frame_base(const ArmDev &A, Frame &F)
{
#pragma unroll
    for (int k = 0; k < 9; ++k) F.R[k] = A.base_R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) F.t[k] = A.base_t[k];
}

// T_i = T_{i-1} Rz(q + theta) Tz(d) Tx(a) Rx(alpha), row by row:
//   u = r0 cos + r1 sin, v = r1 cos - r0 sin,
//   R_i row = (u, v cos(alpha) + r2 sin(alpha), r2 cos(alpha) - v sin(alpha)),
//   t_i = t + a u + d r2.
__device__ __forceinline__ void frame_step(Frame &F, float q, float4 dh, float2 tw)
{
    float s, c;
    sincosf(__fadd_rn(q, dh.w), &s, &c);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float r0 = F.R[3 * r], r1 = F.R[3 * r + 1], r2 = F.R[3 * r + 2];
        const float u = __fmaf_rn(r1, s, __fmul_rn(r0, c));
        const float v = __fmaf_rn(r1, c, -__fmul_rn(r0, s));
        F.R[3 * r] = u;
        F.R[3 * r + 1] = __fmaf_rn(r2, tw.x, __fmul_rn(v, tw.y));
        F.R[3 * r + 2] = __fmaf_rn(r2, tw.y, -__fmul_rn(v, tw.x));
        F.t[r] = __fmaf_rn(dh.y, r2, __fmaf_rn(dh.x, u, F.t[r]));
    }
}

// the same step from the sine and cosine of q + theta computed beforehand
__device__ __forceinline__ void frame_step_sc(Frame &F, float s, float c, float4 dh, float2 tw)
{
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float r0 = F.R[3 * r], r1 = F.R[3 * r + 1], r2 = F.R[3 * r + 2];
        const float u = __fmaf_rn(r1, s, __fmul_rn(r0, c));
        const float v = __fmaf_rn(r1, c, -__fmul_rn(r0, s));
        F.R[3 * r] = u;
        F.R[3 * r + 1] = __fmaf_rn(r2, tw.x, __fmul_rn(v, tw.y));
        F.R[3 * r + 2] = __fmaf_rn(r2, tw.y, -__fmul_rn(v, tw.x));
        F.t[r] = __fmaf_rn(dh.y, r2, __fmaf_rn(dh.x, u, F.t[r]));
    }
}

__device__ __forceinline__ float3 sphere_centre(const Frame &F, float4 p)
{
    float3 c;
    c.x = __fmaf_rn(F.R[0], p.x, __fmaf_rn(F.R[1], p.y, __fmaf_rn(F.R[2], p.z, F.t[0])));
    c.y = __fmaf_rn(F.R[3], p.x, __fmaf_rn(F.R[4], p.y, __fmaf_rn(F.R[5], p.z, F.t[1])));
    c.z = __fmaf_rn(F.R[6], p.x, __fmaf_rn(F.R[7], p.y, __fmaf_rn(F.R[8], p.z, F.t[2])));
    return c;
}

// Semi-implicit Euler step of one joint: qd += u dt; q += qd dt.
__device__ __forceinline__ void integrate(float &q, float &qd, float u, float dt)
{
    qd = __fmaf_rn(u, dt, qd);
    q = __fmaf_rn(qd, dt, q);
}

// Pose cost: ||p - g_p|| + w_rot (3 - tr(R_g^T R)) / 2.
__device__ __forceinline__ float pose_cost(const Frame &F, const float *gp, const float *gR,
                                           float w_rot)
{
    const float dx = __fsub_rn(F.t[0], gp[0]), dy = __fsub_rn(F.t[1], gp[1]),
                dz = __fsub_rn(F.t[2], gp[2]);
    const float dist = sqrtf(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
    float tr = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) tr = __fmaf_rn(gR[k], F.R[k], tr);
    return __fmaf_rn(w_rot * 0.5f, __fsub_rn(3.0f, tr), dist);
}

__device__ __forceinline__ float hinge2(float e) { return e > 0.f ? __fmul_rn(e, e) : 0.f; }

// max(0, 1 - dist / B)
__device__ __forceinline__ float ramp(float dist, float B)
{
    // at or beyond the buffer (also +inf, no pair inside) the value is 0:
    // dist / B rounds to at least 1 there, so skipping the division (whose
    // special-value path +inf would take) changes no result
    if (!(dist < B)) return 0.f;
    const float c = __fsub_rn(1.0f, __fdiv_rn(dist, B));
    return c > 0.f ? c : 0.f;
}

// Signed distance of a sphere (centre c, radius r) to a box (centre, half).
__device__ __forceinline__ float sphere_aabb(float3 c, float r, float4 bc, float4 bh)
{
    const float qx = __fsub_rn(fabsf(__fsub_rn(c.x, bc.x)), bh.x);
    const float qy = __fsub_rn(fabsf(__fsub_rn(c.y, bc.y)), bh.y);
    const float qz = __fsub_rn(fabsf(__fsub_rn(c.z, bc.z)), bh.z);
    const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
    const float out = sqrtf(__fmaf_rn(mz, mz, __fmaf_rn(my, my, __fmul_rn(mx, mx))));
    const float in = fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
    return __fsub_rn(__fadd_rn(out, in), r);
}

// Order-preserving map float -> int, so integer atomicMin is a float min.
__device__ __forceinline__ int float_to_ordered(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_to_float(int i)
{
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// alpha^(j,i) = ((e_j + 1e-4) / (e_i + 1e-4))^tau clamped to [1e-6, 1e6].
__device__ __forceinline__ float priority(float e_self, float e_other, float tau)
{
    float a = powf(__fdiv_rn(e_self + 1e-4f, e_other + 1e-4f), tau);
    return fminf(fmaxf(a, 1e-6f), 1e6f);
}

}  // namespace mrs
