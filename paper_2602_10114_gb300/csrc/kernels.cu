// kernels.cu -- the sm_103a kernels of one MR-STORM control cycle.
//
// Per cycle (Algorithm 1 of arxiv 2602.10114, all arms batched):
//   k_prep     Sense + Shift: distance-to-goal, priority weights alpha^(j,i)
//              (Sec. IV-B), left shift of phi (Sec. III-A), Cholesky L_h.
//   per optimisation iteration:
//     k_sample   SampleControls: Philox normals, eps = L_h z, U = mu + eps,
//                semi-implicit Euler integration, stop/joint-limit terms.
//     k_rollout  Rollout: DH kinematics of the collision spheres and the
//                world / self / coordination clearance terms (Eq. 5,
//                Sec. IV-A), stage cost C_{n,h}.
//     k_costs    Eq. 1: discounted sum over the horizon (compensated).
//     k_update   Eqs. 2-4: log-sum-exp weights, weighted mean/covariance,
//                EMA; PickBest (U_*) on the last iteration.
//   k_toplan   ToPlan + Publish: zero-noise rollout of the updated mean to the
//              anticipated plan on the board (Sec. IV-A).
#include <cstdio>

#include "kernels.cuh"

namespace mrs {

constexpr int kMaxWorld = MRS_MAX_WORLD_SPHERES;
constexpr int kMaxAabb = MRS_MAX_AABBS;

// ---------------------------------------------------------------------------
// set-up

__global__ void k_init_arms(ArmDev *arms)
{
    ArmDev &A = arms[blockIdx.x];
    const int t = threadIdx.x;
    if (t == 0) {
        float w = A.base_pose[3], x = A.base_pose[4], y = A.base_pose[5], z = A.base_pose[6];
        const float n = sqrtf(w * w + x * x + y * y + z * z);
        w /= n; x /= n; y /= n; z /= n;
        A.base_R[0] = 1.f - 2.f * (y * y + z * z);
        A.base_R[1] = 2.f * (x * y - w * z);
        A.base_R[2] = 2.f * (x * z + w * y);
        A.base_R[3] = 2.f * (x * y + w * z);
        A.base_R[4] = 1.f - 2.f * (x * x + z * z);
        A.base_R[5] = 2.f * (y * z - w * x);
        A.base_R[6] = 2.f * (x * z - w * y);
        A.base_R[7] = 2.f * (y * z + w * x);
        A.base_R[8] = 1.f - 2.f * (x * x + y * y);
        A.base_t[0] = A.base_pose[0];
        A.base_t[1] = A.base_pose[1];
        A.base_t[2] = A.base_pose[2];
    }
    if (t < A.dof) {
        float s, c;
        sincosf(A.dh[t].z, &s, &c);
        A.twist[t] = make_float2(s, c);
    }
}

// mu = 0, Sigma = sigma^2 I, empty board, clocks at zero.
__global__ void k_reset(Params P, Dev D, int total_hdd, int total_hd)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int i = tid; i < total_hd; i += stride) D.mu[i] = 0.f;
    const float s2 = P.sigma_init * P.sigma_init;
    for (int a = 0; a < P.n_arms; ++a) {
        const ArmDev &A = D.arms[a];
        const int dd = A.dof * A.dof;
        for (int i = tid; i < A.H * dd; i += stride) {
            const int k = i % dd;
            D.Sigma[A.off_hdd + i] = (k % (A.dof + 1) == 0) ? s2 : 0.f;
        }
    }
    for (int i = tid; i < P.n_arms; i += stride) {
        D.board_valid[i] = 0;
        D.board_stamp[i] = -1;
        D.board_dist[i] = 0.f;
        D.e_now[i] = 0.f;
        D.n_star[i] = 0;
    }
    if (tid == 0) {
        *D.cycle = 0;
        *D.world_t = 0.f;
        *D.err = 0;
        D.world_n[0] = 0;
        D.world_n[1] = 0;
    }
}

// ---------------------------------------------------------------------------
// Sense + Shift + Cholesky (one block per arm)

__device__ void cholesky_fp32(int d, const float *S, float *L)
{
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            float s = S[i * d + j];
            if (i == j) s = __fadd_rn(s, 1e-8f);
            for (int k = 0; k < j; ++k) s = __fmaf_rn(-L[i * d + k], L[j * d + k], s);
            if (i == j)
                L[i * d + i] = sqrtf(s > 1e-12f ? s : 1e-12f);
            else
                L[i * d + j] = __fdiv_rn(s, L[j * d + j]);
        }
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) L[i * d + j] = 0.f;
}

__global__ void k_prep(Params P, Dev D)
{
    extern __shared__ float sm[];
    const int a = blockIdx.x;
    const ArmDev &A = D.arms[a];
    const int d = A.dof, H = A.H, dd = d * d;
    const long long cycle = *D.cycle;
    float *Sig = D.Sigma + A.off_hdd;
    float *mu = D.mu + A.off_hd;

    // Shift (not before the first cycle): phi_h <- phi_{h+1}; the last step
    // keeps its mean and restarts from sigma_init^2 I.
    if (cycle > 0) {
        float *sS = sm, *sM = sm + H * dd;
        for (int i = threadIdx.x; i < H * dd; i += blockDim.x) sS[i] = Sig[i];
        for (int i = threadIdx.x; i < H * d; i += blockDim.x) sM[i] = mu[i];
        __syncthreads();
        const float s2 = P.sigma_init * P.sigma_init;
        for (int i = threadIdx.x; i < H * dd; i += blockDim.x) {
            const int h = i / dd, k = i % dd;
            Sig[i] = (h + 1 < H) ? sS[i + dd] : ((k % (d + 1) == 0) ? s2 : 0.f);
        }
        for (int i = threadIdx.x; i < H * d; i += blockDim.x) {
            const int h = i / d;
            mu[i] = (h + 1 < H) ? sM[i + d] : sM[i];
        }
        __syncthreads();
    }
    // Cholesky factor of every step's covariance.
    for (int h = threadIdx.x; h < H; h += blockDim.x)
        cholesky_fp32(d, Sig + h * dd, D.L + A.off_hdd + h * dd);

    // Sense: distance of the end effector to the goal, from the measured q.
    __shared__ float e_self;
    if (threadIdx.x == 0) {
        const float *in = D.input + A.off_in;
        Frame F;
        frame_base(A, F);
        for (int i = 0; i < d; ++i) frame_step(F, in[i], A.dh[i], A.twist[i]);
        const float *gp = in + 2 * d;
        const float dx = __fsub_rn(F.t[0], gp[0]), dy = __fsub_rn(F.t[1], gp[1]),
                    dz = __fsub_rn(F.t[2], gp[2]);
        e_self = sqrtf(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
        D.e_now[a] = e_self;
    }
    __syncthreads();
    // Priority of every neighbour with a published plan (Sec. IV-B), from the
    // own sensed distance and the neighbour's published one.
    for (int i = threadIdx.x; i < P.n_arms; i += blockDim.x)
        D.alpha[a * P.n_arms + i] = (i != a && D.board_valid[i])
                                        ? priority(e_self, D.board_dist[i], P.tau)
                                        : 0.f;
}

// ---------------------------------------------------------------------------
// SampleControls + integration (one block per (arm, 32 samples))

__global__ void __launch_bounds__(256) k_sample(Params P, Dev D, const SampleTile *tiles, int iter)
{
    extern __shared__ float sm[];
    const SampleTile T = tiles[blockIdx.x];
    const ArmDev &A = D.arms[T.arm];
    const int d = A.dof, H = A.H, K = A.K, dd = d * d;
    float *sL = sm;                 // [H][d][d]
    float *sU = sL + H * dd;        // [H][d][32]: U, then the joint-limit terms
    float *sS = sU + H * d * 32;    // [H][d][32]: stop terms
    for (int i = threadIdx.x; i < H * dd; i += blockDim.x) sL[i] = D.L[A.off_hdd + i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = T.n0 + lane;
    const bool valid = n < K;
    const long long cycle = *D.cycle;
    const float *mu = D.mu + A.off_hd;
    float *eps_out = D.eps + A.off_khd;

    for (int h = warp; h < H; h += blockDim.x >> 5) {
        float z[kMaxDof];
        normals(P.seed, T.arm, cycle, iter, n, h, d, z);
        const float *Lh = sL + h * dd;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            if (j < d) {
                float e = 0.f;
#pragma unroll
                for (int c = 0; c <= j; ++c) e = __fmaf_rn(Lh[j * d + c], z[c], e);
                if (P.zero_noise) e = 0.f;
                sU[(h * d + j) * 32 + lane] = __fadd_rn(mu[h * d + j], e);
                if (valid) eps_out[(long long)(h * d + j) * K + n] = e;
            }
        }
    }
    __syncthreads();

    // Integration, one thread per (sample, joint), sequential over the horizon.
    const float *in = D.input + A.off_in;
    float *traj = D.traj + A.off_khd;
    for (int t = threadIdx.x; t < 32 * d; t += blockDim.x) {
        const int l = t & 31, j = t >> 5;
        const int nn = T.n0 + l;
        float q = in[j], qd = in[d + j];
        const float hi = __fsub_rn(A.q_hi[j], P.q_margin), lo = __fadd_rn(A.q_lo[j], P.q_margin);
        for (int h = 0; h < H; ++h) {
            const int idx = (h * d + j) * 32 + l;
            integrate(q, qd, sU[idx], P.dt);
            if (nn < K) traj[(long long)(h * d + j) * K + nn] = q;
            sS[idx] = hinge2(__fsub_rn(fabsf(qd), A.qd_max[j]));
            sU[idx] = __fadd_rn(hinge2(__fsub_rn(q, hi)), hinge2(__fsub_rn(lo, q)));
        }
    }
    __syncthreads();
    float *lim = D.stage_lim + A.off_kh;
    for (int t = threadIdx.x; t < 32 * H; t += blockDim.x) {
        const int l = t & 31, h = t >> 5;
        const int nn = T.n0 + l;
        if (nn >= K) continue;
        float s = 0.f, jc = 0.f;
        for (int j = 0; j < d; ++j) {
            s = __fadd_rn(s, sS[(h * d + j) * 32 + l]);
            jc = __fadd_rn(jc, sU[(h * d + j) * 32 + l]);
        }
        lim[(long long)h * K + nn] = __fmaf_rn(P.w_joint, jc, __fmul_rn(P.w_stop, s));
    }
}

// ---------------------------------------------------------------------------
// Rollout costs (one block per (arm, step h, 32 samples); warp g owns sphere
// group g = spheres [g*spg, (g+1)*spg) of those 32 rollout steps)

struct RolloutSmem {
    float4 *sph;      // [ns] local centre + radius
    int *frame;       // [ns]
    int *start;       // [ns] self-pair start
    float4 *world;    // [n_world] at the step's time
    float4 *aabb;     // [2 * n_aabb]
    float4 *plan;     // neighbours' plan spheres at step h, concatenated
    int *nb_start;    // [n_nb + 1]
    float *nb_alpha;  // [n_nb]
    float *own;       // [ns][3][32] own sphere centres
    int *red;         // [(2 + n_nb) * 32] ordered-int minima: world, self, neighbours
};

// Candidate test of one pair: only pairs within the ramp of the cost
// (centre distance < r1 + r2 + B) can change it; those get the exact
// distance.  m is the running minimum of the signed distance.
__device__ __forceinline__ void pair_min(float3 c, float rB, float r, float4 p, float &m)
{
    const float dx = __fsub_rn(p.x, c.x), dy = __fsub_rn(p.y, c.y), dz = __fsub_rn(p.z, c.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    const float t = __fadd_rn(rB, p.w);
    if (d2 < __fmul_rn(t, t)) m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), r), p.w));
}

template <int SPG>
__device__ __forceinline__ void rollout_group(const Params &P, const Dev &D, const ArmDev &A,
                                              const RolloutSmem &S, int h, int n, bool valid,
                                              int g, int lane, int n_world, int n_aabb, int n_nb,
                                              float *pose_out)
{
    const int d = A.dof, ns = A.ns, K = A.K;
    const int s0 = g * SPG;
    const int cnt = max(0, min(SPG, ns - s0));
    // joint positions of this rollout step, read per frame (coalesced over n)
    const float *qh = D.traj + A.off_khd + (long long)h * d * K + (valid ? n : 0);

    // DH chain up to the last frame this group needs (the last group always
    // runs to the end effector for the pose cost).
    float cx[SPG], cy[SPG], cz[SPG], rr[SPG];
    Frame F;
    frame_base(A, F);
    int f = 0;
#pragma unroll
    for (int s = 0; s < SPG; ++s) {
        if (s < cnt) {
            const int fs = S.frame[s0 + s];
            while (f < fs) {
                frame_step(F, qh[(long long)f * K], A.dh[f], A.twist[f]);
                ++f;
            }
            const float4 p = S.sph[s0 + s];
            const float3 c = sphere_centre(F, p);
            cx[s] = c.x; cy[s] = c.y; cz[s] = c.z; rr[s] = p.w;
            S.own[((s0 + s) * 3 + 0) * 32 + lane] = c.x;
            S.own[((s0 + s) * 3 + 1) * 32 + lane] = c.y;
            S.own[((s0 + s) * 3 + 2) * 32 + lane] = c.z;
        } else {
            cx[s] = cy[s] = cz[s] = 1e15f;
            rr[s] = 0.f;
        }
    }
    if (g == kGroups - 1) {
        while (f < d) {
            frame_step(F, qh[(long long)f * K], A.dh[f], A.twist[f]);
            ++f;
        }
        const float *in = D.input + A.off_in;
        *pose_out = pose_cost(F, in + 2 * d, in + 2 * d + 3, P.w_rot);
    }

    // world clearance: spheres, then boxes
    if (cnt > 0) {
        float m = kInf;
        float rB[SPG];
#pragma unroll
        for (int s = 0; s < SPG; ++s) rB[s] = __fadd_rn(rr[s], P.B_world);
        for (int k = 0; k < n_world; ++k) {
            const float4 o = S.world[k];
#pragma unroll
            for (int s = 0; s < SPG; ++s) pair_min(make_float3(cx[s], cy[s], cz[s]), rB[s], rr[s], o, m);
        }
        for (int b = 0; b < n_aabb; ++b) {
            const float4 bc = S.aabb[2 * b], bh = S.aabb[2 * b + 1];
#pragma unroll
            for (int s = 0; s < SPG; ++s)
                if (s < cnt) m = fminf(m, sphere_aabb(make_float3(cx[s], cy[s], cz[s]), rr[s], bc, bh));
        }
        if (m < P.B_world) atomicMin(&S.red[0 * 32 + lane], float_to_ordered(m));

        // coordination: every published neighbour plan at this step
#pragma unroll
        for (int s = 0; s < SPG; ++s) rB[s] = __fadd_rn(rr[s], P.B);
        for (int nb = 0; nb < n_nb; ++nb) {
            float mn = kInf;
            const int k1 = S.nb_start[nb + 1];
            for (int k = S.nb_start[nb]; k < k1; ++k) {
                const float4 p = S.plan[k];
#pragma unroll
                for (int s = 0; s < SPG; ++s) pair_min(make_float3(cx[s], cy[s], cz[s]), rB[s], rr[s], p, mn);
            }
            if (mn < P.B) atomicMin(&S.red[(2 + nb) * 32 + lane], float_to_ordered(mn));
        }
    }
    __syncthreads();   // own sphere centres of all groups are in shared memory

    // self collision: own spheres against later spheres on bodies >= 3 apart
    if (cnt > 0) {
        float m = kInf;
#pragma unroll
        for (int s = 0; s < SPG; ++s) {
            if (s < cnt) {
                const float rB = __fadd_rn(rr[s], P.B_self);
                const float3 c = make_float3(cx[s], cy[s], cz[s]);
                for (int k = S.start[s0 + s]; k < ns; ++k) {
                    const float4 p = make_float4(S.own[(k * 3 + 0) * 32 + lane],
                                                 S.own[(k * 3 + 1) * 32 + lane],
                                                 S.own[(k * 3 + 2) * 32 + lane], S.sph[k].w);
                    pair_min(c, rB, rr[s], p, m);
                }
            }
        }
        if (m < P.B_self) atomicMin(&S.red[1 * 32 + lane], float_to_ordered(m));
    }
}

__global__ void __launch_bounds__(kRolloutThreads) k_rollout(Params P, Dev D,
                                                             const RolloutTile *tiles, int iter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const RolloutTile T = tiles[blockIdx.x];
    const ArmDev &A = D.arms[T.arm];
    const int ns = A.ns, h = T.h;
    const int n_world = D.world_n[0], n_aabb = D.world_n[1];
    const int NA = P.n_arms;

    // shared-memory carve (sizes bounded by the build limits)
    RolloutSmem S;
    unsigned char *p = smraw;
    S.world = (float4 *)p;  p += sizeof(float4) * kMaxWorld;
    S.aabb = (float4 *)p;   p += sizeof(float4) * 2 * kMaxAabb;
    S.sph = (float4 *)p;    p += sizeof(float4) * kMaxSpheres;
    S.plan = (float4 *)p;   p += sizeof(float4) * (size_t)P.max_ns * NA;
    S.own = (float *)p;     p += sizeof(float) * kMaxSpheres * 3 * 32;
    S.frame = (int *)p;     p += sizeof(int) * kMaxSpheres;
    S.start = (int *)p;     p += sizeof(int) * kMaxSpheres;
    S.nb_start = (int *)p;  p += sizeof(int) * (MRS_MAX_ARMS + 1);
    S.nb_alpha = (float *)p; p += sizeof(float) * MRS_MAX_ARMS;
    S.red = (int *)p;

    __shared__ int s_nb_arm[MRS_MAX_ARMS];
    __shared__ int s_nnb;
    if (threadIdx.x == 0) {
        int nnb = 0, tot = 0;
        for (int i = 0; i < NA; ++i) {
            if (i == T.arm || !D.board_valid[i]) continue;
            const ArmDev &Ai = D.arms[i];
            if (h >= Ai.H) continue;                 // min(H_j, H_i) rule
            s_nb_arm[nnb] = i;
            S.nb_start[nnb] = tot;
            S.nb_alpha[nnb] = D.alpha[T.arm * NA + i];
            tot += Ai.ns;
            ++nnb;
        }
        S.nb_start[nnb] = tot;
        s_nnb = nnb;
    }
    const float t_h = __fmaf_rn((float)(h + 1), P.dt, *D.world_t);
    for (int k = threadIdx.x; k < n_world; k += blockDim.x) {
        const float4 o = D.world[k], v = D.world_vel[k];
        S.world[k] = make_float4(__fmaf_rn(v.x, t_h, o.x), __fmaf_rn(v.y, t_h, o.y),
                                 __fmaf_rn(v.z, t_h, o.z), o.w);
    }
    for (int k = threadIdx.x; k < 2 * n_aabb; k += blockDim.x) S.aabb[k] = D.aabb[k];
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        S.sph[k] = A.sph[k];
        S.frame[k] = A.frame[k];
        S.start[k] = A.self_start[k];
    }
    __syncthreads();
    const int n_nb = s_nnb;
    for (int nb = 0; nb < n_nb; ++nb) {
        const ArmDev &Ai = D.arms[s_nb_arm[nb]];
        const float4 *src = D.board_sph + (Ai.off_hs >> 2) + (size_t)h * Ai.ns;
        for (int k = threadIdx.x; k < Ai.ns; k += blockDim.x) S.plan[S.nb_start[nb] + k] = src[k];
    }
    for (int k = threadIdx.x; k < (2 + n_nb) * 32; k += blockDim.x) S.red[k] = float_to_ordered(kInf);
    __syncthreads();

    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = T.n0 + lane;
    const bool valid = n < A.K;
    __shared__ float s_pose[32];
    float pose = 0.f;
    switch (A.spg) {
        case 1: rollout_group<1>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 2: rollout_group<2>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 3: rollout_group<3>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 4: rollout_group<4>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 5: rollout_group<5>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 6: rollout_group<6>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        case 7: rollout_group<7>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
        default: rollout_group<8>(P, D, A, S, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
    }
    if (g == kGroups - 1) s_pose[lane] = pose;
    __syncthreads();

    // stage cost of Eq. 5 plus the prioritised coordination term
    if (g == 0 && valid) {
        const long long idx = A.off_kh + (long long)h * A.K + n;
        const float dw = ordered_to_float(S.red[0 * 32 + lane]);
        const float dsf = ordered_to_float(S.red[1 * 32 + lane]);
        float dyn = 0.f;
        for (int nb = 0; nb < n_nb; ++nb) {
            const float rho = fmaxf(ordered_to_float(S.red[(2 + nb) * 32 + lane]), 0.f);
            dyn = __fmaf_rn(S.nb_alpha[nb], ramp(rho, P.B), dyn);
        }
        float c = __fmul_rn(P.w_pose, s_pose[lane]);
        c = __fadd_rn(c, D.stage_lim[idx]);
        c = __fmaf_rn(P.w_coll, ramp(dw, P.B_world), c);
        c = __fmaf_rn(P.w_self, ramp(dsf, P.B_self), c);
        c = __fmaf_rn(P.w_dyn, dyn, c);
        D.stage[idx] = c;
    }
    (void)iter;
}

// ---------------------------------------------------------------------------
// Eq. 1: C_n = sum_h gamma^h C_{n,h}, compensated (Kahan) summation.

__global__ void __launch_bounds__(256) k_costs(Params P, Dev D, const CostTile *tiles)
{
    const CostTile T = tiles[blockIdx.x];
    const ArmDev &A = D.arms[T.arm];
    const int n = T.n0 + threadIdx.x;
    if (n >= A.K) return;
    const float *st = D.stage + A.off_kh;
    float s = 0.f, c = 0.f;
    for (int h = 0; h < A.H; ++h) {
        const float gh = (P.gamma == 1.f) ? 1.f : powf(P.gamma, (float)h);
        const float y = __fsub_rn(__fmul_rn(gh, st[(long long)h * A.K + n]), c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    D.costs[A.off_k + n] = s;
}

// ---------------------------------------------------------------------------
// Eqs. 2-4 for one (arm, step h).  Every block recomputes the arm's minimum
// cost and normaliser (identical, deterministic reductions), then reduces the
// weighted first and second moments of eps at its step:
//   mu~ = mu + S1/Z,  Sigma~ = S2/Z - (S1/Z)(S1/Z)^T,
// which equals Eq. 3 since U - mu~ = eps - S1/Z.

constexpr int kMoments = kMaxDof + kMaxDof * (kMaxDof + 1) / 2;  // 54

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(256) k_update(Params P, Dev D, const UpdateTile *tiles, int last)
{
    const UpdateTile T = tiles[blockIdx.x];
    const ArmDev &A = D.arms[T.arm];
    const int d = A.dof, K = A.K, h = T.h, dd = d * d;
    const float *C = D.costs + A.off_k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ float s_v[32];
    __shared__ int s_i[32];
    __shared__ float s_beta, s_Z;
    __shared__ int s_best;
    __shared__ float s_mom[8][kMoments];

    // minimum cost and its lowest index
    float bv = kInf;
    int bi = 0x7fffffff;
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
        const float v = C[n];
        if (v < bv || (v == bv && n < bi)) { bv = v; bi = n; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_v[warp] = bv; s_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = s_v[0];
        int i = s_i[0];
        for (int w = 1; w < nw; ++w)
            if (s_v[w] < v || (s_v[w] == v && s_i[w] < i)) { v = s_v[w]; i = s_i[w]; }
        s_beta = v;
        s_best = i;
    }
    __syncthreads();
    const float beta = s_beta;
    const float inv_lambda = __frcp_rn(P.lambda);

    // normaliser Z = sum_n exp(-(C_n - beta)/lambda) and the moments of eps
    float z = 0.f;
    float m1[kMaxDof], m2[kMoments - kMaxDof];
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) m1[j] = 0.f;
#pragma unroll
    for (int k = 0; k < kMoments - kMaxDof; ++k) m2[k] = 0.f;
    const float *eps = D.eps + A.off_khd + (long long)h * d * K;
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
        const float w = expf(-__fmul_rn(__fsub_rn(C[n], beta), inv_lambda));
        z = __fadd_rn(z, w);
        float e[kMaxDof];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) e[j] = (j < d) ? eps[(long long)j * K + n] : 0.f;
        int k = 0;
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) {
            m1[j] = __fmaf_rn(w, e[j], m1[j]);
            const float we = __fmul_rn(w, e[j]);
#pragma unroll
            for (int c = 0; c <= j; ++c) {
                m2[k] = __fmaf_rn(we, e[c], m2[k]);
                ++k;
            }
        }
    }
    z = warp_sum(z);
    if (lane == 0) s_v[warp] = z;
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) {
        const float v = warp_sum(m1[j]);
        if (lane == 0) s_mom[warp][j] = v;
    }
#pragma unroll
    for (int k = 0; k < kMoments - kMaxDof; ++k) {
        const float v = warp_sum(m2[k]);
        if (lane == 0) s_mom[warp][kMaxDof + k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float Z = 0.f;
        for (int w = 0; w < nw; ++w) Z = __fadd_rn(Z, s_v[w]);
        s_Z = Z;
    }
    if (threadIdx.x < kMoments) {
        float v = 0.f;
        for (int w = 0; w < nw; ++w) v = __fadd_rn(v, s_mom[w][threadIdx.x]);
        s_mom[0][threadIdx.x] = v;
    }
    __syncthreads();

    if (threadIdx.x == 0) {
        const float invZ = __frcp_rn(s_Z);
        float *mu = D.mu + A.off_hd + h * d;
        float *Sig = D.Sigma + A.off_hdd + h * dd;
        float delta[kMaxDof];
        for (int j = 0; j < d; ++j) delta[j] = __fmul_rn(s_mom[0][j], invZ);
        // PickBest on the last iteration: U_* = mu_1 + eps_{n*,1} (old mean)
        if (last && h == 0) {
            const float *e0 = D.eps + A.off_khd;
            for (int j = 0; j < d; ++j)
                D.out[D.out_u + A.off_d + j] = __fadd_rn(mu[j], e0[(long long)j * K + s_best]);
            D.out[D.out_min + T.arm] = beta;
            D.n_star[T.arm] = s_best;
        }
        for (int j = 0; j < d; ++j) mu[j] = __fmaf_rn(P.alpha_mu, delta[j], mu[j]);
        int k = 0;
        for (int j = 0; j < d; ++j)
            for (int c = 0; c <= j; ++c) {
                const float st = __fsub_rn(__fmul_rn(s_mom[0][kMaxDof + k], invZ),
                                           __fmul_rn(delta[j], delta[c]));
                const float nv = __fmaf_rn(P.alpha_sigma, st,
                                           __fmul_rn(1.f - P.alpha_sigma, Sig[j * d + c]));
                Sig[j * d + c] = nv;
                Sig[c * d + j] = nv;
                ++k;
            }
        if (!last) cholesky_fp32(d, Sig, D.L + A.off_hdd + h * dd);
    }
}

// ---------------------------------------------------------------------------
// ToPlan + Publish (one block per arm): integrate the updated mean from the
// sensed state, kinematics of every sphere at every step, into the board.
// The last block to finish advances the cycle counter and the world clock.

__global__ void k_toplan(Params P, Dev D, int *done_counter)
{
    extern __shared__ float sq[];   // [H][d]
    const int a = blockIdx.x;
    const ArmDev &A = D.arms[a];
    const int d = A.dof, H = A.H, ns = A.ns;
    const float *mu = D.mu + A.off_hd;
    const float *in = D.input + A.off_in;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        float q = in[j], qd = in[d + j];
        for (int h = 0; h < H; ++h) {
            integrate(q, qd, mu[h * d + j], P.dt);
            sq[h * d + j] = q;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H * d; i += blockDim.x) {
        D.board_q[A.off_hd + i] = sq[i];
        D.out[D.out_q + A.off_hd + i] = sq[i];
        D.out[D.out_mean + A.off_hd + i] = mu[i];
    }
    float4 *board = D.board_sph + (A.off_hs >> 2);
    float4 *outs = (float4 *)(D.out + D.out_sph) + (A.off_hs >> 2);
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        Frame F;
        frame_base(A, F);
        int f = 0;
        for (int s = 0; s < ns; ++s) {
            const int fs = A.frame[s];
            while (f < fs) {
                frame_step(F, sq[h * d + f], A.dh[f], A.twist[f]);
                ++f;
            }
            const float4 p = A.sph[s];
            const float3 c = sphere_centre(F, p);
            const float4 v = make_float4(c.x, c.y, c.z, p.w);
            board[h * ns + s] = v;
            outs[h * ns + s] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        D.board_valid[a] = 1;
        D.board_stamp[a] = *D.cycle;
        D.board_dist[a] = D.e_now[a];
        D.out[D.out_dist + a] = D.e_now[a];
        __threadfence();
        const int prev = atomicAdd(done_counter, 1);
        if (prev == gridDim.x - 1) {
            *D.cycle = *D.cycle + 1;
            *D.world_t = __fadd_rn(*D.world_t, P.dt);
            *done_counter = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// utility kernels

__global__ void k_fk(Dev D, int arm, int n, const float *q, float *ee, float *spheres)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ArmDev &A = D.arms[arm];
    const int d = A.dof;
    Frame F;
    frame_base(A, F);
    int f = 0;
    for (int s = 0; s < A.ns; ++s) {
        const int fs = A.frame[s];
        while (f < fs) {
            frame_step(F, q[(size_t)i * d + f], A.dh[f], A.twist[f]);
            ++f;
        }
        if (spheres) {
            const float4 p = A.sph[s];
            const float3 c = sphere_centre(F, p);
            ((float4 *)spheres)[(size_t)i * A.ns + s] = make_float4(c.x, c.y, c.z, p.w);
        }
    }
    while (f < d) {
        frame_step(F, q[(size_t)i * d + f], A.dh[f], A.twist[f]);
        ++f;
    }
    for (int k = 0; k < 9; ++k) ee[(size_t)i * 12 + k] = F.R[k];
    for (int k = 0; k < 3; ++k) ee[(size_t)i * 12 + 9 + k] = F.t[k];
}

__global__ void k_debug_spheres(Dev D, int n_req, const int *anh, float *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_req) return;
    const int a = anh[3 * r], n = anh[3 * r + 1], h = anh[3 * r + 2];
    const ArmDev &A = D.arms[a];
    const int d = A.dof;
    float q[kMaxDof];
    for (int j = 0; j < d; ++j) q[j] = D.traj[A.off_khd + (long long)(h * d + j) * A.K + n];
    Frame F;
    frame_base(A, F);
    int f = 0;
    for (int s = 0; s < A.ns; ++s) {
        const int fs = A.frame[s];
        while (f < fs) {
            frame_step(F, q[f], A.dh[f], A.twist[f]);
            ++f;
        }
        const float4 p = A.sph[s];
        const float3 c = sphere_centre(F, p);
        ((float4 *)out)[(size_t)r * kMaxSpheres + s] = make_float4(c.x, c.y, c.z, p.w);
    }
}

__global__ void k_philox(int n, const uint4 *ctr, uint2 key, uint4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

// ---------------------------------------------------------------------------
// host wrappers

cudaError_t configure_kernels(const LaunchPlan &L)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_rollout)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_sample)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.smem_prep)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t enqueue_init(const Params &P, const Dev &D, int n_arms, int total_hdd, int total_hd,
                         cudaStream_t s)
{
    k_init_arms<<<n_arms, 32, 0, s>>>(D.arms);
    k_reset<<<32, 256, 0, s>>>(P, D, total_hdd, total_hd);
    return cudaGetLastError();
}

cudaError_t enqueue_cycle(const Params &P, const Dev &D, const LaunchPlan &L, cudaStream_t s,
                          cudaEvent_t *events, bool capturing)
{
    int ev = 0;
    cudaError_t rec = cudaSuccess;
    auto mark = [&]() {
        if (!events || rec != cudaSuccess) return;
        rec = capturing ? cudaEventRecordWithFlags(events[ev++], s, cudaEventRecordExternal)
                        : cudaEventRecord(events[ev++], s);
    };
    mark();
    k_prep<<<L.n_arms, 256, L.smem_prep, s>>>(P, D);
    mark();
    for (int it = 0; it < P.iterations; ++it) {
        const int last = (it == P.iterations - 1);
        k_sample<<<L.n_sample_tiles, 256, L.smem_sample, s>>>(P, D, L.sample_tiles, it);
        mark();
        k_rollout<<<L.n_rollout_tiles, kRolloutThreads, L.smem_rollout, s>>>(P, D, L.rollout_tiles,
                                                                            it);
        mark();
        k_costs<<<L.n_cost_tiles, 256, 0, s>>>(P, D, L.cost_tiles);
        mark();
        k_update<<<L.n_update_tiles, 256, 0, s>>>(P, D, L.update_tiles, last);
        mark();
    }
    k_toplan<<<L.n_arms, 128, L.smem_toplan, s>>>(P, D, L.done_counter);
    mark();
    if (rec != cudaSuccess) return rec;
    return cudaGetLastError();
}

cudaError_t enqueue_fk(const Dev &D, int arm, int n, const float *q, float *ee, float *spheres,
                       cudaStream_t s)
{
    k_fk<<<(n + 127) / 128, 128, 0, s>>>(D, arm, n, q, ee, spheres);
    return cudaGetLastError();
}

cudaError_t enqueue_debug_spheres(const Dev &D, int n_req, const int *anh, float *out,
                                  cudaStream_t s)
{
    k_debug_spheres<<<(n_req + 63) / 64, 64, 0, s>>>(D, n_req, anh, out);
    return cudaGetLastError();
}

cudaError_t enqueue_philox(int n, const uint4 *ctr, uint2 key, uint4 *out, cudaStream_t s)
{
    k_philox<<<(n + 127) / 128, 128, 0, s>>>(n, ctr, key, out);
    return cudaGetLastError();
}

}  // namespace mrs
