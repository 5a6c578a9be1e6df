// kernels.cu -- the sm_103a kernels of one MR-STORM control cycle.
//
// Per cycle (Algorithm 1 of arxiv 2602.10114, all arms batched):
//   per optimisation iteration:
//     k_sample   SampleControls: Philox normals, eps = L_h z, U = mu + eps,
//                semi-implicit Euler integration, stop/joint-limit terms;
//                on the first iteration also Sense + Shift: distance-to-goal,
//                priority weights alpha^(j,i) (Sec. IV-B), left shift of phi
//                (Sec. III-A), Cholesky L_h.
//     k_rollout  Rollout: DH kinematics of the collision spheres and the
//                world / self / coordination clearance terms (Eq. 5,
//                Sec. IV-A), stage cost C_{n,h}.
//     k_costs    Eq. 1: discounted sum over the horizon (compensated).
//     k_update   Eqs. 2-4: log-sum-exp weights, weighted mean/covariance,
//                EMA; PickBest (U_*) on the last iteration.
//   k_toplan   ToPlan + Publish: zero-noise rollout of the updated mean to the
//              anticipated plan on the board (Sec. IV-A).
#include <cstdio>

#include <mutex>

#include "kernels.cuh"

namespace mrs {

// ---------------------------------------------------------------------------
// set-up

__global__ void k_init_arms(ArmDev *arms)
{
    ArmDev &A = arms[blockIdx.x];
    const int t = threadIdx.x;
    if (t == 0) {
        quat_to_R(A.base_pose[3], A.base_pose[4], A.base_pose[5], A.base_pose[6], A.base_R);
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
    for (int i = tid; i < P.n_arms * P.n_arms; i += stride) D.alpha[i] = 0.f;
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

// Cholesky factor L of S + 1e-8 I (the diagonal clamped at 1e-6) by one
// warp: lane l holds the lower-triangle elements e = l and l + 32 (e = i(i+1)/2
// + j, i >= j) and the columns are finished left to right; after column k
// every element (i, j) with j > k takes its update -L[i][k] L[j][k], the two
// factors fetched from their lanes by shuffles.  Each element thus sees the
// same fused multiply-adds in the same order (k ascending) as the row-by-row
// algorithm, then the same correctly rounded square root or division: the
// factor is bitwise the same, with a dependent chain of d columns instead of
// d(d+1)/2 elements.  S and Lout are row-major [d][d] (S in shared or global
// memory, visible to the whole warp); the upper triangle of Lout is zeroed.
// All 32 lanes must call it together.
__device__ __forceinline__ void cholesky_warp(int d, const float *S, float *Lout, int lane)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int nel = d * (d + 1) / 2;   // <= 45 for d <= 9
    int ri[2], ci[2];
    float v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int e = lane + 32 * u;
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        ri[u] = i;
        ci[u] = e - i * (i + 1) / 2;
        v[u] = 0.f;
        if (e < nel) {
            v[u] = S[i * d + ci[u]];
            if (i == ci[u]) v[u] = __fadd_rn(v[u], 1e-8f);
        }
    }
    for (int k = 0; k < d; ++k) {
        // the diagonal element (k, k), then the rest of column k
        const int ekk = k * (k + 1) / 2 + k;
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (lane + 32 * u == ekk) v[u] = sqrtf(v[u] > 1e-12f ? v[u] : 1e-12f);
        const float a0 = __shfl_sync(kAll, v[0], ekk & 31), a1 = __shfl_sync(kAll, v[1], ekk & 31);
        const float lkk = (ekk >> 5) ? a1 : a0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (lane + 32 * u < nel && ci[u] == k && ri[u] > k) v[u] = __fdiv_rn(v[u], lkk);
        // trailing update of the elements (i, j), j > k
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const bool upd = lane + 32 * u < nel && ci[u] > k;
            const int ei = ri[u] * (ri[u] + 1) / 2 + k, ej = ci[u] * (ci[u] + 1) / 2 + k;
            const int si = upd ? ei : 0, sj = upd ? ej : 0;
            const float x0 = __shfl_sync(kAll, v[0], si & 31), x1 = __shfl_sync(kAll, v[1], si & 31);
            const float y0 = __shfl_sync(kAll, v[0], sj & 31), y1 = __shfl_sync(kAll, v[1], sj & 31);
            const float lik = (si >> 5) ? x1 : x0, ljk = (sj >> 5) ? y1 : y0;
            if (upd) v[u] = __fmaf_rn(-lik, ljk, v[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (lane + 32 * u < nel) Lout[ri[u] * d + ci[u]] = v[u];
    for (int e = lane; e < d * d; e += 32)
        if (e % d > e / d) Lout[e] = 0.f;
}

// Sense + Shift as a kernel of its own (one block per arm), for workloads
// whose arms have many sample blocks: distance-to-goal, priority weights
// alpha^(j,i) (Sec. IV-B), the shifted state (Sec. III-A) into this cycle's
// buffer and the shifted Cholesky factors L_h.
__global__ void k_prep(Params P, Dev D)
{
    extern __shared__ float sm[];
    const int a = blockIdx.x, t = threadIdx.x;
    const ArmDev &A = D.arms[a];
    pdl_trigger();   // first kernel of the cycle, launched after the full predecessor
    __shared__ float s_in[2 * kMaxDof + 12];
    __shared__ float4 s_dh[kMaxDof];
    __shared__ float2 s_tw[kMaxDof];
    __shared__ float s_base[12];
    __shared__ float s_bdist[MRS_MAX_ARMS];
    __shared__ int s_bvalid[MRS_MAX_ARMS];   // usable: published and fresh enough
    __shared__ float e_self;

    // first wave of loads, none depending on another: the cycle, the arm's
    // header and kinematic constants, the board's published distances
    const long long cycle = *D.cycle;
    const int external = A.external, d = A.dof, H = A.H, dd = d * d;
    const int off_hdd = A.off_hdd, off_hd = A.off_hd, off_in = A.off_in;
    if (t < kMaxDof) {
        s_dh[t] = A.dh[t];
        s_tw[t] = A.twist[t];
    }
    if (t < 9) s_base[t] = A.base_R[t];
    else if (t < 12) s_base[t] = A.base_t[t - 9];
    if (t < P.n_arms) {
        s_bvalid[t] = plan_usable(P, D.board_valid[t], D.board_stamp[t], cycle) ? 1 : 0;
        s_bdist[t] = D.board_dist[t];
    }
    if (external) return;   // optimised elsewhere (uniform over the block)
    const float *Sig = sigma_buf(D, cycle) + off_hdd;   // the previous cycle's state
    const float *mu = mu_buf(D, cycle) + off_hd;
    float *Sig_cur = sigma_buf(D, cycle + 1) + off_hdd;  // this cycle's
    float *mu_cur = mu_buf(D, cycle + 1) + off_hd;
    float *sS = sm, *sL = sm + H * dd, *sM = sm + 2 * H * dd;

    // second wave: the shifted distribution (Shift, Sec. III-A: phi_h <-
    // phi_{h+1}, the last step keeps its mean and restarts from
    // sigma_init^2 I; not before the first cycle), with the state's Cholesky
    // factors shifted alike (the restart's factor is diagonal, the value the
    // factorisation gives), and the sensed input
    const bool shift = cycle > 0;
    const float s2 = P.sigma_init * P.sigma_init;
    const float x2 = __fadd_rn(s2, 1e-8f), l_last = sqrtf(x2 > 1e-12f ? x2 : 1e-12f);
    const float *Lf = lst_buf(D, cycle) + off_hdd;
#pragma unroll 4
    for (int i = t; i < H * dd; i += blockDim.x) {
        const int h = i / dd, k = i % dd;
        const int src = !shift ? i : (h + 1 < H ? i + dd : -1);
        const bool dg = k % (d + 1) == 0;
        sS[i] = src >= 0 ? Sig[src] : (dg ? s2 : 0.f);
        sL[i] = src >= 0 ? Lf[src] : (dg ? l_last : 0.f);
    }
#pragma unroll 4
    for (int i = t; i < H * d; i += blockDim.x) {
        const int h = i / d;
        sM[i] = (shift && h + 1 < H) ? mu[i + d] : mu[i];
    }
    if (t < 2 * d + 12) s_in[t] = D.input[off_in + t];
    __syncthreads();
    for (int i = t; i < H * dd; i += blockDim.x) Sig_cur[i] = sS[i];
    for (int i = t; i < H * d; i += blockDim.x) mu_cur[i] = sM[i];
    // Sense, on the last thread: the end effector's distance to the goal
    if (t == blockDim.x - 1) {
        Frame F;
        for (int k = 0; k < 9; ++k) F.R[k] = s_base[k];
        for (int k = 0; k < 3; ++k) F.t[k] = s_base[9 + k];
        for (int i = 0; i < d; ++i) frame_step(F, s_in[i], s_dh[i], s_tw[i]);
        const float *gp = s_in + 2 * d;
        const float dx = __fsub_rn(F.t[0], gp[0]), dy = __fsub_rn(F.t[1], gp[1]),
                    dz = __fsub_rn(F.t[2], gp[2]);
        e_self = sqrtf(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
        D.e_now[a] = e_self;
    }
    __syncthreads();
    for (int i = t; i < H * dd; i += blockDim.x) D.L[off_hdd + i] = sL[i];
    // Priority of every neighbour with a published plan (Sec. IV-B), from the
    // own sensed distance and the neighbour's published one.
    for (int i = t; i < P.n_arms; i += blockDim.x)
        D.alpha[a * P.n_arms + i] =
            (i != a && s_bvalid[i]) ? priority(e_self, s_bdist[i], P.tau) : 0.f;
}

// ---------------------------------------------------------------------------
// SampleControls + integration (one block per (arm, NS samples)).  With
// with_prep (first iteration, every arm of at most 1024 samples) the launch is
// also the cycle's Sense + Shift: every block
// shifts the previous state (Shift, Sec. III-A: phi_h <- phi_{h+1}, the last
// step keeps its mean and restarts from sigma_init^2 I; not before the first
// cycle) and the state's Cholesky factors with it, chunk by chunk, into
// shared memory; the arm's first block (n0 = 0) publishes the shifted state
// and factors into the cycle's buffers, and computes the sensed distance to
// the goal and the priorities alpha^(j,i) (Sec. IV-B).

// NS = 32 runs on the large workloads, whose grids fill the GPU: two resident
// blocks per SM (at most 64 registers).
template <int NS>
__global__ void __launch_bounds__(512, NS == 32 ? 2 : 1)
    k_sample(Params P, Dev D, const SampleTile *tiles, int iter, int smem_floats, int with_prep)
{
    extern __shared__ float sm[];
    __shared__ float s_bdist[MRS_MAX_ARMS];
    __shared__ int s_bvalid[MRS_MAX_ARMS];   // usable: published and fresh enough
    __shared__ float s_e;
    const SampleTile T = tiles[blockIdx.x];
    const long long cycle = *D.cycle;
    const ArmDev &A = D.arms[T.arm];
    const int d = A.dof, H = A.H, K = A.K, dd = d * d;
    const int off_hdd = A.off_hdd, off_hd = A.off_hd;
    const bool prep = with_prep != 0, leader = prep && T.n0 == 0;
    const float *mu_prev = mu_buf(D, cycle) + off_hd, *sig_prev = sigma_buf(D, cycle) + off_hdd;
    float *mu_cur = mu_buf(D, cycle + 1) + off_hd, *sig_cur = sigma_buf(D, cycle + 1) + off_hdd;
    // the horizon in chunks of Hc steps that fit the block's shared memory
    const int Hc = max(1, min(H, smem_floats / (dd + d + 2 * d * NS)));
    float *sL = sm;                 // [Hc][d][d]
    float *sMu = sL + Hc * dd;      // [Hc][d]
    float *sU = sMu + Hc * d;       // [Hc][d][NS]: U, then the joint-limit terms
    float *sS = sU + Hc * d * NS;   // [Hc][d][NS]: stop terms

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // lane l draws sample n0 + l % NS at step slot warp * 32 / NS + l / NS
    const int sl = lane % NS, slot = warp * (32 / NS) + lane / NS, nslot = 512 / NS;   // 512 threads
    const int n = T.n0 + sl;
    const bool valid = n < K;
    float *eps_out = D.eps + A.off_khd;
    const float *in = D.input + A.off_in;
    float *traj = D.traj + A.off_khd;
    float *lim = D.stage_lim + A.off_kh;

    // integration state and constants of this thread's (sample, joint),
    // carried across chunks; loaded in the same wave as the first chunk
    const int ti = threadIdx.x, il = ti % NS, ij = ti / NS;
    const bool integrates = ti < NS * d;
    float q = 0.f, qd = 0.f, hi = 0.f, lo = 0.f, vmax = 0.f;
    if (integrates) {
        q = in[ij];
        qd = in[d + ij];
        hi = __fsub_rn(A.q_hi[ij], P.q_margin);
        lo = __fadd_rn(A.q_lo[ij], P.q_margin);
        vmax = A.qd_max[ij];
    }
    if (leader && ti < P.n_arms) {   // the board's published distances, for the priorities
        s_bvalid[ti] = plan_usable(P, D.board_valid[ti], D.board_stamp[ti], cycle) ? 1 : 0;
        s_bdist[ti] = D.board_dist[ti];
    }
    pdl_wait();      // later iterations: L and mu come from the previous update
    pdl_trigger();
    const bool shift = cycle > 0;
    const float s2 = P.sigma_init * P.sigma_init;
    const float x2 = __fadd_rn(s2, 1e-8f), l_last = sqrtf(x2 > 1e-12f ? x2 : 1e-12f);

    for (int h0 = 0; h0 < H; h0 += Hc) {
        const int nh = min(Hc, H - h0);
        if (prep) {
            // the state's Cholesky factors (taken beside the previous ToPlan)
            // shift with the covariances; the restart's factor is diagonal,
            // the value the factorisation gives
            const float *Lf = lst_buf(D, cycle) + off_hdd;
#pragma unroll 4
            for (int i = threadIdx.x; i < nh * dd; i += blockDim.x) {
                const int hl = i / dd, k = i - hl * dd, h = h0 + hl;
                const int src = !shift ? h * dd + k : (h + 1 < H ? (h + 1) * dd + k : -1);
                const bool dg = k % (d + 1) == 0;
                const float lf = src >= 0 ? Lf[src] : (dg ? l_last : 0.f);
                sL[i] = lf;
                if (leader) {   // the cycle's shifted state and factors
                    sig_cur[h0 * dd + i] = src >= 0 ? sig_prev[src] : (dg ? s2 : 0.f);
                    D.L[off_hdd + (long long)h0 * dd + i] = lf;
                }
            }
            for (int i = threadIdx.x; i < nh * d; i += blockDim.x) {
                const int h = h0 + i / d, src = h0 * d + i;
                sMu[i] = (shift && h + 1 < H) ? mu_prev[src + d] : mu_prev[src];
                if (leader) mu_cur[h0 * d + i] = sMu[i];
            }
            __syncthreads();
        } else {
#pragma unroll 4
            for (int i = threadIdx.x; i < nh * dd; i += blockDim.x)
                sL[i] = D.L[off_hdd + (long long)h0 * dd + i];
            for (int i = threadIdx.x; i < nh * d; i += blockDim.x) sMu[i] = mu_cur[h0 * d + i];
            __syncthreads();
        }

#pragma unroll 1
        for (int hl = slot; hl < nh; hl += nslot) {
            const int h = h0 + hl;
            float z[kMaxDof];
            normals(P.seed, T.arm, cycle, iter, n, h, d, z);
            const float *Lh = sL + hl * dd;
#pragma unroll
            for (int j = 0; j < kMaxDof; ++j) {
                if (j < d) {
                    float e = 0.f;
#pragma unroll
                    for (int c = 0; c <= j; ++c) e = __fmaf_rn(Lh[j * d + c], z[c], e);
                    if (P.zero_noise) e = 0.f;
                    sU[(hl * d + j) * NS + sl] = __fadd_rn(sMu[hl * d + j], e);
                    if (valid) eps_out[(long long)(h * d + j) * K + n] = e;
                }
            }
        }
        __syncthreads();

        // Integration, one thread per (sample, joint), sequential over the
        // horizon; the controls are read 8 steps ahead, so that the chain
        // does not wait on shared memory at every step.
        if (integrates) {
            const int nn = T.n0 + il;
            for (int hb = 0; hb < nh; hb += 8) {
                float u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    u[k] = (hb + k < nh) ? sU[((hb + k) * d + ij) * NS + il] : 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int hl = hb + k;
                    if (hl >= nh) break;
                    const int h = h0 + hl;
                    const int idx = (hl * d + ij) * NS + il;
                    integrate(q, qd, u[k], P.dt);
                    if (nn < K) traj[(long long)(h * d + ij) * K + nn] = q;
                    sS[idx] = hinge2(__fsub_rn(fabsf(qd), vmax));
                    sU[idx] = __fadd_rn(hinge2(__fsub_rn(q, hi)), hinge2(__fsub_rn(lo, q)));
                }
            }
        } else if (leader && h0 == 0 && ti == blockDim.x - 1) {
            // Sense, on an idle warp: the end effector's distance to the goal
            Frame F;
            frame_base(A, F);
            for (int i = 0; i < d; ++i) frame_step(F, in[i], A.dh[i], A.twist[i]);
            const float *gp = in + 2 * d;
            const float dx = __fsub_rn(F.t[0], gp[0]), dy = __fsub_rn(F.t[1], gp[1]),
                        dz = __fsub_rn(F.t[2], gp[2]);
            s_e = sqrtf(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
            D.e_now[T.arm] = s_e;
        }
        __syncthreads();
        if (leader && h0 == 0)
            // Priority of every neighbour with a published plan (Sec. IV-B),
            // from the own sensed distance and the neighbour's published one.
            for (int i = ti; i < P.n_arms; i += blockDim.x)
                D.alpha[T.arm * P.n_arms + i] =
                    (i != T.arm && s_bvalid[i]) ? priority(s_e, s_bdist[i], P.tau) : 0.f;
        for (int t = threadIdx.x; t < NS * nh; t += blockDim.x) {
            const int l = t % NS, hl = t / NS;
            const int nn = T.n0 + l;
            if (nn >= K) continue;
            float s = 0.f, jc = 0.f;
            for (int j = 0; j < d; ++j) {
                s = __fadd_rn(s, sS[(hl * d + j) * NS + l]);
                jc = __fadd_rn(jc, sU[(hl * d + j) * NS + l]);
            }
            lim[(long long)(h0 + hl) * K + nn] = __fmaf_rn(P.w_joint, jc, __fmul_rn(P.w_stop, s));
        }
        __syncthreads();   // the chunk's shared memory is reused by the next
    }
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
    pdl_wait();      // the stage costs come from the rollout
    pdl_trigger();
    float s = 0.f, c = 0.f;
    for (int h0 = 0; h0 < A.H; h0 += 32) {
        float v[32];
#pragma unroll
        for (int u = 0; u < 32; ++u)      // loads first (one round trip), then the ordered sum
            v[u] = (h0 + u < A.H) ? st[(long long)(h0 + u) * A.K + n] : 0.f;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            if (h0 + u >= A.H) break;
            const float gh = (P.gamma == 1.f) ? 1.f : powf(P.gamma, (float)(h0 + u));
            const float y = __fsub_rn(__fmul_rn(gh, v[u]), c);
            const float t = __fadd_rn(s, y);
            c = __fsub_rn(__fsub_rn(t, s), y);
            s = t;
        }
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

constexpr int kUpdateThreads = 256;
constexpr size_t kUpdateSmem = sizeof(float) * (kMoments + 1) * (kUpdateThreads + 1);

__global__ void __launch_bounds__(kUpdateThreads) k_update(Params P, Dev D, const UpdateTile *tiles,
                                                           int last)
{
    constexpr int NT = kUpdateThreads;
    constexpr int kM2 = kMoments - kMaxDof;
    const UpdateTile T = tiles[blockIdx.x];
    const ArmDev &A = D.arms[T.arm];
    const long long cycle = *D.cycle;
    const int d = A.dof, K = A.K, h = T.h, dd = d * d;
    const float *C = D.costs + A.off_k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NT >> 5;
    __shared__ float s_v[32];
    __shared__ int s_i[32];
    __shared__ float s_beta, s_Z;
    __shared__ int s_best;
    // per-thread partial moments and Z, [kMoments + 1][NT + 1] (dynamic)
    extern __shared__ float s_dyn[];
    float (*s_part)[NT + 1] = reinterpret_cast<float (*)[NT + 1]>(s_dyn);
    __shared__ float s_mom[kMoments + 1];
    // the first sample's noise of this thread (e_first) is loaded before the
    // wait: the sample kernel that wrote it finished before the costs kernel
    // could start, and the minimum below does not need it
    const float *eps = D.eps + A.off_khd + (long long)h * d * K;
    float e_first[kMaxDof];
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j)
        e_first[j] = (j < d && (int)threadIdx.x < K) ? eps[(long long)j * K + threadIdx.x] : 0.f;
    // so are this step's current mean and covariance entries (one per
    // thread: mean j = thread, covariance entry (j, c) of the lower triangle
    // number t = thread; d (d + 1) / 2 <= 45 < NT), written before the
    // sample kernel ran
    static_assert(kMaxDof * (kMaxDof + 1) / 2 <= NT, "one covariance entry per thread");
    float *mu = mu_buf(D, cycle + 1) + A.off_hd + h * d;          // the cycle's state
    float *Sig = sigma_buf(D, cycle + 1) + A.off_hdd + h * dd;
    const int tcov = threadIdx.x;
    int jt = 0;
    while ((jt + 1) * (jt + 2) / 2 <= tcov && jt < kMaxDof) ++jt;
    const int ct = tcov - jt * (jt + 1) / 2;
    const bool has_cov = tcov < d * (d + 1) / 2;
    const float mu_old = (int)threadIdx.x < d ? mu[threadIdx.x] : 0.f;
    const float sig_old = has_cov ? Sig[jt * d + ct] : 0.f;
    pdl_wait();      // the totals come from the costs kernel
    pdl_trigger();

    // minimum cost and its lowest index
    float bv = kInf;
    int bi = 0x7fffffff;
#pragma unroll 4
    for (int n = threadIdx.x; n < K; n += NT) {
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

    // per-thread partial normaliser Z = sum_n exp(-(C_n - beta)/lambda) and
    // weighted moments of eps at this step
    float z = 0.f;
    float m1[kMaxDof], m2[kM2];
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) m1[j] = 0.f;
#pragma unroll
    for (int k = 0; k < kM2; ++k) m2[k] = 0.f;
#pragma unroll 2
    for (int n = threadIdx.x; n < K; n += NT) {
        const float w = expf(-__fmul_rn(__fsub_rn(C[n], beta), inv_lambda));
        z = __fadd_rn(z, w);
        float e[kMaxDof];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j)
            e[j] = (n == (int)threadIdx.x) ? e_first[j] : ((j < d) ? eps[(long long)j * K + n] : 0.f);
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
    // block reduction through shared memory, in a fixed order
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) s_part[j][threadIdx.x] = m1[j];
#pragma unroll
    for (int k = 0; k < kM2; ++k) s_part[kMaxDof + k][threadIdx.x] = m2[k];
    s_part[kMoments][threadIdx.x] = z;
    __syncthreads();
    for (int c = warp; c <= kMoments; c += nw) {
        float v = 0.f;
        for (int t = lane; t < NT; t += 32) v = __fadd_rn(v, s_part[c][t]);
        v = warp_sum(v);
        if (lane == 0) s_mom[c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_Z = s_mom[kMoments];
    __syncthreads();

    const float invZ = __frcp_rn(s_Z);
    // PickBest on the last iteration: U_* = mu_1 + eps_{n*,1} (before the update)
    if (last && h == 0 && threadIdx.x < d) {
        const int j = threadIdx.x;
        const float *e0 = D.eps + A.off_khd;
        D.out[D.out_u + A.off_d + j] = __fadd_rn(mu_old, e0[(long long)j * K + s_best]);
        if (j == 0) {
            D.out[D.out_min + T.arm] = beta;
            D.n_star[T.arm] = s_best;
        }
    }
    __syncthreads();
    // Eq. 4 with Eq. 3 written through eps: delta = S1/Z, Sigma~ = S2/Z - delta delta^T
    if (threadIdx.x < d) {
        const int j = threadIdx.x;
        mu[j] = __fmaf_rn(P.alpha_mu, __fmul_rn(s_mom[j], invZ), mu_old);
    }
    if (has_cov) {
        const int t = tcov, j = jt, c = ct;
        const float dj = __fmul_rn(s_mom[j], invZ), dc = __fmul_rn(s_mom[c], invZ);
        const float st = __fsub_rn(__fmul_rn(s_mom[kMaxDof + t], invZ), __fmul_rn(dj, dc));
        const float nv = __fmaf_rn(P.alpha_sigma, st, __fmul_rn(1.f - P.alpha_sigma, sig_old));
        Sig[j * d + c] = nv;
        Sig[c * d + j] = nv;
    }
    if (!last) {
        __syncthreads();
        if (warp == 0) cholesky_warp(d, Sig, D.L + A.off_hdd + h * dd, lane);
    }
}

// Cholesky factor of the state's covariance at work item w (arm, step) in
// the buffers of the given parity, by one warp.  The cycle takes them in
// ToPlan's launch, after the last update, and the next cycle's Shift moves
// them with the covariances, so the sampling never factors on its critical
// path; k_chol takes them after an initialisation or a state load.
__device__ __forceinline__ void state_factor(const Dev &D, const UpdateTile *tiles, int w,
                                             long long parity, int lane)
{
    const UpdateTile T = tiles[w];
    const ArmDev &A = D.arms[T.arm];
    const int d = A.dof;
    const long long o = A.off_hdd + (long long)T.h * d * d;
    cholesky_warp(d, sigma_buf(D, parity) + o, lst_buf(D, parity) + o, lane);
}

__global__ void __launch_bounds__(256) k_chol(Dev D, const UpdateTile *tiles, int n_tiles, int parity)
{
    const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (w < n_tiles) state_factor(D, tiles, w, parity, threadIdx.x & 31);   // uniform over the warp
}

// ---------------------------------------------------------------------------
// ToPlan + Publish (one block per arm): integrate the updated mean from the
// sensed state, kinematics of every sphere at every step, into the board.
// The last block to finish advances the cycle counter and the world clock.
//
// Latency layout: every global read is issued in two waves (the arm's
// constants with its header, then the mean, the sensed state, the cycle and
// the sensed distance); the sines and cosines of q_h + theta are taken in
// parallel, one (step, joint) per thread, so that the kinematics chains run
// from shared memory only.  frame_step_sc from sincosf(q + theta) is the
// rollout's frame_step, so a zero-noise rollout still reproduces the plan
// bit for bit.

// The last block of ToPlan's launch to finish advances the cycle counter and
// the world clock and clears the next cycle's work counters.
__device__ __forceinline__ void toplan_done(const Params &P, const Dev &D, int *done_counter,
                                            long long cyc)
{
    __threadfence();
    const int prev = atomicAdd(done_counter, 1);
    if (prev == gridDim.x - 1) {
        *D.cycle = cyc + 1;
        *D.world_t = __fadd_rn(*D.world_t, P.dt);
        *done_counter = 0;
        for (int i = 0; i < P.iterations; ++i) D.work[i] = 0;   // the next cycle's tile counters
    }
}

// The rollout's copy of the world (Dev::world_s, world_vel_s): the spheres
// sorted by the Morton code of their centres at the next cycle's
// mid-horizon time (t_next: the next cycle's world time), so that the
// rollout's clusters of 8 consecutive spheres are compact.  Only the order
// changes, never a sphere, so no result depends on it.  One block of 256
// threads: block-wide bounding box, 10-bit codes per axis, a bitonic sort of
// (code, index) keys in shared memory, then the gather.
__device__ void world_order_block(const Params &P, const Dev &D, float t_next)
{
    __shared__ unsigned long long key[MRS_MAX_WORLD_SPHERES];
    __shared__ float s_box[8][6];
    const int n = D.world_n[0], t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (n <= 0) return;
    int hmax = 1;
    for (int i = 0; i < P.n_arms; ++i) hmax = max(hmax, D.arms[i].H);
    const float tr = t_next + P.dt * (0.5f * (float)hmax + 1.f);
    auto pos = [&](int k) {
        const float4 o = D.world[k], v = D.world_vel[k];
        return make_float3(o.x + v.x * tr, o.y + v.y * tr, o.z + v.z * tr);
    };
    float lo[3] = {kInf, kInf, kInf}, hi[3] = {-kInf, -kInf, -kInf};
    for (int k = t; k < n; k += blockDim.x) {
        const float3 p = pos(k);
        lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
    }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if (lane == 0) {
            s_box[w][a] = lo[a];
            s_box[w][3 + a] = hi[a];
        }
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            lo[a] = fminf(lo[a], s_box[i][a]);
            hi[a] = fmaxf(hi[a], s_box[i][3 + a]);
        }
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int k = t; k < n2; k += blockDim.x) {
        unsigned long long kk = ~0ull;
        if (k < n) {
            const float3 p = pos(k);
            const float c[3] = {p.x, p.y, p.z};
            unsigned code = 0;
            for (int a = 0; a < 3; ++a) {
                const float ext = fmaxf(hi[a] - lo[a], 1e-6f);
                const unsigned q = (unsigned)fminf(fmaxf((c[a] - lo[a]) * (1023.f / ext), 0.f), 1023.f);
                for (int b = 0; b < 10; ++b) code |= ((q >> b) & 1u) << (3 * b + a);
            }
            kk = ((unsigned long long)code << 32) | (unsigned)k;
        }
        key[k] = kk;
    }
    __syncthreads();
    for (int size = 2; size <= n2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < n2 / 2; i += blockDim.x) {
                const int a = ((i & ~(stride - 1)) << 1) | (i & (stride - 1)), b = a + stride;
                const unsigned long long ka = key[a], kb = key[b];
                if ((ka > kb) == ((a & size) == 0)) {
                    key[a] = kb;
                    key[b] = ka;
                }
            }
            __syncthreads();
        }
    for (int i = t; i < n; i += blockDim.x) {
        const int k = (int)(unsigned)(key[i] & 0xffffffffull);
        D.world_s[i] = D.world[k];
        D.world_vel_s[i] = D.world_vel[k];
    }
}

__global__ void __launch_bounds__(256) k_world_order(Params P, Dev D)
{
    world_order_block(P, D, *D.world_t);
}

cudaError_t enqueue_world_order(const Params &P, const Dev &D, cudaStream_t s)
{
    k_world_order<<<1, 256, 0, s>>>(P, D);
    return cudaGetLastError();
}

// ToPlan (one block per arm), the next cycle's state factors (the blocks
// after them) and the world's order for the next cycle (the last block)
__global__ void __launch_bounds__(256) k_toplan(Params P, Dev D, int *done_counter,
                                                const UpdateTile *ftiles, int n_ftiles)
{
    if ((int)blockIdx.x == (int)gridDim.x - 1) {   // uniform over the block
        // the world time is advanced only by the last block past toplan_done,
        // so it is still this cycle's here; the current rollout has finished
        // with the copy (the wait below covers every earlier kernel)
        const long long cyc = *D.cycle;
        const float t_next = __fadd_rn(*D.world_t, P.dt);
        pdl_wait();
        pdl_trigger();
        world_order_block(P, D, t_next);
        __syncthreads();
        if (threadIdx.x == 0) toplan_done(P, D, done_counter, cyc);
        return;
    }
    if ((int)blockIdx.x >= P.n_arms) {   // uniform over the block
        // the next cycle's factors: the state the update just wrote is in the
        // buffer of parity cycle + 1 (the counter advances only once every
        // block of this launch has passed its end)
        const long long cyc = *D.cycle;
        pdl_wait();
        pdl_trigger();
        const int w = ((int)blockIdx.x - P.n_arms) * 8 + (threadIdx.x >> 5);
        if (w < n_ftiles) state_factor(D, ftiles, w, cyc + 1, threadIdx.x & 31);
        __syncthreads();
        if (threadIdx.x == 0) toplan_done(P, D, done_counter, cyc);
        return;
    }
    extern __shared__ float sq[];   // [H][d] plan joints, mean, sin(q + theta), cos(q + theta)
    __shared__ float4 s_sph[kMaxSpheres];
    __shared__ int s_frame[kMaxSpheres];
    __shared__ float4 s_dh[kMaxDof];
    __shared__ float2 s_tw[kMaxDof];
    __shared__ float s_base[12];
    __shared__ float s_in[2 * kMaxDof];
    __shared__ long long s_cycle;
    __shared__ float s_e;
    const int a = blockIdx.x, t = threadIdx.x;
    const ArmDev &A = D.arms[a];
    const long long cyc = *D.cycle;
    // wave 1: header and constants (fixed extents, no dependence on the header)
    const int d = A.dof, H = A.H, ns = A.ns, off_hd = A.off_hd, off_in = A.off_in;
    const bool local = !A.external;   // external arms keep the plan they were given
    if (t < kMaxSpheres) {
        s_sph[t] = A.sph[t];
        s_frame[t] = A.frame[t];
    }
    if (t < kMaxDof) {
        s_dh[t] = A.dh[t];
        s_tw[t] = A.twist[t];
    }
    if (t < 9) s_base[t] = A.base_R[t];
    else if (t < 12) s_base[t] = A.base_t[t - 9];
    const int Hd = H * d;
    float *smu = sq + Hd, *ssn = sq + 2 * Hd, *scs = sq + 3 * Hd;
    // wave 2: sensed state, cycle and sensed distance, then (once the update
    // has finished) the mean
    if (local && t < 2 * d) s_in[t] = D.input[off_in + t];
    if (t == 0) {
        s_cycle = *D.cycle;
        s_e = D.e_now[a];
    }
    pdl_wait();
    pdl_trigger();
    if (local) {
        const float *mu = mu_buf(D, cyc + 1) + off_hd;   // the cycle's updated mean
#pragma unroll 4
        for (int i = t; i < Hd; i += blockDim.x) smu[i] = mu[i];
    }
    __syncthreads();
    if (local) {
        // integration, one thread per joint, sequential over the horizon
        // (the mean read 8 steps ahead)
        if (t < d) {
            float q = s_in[t], qd = s_in[d + t];
            for (int hb = 0; hb < H; hb += 8) {
                float u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) u[k] = (hb + k < H) ? smu[(hb + k) * d + t] : 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (hb + k >= H) break;
                    integrate(q, qd, u[k], P.dt);
                    sq[(hb + k) * d + t] = q;
                }
            }
        }
        for (int i = t; i < Hd; i += blockDim.x) D.out[D.out_mean + off_hd + i] = smu[i];
        __syncthreads();
        for (int i = t; i < Hd; i += blockDim.x) {
            const float q = sq[i];
            float sn, cs;
            sincosf(__fadd_rn(q, s_dh[i % d].w), &sn, &cs);
            ssn[i] = sn;
            scs[i] = cs;
            D.board_q[off_hd + i] = q;
            D.out[D.out_q + off_hd + i] = q;
        }
        __syncthreads();
        // kinematics: one thread per (step, group of 8 spheres), the same
        // chain and sphere arithmetic as the rollout
        float4 *board = D.board_sph + (A.off_hs >> 2);
        float4 *outs = (float4 *)(D.out + D.out_sph) + (A.off_hs >> 2);
        const int ng = (ns + 7) / 8;
        for (int u = t; u < H * ng; u += blockDim.x) {
            const int h = u / ng, s0 = (u % ng) * 8, s1 = min(ns, s0 + 8);
            Frame F;
#pragma unroll
            for (int k = 0; k < 9; ++k) F.R[k] = s_base[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) F.t[k] = s_base[9 + k];
            int f = 0;
            for (int s = s0; s < s1; ++s) {
                const int fs = s_frame[s];
                while (f < fs) {
                    frame_step_sc(F, ssn[h * d + f], scs[h * d + f], s_dh[f], s_tw[f]);
                    ++f;
                }
                const float4 p = s_sph[s];
                const float3 c = sphere_centre(F, p);
                const float4 v = make_float4(c.x, c.y, c.z, p.w);
                board[h * ns + s] = v;
                outs[h * ns + s] = v;
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        if (local) {
            D.board_valid[a] = 1;
            D.board_stamp[a] = s_cycle;
            D.board_dist[a] = s_e;
            D.out[D.out_dist + a] = s_e;
        }
        toplan_done(P, D, done_counter, s_cycle);
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

// C_manip of Eq. 5 for every rollout step (w_manip > 0 only): FK frames of
// the sampled joints, the end-effector geometric Jacobian (joint i: axis z
// and origin o of the frame before it; column (z x (o_ee - o), z)), its
// Gram matrix (J J^T for d >= 6, J^T J below), the determinant by Cholesky
// (a non-positive pivot: singular), w = sqrt(det) and max(0, 1 - w / w0),
// added with weight w_manip to the stop + joint-limit term of the step.
__global__ void k_manip(Params P, Dev D, int total_kh)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_kh) return;
    int a = 0;
    while (a + 1 < P.n_arms && r >= D.arms[a + 1].off_kh) ++a;
    const ArmDev &A = D.arms[a];
    if (A.external) return;
    const int d = A.dof, K = A.K;
    const int loc = r - (int)A.off_kh, h = loc / K, n = loc - h * K;
    const float *qh = D.traj + A.off_khd + (long long)h * d * K + n;
    float z[kMaxDof][3], o[kMaxDof][3];
    Frame F;
    frame_base(A, F);
    for (int j = 0; j < d; ++j) {
        z[j][0] = F.R[2]; z[j][1] = F.R[5]; z[j][2] = F.R[8];
        o[j][0] = F.t[0]; o[j][1] = F.t[1]; o[j][2] = F.t[2];
        frame_step(F, qh[(long long)j * K], A.dh[j], A.twist[j]);
    }
    float J[6][kMaxDof];
    for (int j = 0; j < d; ++j) {
        const float rx = F.t[0] - o[j][0], ry = F.t[1] - o[j][1], rz = F.t[2] - o[j][2];
        J[0][j] = z[j][1] * rz - z[j][2] * ry;
        J[1][j] = z[j][2] * rx - z[j][0] * rz;
        J[2][j] = z[j][0] * ry - z[j][1] * rx;
        J[3][j] = z[j][0];
        J[4][j] = z[j][1];
        J[5][j] = z[j][2];
    }
    const int m = d >= 6 ? 6 : d;
    float G[6][6];
    for (int u = 0; u < m; ++u)
        for (int v = 0; v <= u; ++v) {
            float s = 0.f;
            if (d >= 6)
                for (int k = 0; k < d; ++k) s = fmaf(J[u][k], J[v][k], s);
            else
                for (int k = 0; k < 6; ++k) s = fmaf(J[k][u], J[k][v], s);
            G[u][v] = s;
        }
    // Cholesky in place (lower triangle); det = prod L_kk^2
    float det = 1.f;
    for (int k = 0; k < m && det > 0.f; ++k) {
        float p = G[k][k];
        for (int t = 0; t < k; ++t) p -= G[k][t] * G[k][t];
        if (!(p > 0.f)) {
            det = 0.f;
            break;
        }
        const float l = sqrtf(p);
        G[k][k] = l;
        det *= p;
        for (int i = k + 1; i < m; ++i) {
            float s = G[i][k];
            for (int t = 0; t < k; ++t) s -= G[i][t] * G[k][t];
            G[i][k] = s / l;
        }
    }
    const float w = sqrtf(det);
    const float c = fmaxf(0.f, 1.f - w / P.manip_w0);
    D.stage_lim[A.off_kh + (long long)h * K + n] += P.w_manip * c;
}

cudaError_t raise_smem_limit(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t configure_kernels(const LaunchPlan &L)
{
    cudaError_t e;
    if ((e = configure_rollout(L)) != cudaSuccess) return e;
    const void *sample = L.sample_tile == 16 ? (const void *)k_sample<16> : (const void *)k_sample<32>;
    if ((e = raise_smem_limit(sample, L.smem_sample)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void *)k_prep, L.smem_prep)) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void *)k_update, kUpdateSmem)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t enqueue_init(const Params &P, const Dev &D, int n_arms, int total_hdd, int total_hd,
                         cudaStream_t s)
{
    k_init_arms<<<n_arms, 32, 0, s>>>(D.arms);
    k_reset<<<32, 256, 0, s>>>(P, D, total_hdd, total_hd);
    return cudaGetLastError();
}

cudaError_t enqueue_state_factors(const Dev &D, const LaunchPlan &L, int parity, cudaStream_t s)
{
    if (L.n_update_tiles > 0)
        k_chol<<<(L.n_update_tiles + 7) / 8, 256, 0, s>>>(D, L.update_tiles, L.n_update_tiles, parity);
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
    // programmatic dependent launch between consecutive cycle kernels (not
    // with timing events between them)
    const bool pdl = events == nullptr;
    mark();
    if (!L.merge_prep) k_prep<<<L.n_arms, 512, L.smem_prep, s>>>(P, D);
    mark();   // with merge_prep, Sense + Shift run in the first sample launch
    for (int it = 0; it < P.iterations; ++it) {
        const int last = (it == P.iterations - 1);
        // with merge_prep the first sample launch opens the cycle (no kernel before it)
        const int with_prep = (it == 0 && L.merge_prep) ? 1 : 0;
        if ((rec = launch_k(L.sample_tile == 16 ? k_sample<16> : k_sample<32>, L.n_sample_tiles,
                            512, L.smem_sample, s, pdl && !with_prep, P, D,
                            L.sample_tiles, it, (int)(L.smem_sample / sizeof(float)), with_prep)) !=
            cudaSuccess)
            return rec;
        if (P.w_manip > 0.f)
            k_manip<<<(L.total_kh + 127) / 128, 128, 0, s>>>(P, D, L.total_kh);
        mark();
        // the rollout follows the sample kernel directly unless a manipulability
        // or surrogate stage sits between them
        const bool pdl_roll = pdl && !(P.w_manip > 0.f) && L.n_groups == 0 && L.n_pair_groups == 0;
        for (int i = 0; i < L.n_groups; ++i)   // learned self clearance of every step
            if ((rec = enqueue_self_surrogate(D, L.groups[i], s)) != cudaSuccess) return rec;
        if (L.n_pair_groups > 0 && it == 0 && D.pair_board &&
            (rec = cudaMemcpyAsync(D.pair_board, D.board_sph, L.board_bytes,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return rec;
        for (int i = 0; i < L.n_pair_groups; ++i)   // learned clearance to the neighbours' plans
            if ((rec = enqueue_pair_surrogate(D, L.pair_groups[i], s)) != cudaSuccess) return rec;
        mark();
        if ((rec = launch_rollout(P, D, L, it, s, pdl_roll)) != cudaSuccess) return rec;
        mark();
        if ((rec = launch_k(k_costs, L.n_cost_tiles, 256, 0, s, pdl, P, D, L.cost_tiles)) !=
            cudaSuccess)
            return rec;
        mark();
        if ((rec = launch_k(k_update, L.n_update_tiles, kUpdateThreads, kUpdateSmem, s, pdl, P, D,
                            L.update_tiles, last)) != cudaSuccess)
            return rec;
        mark();
    }
    // ToPlan on one block per arm, the next cycle's factors on the blocks after them, the
    // world's order for the next cycle on the last
    if ((rec = launch_k(k_toplan, L.n_arms + (L.n_update_tiles + 7) / 8 + 1, 256, L.smem_toplan, s, pdl,
                        P, D, L.done_counter, L.update_tiles, L.n_update_tiles)) != cudaSuccess)
        return rec;
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
