// surrogate.cu -- the learned self-collision clearance inside the control
// cycle (the paper has no network: this is a library extension).
//
//  * k_self_dataset   training data: joint vectors uniform within the limits
//                     (Philox), sin/cos features and the exact clearance label;
//  * k_self_clearance exact self-collision clearance of given joint vectors,
//                     or of every rollout step of the last cycle (evaluation);
//  * k_pair_dataset   arm-pair training data: two joint vectors, a relative
//                     base pose, the exact clearance between the two arms;
//  * k_pair_clearance_traj  exact clearance of every rollout step of an arm
//                     to a neighbour's published plan (evaluation).
// The surrogates' own inference (features, layers, output) is one fused
// kernel of mlp_fused.cuh.
// The clearance is the minimum over the arm's self-collision pairs (bodies at
// least three apart, clear of the B_self band at the rest pose) of
// sqrt(d2) - r1 - r2, with the rollout's kinematics and pair arithmetic (same
// functions, same operation order).
#include "kernels.cuh"

namespace mrs {

__device__ float self_clearance(const Dev &D, const ArmDev &A, const float *q, int q_stride)
{
    float3 c[kMaxSpheres];
    Frame F;
    frame_base(A, F);
    int f = 0;
    for (int s = 0; s < A.ns; ++s) {
        const int fs = A.frame[s];
        while (f < fs) {
            frame_step(F, q[f * q_stride], A.dh[f], A.twist[f]);
            ++f;
        }
        c[s] = sphere_centre(F, A.sph[s]);
    }
    float m = kInf;
    const int *pairs = D.self_pairs + A.self_off;
    for (int i = 0; i < A.n_self; ++i) {
        const int a1 = pairs[i] & 0xff, a2 = pairs[i] >> 8;
        const float dx = __fsub_rn(c[a2].x, c[a1].x), dy = __fsub_rn(c[a2].y, c[a1].y),
                    dz = __fsub_rn(c[a2].z, c[a1].z);
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), A.sph[a1].w), A.sph[a2].w));
    }
    return m;
}

__global__ void k_self_dataset(Dev D, int arm, int n, unsigned long long seed, float *x, float *t,
                               float *q_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ArmDev &A = D.arms[arm];
    const int d = A.dof;
    float q[kMaxDof];
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int b = 0; 4 * b < d; ++b) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)b, 0x5e1fda7au, (uint32_t)arm), key);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
        for (int k = 0; k < 4 && 4 * b + k < d; ++k) {
            const int j = 4 * b + k;
            q[j] = __fmaf_rn(A.q_hi[j] - A.q_lo[j], uniform23(w[k]), A.q_lo[j]);
        }
    }
    for (int j = 0; j < d; ++j) {
        float s, co;
        sincosf(q[j], &s, &co);
        x[(size_t)i * 2 * d + 2 * j] = s;
        x[(size_t)i * 2 * d + 2 * j + 1] = co;
        if (q_out) q_out[(size_t)i * d + j] = q[j];
    }
    t[i] = self_clearance(D, A, q, 1);
}

// q rows [n][dof]
__global__ void k_self_clearance_rows(Dev D, int arm, int n, const float *q, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ArmDev &A = D.arms[arm];
    out[i] = self_clearance(D, A, q + (size_t)i * A.dof, 1);
}

// every rollout step of the last cycle, out [H][K]
__global__ void k_self_clearance_traj(Dev D, int arm, float *out)
{
    const ArmDev &A = D.arms[arm];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= A.H * A.K) return;
    const int h = r / A.K, n = r % A.K;
    out[r] = self_clearance(D, A, D.traj + A.off_khd + (size_t)h * A.dof * A.K + n, A.K);
}

// Sphere centres of an arm at joints q (stride q_stride) with the base frame F
// given; c must hold A.ns entries.
__device__ void arm_spheres(const ArmDev &A, Frame F, const float *q, int q_stride, float3 *c)
{
    int f = 0;
    for (int s = 0; s < A.ns; ++s) {
        const int fs = A.frame[s];
        while (f < fs) {
            frame_step(F, q[f * q_stride], A.dh[f], A.twist[f]);
            ++f;
        }
        c[s] = sphere_centre(F, A.sph[s]);
    }
}

// minimum over all sphere pairs of centre distance minus radii (the pair
// arithmetic of the rollout's exact pass)
__device__ float pair_min(const ArmDev &Aa, const float3 *ca, const ArmDev &Ab, const float3 *cb)
{
    float m = kInf;
    for (int i = 0; i < Aa.ns; ++i)
        for (int k = 0; k < Ab.ns; ++k) {
            const float dx = __fsub_rn(cb[k].x, ca[i].x), dy = __fsub_rn(cb[k].y, ca[i].y),
                        dz = __fsub_rn(cb[k].z, ca[i].z);
            const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), Aa.sph[i].w), Ab.sph[k].w));
        }
    return m;
}

__global__ void k_pair_dataset(Dev D, int a, int b, int n, unsigned long long seed,
                               const float *poses, int n_pose, float jit_t, float jit_yaw,
                               float *x, float *t, float *qa_out, float *qb_out, float *pose_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ArmDev &Aa = D.arms[a], &Ab = D.arms[b];
    const int da = Aa.dof, db = Ab.dof;
    // uniforms: d_a + d_b joints, the pose index, 3 translation and 1 yaw jitters
    float u[2 * kMaxDof + 5];
    const int nu = da + db + 5;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int blk = 0; 4 * blk < nu; ++blk) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)blk, 0x9a1e5u,
                                                 (uint32_t)(a | (b << 8))), key);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
        for (int k = 0; k < 4 && 4 * blk + k < nu; ++k) u[4 * blk + k] = uniform23(w[k]);
    }
    float qa[kMaxDof], qb[kMaxDof];
    for (int j = 0; j < da; ++j) qa[j] = __fmaf_rn(Aa.q_hi[j] - Aa.q_lo[j], u[j], Aa.q_lo[j]);
    for (int j = 0; j < db; ++j) qb[j] = __fmaf_rn(Ab.q_hi[j] - Ab.q_lo[j], u[da + j], Ab.q_lo[j]);
    const int pi = min(n_pose - 1, (int)(u[da + db] * (float)n_pose));
    const float *p0 = poses + 7 * pi;
    float pose[7];
    for (int k = 0; k < 3; ++k) pose[k] = p0[k] + jit_t * (2.f * u[da + db + 1 + k] - 1.f);
    {
        // compose the base rotation with a yaw about its own z
        float sy, cy;
        sincosf(0.5f * jit_yaw * (2.f * u[da + db + 4] - 1.f), &sy, &cy);
        const float w = p0[3], xq = p0[4], yq = p0[5], zq = p0[6];
        pose[3] = w * cy - zq * sy;
        pose[4] = xq * cy + yq * sy;
        pose[5] = yq * cy - xq * sy;
        pose[6] = zq * cy + w * sy;
    }
    // features
    float *xr = x + (size_t)i * (2 * da + 2 * db + 7);
    for (int j = 0; j < da; ++j) sincosf(qa[j], &xr[2 * j], &xr[2 * j + 1]);
    for (int j = 0; j < db; ++j) sincosf(qb[j], &xr[2 * da + 2 * j], &xr[2 * da + 2 * j + 1]);
    for (int k = 0; k < 7; ++k) xr[2 * da + 2 * db + k] = pose[k];
    if (qa_out) for (int j = 0; j < da; ++j) qa_out[(size_t)i * da + j] = qa[j];
    if (qb_out) for (int j = 0; j < db; ++j) qb_out[(size_t)i * db + j] = qb[j];
    if (pose_out) for (int k = 0; k < 7; ++k) pose_out[(size_t)i * 7 + k] = pose[k];
    // label: arm a at the identity, arm b at the pose
    Frame Fa, Fb;
    for (int k = 0; k < 9; ++k) Fa.R[k] = (k % 4 == 0) ? 1.f : 0.f;
    Fa.t[0] = Fa.t[1] = Fa.t[2] = 0.f;
    quat_to_R(pose[3], pose[4], pose[5], pose[6], Fb.R);
    Fb.t[0] = pose[0]; Fb.t[1] = pose[1]; Fb.t[2] = pose[2];
    float3 ca[kMaxSpheres], cb[kMaxSpheres];
    arm_spheres(Aa, Fa, qa, 1, ca);
    arm_spheres(Ab, Fb, qb, 1, cb);
    t[i] = pair_min(Aa, ca, Ab, cb);
}

// every rollout step of arm a (world frame) against arm b's published plan
// spheres at step min(h, H_b - 1) as the last cycle read them; out [H][K]
__global__ void k_pair_clearance_traj(Dev D, int a, int b, float *out)
{
    const ArmDev &Aa = D.arms[a], &Ab = D.arms[b];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Aa.H * Aa.K) return;
    const int h = r / Aa.K, n = r % Aa.K;
    Frame F;
    frame_base(Aa, F);
    float3 ca[kMaxSpheres], cb[kMaxSpheres];
    arm_spheres(Aa, F, D.traj + Aa.off_khd + (size_t)h * Aa.dof * Aa.K + n, Aa.K, ca);
    const float4 *board = D.pair_board ? D.pair_board : D.board_sph;
    const float4 *pl = board + (Ab.off_hs >> 2) + (size_t)min(h, Ab.H - 1) * Ab.ns;
    for (int k = 0; k < Ab.ns; ++k) {
        const float4 p = pl[k];
        cb[k] = make_float3(p.x, p.y, p.z);
    }
    out[r] = pair_min(Aa, ca, Ab, cb);
}

cudaError_t enqueue_pair_dataset(const Dev &D, int a, int b, int n, unsigned long long seed,
                                 const float *poses, int n_pose, float jit_t, float jit_yaw,
                                 float *x, float *t, float *qa, float *qb, float *pose_out,
                                 cudaStream_t s)
{
    k_pair_dataset<<<(n + 127) / 128, 128, 0, s>>>(D, a, b, n, seed, poses, n_pose, jit_t, jit_yaw,
                                                   x, t, qa, qb, pose_out);
    return cudaGetLastError();
}

cudaError_t enqueue_pair_clearance_traj(const Dev &D, int a, int b, int rows, float *out,
                                        cudaStream_t s)
{
    k_pair_clearance_traj<<<(rows + 127) / 128, 128, 0, s>>>(D, a, b, out);
    return cudaGetLastError();
}

cudaError_t enqueue_pair_surrogate(const Dev &D, const PairGroup &g, cudaStream_t s)
{
    return mlp_infer_pairs(g.net, D.traj, D.board_q, g.segs, D.rhohat, D.err, s);
}

cudaError_t enqueue_self_dataset(const Dev &D, int arm, int n, unsigned long long seed, float *x,
                                 float *t, float *q, cudaStream_t s)
{
    k_self_dataset<<<(n + 127) / 128, 128, 0, s>>>(D, arm, n, seed, x, t, q);
    return cudaGetLastError();
}

cudaError_t enqueue_self_clearance_rows(const Dev &D, int arm, int n, const float *q, float *out,
                                        cudaStream_t s)
{
    k_self_clearance_rows<<<(n + 127) / 128, 128, 0, s>>>(D, arm, n, q, out);
    return cudaGetLastError();
}

cudaError_t enqueue_self_clearance_traj(const Dev &D, int arm, int rows, float *out, cudaStream_t s)
{
    k_self_clearance_traj<<<(rows + 127) / 128, 128, 0, s>>>(D, arm, out);
    return cudaGetLastError();
}

// Surrogate inference inside the cycle for the arms sharing one network:
// features, hidden layers and output of every rollout step in one fused
// launch, into each arm's slice of dhat ([H][K] order).
cudaError_t enqueue_self_surrogate(const Dev &D, const SurrogateGroup &g, cudaStream_t s)
{
    return mlp_infer_trajs(g.net, D.traj, g.segs, D.dhat, D.err, s);
}

}  // namespace mrs
