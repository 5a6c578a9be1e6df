// surrogate.cu -- the learned self-collision clearance inside the control
// cycle (the paper has no network: this is a library extension).
//
//  * k_self_dataset   training data: joint vectors uniform within the limits
//                     (Philox), sin/cos features and the exact clearance label;
//  * k_self_clearance exact self-collision clearance of given joint vectors,
//                     or of every rollout step of the last cycle (evaluation);
// The surrogate's own inference (features, layers, output) is one fused
// kernel of mlp_fused.cuh.
// The clearance is the minimum over the arm's sphere pairs on bodies at least
// three apart of sqrt(d2) - r1 - r2, with the rollout's kinematics and pair
// arithmetic (same functions, same operation order).
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
