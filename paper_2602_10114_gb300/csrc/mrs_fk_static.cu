// mrs_fk_static.cu -- forward kinematics that allocates no device memory.
//
// mrs_fk stages the joint vectors and its results in device buffers that it
// allocates and frees on every call.  Some callers cannot do that: a control
// loop with a hard period must not call cudaMalloc/cudaFree (they can block
// and synchronise the whole device), and a process whose device memory is
// owned by another allocator may forbid them outright.  This file gives those
// callers the same computation with its staging in one fixed, file-scope
// device array that every GPU loading the library holds until exit.
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace mrs {

// Static scratch: the joint vectors, end-effector poses and sphere centres of
// one call, each part starting on a 16-byte boundary.  2^20 floats = 4 MiB.
constexpr size_t kFkStaticFloats = size_t(1) << 20;
static __device__ __align__(256) float g_fk_scratch[kFkStaticFloats];

// Device address of g_fk_scratch per device ordinal, looked up once per device
// (host code cannot use the array's name as a device address).
constexpr int kMaxDevices = 64;
static float *g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static size_t pad4(size_t n) { return (n + 3) / 4 * 4; }

// Same arithmetic, in the same order, as the rollout's kinematics.
__global__ void k_fk_static(Dev D, int arm, int n, const float *q, float *ee, float4 *spheres)
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
        const float4 p = A.sph[s];
        const float3 c = sphere_centre(F, p);
        spheres[(size_t)i * A.ns + s] = make_float4(c.x, c.y, c.z, p.w);
    }
    while (f < d) {
        frame_step(F, q[(size_t)i * d + f], A.dh[f], A.twist[f]);
        ++f;
    }
    for (int k = 0; k < 9; ++k) ee[(size_t)i * 12 + k] = F.R[k];
    for (int k = 0; k < 3; ++k) ee[(size_t)i * 12 + 9 + k] = F.t[k];
}

size_t fk_static_capacity_floats() { return kFkStaticFloats; }

// Host side of mrs_fk_static.  Returns cudaSuccess, or an error with `why`
// set; a request larger than the scratch is rejected before any CUDA call.
cudaError_t fk_static(const Dev &D, int arm, int dof, int ns, int n, const float *q_host,
                      float *ee_host, float *spheres_host, cudaStream_t s, std::string &why,
                      bool &too_large)
{
    too_large = false;
    const size_t nq = pad4((size_t)n * dof), ne = (size_t)n * 12, nsph = (size_t)n * ns * 4;
    if (nq + ne + nsph > kFkStaticFloats) {
        too_large = true;
        why = "request needs " + std::to_string(nq + ne + nsph) + " floats of static scratch; the "
              "limit is " + std::to_string(kFkStaticFloats);
        return cudaErrorInvalidValue;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return why = "cudaGetDevice", e;
    if (dev < 0 || dev >= kMaxDevices) return why = "device ordinal out of range", cudaErrorInvalidDevice;
    float *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device (the device is current): look up the
            // device address of the static array
            float *p = nullptr;
            e = cudaGetSymbolAddress((void **)&p, g_fk_scratch);
            if (e != cudaSuccess) return why = "cudaGetSymbolAddress", e;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    float *dq = base, *dee = base + nq;
    float4 *dsph = (float4 *)(dee + ne);
    // every element copied back below is written by the kernel, so nothing in
    // the scratch needs to start at zero
    if ((e = cudaMemcpyAsync(dq, q_host, sizeof(float) * n * dof, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return why = "upload", e;
    k_fk_static<<<(n + 127) / 128, 128, 0, s>>>(D, arm, n, dq, dee, dsph);
    if ((e = cudaGetLastError()) != cudaSuccess) return why = "launch", e;
    if ((e = cudaMemcpyAsync(ee_host, dee, sizeof(float) * ne, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return why = "download", e;
    if (spheres_host &&
        (e = cudaMemcpyAsync(spheres_host, dsph, sizeof(float) * nsph, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
        return why = "download", e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return why = "sync", e;
    return cudaSuccess;
}

}  // namespace mrs
