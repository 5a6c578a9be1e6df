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

size_t fk_static_capacity_floats() { return kFkStaticFloats; }

// Host side of mrs_fk_static, on `device` (the context's device, current
// during the call).  The kinematics are mrs_fk's own kernel (enqueue_fk) run
// on slices of the static scratch.  Returns cudaSuccess, or an error with
// `why` set; a request larger than the scratch is rejected before any CUDA
// call.
cudaError_t fk_static(const Dev &D, int device, int arm, int dof, int ns, int n,
                      const float *q_host, float *ee_host, float *spheres_host, cudaStream_t s,
                      std::string &why, bool &too_large)
{
    too_large = false;
    const size_t nq = pad4((size_t)n * dof), ne = (size_t)n * 12, nsph = (size_t)n * ns * 4;
    if (nq + ne + nsph > kFkStaticFloats) {
        too_large = true;
        why = "request needs " + std::to_string(nq + ne + nsph) + " floats of static scratch; the "
              "limit is " + std::to_string(kFkStaticFloats);
        return cudaErrorInvalidValue;
    }
    const int dev = device;
    cudaError_t e = cudaSuccess;
    if (dev < 0 || dev >= kMaxDevices) return why = "device ordinal out of range", cudaErrorInvalidDevice;
    float *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device (made current by the caller): look
            // up the device address of the static array
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
    if ((e = enqueue_fk(D, arm, n, dq, dee, (float *)dsph, s)) != cudaSuccess)
        return why = "launch", e;
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
