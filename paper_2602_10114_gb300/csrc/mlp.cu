// mlp.cu -- learned clearance surrogate: a small MLP (sin/cos joint features
// in, signed clearance out, SiLU hidden layers) with BF16 weights and
// activations and FP32 accumulation on the tcgen05 tensor cores, trained by
// this file's forward / backward / Adam kernels.  The paper has no network;
// the surrogate stands in for the exact self-collision distance (Eq. 5,
// C_self) with an exact fallback near contact.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "mrs.h"
#include "mlp_fused.cuh"
#include "tc_gemm.cuh"

namespace mrs {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// epilogues of the tensor-core GEMM

struct EpiStoreF32 {
    float *C;
    int ldc;
    __device__ void operator()(int r, int c0, const float (&v)[16]) const
    {
#pragma unroll
        for (int i = 0; i < 16; ++i) C[(size_t)r * ldc + c0 + i] = v[i];
    }
};

struct EpiAtomicF32 {   // split-K accumulation
    float *C;
    int ldc, ncols;
    __device__ void operator()(int r, int c0, const float (&v)[16]) const
    {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (c0 + i < ncols) atomicAdd(&C[(size_t)r * ldc + c0 + i], v[i]);
    }
};

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// z = acc + bias; H = bf16(silu(z)); optionally keep z for the backward pass
struct EpiBiasSilu {
    const float *bias;
    float *Z;     // may be null (inference)
    bf16 *H;
    int ld;
    __device__ void operator()(int r, int c0, const float (&v)[16]) const
    {
        __align__(16) bf16 h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float z = v[i] + bias[c0 + i];
            if (Z) Z[(size_t)r * ld + c0 + i] = z;
            h[i] = __float2bfloat16_rn(z * sigmoidf_(z));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(H + (size_t)r * ld + c0);
        dst[0] = *reinterpret_cast<const uint4 *>(&h[0]);
        dst[1] = *reinterpret_cast<const uint4 *>(&h[8]);
    }
};

template <int BK, class Epi>
__global__ void __launch_bounds__(tc::kThreads) k_gemm(const bf16 *A, int lda, const bf16 *B,
                                                       int ldb, int M, int N, int K, int *err,
                                                       Epi epi)
{
    __shared__ tc::GemmSmem<BK> S;
    const int m0 = blockIdx.x * 128;
    const int slice = ((K + gridDim.y - 1) / gridDim.y + BK - 1) / BK * BK;
    const int kb = blockIdx.y * slice, ke = min(K, kb + slice);
    if (kb >= ke) return;
    tc::gemm_tile<BK>(A, lda, B, ldb, M, N, kb, ke, m0, S, err, epi);
}

template <class Epi>
static cudaError_t gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
                        int ksplit, int *err, Epi epi, cudaStream_t s)
{
    dim3 grid((M + 127) / 128, ksplit);
    if (K <= 16)
        k_gemm<16, Epi><<<grid, tc::kThreads, 0, s>>>(A, lda, B, ldb, M, N, K, err, epi);
    else
        k_gemm<32, Epi><<<grid, tc::kThreads, 0, s>>>(A, lda, B, ldb, M, N, K, err, epi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// elementwise and reduction kernels

__global__ void k_to_bf16_pad(const float *x, int n, int in_dim, int in_pad, bf16 *X)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * in_pad) return;
    const int r = (int)(i / in_pad), c = (int)(i % in_pad);
    X[i] = __float2bfloat16_rn(c < in_dim ? x[(size_t)r * in_dim + c] : 0.f);
}

// y[r] = H[r] . w + b (one warp per row)
__global__ void k_out_layer(const bf16 *H, int width, const float *w, const float *b, int n,
                            float *y)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    float s = 0.f;
    for (int c = lane; c < width; c += 32)
        s = fmaf(__bfloat162float(H[(size_t)r * width + c]), w[c], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] = s + b[0];
}

// squared error on clipped targets, an over-prediction (y above the target)
// weighted by over_w: dy = 2 w (y - t) / n, loss += w (y - t)^2 / n
__global__ void k_loss(const float *y, const float *t, int n, float lo, float hi, float over_w,
                       float *dy, float *loss)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f, w = 1.f;
    if (r < n) {
        const float tc = fminf(fmaxf(t[r], lo), hi);
        e = y[r] - tc;
        w = e > 0.f ? over_w : 1.f;
        dy[r] = 2.f * w * e / (float)n;
    }
    float s = w * e * e / (float)n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// output layer backward: dH[r][c] = dy[r] w[c]; dw[c] += sum_r dy[r] H[r][c];
// db += sum_r dy[r]   (block per 32 rows, thread per column)
__global__ void k_out_back(const bf16 *H, int width, const float *w, const float *dy, int n,
                           float *dH, float *dw, float *db)
{
    const int c = threadIdx.x;   // blockDim.x == width
    const int r0 = blockIdx.x * 32;
    float acc = 0.f, accb = 0.f;
    for (int r = r0; r < min(n, r0 + 32); ++r) {
        const float g = dy[r];
        dH[(size_t)r * width + c] = g * w[c];
        acc = fmaf(g, __bfloat162float(H[(size_t)r * width + c]), acc);
        accb += g;
    }
    atomicAdd(&dw[c], acc);
    if (c == 0) atomicAdd(db, accb);
}

// through SiLU: dZ = dH * silu'(Z) -> bf16, and column sums into db
__global__ void k_silu_back(const float *dH, const float *Z, int n, int width, bf16 *dZ, float *db)
{
    const int c = threadIdx.x;   // blockDim.x == width
    const int r0 = blockIdx.x * 32;
    float acc = 0.f;
    for (int r = r0; r < min(n, r0 + 32); ++r) {
        const size_t i = (size_t)r * width + c;
        const float z = Z[i], sg = sigmoidf_(z);
        const float g = dH[i] * sg * (1.f + z * (1.f - sg));
        const bf16 gb = __float2bfloat16_rn(g);
        dZ[i] = gb;
        acc += __bfloat162float(gb);
    }
    atomicAdd(&db[c], acc);
}

// out[c][r] = in[r][c] for a [rows][cols] BF16 matrix (32 x 32 tiles)
__global__ void k_transpose_bf16(const bf16 *in, int rows, int cols, bf16 *out)
{
    __shared__ bf16 t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + j, c = bx + threadIdx.x;
        t[j][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = bx + j, r = by + threadIdx.x;
        if (c < cols && r < rows) out[(size_t)c * rows + r] = t[threadIdx.x][j];
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters
__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of a weight matrix W [rows][cols] and of its transpose
__global__ void k_weights_bf16(const float *W, int rows, int cols, bf16 *Wb, bf16 *WbT)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const bf16 b = __float2bfloat16_rn(W[i]);
    Wb[i] = b;
    WbT[(size_t)c * rows + r] = b;
}

// W [rows][cols] (cols a multiple of 16) into 16-column chunks in the
// canonical K-major layout of a tcgen05 B operand: within a chunk, element
// (n, k) at byte (n / 8) * 256 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2.
__global__ void k_pack_chunks(const float *W, int rows, int cols, unsigned char *dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int n = i / cols, k = i % cols, c = k >> 4, kk = k & 15;
    const size_t off = (size_t)c * rows * 32 + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 +
                       (kk & 7) * 2;
    *reinterpret_cast<bf16 *>(dst + off) = __float2bfloat16_rn(W[i]);
}

// uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from Philox, zero biases
__global__ void k_init_param(float *p, size_t n, float scale, unsigned long long seed,
                             unsigned tensor)
{
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)i, tensor, 0x6d6c70u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    p[i] = scale * (2.f * uniform23(x.x) - 1.f);
}

}  // namespace mrs

using namespace mrs;

struct mrs_mlp {
    int in_dim = 0, in_pad = 0, width = 0, layers = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // parameters (FP32 master), Adam moments, gradients: one flat vector each
    std::vector<size_t> offW, offB;   // per hidden layer
    size_t offWo = 0, offBo = 0, n_params = 0;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    long long step = 0;
    float over_weight = 1.f;   // loss weight of over-predictions
    std::vector<bf16 *> Wb, WbT;
    // training buffers (capacity `cap` rows)
    int cap = 0;
    bf16 *X = nullptr;
    std::vector<float *> Z;
    std::vector<bf16 *> Hs;
    float *y = nullptr, *dy = nullptr, *dH = nullptr, *loss = nullptr;
    bf16 *dZ = nullptr, *dZT = nullptr, *HT = nullptr;
    // fused inference: packed BF16 weight chunks and the kernel's set-up
    unsigned char *wpack = nullptr;
    fused::Net fnet{};
    int per_sm_rows = 0, per_sm_traj = 0, per_sm_pair = 0, num_sms = 0;
    size_t fnet_smem = 0;
    int *err = nullptr;
    std::string msg;
};

static size_t pad16(size_t x) { return (x + 15) / 16 * 16; }

// K chunks of 16 per weight-ring slot of the fused inference kernel: the
// chunks of a slot share one barrier wait and one commit of the thread that
// issues the MMAs
static constexpr int kFusedGroup = 2;

static mrs_status mlp_fail(mrs_mlp *m, mrs_status s, const std::string &why)
{
    if (m) m->msg = why;
    return s;
}

#define MCK(call, what)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return mlp_fail(m, MRS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int in_of(const mrs_mlp *m, int l) { return l == 0 ? m->in_pad : m->width; }

// index of the first 16-column weight chunk of layer l
static int chunk_index(const mrs_mlp *m, int l)
{
    int c = 0;
    for (int i = 0; i < l; ++i) c += in_of(m, i) / 16;
    return c;
}

// Shared memory, ring depth and occupancy of the fused inference kernel.
// Two CTAs per SM when the width allows (about 110 KB each); the ring takes
// what the layer input leaves.  More CTAs per SM than the tensor memory
// holds (512 columns) would wait in tcgen05.alloc, so the shared memory is
// padded until they cannot be resident.
template <class In>
static cudaError_t configure_fused(mrs_mlp *m, int *per_sm)
{
    fused::Net &n = m->fnet;
    const size_t smem = fused::smem_bytes(n);
    const int max_ctas = 512 / (int)n.tmem_cols;
    size_t need = smem;
    const size_t sm_bytes = 228 * 1024, reserve = 1024;
    if ((size_t)(max_ctas + 1) * (smem + reserve) <= sm_bytes)
        need = sm_bytes / (size_t)(max_ctas + 1) - reserve + 16;
    need = (need + 15) / 16 * 16;
    cudaError_t e = raise_smem_limit((const void *)fused::k_mlp_fused<In>, need);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fused::k_mlp_fused<In>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the kernel's own limits (shared memory with
    // the 1 KB the driver reserves per CTA, registers allocated per warp in
    // units of 256, threads, tensor-memory columns); the occupancy query
    // answered 1 where two fit
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fused::k_mlp_fused<In>);
    if (e != cudaSuccess) return e;
    const int warps = fused::kThreads / 32;
    const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int fit = (int)(sm_bytes / (need + reserve));
    fit = std::min(fit, 65536 / (regs_per_warp * warps));
    fit = std::min(fit, 2048 / fused::kThreads);
    fit = std::min(fit, max_ctas);
    *per_sm = fit;
    if (*per_sm < 1) return cudaErrorInvalidConfiguration;
    m->fnet_smem = need;
    return cudaSuccess;
}

template <class In>
static cudaError_t launch_fused(mrs_mlp *m, const In &in, int rows, float *y, int *err, int per_sm,
                                cudaStream_t s)
{
    const int tiles = (rows + 127) / 128;
    const int grid = std::min(tiles, per_sm * m->num_sms);
    fused::k_mlp_fused<In><<<grid, fused::kThreads, m->fnet_smem, s>>>(m->fnet, in, rows, y, err);
    return cudaGetLastError();
}

static mrs_status mlp_refresh_bf16(mrs_mlp *m)
{
    for (int l = 0; l < m->layers; ++l) {
        const int rows = m->width, cols = in_of(m, l);
        k_weights_bf16<<<(rows * cols + 255) / 256, 256, 0, m->stream>>>(
            m->params + m->offW[l], rows, cols, m->Wb[l], m->WbT[l]);
        k_pack_chunks<<<(rows * cols + 255) / 256, 256, 0, m->stream>>>(
            m->params + m->offW[l], rows, cols,
            m->wpack + (size_t)m->fnet.chunk_bytes * chunk_index(m, l));
    }
    MCK(cudaGetLastError(), "bf16 weights");
    return MRS_OK;
}

static mrs_status mlp_reserve(mrs_mlp *m, int n)
{
    if (n <= m->cap) return MRS_OK;
    const int c = (n + 127) / 128 * 128;
    cudaFree(m->X);
    for (auto p : m->Z) cudaFree(p);
    for (auto p : m->Hs) cudaFree(p);
    cudaFree(m->y); cudaFree(m->dy); cudaFree(m->dH); cudaFree(m->dZ); cudaFree(m->dZT); cudaFree(m->HT);
    const size_t W = m->width;
    MCK(cudaMalloc(&m->X, sizeof(bf16) * c * m->in_pad), "alloc");
    for (int l = 0; l < m->layers; ++l) {
        MCK(cudaMalloc(&m->Z[l], sizeof(float) * c * W), "alloc");
        MCK(cudaMalloc(&m->Hs[l], sizeof(bf16) * c * W), "alloc");
    }
    MCK(cudaMalloc(&m->y, sizeof(float) * c), "alloc");
    MCK(cudaMalloc(&m->dy, sizeof(float) * c), "alloc");
    MCK(cudaMalloc(&m->dH, sizeof(float) * c * W), "alloc");
    MCK(cudaMalloc(&m->dZ, sizeof(bf16) * c * W), "alloc");
    MCK(cudaMalloc(&m->dZT, sizeof(bf16) * c * W), "alloc");
    MCK(cudaMalloc(&m->HT, sizeof(bf16) * c * std::max<size_t>(W, m->in_pad)), "alloc");
    m->cap = c;
    return MRS_OK;
}

// forward over n rows already in m->X; keeps Z and H for the backward pass
static mrs_status mlp_forward_train(mrs_mlp *m, int n)
{
    const bf16 *in = m->X;
    for (int l = 0; l < m->layers; ++l) {
        EpiBiasSilu e{m->params + m->offB[l], m->Z[l], m->Hs[l], m->width};
        MCK(gemm(in, in_of(m, l), m->Wb[l], in_of(m, l), n, m->width, in_of(m, l), 1, m->err, e,
                 m->stream), "forward gemm");
        in = m->Hs[l];
    }
    k_out_layer<<<(n + 7) / 8, 256, 0, m->stream>>>(in, m->width, m->params + m->offWo,
                                                    m->params + m->offBo, n, m->y);
    MCK(cudaGetLastError(), "output layer");
    return MRS_OK;
}

// gradients of the clipped-target MSE into m->grads (zeroed here)
static mrs_status mlp_backward(mrs_mlp *m, const float *t, int n)
{
    const int W = m->width;
    MCK(cudaMemsetAsync(m->grads, 0, sizeof(float) * m->n_params, m->stream), "memset");
    MCK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream), "memset");
    k_loss<<<(n + 255) / 256, 256, 0, m->stream>>>(m->y, t, n, -0.1f, 0.3f, m->over_weight, m->dy,
                                                   m->loss);
    k_out_back<<<(n + 31) / 32, W, 0, m->stream>>>(m->Hs[m->layers - 1], W, m->params + m->offWo,
                                                   m->dy, n, m->dH, m->grads + m->offWo,
                                                   m->grads + m->offBo);
    MCK(cudaGetLastError(), "loss / output backward");
    const int ksplit = std::max(1, std::min(32, n / 256));
    for (int l = m->layers - 1; l >= 0; --l) {
        const int in = in_of(m, l);
        k_silu_back<<<(n + 31) / 32, W, 0, m->stream>>>(m->dH, m->Z[l], n, W, m->dZ,
                                                        m->grads + m->offB[l]);
        const bf16 *Hprev = (l == 0) ? m->X : m->Hs[l - 1];
        dim3 tb(32, 8);
        k_transpose_bf16<<<dim3((W + 31) / 32, (n + 31) / 32), tb, 0, m->stream>>>(m->dZ, n, W, m->dZT);
        k_transpose_bf16<<<dim3((in + 31) / 32, (n + 31) / 32), tb, 0, m->stream>>>(Hprev, n, in, m->HT);
        MCK(cudaGetLastError(), "backward elementwise");
        // dW_l [W][in] = dZ^T [W][n] * (H_{l-1}^T [in][n])^T  (split over the batch)
        EpiAtomicF32 e{m->grads + m->offW[l], in, in};
        MCK(gemm(m->dZT, n, m->HT, n, W, (int)pad16(in), n, ksplit, m->err, e, m->stream),
            "weight-gradient gemm");
        if (l > 0) {
            // dH_{l-1} [n][in] = dZ [n][W] * W_l [W][in]  (B operand = W_l^T [in][W])
            EpiStoreF32 e2{m->dH, in};
            MCK(gemm(m->dZ, W, m->WbT[l], W, n, in, W, 1, m->err, e2, m->stream), "input-gradient gemm");
        }
    }
    return MRS_OK;
}

static mrs_status load_x(mrs_mlp *m, const float *d_x, int n)
{
    const long long tot = (long long)n * m->in_pad;
    k_to_bf16_pad<<<(unsigned)((tot + 255) / 256), 256, 0, m->stream>>>(d_x, n, m->in_dim, m->in_pad, m->X);
    MCK(cudaGetLastError(), "features");
    return MRS_OK;
}

static mrs_status check_err(mrs_mlp *m)
{
    int e = 0;
    MCK(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "error word");
    MCK(cudaStreamSynchronize(m->stream), "sync");
    if (e) return mlp_fail(m, MRS_ETIMEOUT, "a tensor-core wait gave up");
    return MRS_OK;
}

namespace mrs {

int mlp_in_dim(const mrs_mlp *m) { return m->in_dim; }

// surrogate inference over every rollout step of a set of arms (segments of
// the trajectory array) into their slices of dhat, in one fused launch
cudaError_t mlp_infer_trajs(mrs_mlp *m, const float *traj, const fused::TrajSegs &segs,
                            float *dhat, int *err, cudaStream_t s)
{
    return launch_fused(m, fused::InTrajSet{traj, segs}, segs.row_start[segs.n], dhat, err,
                        m->per_sm_traj, s);
}

// arm-pair surrogate over every rollout step of a set of (a, b) segments
cudaError_t mlp_infer_pairs(mrs_mlp *m, const float *traj, const float *plan,
                            const fused::PairSegs &segs, float *rhohat, int *err, cudaStream_t s)
{
    return launch_fused(m, fused::InPairSet{traj, plan, segs}, segs.row_start[segs.n], rhohat,
                        err, m->per_sm_pair, s);
}

}  // namespace mrs

extern "C" {

mrs_status mrs_mlp_create(int in_dim, int width, int layers, unsigned long long seed, void *stream,
                          mrs_mlp **out)
{
    if (!out || in_dim < 1 || in_dim > 256 || width < 16 || width > 256 || width % 16 ||
        layers < 1 || layers > 8)
        return MRS_EINVAL;
    mrs_mlp *m = new (std::nothrow) mrs_mlp();
    if (!m) return MRS_ENOMEM;
    m->in_dim = in_dim;
    m->in_pad = (int)pad16(in_dim);
    m->width = width;
    m->layers = layers;
    size_t o = 0;
    for (int l = 0; l < layers; ++l) {
        m->offW.push_back(o);
        o += (size_t)width * in_of(m, l);
        m->offB.push_back(o);
        o += width;
    }
    m->offWo = o;
    o += width;
    m->offBo = o;
    o += 1;
    m->n_params = o;
    m->Z.assign(layers, nullptr);
    m->Hs.assign(layers, nullptr);
    m->Wb.assign(layers, nullptr);
    m->WbT.assign(layers, nullptr);
    if (stream) {
        m->stream = (cudaStream_t)stream;
    } else if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete m;
        return MRS_ECUDA;
    } else {
        m->own_stream = true;
    }
    bool okk = cudaMalloc(&m->params, sizeof(float) * o) == cudaSuccess &&
               cudaMalloc(&m->grads, sizeof(float) * o) == cudaSuccess &&
               cudaMalloc(&m->am, sizeof(float) * o) == cudaSuccess &&
               cudaMalloc(&m->av, sizeof(float) * o) == cudaSuccess &&
               cudaMalloc(&m->loss, sizeof(float)) == cudaSuccess &&
               cudaMalloc(&m->err, sizeof(int)) == cudaSuccess;
    for (int l = 0; okk && l < layers; ++l)
        okk = cudaMalloc(&m->Wb[l], sizeof(bf16) * width * in_of(m, l)) == cudaSuccess &&
              cudaMalloc(&m->WbT[l], sizeof(bf16) * width * in_of(m, l)) == cudaSuccess;
    const int n_chunks = chunk_index(m, layers);
    if (okk) okk = cudaMalloc(&m->wpack, (size_t)n_chunks * width * 32) == cudaSuccess;
    if (!okk) {
        mrs_mlp_destroy(m);
        return MRS_ENOMEM;
    }
    // fused inference set-up
    {
        fused::Net &n = m->fnet;
        n.wpack = m->wpack;
        n.params = m->params;
        n.offB0 = (int)m->offB[0];
        for (int l = 1; l < layers; ++l)
            if (m->offB[l] != m->offB[0] + (size_t)l * (width * width + width)) {
                mrs_mlp_destroy(m);
                return MRS_EINVAL;
            }
        n.offWo = (int)m->offWo;
        n.offBo = (int)m->offBo;
        n.in_pad = m->in_pad;
        n.width = width;
        n.layers = layers;
        n.chunk_bytes = (unsigned)width * 32u;
        n.group = kFusedGroup;
        n.slot_bytes = (unsigned)n.group * n.chunk_bytes;
        n.a_bytes = 128u * 2u * (unsigned)std::max(m->in_pad, width);
        n.tmem_cols = 32;
        while ((int)n.tmem_cols < width) n.tmem_cols *= 2;
        n.p_floats = (unsigned)(layers * width + width + 1);
        const long budget = 110 * 1024 - (long)n.a_bytes - (long)sizeof(fused::Ctl) -
                            (long)n.p_floats * 4 - 16;
        n.slots = (int)std::max(2L, std::min((long)fused::kMaxSlots, budget / (long)n.slot_bytes));
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            configure_fused<fused::InRows>(m, &m->per_sm_rows) != cudaSuccess ||
            configure_fused<fused::InTrajSet>(m, &m->per_sm_traj) != cudaSuccess ||
            configure_fused<fused::InPairSet>(m, &m->per_sm_pair) != cudaSuccess) {
            mrs_mlp_destroy(m);
            return MRS_ECUDA;
        }
    }
    cudaMemsetAsync(m->params, 0, sizeof(float) * o, m->stream);
    cudaMemsetAsync(m->am, 0, sizeof(float) * o, m->stream);
    cudaMemsetAsync(m->av, 0, sizeof(float) * o, m->stream);
    cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
    for (int l = 0; l < layers; ++l) {
        const size_t n = (size_t)width * in_of(m, l);
        k_init_param<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(
            m->params + m->offW[l], n, 1.f / std::sqrt((float)(l == 0 ? in_dim : width)), seed, l);
    }
    k_init_param<<<1, 256, 0, m->stream>>>(m->params + m->offWo, width, 1.f / std::sqrt((float)width),
                                           seed, layers);
    if (mlp_refresh_bf16(m) != MRS_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) {
        mrs_mlp_destroy(m);
        return MRS_ECUDA;
    }
    *out = m;
    return MRS_OK;
}

void mrs_mlp_destroy(mrs_mlp *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->params); cudaFree(m->grads); cudaFree(m->am); cudaFree(m->av);
    cudaFree(m->loss); cudaFree(m->err);
    for (auto p : m->Wb) cudaFree(p);
    for (auto p : m->WbT) cudaFree(p);
    cudaFree(m->X);
    for (auto p : m->Z) cudaFree(p);
    for (auto p : m->Hs) cudaFree(p);
    cudaFree(m->y); cudaFree(m->dy); cudaFree(m->dH); cudaFree(m->dZ); cudaFree(m->dZT); cudaFree(m->HT);
    cudaFree(m->wpack);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

const char *mrs_mlp_last_error(const mrs_mlp *m) { return m ? m->msg.c_str() : "null network"; }

mrs_status mrs_mlp_param_count(const mrs_mlp *m, size_t *n)
{
    if (!m || !n) return MRS_EINVAL;
    *n = m->n_params;
    return MRS_OK;
}

mrs_status mrs_mlp_set_loss(mrs_mlp *m, float over_weight)
{
    if (!m || !std::isfinite(over_weight) || over_weight < 1.f) return MRS_EINVAL;
    m->over_weight = over_weight;
    return MRS_OK;
}

mrs_status mrs_mlp_launch_info(const mrs_mlp *m, int *info, int n)
{
    if (!m || !info || n < 5) return MRS_EINVAL;
    info[0] = m->per_sm_rows;
    info[1] = m->per_sm_traj;
    info[2] = m->fnet.slots;
    info[3] = (int)m->fnet_smem;
    info[4] = m->num_sms;
    return MRS_OK;
}

mrs_status mrs_mlp_get_params(mrs_mlp *m, float *host, size_t n)
{
    if (!m || !host || n < m->n_params) return MRS_EINVAL;
    MCK(cudaMemcpyAsync(host, m->params, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost,
                        m->stream), "download");
    MCK(cudaStreamSynchronize(m->stream), "sync");
    return MRS_OK;
}

mrs_status mrs_mlp_set_params(mrs_mlp *m, const float *host, size_t n)
{
    if (!m || !host || n < m->n_params) return MRS_EINVAL;
    for (size_t i = 0; i < m->n_params; ++i)
        if (!std::isfinite(host[i])) return mlp_fail(m, MRS_EINVAL, "non-finite parameter");
    MCK(cudaMemcpyAsync(m->params, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice,
                        m->stream), "upload");
    mrs_status st = mlp_refresh_bf16(m);
    if (st != MRS_OK) return st;
    MCK(cudaStreamSynchronize(m->stream), "sync");
    return MRS_OK;
}

mrs_status mrs_mlp_forward(mrs_mlp *m, const float *d_x, int n, float *d_y)
{
    if (!m || !d_x || !d_y || n < 1) return MRS_EINVAL;
    MCK(launch_fused(m, fused::InRows{d_x, m->in_dim}, n, d_y, m->err, m->per_sm_rows, m->stream),
        "fused forward");
    return check_err(m);
}

mrs_status mrs_mlp_grads(mrs_mlp *m, const float *d_x, const float *d_t, int n, float *host_grads,
                         float *host_loss)
{
    if (!m || !d_x || !d_t || n < 1) return MRS_EINVAL;
    mrs_status st = mlp_reserve(m, n);
    if (st != MRS_OK) return st;
    if ((st = load_x(m, d_x, n)) != MRS_OK) return st;
    if ((st = mlp_forward_train(m, n)) != MRS_OK) return st;
    if ((st = mlp_backward(m, d_t, n)) != MRS_OK) return st;
    if (host_grads)
        MCK(cudaMemcpyAsync(host_grads, m->grads, sizeof(float) * m->n_params,
                            cudaMemcpyDeviceToHost, m->stream), "download");
    if (host_loss)
        MCK(cudaMemcpyAsync(host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream),
            "download");
    return check_err(m);
}

mrs_status mrs_mlp_train_step(mrs_mlp *m, const float *d_x, const float *d_t, int n, float lr,
                              float *host_loss)
{
    if (!m || !d_x || !d_t || n < 1 || !(lr > 0.f)) return MRS_EINVAL;
    mrs_status st = mlp_reserve(m, n);
    if (st != MRS_OK) return st;
    if ((st = load_x(m, d_x, n)) != MRS_OK) return st;
    if ((st = mlp_forward_train(m, n)) != MRS_OK) return st;
    if ((st = mlp_backward(m, d_t, n)) != MRS_OK) return st;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    k_adam<<<(unsigned)((m->n_params + 255) / 256), 256, 0, m->stream>>>(
        m->params, m->grads, m->am, m->av, m->n_params, lr, b1, b2, 1e-8f, c1, c2);
    MCK(cudaGetLastError(), "adam");
    if ((st = mlp_refresh_bf16(m)) != MRS_OK) return st;
    if (host_loss)
        MCK(cudaMemcpyAsync(host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream),
            "download");
    return check_err(m);
}

mrs_status mrs_selftest_gemm(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *C)
{
    if (M < 1 || N < 16 || N > 256 || N % 16 || K < 8 || K % 8 || !A || !B || !C) return MRS_EINVAL;
    bf16 *dA = nullptr, *dB = nullptr;
    float *dC = nullptr;
    int *err = nullptr;
    cudaError_t e = cudaMalloc(&dA, sizeof(bf16) * M * K);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(bf16) * N * K);
    if (e == cudaSuccess) e = cudaMalloc(&dC, sizeof(float) * M * N);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, sizeof(bf16) * M * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, sizeof(bf16) * N * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = gemm(dA, K, dB, K, M, N, K, 1, err, EpiStoreF32{dC, N}, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(C, dC, sizeof(float) * M * N, cudaMemcpyDeviceToHost);
    cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(err);
    if (e != cudaSuccess) return MRS_ECUDA;
    return h_err ? MRS_ETIMEOUT : MRS_OK;
}

}  // extern "C"
