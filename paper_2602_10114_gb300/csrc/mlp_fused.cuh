// mlp_fused.cuh -- fused inference of the clearance surrogate: input
// features, every hidden layer and the output layer of 128 rows in one CTA,
// activations never leaving the SM.
//
// Per 128-row tile the CTA keeps the layer input A [128][K] (BF16, canonical
// K-major layout without swizzle) in shared memory and the layer's
// accumulator [128][width] (FP32) in tensor memory.  The weights stream
// through a ring of shared-memory slots, each holding `group` consecutive
// 16-wide K chunks of one layer (fewer at the end of a layer), pre-packed in
// global memory in the same canonical layout so that one cp.async.bulk
// fills a slot.  One thread issues every MMA of the CTA, and each chunk costs
// it a few hundred cycles of dependent instruction latency when it waits and
// commits per chunk, longer than the tensor core takes for the chunk
// (M = 128, N = 256, K = 16): a slot's chunks share one wait and one commit.
// Warp roles (320 threads):
//   warps 0-7  features of the tile into A; after each layer, bias + SiLU
//              of the accumulator back into A (hidden layers) or the dot
//              product with the output weights (last layer).  Warp w reads
//              TMEM lanes 32 (w % 4) .. + 31 (one row per thread) and every
//              other 16-column chunk, starting at chunk w / 4.
//   warp 8     producer: the slot sequence (tile, layer, chunk group) into
//              the ring, an mbarrier pair (full / empty) per slot.
//   warp 9     owns the TMEM allocation; one lane issues tcgen05.mma
//              (M = 128, N = width, K = 16) per chunk, commits each slot to
//              its empty barrier and each layer to acc_full.
// The weight sequence does not depend on the data, so the producer runs
// ahead across layer and tile boundaries, bounded only by the ring depth.
// Every wait is bounded; a timeout sets the error word and the shared abort
// flag, which every role polls, then the producer waits for its copies in
// flight, the issuer for its MMAs, and the CTA frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "tc_gemm.cuh"

namespace mrs {
namespace fused {

constexpr int kEpiWarps = 8;
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kThreads = 320;
constexpr int kMaxLayers = 8;
constexpr int kMaxSlots = 16;

struct Net {
    const unsigned char *wpack;   // chunks of all layers in order, chunk_bytes each
    const float *params;          // FP32 master parameters (biases, output layer)
    int offB0;                    // bias of layer 0; layer l's at offB0 + l (width^2 + width)
    int offWo, offBo;
    int in_pad, width, layers;
    int slots;                    // ring depth
    int group;                    // K chunks per slot
    unsigned chunk_bytes;         // width * 16 * 2
    unsigned slot_bytes;          // group * chunk_bytes
    unsigned a_bytes;             // 128 * max(in_pad, width) * 2
    unsigned tmem_cols;           // power of two >= max(32, width)
    unsigned p_floats;            // biases, output weights and bias: layers * width + width + 1
};

struct alignas(16) Ctl {          // follows the A buffer and the ring
    uint64_t full[kMaxSlots], empty[kMaxSlots];
    uint64_t acc_full, a_ready, part_full, drain;
    float part[128];
    uint32_t tmem;
    int abort;
};

// A buffer, weight ring, control block, then the FP32 halved biases and the
// output layer (16-byte aligned: the control block's size is a multiple of 16)
__host__ __device__ inline size_t smem_bytes(const Net &n)
{
    return (size_t)n.a_bytes + (size_t)n.slots * n.slot_bytes + sizeof(Ctl) +
           ((size_t)n.p_floats * 4 + 15) / 16 * 16;
}

__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(tc::smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    for (unsigned it = 0; it < tc::kWaitLimit; ++it) {
        if (try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tc::smem_u32(dst_smem)), "l"(__cvta_generic_to_global(src_gmem)), "r"(bytes),
                   "r"(tc::smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fail(Ctl &C, int *err)
{
    C.abort = 1;
    atomicExch(err, 1);
}

// z sigmoid(z) = h (1 + tanh h) with h = z / 2: one hardware tanh (relative
// error about 2^-11, an absolute error of the result below 2^-12 |z|, the
// order of the BF16 rounding that follows) instead of an exponential and a
// reciprocal, which halves the special-function work of the epilogue.  The
// caller passes h = acc / 2 + bias / 2 (one FMA, the halved biases kept in
// shared memory).
__device__ __forceinline__ float silu_half(float h)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// two floats as BF16 (round to nearest even), a in the low half
__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ int in_of(const Net &n, int l) { return l == 0 ? n.in_pad : n.width; }

// Features of plain FP32 rows x [rows][in_dim].
struct InRows {
    const float *x;
    int in_dim;
    using Row = int;
    __device__ __forceinline__ Row at(int row) const { return row; }
    __device__ __forceinline__ void operator()(Row row, int g, float (&v)[8]) const
    {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * g + i;
            v[i] = k < in_dim ? x[(size_t)row * in_dim + k] : 0.f;
        }
    }
    __device__ __forceinline__ size_t out(Row row) const { return (size_t)row; }
};

// sin, cos of each joint of every rollout step of a set of arms that share
// one network: segment s covers rows [row_start[s], row_start[s+1]) of arm
// trajectories traj + off_khd[s] ([H][dof][K], local row = h K + n), its
// outputs go to off_kh[s] + local row; feature 2j = sin q_j, 2j+1 = cos q_j.
constexpr int kMaxSegs = 32;
struct TrajSegs {
    int n;
    int row_start[kMaxSegs + 1];
    int K[kMaxSegs], dof[kMaxSegs];
    long long off_khd[kMaxSegs], off_kh[kMaxSegs];
};

struct InTrajSet {
    const float *traj;
    TrajSegs seg;
    struct Row {
        int s, r;                 // segment, row within it
    };
    __device__ __forceinline__ Row at(int row) const
    {
        int s = 0;
        while (s + 1 < seg.n && row >= seg.row_start[s + 1]) ++s;
        return Row{s, row - seg.row_start[s]};
    }
    // The features are rounded to BF16 (8 significant bits) before the first
    // layer, so the fast sine and cosine (absolute error near 1e-6 for the
    // joint ranges of an arm) change none beyond that rounding's last step.
    __device__ __forceinline__ void operator()(Row w, int g, float (&v)[8]) const
    {
        const int K = seg.K[w.s], dof = seg.dof[w.s];
        const int h = w.r / K, n = w.r - h * K;
        const float *qh = traj + seg.off_khd[w.s] + (size_t)h * dof * K + n;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int j = 4 * g + p;
            float sn = 0.f, cs = 0.f;
            if (j < dof) __sincosf(qh[(size_t)j * K], &sn, &cs);
            v[2 * p] = sn;
            v[2 * p + 1] = cs;
        }
    }
    __device__ __forceinline__ size_t out(Row w) const { return (size_t)(seg.off_kh[w.s] + w.r); }
};

// Features of the arm-pair surrogate for every rollout step of arm a against
// the published plan of arm b, for a set of (a, b) segments sharing one
// network: row = h K_a + n of segment s; features 2j, 2j+1 = sin, cos of
// arm a's joint j at the sampled step (trajectory traj + off_khd[s],
// [H][d_a][K_a]), then sin, cos of arm b's plan joints at step min(h,
// H_b - 1) (plan + off_hd[s], [H_b][d_b]), then the 7 numbers of arm b's
// base pose in arm a's base frame (xyz, quaternion w x y z); outputs to
// off_out[s] + row within the segment.
struct PairSegs {
    int n;
    int row_start[kMaxSegs + 1];
    int K[kMaxSegs], Hb[kMaxSegs], da[kMaxSegs], db[kMaxSegs];
    long long off_khd[kMaxSegs], off_hd[kMaxSegs], off_out[kMaxSegs];
    float pose[kMaxSegs][7];
};

struct InPairSet {
    const float *traj, *plan;
    PairSegs seg;
    struct Row {
        int s, r;                 // segment, row within it
    };
    __device__ __forceinline__ Row at(int row) const
    {
        int s = 0;
        while (s + 1 < seg.n && row >= seg.row_start[s + 1]) ++s;
        return Row{s, row - seg.row_start[s]};
    }
    // fast sine and cosine, as for InTrajSet: the features are rounded to BF16
    __device__ __forceinline__ void operator()(Row w, int g, float (&v)[8]) const
    {
        const int s = w.s, K = seg.K[s], da = seg.da[s], db = seg.db[s];
        const int r = w.r, h = r / K, n = r - h * K;
        const float *qa = traj + seg.off_khd[s] + (size_t)h * da * K + n;
        const float *qb = plan + seg.off_hd[s] + (size_t)min(h, seg.Hb[s] - 1) * db;
#pragma unroll
        for (int p = 0; p < 8; p += 2) {
            const int f = 8 * g + p;                 // even: (sin, cos) pairs stay together
            float a = 0.f, b = 0.f;
            if (f < 2 * da) {
                __sincosf(qa[(size_t)(f >> 1) * K], &a, &b);
            } else if (f < 2 * da + 2 * db) {
                __sincosf(qb[(f - 2 * da) >> 1], &a, &b);
            } else {
                const int k = f - 2 * da - 2 * db;
                a = k < 7 ? seg.pose[s][k] : 0.f;
                b = k + 1 < 7 ? seg.pose[s][k + 1] : 0.f;
            }
            v[p] = a;
            v[p + 1] = b;
        }
    }
    __device__ __forceinline__ size_t out(Row w) const { return (size_t)(seg.off_out[w.s] + w.r); }
};

// Input functor interface: in.at(row) locates a valid row (row < rows) once,
// in(at, g, v) fills its 8 features 8g .. 8g+7, features at or beyond the
// input width 0, and the row's output goes to y[in.out(at)].
template <class In>
__global__ void __launch_bounds__(kThreads, 2)
k_mlp_fused(Net net, In in, int rows, float *y, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *ring = smem + net.a_bytes;
    Ctl &C = *reinterpret_cast<Ctl *>(ring + (size_t)net.slots * net.slot_bytes);
    float *Ps = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(&C) + sizeof(Ctl));
    volatile int *abort = &C.abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (rows + 127) / 128;
    const int S = net.slots, G = net.group;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&C.full[s], 1);
            tc::mbar_init(&C.empty[s], 1);
        }
        tc::mbar_init(&C.acc_full, 1);
        tc::mbar_init(&C.a_ready, kEpiWarps * 32);
        tc::mbar_init(&C.part_full, 4 * 32);
        tc::mbar_init(&C.drain, 1);
        C.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tc::tmem_alloc(&C.tmem, net.tmem_cols);
    {
        // halved biases of every layer (the SiLU takes z / 2), output weights
        // and bias, read by the epilogue
        const int W = net.width, LW = net.layers * W;
        for (int i = threadIdx.x; i < (int)net.p_floats; i += kThreads) {
            float v;
            if (i < LW)
                v = 0.5f * net.params[net.offB0 + (size_t)(i / W) * (W * W + W) + i % W];
            else if (i < LW + W)
                v = net.params[net.offWo + i - LW];
            else
                v = net.params[net.offBo];
            Ps[i] = v;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = C.tmem;

    if (warp == kProducerWarp) {
        if (lane == 0) {
            uint32_t cnt = 0, s = 0, phase = 0;   // slots filled, ring position, its wrap parity
            bool ok = true;
            for (int t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
                const unsigned char *src = net.wpack;
                for (int l = 0; ok && l < net.layers; ++l) {
                    const int nch = in_of(net, l) / 16;
                    for (int c = 0; c < nch; c += G) {
                        const uint32_t bytes = (uint32_t)min(G, nch - c) * net.chunk_bytes;
                        if (!wait_or_abort(&C.empty[s], phase ^ 1u, abort)) {
                            fail(C, err);
                            ok = false;
                            break;
                        }
                        arrive_expect_tx(&C.full[s], bytes);
                        bulk_copy(ring + (size_t)s * net.slot_bytes, src, bytes, &C.full[s]);
                        src += bytes;
                        ++cnt;
                        if (++s == (uint32_t)S) {
                            s = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // no copy may still be landing in shared memory when the CTA exits
            const uint32_t first = cnt > (uint32_t)S ? cnt - S : 0u;
            for (uint32_t k = first; k < cnt; ++k)
                if (!tc::mbar_wait(&C.full[k % S], (k / S) & 1u)) atomicExch(err, 1);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            uint32_t s = 0, phase = 0, v = 0;
            bool ok = true;
            const uint32_t idesc = tc::idesc_bf16_f32(128, net.width);
            const uint32_t a0 = tc::smem_u32(Abuf);
            const uint64_t bd0 = tc::smem_desc(tc::smem_u32(ring), 128u, 256u);
            for (int t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
                for (int l = 0; ok && l < net.layers; ++l) {
                    if (!wait_or_abort(&C.a_ready, (v++) & 1u, abort)) {
                        fail(C, err);
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int K = in_of(net, l), nch = K / 16;
                    // descriptors of chunk 0 of A and of slot 0; a chunk
                    // further on adds its byte offset / 16 to the address
                    // field (shared addresses stay below 2^18 bytes: no carry)
                    const uint64_t ad0 = tc::smem_desc(a0, 128u, (uint32_t)(K / 8) * 128u);
                    for (int c = 0; c < nch; c += G) {
                        if (!wait_or_abort(&C.full[s], phase, abort)) {
                            fail(C, err);
                            ok = false;
                            break;
                        }
                        const int g = min(G, nch - c);
                        const uint64_t bd = bd0 + (uint64_t)((s * net.slot_bytes) >> 4);
                        for (int j = 0; j < g; ++j)
                            tc::mma_bf16(tmem, ad0 + (uint64_t)((c + j) * 16),
                                         bd + (uint64_t)(j * (net.chunk_bytes >> 4)), idesc,
                                         (c + j) > 0 ? 1u : 0u);
                        tc::mma_commit(&C.empty[s]);
                        if (++s == (uint32_t)S) {
                            s = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) tc::mma_commit(&C.acc_full);
                }
            }
            // every MMA issued has completed before the TMEM is freed
            tc::mma_commit(&C.drain);
            if (!tc::mbar_wait(&C.drain, 0)) atomicExch(err, 1);
        }
    } else {
        // epilogue warps
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const int W = net.width;
        const float *w_out = Ps + net.layers * W;
        const float b_out = Ps[net.layers * W + W];
        uint32_t u = 0, pp = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
            const int row = t * 128 + m;
            const bool valid = row < rows;
            const typename In::Row at = in.at(valid ? row : 0);
            // features of this row into A (layout of K = in_pad)
            {
                const uint32_t sbo = (uint32_t)(net.in_pad / 8) * 128u;
                for (int g = half; g < net.in_pad / 8; g += 2) {
                    float v[8];
                    if (valid) {
                        in(at, g, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = 0.f;
                    }
                    *reinterpret_cast<uint4 *>(Abuf + (m >> 3) * sbo + g * 128 + (m & 7) * 16) =
                        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                                   pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
                }
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            arrive(&C.a_ready);
            float part = 0.f;
            for (int l = 0; l < net.layers; ++l) {
                const bool got = wait_or_abort(&C.acc_full, (u++) & 1u, abort);
                if (!__all_sync(0xffffffffu, got)) {
                    fail(C, err);
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const bool last = l == net.layers - 1;
                const float *hbias = Ps + l * W;
                const uint32_t sbo = (uint32_t)(W / 8) * 128u;
                // this thread's 16-column chunks cc = half, half + 2, ..., two
                // loads in flight per wait
                auto finish = [&](int cc, const uint32_t (&r)[16]) {
                    uint32_t pk[8];
                    const float4 *hb = reinterpret_cast<const float4 *>(hbias + cc * 16);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 b = hb[i];
                        pk[2 * i] = pack_bf16(silu_half(fmaf(__uint_as_float(r[4 * i]), 0.5f, b.x)),
                                              silu_half(fmaf(__uint_as_float(r[4 * i + 1]), 0.5f, b.y)));
                        pk[2 * i + 1] =
                            pack_bf16(silu_half(fmaf(__uint_as_float(r[4 * i + 2]), 0.5f, b.z)),
                                      silu_half(fmaf(__uint_as_float(r[4 * i + 3]), 0.5f, b.w)));
                    }
                    if (!last) {
                        unsigned char *dst = Abuf + (m >> 3) * sbo + (2 * cc) * 128 + (m & 7) * 16;
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        *reinterpret_cast<uint4 *>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
                        const float4 *wo = reinterpret_cast<const float4 *>(w_out + cc * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 w = wo[i];
                            part = fmaf(__uint_as_float(pk[2 * i] << 16), w.x, part);
                            part = fmaf(__uint_as_float(pk[2 * i] & 0xffff0000u), w.y, part);
                            part = fmaf(__uint_as_float(pk[2 * i + 1] << 16), w.z, part);
                            part = fmaf(__uint_as_float(pk[2 * i + 1] & 0xffff0000u), w.w, part);
                        }
                    }
                };
                const int nc = W / 16;
                for (int cc = half; cc < nc; cc += 4) {
                    uint32_t r0[16], r1[16];
                    const bool two = cc + 2 < nc;      // uniform over the warp
                    tc::tmem_ld16_async(lane_base + (uint32_t)(cc * 16), r0);
                    if (two) tc::tmem_ld16_async(lane_base + (uint32_t)((cc + 2) * 16), r1);
                    tc::tmem_wait_ld();
                    finish(cc, r0);
                    if (two) finish(cc + 2, r1);
                }
                tc::fence_before_sync();
                if (!last) {
                    tc::fence_async_smem();
                    arrive(&C.a_ready);
                }
            }
            if (!ok) break;
            // output: the two column halves of a row meet in shared memory
            if (half == 1) {
                C.part[m] = part;
                arrive(&C.part_full);
            } else {
                const bool got = wait_or_abort(&C.part_full, (pp++) & 1u, abort);
                if (!got) {
                    fail(C, err);
                    ok = false;
                } else if (valid) {
                    y[in.out(at)] = part + C.part[m] + b_out;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, net.tmem_cols);
    }
}

}  // namespace fused
}  // namespace mrs
