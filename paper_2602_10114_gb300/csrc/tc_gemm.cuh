// tc_gemm.cuh -- BF16 tensor-core GEMM on sm_103a with tcgen05 (5th-gen
// tensor cores), used by the learned clearance surrogates.
//
//   C[M][N] = A[M][K] * B[N][K]^T      (A, B row-major BF16, K contiguous)
//
// One CTA of 128 threads computes a 128 x N tile (N <= 256, multiple of 16)
// with the FP32 accumulator in tensor memory (TMEM).  Per K chunk the four
// warps copy the A and B tiles into shared memory in the canonical K-major
// layout without swizzle (8-row x 16-byte core matrices; consecutive core
// matrices along K are LBO = 128 B apart, consecutive 8-row groups SBO =
// (BK / 8) * 128 B apart), fence them to the async proxy, and one elected
// thread issues BK / 16 tcgen05.mma instructions (M = 128, N, K = 16) and
// commits them to an mbarrier.  Every wait on the mbarrier is bounded; on
// timeout the kernel sets the error word and abandons the tile.  The epilogue
// reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// one output row per thread) and hands each row to a functor.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace mrs {
namespace tc {

constexpr int kThreads = 128;
constexpr unsigned kWaitLimit = 1u << 22;   // polls of a bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, LBO >> 4
// in 16-29, SBO >> 4 in 32-45, descriptor version 1 in bits 46-47, base
// offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// true when phase `parity` of the barrier has completed within `limit`
// polls (none at all for limit = 0); bounded
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned limit = kWaitLimit)
{
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(dst_smem)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting:
// the registers are valid after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy rows [r0, r0 + R) x K columns [k0, k0 + BK) of a row-major BF16 matrix
// (ld elements per row, `rows` valid rows, zero fill beyond) into the
// canonical K-major no-swizzle layout at dst.
template <int BK>
__device__ __forceinline__ void load_tile_kmajor(const __nv_bfloat16 *src, int ld, int rows, int r0,
                                                 int R, int k0, int K, unsigned char *dst)
{
    constexpr int kVec = BK / 8;                    // 16-byte vectors per tile row
    const int total = R * kVec;
    for (int i = threadIdx.x; i < total; i += kThreads) {
        const int r = i / kVec, kc = i % kVec;
        const int gr = r0 + r, gk = k0 + kc * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < rows && gk < K) v = *reinterpret_cast<const uint4 *>(src + (size_t)gr * ld + gk);
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * (kVec * 128) + kc * 128 + (r & 7) * 16) = v;
    }
}

// Shared memory of one CTA: A tile, B tile, barrier, TMEM address.
template <int BK>
struct GemmSmem {
    alignas(128) unsigned char a[128 * BK * 2];
    alignas(128) unsigned char b[256 * BK * 2];
    alignas(8) uint64_t bar;
    uint32_t tmem;
};

// Epilogue functor interface: f(row, col0, v[16]) for 16 consecutive columns
// of one row (row < M guaranteed, col0 + 16 <= N).  A is [M][lda], B is
// [N][ldb]; the product runs over K columns [k_begin, k_end) (a multiple of 8
// wide; a split-K slice when several CTAs share one output tile).
template <int BK, class Epi>
__device__ __forceinline__ void gemm_tile(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
                                          int ldb, int M, int N, int k_begin, int k_end, int m0,
                                          GemmSmem<BK> &S, int *err, Epi &epi)
{
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(&S.tmem, 256);
    if (threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t idesc = idesc_bf16_f32(128, N);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = k_begin; k0 < k_end; k0 += BK) {
        load_tile_kmajor<BK>(A, lda, M, m0, 128, k0, k_end, S.a);
        load_tile_kmajor<BK>(B, ldb, N, 0, N, k0, k_end, S.b);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after_sync();
            const uint32_t a0 = smem_u32(S.a), b0 = smem_u32(S.b);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, (BK / 8) * 128);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, (BK / 8) * 128);
                mma_bf16(tmem, ad, bd, idesc, (k0 > k_begin || kk > 0) ? 1u : 0u);
            }
            mma_commit(&S.bar);
        }
        // the tiles may be overwritten only after the MMAs that read them
        if (!mbar_wait(&S.bar, phase)) {
            ok = false;
            atomicExch(err, 1);
        }
        phase ^= 1u;
        fence_after_sync();
        if (!__syncthreads_and(ok)) break;
    }
    if (__syncthreads_and(ok)) {
        const int row = m0 + threadIdx.x;   // warp w: TMEM lanes 32w .. 32w+31
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)c0, v);
            if (row < M) epi(row, c0, v);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace tc
}  // namespace mrs
