// rollout_kernel.cuh -- the Rollout step of Algorithm 1 for every arm: kinematics of
// the collision spheres at each sampled state and the stage cost of Eq. 5
// with the prioritised coordination term of Eq. 9 (Sec. IV-A/B).
//
// Work unit (tile): (arm, step h, 32 nsub samples).  A persistent grid of
// 256-thread blocks takes tiles from an atomic counter and stages the tile's
// inputs (world at the step's time, the neighbours' plan spheres at step h --
// copied from the plan board by the bulk-copy engine, cp.async.bulk on an
// mbarrier -- and the arm's constants) once; the samples then pass through in
// sub-batches of 32.  Warp g of a block owns sphere group g (spheres [g*spg, (g+1)*spg),
// spg = ceil(N_S / 8)) of the sub-batch's 32 rollout steps, one sample per
// lane.  The samples per tile, the tile order and the resident blocks per SM
// are chosen at run time (mrs_autotune).
//
// Pair tests.  A pair (own sphere c, radius r; other sphere p, radius r_p)
// can change a ramp cost max(0, 1 - dist/B) only if |c - p| < r + r_p + B.
// The other spheres of a unit -- the world at the step's time, then each
// neighbour's plan slice -- form clusters of up to 8 consecutive spheres,
// each with its box (the world is kept in a spatial order, refreshed every
// cycle, so that its clusters are compact).  A warp narrows the pairs in
// three box tests, each conservative (it never drops a pair inside the
// ramp): the cluster boxes against the box of the warp's own spheres over
// its 32 samples; the spheres of the near clusters against that box; every
// (candidate, own sphere) pair against that own sphere's box over the
// samples.  The pairs left get the exact distance of every sample, the
// square root only inside the ramp.  Since the cost is zero outside the
// ramp, the result equals the brute-force minimum of Eq. 6 restricted to the
// ramp, whatever the order of the spheres.
#pragma once

#include <algorithm>

#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace mrs {

// slack of every box test (m): far above the rounding of the coordinates
// (a few 1e-7 m over the workspace), so that no test drops a pair the exact
// distance keeps
constexpr float kCullMargin = 1e-3f;

// every sphere-group size (bits 1 .. 8) for the build that serves any arms
constexpr unsigned kAllSizes = 0x1FEu;

// the size of a build that holds one sphere-group size, else 0
constexpr int single_size(unsigned sizes)
{
    for (int s = 1; s <= 8; ++s)
        if (sizes == (1u << s)) return s;
    return 0;
}

// capacity of the block's list of obstacle pairs per sub-batch (a warp tests
// the pairs that do not fit itself)
constexpr int kObstaclePairCap = 512;

// The unit arm's scalars, staged in shared memory once per unit (the
// ArmDev record in global memory would be re-read after the unit's stores)
struct ArmHdr {
    int dof, K, ns, n_self, learned, H;
    unsigned pair_mask;
    float pair_margin, self_margin;
    int spg;
    long long off_kh, off_khd;
};

struct RolloutSmem {
    float4 *other;     // world spheres at the step's time, then neighbours' plan spheres
    unsigned char *seg;     // [n_other] set of each plan sphere: 2 + its neighbour slot
    float4 *cbox;      // [2 * n_cl] box of each cluster: lo, hi (w unused)
    int *cinfo;        // [n_cl] first sphere | count << 16 | set << 20 (0 world, 2 + nb)
    float4 *aabb;      // [2 * n_aabb] centre, half extents
    float4 *sph;       // [ns] local centre + radius
    int *frame;        // [ns]
    int2 *pairs;       // [n_self] byte offsets of both spheres in own (o1 | o2 << 16),
                       // and (r1 + B_self + r2)^2 as float bits
    float4 *own;       // [ns][32] own sphere centre and radius of each sample
    int *red;          // [(2 + n_nb) * 32] ordered-int minima: world, self, neighbours
    int *nb_start;     // [n_nb + 1] ranges in `other` (after the world spheres)
    int *nb_cstart;    // [n_nb] first cluster of each neighbour
    float *nb_alpha;   // [n_nb]
    int *nb_arm;       // [n_nb] arm index of each neighbour
    unsigned short *cand;   // [kGroups][cand_cap] per-warp candidate lists
    int cand_cap;
    int2 *opairs;           // [kObstaclePairCap] the sub-batch's obstacle pairs left by the
                            // box tests: own sphere | other << 6 | set << 18, (r + B + r_p)^2
    int *opn;               // the count of opairs entries this sub-batch (by sub-batch parity)
    const unsigned *need;   // [32] with an arm-pair surrogate: the neighbours each lane needs
    const unsigned *skip;   // the neighbours no lane needs (this sub-batch's parity)
    float4 *sbox;           // [ns][2] per-sphere bounding box over the sub-batch: lo, hi
    float2 *sc;             // [dof][32] sin, cos of q_j + theta_j of the sub-batch's samples
    float4 *dh;             // [kMaxDof] the arm's DH rows (a, d, alpha, theta)
    float2 *tw;             // [kMaxDof] sin, cos of the twists
    float *base;            // [12] base rotation (row-major) and translation
    float *goal;            // [12] the arm's goal position and rotation (sensed input)
};

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Other spheres of a unit at most (the world, every other arm's plan slice),
// their clusters, and the capacity of a warp's candidate list.
__host__ __device__ inline int rollout_other_cap(const Params &P, int n_arms)
{
    return P.world_cap + P.max_ns * n_arms;
}
__host__ __device__ inline int rollout_cluster_cap(const Params &P, int n_arms)
{
    return (P.world_cap + 7) / 8 + n_arms * ((P.max_ns + 7) / 8);
}
__host__ __device__ inline int rollout_cand_cap(const Params &, int)
{
    return 128;   // a warp's candidate list; when full, its pairs are taken at once
}

// mbarrier arrive with an expected transaction count (the bytes of the bulk
// copies that complete the phase)
__device__ __forceinline__ void fused_bar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}

// bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16) completing on mbarrier bar
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(tc::smem_u32(dst_smem)), "l"(__cvta_generic_to_global(src_gmem)), "r"(bytes),
                   "r"(tc::smem_u32(bar))
                 : "memory");
}

// 4-byte asynchronous copy global -> shared (one group per call) and the
// wait for all of the calling thread's copies
__device__ __forceinline__ void cp_async4(float *dst_smem, const float *src_gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n cp.async.commit_group;"
                 ::"r"(tc::smem_u32(dst_smem)), "l"(__cvta_generic_to_global(src_gmem)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// minimum / maximum of a float over the full warp (sm_100+ floating-point
// warp reduction; exact)
__device__ __forceinline__ float warp_min(float v)
{
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v)
{
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// box lo / hi reduced over aligned groups of 8 lanes (every lane gets its
// group's; exact)
__device__ __forceinline__ void cluster_box(float3 &lo, float3 &hi)
{
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
}

// squared gap between a point and a box (0 inside)
__device__ __forceinline__ float gap2(float4 p, float3 lo, float3 hi)
{
    const float gx = fmaxf(fmaxf(lo.x - p.x, p.x - hi.x), 0.f);
    const float gy = fmaxf(fmaxf(lo.y - p.y, p.y - hi.y), 0.f);
    const float gz = fmaxf(fmaxf(lo.z - p.z, p.z - hi.z), 0.f);
    return gx * gx + gy * gy + gz * gz;
}

// The same test for a self pair whose squared ramp bound (r1 + B + r2)^2 was
// computed beforehand with the same sums: sqrt(d2) - r1 - r2 when inside
__device__ __forceinline__ void pair_exact_t2(float4 c1, float4 c2, float t2, float &m)
{
    const float dx = __fsub_rn(c2.x, c1.x), dy = __fsub_rn(c2.y, c1.y), dz = __fsub_rn(c2.z, c1.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (d2 < t2) m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), c1.w), c2.w));
}

// Exact distance of one obstacle pair (own sphere, other sphere p) for this
// lane's sample, the square root only inside the ramp, and its minimum into
// the set's slot of the per-lane minima (world 0, neighbour nb at 2 + nb)
// when inside the set's buffer and the lane needs the set (need_nb: bit nb
// for neighbour nb).  code: own sphere | other << 6 | set << 18; t2: the
// squared ramp bound (r + B + r_p)^2 with the sums in this order.
__device__ __forceinline__ void obstacle_pair(const Params &P, const RolloutSmem &S, int code,
                                              float t2, int lane, unsigned need_nb)
{
    const int set = code >> 18;
    const float4 c = S.own[(code & 63) * 32 + lane];
    const float4 p = S.other[(code >> 6) & 4095];
    const float dx = __fsub_rn(p.x, c.x), dy = __fsub_rn(p.y, c.y), dz = __fsub_rn(p.z, c.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (d2 < t2) {
        const float dist = __fsub_rn(__fsub_rn(sqrtf(d2), c.w), p.w);
        const bool need = set == 0 || ((need_nb >> (set - 2)) & 1u);
        if (need && dist < (set == 0 ? P.B_world : P.B))
            atomicMin(&S.red[set * 32 + lane], float_to_ordered(dist));
    }
}

// The warp's obstacle pairs left by the box tests: each (candidate, own
// sphere) pair, one per lane, is tested against that own sphere's box over
// the sub-batch; the pairs within r_p + B + margin of it are appended to the
// block's list, whose exact distances all warps share after the block
// barrier.  Pairs that do not fit the list are done here.
template <int SPG>
__device__ __forceinline__ void near_pairs(const Params &P, const RolloutSmem &S,
                                           const unsigned short *list, int nc, int n_world,
                                           float tw, float tn, int s0, int cnt, int lane,
                                           unsigned need_nb)
{
    const unsigned below = (1u << lane) - 1u;
    const int np = nc * SPG;
    for (int base = 0; base < np; base += 32) {
        const int e = base + lane;
        bool near = false;
        int code = 0;
        float t2 = 0.f;
        if (e < np) {
            const int j = e / SPG, s = e - j * SPG;
            if (s < cnt) {
                const int k = list[j];
                const float4 p = S.other[k];
                const float4 bl = S.sbox[2 * (s0 + s)], bh = S.sbox[2 * (s0 + s) + 1];
                const bool w = k < n_world;
                const float t = p.w + (w ? tw : tn);
                near = gap2(p, make_float3(bl.x, bl.y, bl.z), make_float3(bh.x, bh.y, bh.z)) < t * t;
                const float tb = __fadd_rn(__fadd_rn(S.sph[s0 + s].w, w ? P.B_world : P.B), p.w);
                t2 = __fmul_rn(tb, tb);
                code = (s0 + s) | (k << 6) | ((w ? 0 : (int)S.seg[k]) << 18);
            }
        }
        const unsigned mk = __ballot_sync(0xffffffffu, near);
        if (!mk) continue;
        int at = 0;
        if (lane == 0) at = atomicAdd(S.opn, __popc(mk));
        at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & below);
        const bool stored = near && at < kObstaclePairCap;
        if (stored) S.opairs[at] = make_int2(code, __float_as_int(t2));
        unsigned left = __ballot_sync(0xffffffffu, near && !stored);
        while (left) {
            const int b = __ffs(left) - 1;
            left &= left - 1u;
            obstacle_pair(P, S, __shfl_sync(0xffffffffu, code, b),
                          __shfl_sync(0xffffffffu, t2, b), lane, need_nb);
        }
    }
}

// The warp's obstacle pairs: candidates first, the other spheres (every set)
// within r_p + B + margin of the warp's box [lo, hi] (each own centre +- its
// radius over the 32 lanes), found cluster by cluster.  A cluster whose box is farther than
// B + margin from the warp's box holds no candidate: each of its spheres
// lies in the cluster box by its radius, so its centre is farther than
// r_p + B + margin from the warp's box.  Near clusters are taken four at a
// time, lanes 8i .. 8i + 7 on the i-th, their spheres tested one per lane.
// Sets that no lane of the warp needs (skip_nb, bit nb for neighbour nb) are
// left out.  The candidates go through near_pairs whenever the warp's list
// is full, and at the end.  tw, tn: B + margin of the world and of the plan
// sets.
template <int SPG>
__device__ __forceinline__ void obstacle_pairs(const Params &P, const RolloutSmem &S, float3 lo,
                                               float3 hi, int n_cl, int n_world, float tw,
                                               float tn, unsigned skip_nb, int s0, int cnt,
                                               int lane, unsigned need_nb, unsigned short *list)
{
    const float tc = fmaxf(tw, tn);
    const float tc2 = tc * tc;
    const unsigned below = (1u << lane) - 1u;
    int nc = 0;
    for (int c0 = 0; c0 < n_cl; c0 += 32) {
        const int c = c0 + lane;
        bool near = false;
        if (c < n_cl) {
            const float4 cl = S.cbox[2 * c], ch = S.cbox[2 * c + 1];
            const float gx = fmaxf(fmaxf(cl.x - hi.x, lo.x - ch.x), 0.f);
            const float gy = fmaxf(fmaxf(cl.y - hi.y, lo.y - ch.y), 0.f);
            const float gz = fmaxf(fmaxf(cl.z - hi.z, lo.z - ch.z), 0.f);
            near = gx * gx + gy * gy + gz * gz < tc2;
            if (skip_nb) {
                const int set = S.cinfo[c] >> 20;
                if (set >= 2 && ((skip_nb >> (set - 2)) & 1u)) near = false;
            }
        }
        unsigned mc = __ballot_sync(0xffffffffu, near);
        while (mc) {
            // the (lane / 8)-th lowest near cluster left, then drop four
            unsigned x = mc;
            const int i = lane >> 3;
            if (i >= 1) x &= x - 1u;
            if (i >= 2) x &= x - 1u;
            if (i >= 3) x &= x - 1u;
            mc &= mc - 1u;
            mc &= mc - 1u;
            mc &= mc - 1u;
            mc &= mc - 1u;
            bool keep = false;
            int k = 0;
            if (x) {
                const int info = S.cinfo[c0 + __ffs(x) - 1];
                const int r = lane & 7;
                if (r < ((info >> 16) & 15)) {
                    k = (info & 0xffff) + r;
                    const float4 p = S.other[k];
                    const float t = p.w + (k < n_world ? tw : tn);
                    keep = gap2(p, lo, hi) < t * t;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) list[nc + __popc(m & below)] = (unsigned short)k;
            nc += __popc(m);
            if (nc > S.cand_cap - 32) {   // no room for another step: take these now
                __syncwarp();
                near_pairs<SPG>(P, S, list, nc, n_world, tw, tn, s0, cnt, lane, need_nb);
                __syncwarp();
                nc = 0;
            }
        }
    }
    __syncwarp();
    if (nc > 0) near_pairs<SPG>(P, S, list, nc, n_world, tw, tn, s0, cnt, lane, need_nb);
}

// With an arm-pair surrogate, a step whose predicted clearance to a
// neighbour's plan is at least B + margin needs no exact pass for it (its
// coordination term is zero); a plan published without joints always takes
// the exact pass.  Warp g decides for neighbours g, g + 8, ... of the
// samples n (lane): the loaded predictions and plan flags (pair_loads), then
// the bits (pair_bits): a cleared bit in need[lane] for a neighbour the lane
// does not need, a set bit in *skip for one no lane needs.  need starts at
// all ones and skip at zero for every sub-batch.
constexpr int kPairPerWarp = (MRS_MAX_ARMS + kGroups - 1) / kGroups;
template <class Arm>
__device__ __forceinline__ void pair_loads(const Params &P, const Dev &D, const Arm &A,
                                           unsigned mask, int n_nb, int h, int n, int g,
                                           float (&rv)[kPairPerWarp], int (&bv)[kPairPerWarp])
{
#pragma unroll
    for (int k = 0; k < kPairPerWarp; ++k) {
        const int nb = g + kGroups * k;
        rv[k] = kInf;
        bv[k] = 1;
        if (nb < n_nb) {
            const int ai = __fns(mask, 0, nb + 1);     // the arm of neighbour nb
            if ((A.pair_mask >> ai) & 1u) {
                bv[k] = D.board_valid[ai];
                if (n < A.K)
                    rv[k] = D.rhohat[A.off_kh * P.n_arms + (long long)ai * A.H * A.K +
                                     (long long)h * A.K + n];
            }
        }
    }
}
template <class Arm>
__device__ __forceinline__ void pair_bits(const Params &P, const Arm &A, unsigned mask, int n_nb,
                                          int n, int g, int lane, const float (&rv)[kPairPerWarp],
                                          const int (&bv)[kPairPerWarp], unsigned *need,
                                          unsigned *skip)
{
#pragma unroll
    for (int k = 0; k < kPairPerWarp; ++k) {
        const int nb = g + kGroups * k;
        if (nb < n_nb && ((A.pair_mask >> __fns(mask, 0, nb + 1)) & 1u)) {
            const bool nd = n < A.K && (bv[k] != 1 || rv[k] < P.B + A.pair_margin);
            if (!nd) atomicAnd(&need[lane], ~(1u << nb));
            if (!__any_sync(0xffffffffu, nd) && lane == 0) atomicOr(skip, 1u << nb);
        }
    }
}

// pair_loads then pair_bits, out of line: the exact mode never calls it, so
// that its code stays out of the hot loop's instruction footprint
template <class Arm>
__device__ __noinline__ void pair_masks(const Params &P, const Dev &D, const Arm &A, unsigned mask,
                                        int n_nb, int h, int n, int g, int lane, unsigned *need,
                                        unsigned *skip)
{
    float rv[kPairPerWarp];
    int bv[kPairPerWarp];
    pair_loads(P, D, A, mask, n_nb, h, n, g, rv, bv);
    pair_bits(P, A, mask, n_nb, n, g, lane, rv, bv, need, skip);
}

template <int SPG>
__device__ __forceinline__ void rollout_group(const Params &P, const Dev &D, const ArmHdr &A,
                                              const RolloutSmem &S, int h, int n, bool valid,
                                              int g, int lane, int n_world, int n_aabb, int n_nb,
                                              int n_cl, float *pose_out)
{
    const int d = A.dof, K = A.K;
    const int s0 = g * SPG;
    const int cnt = max(0, min(SPG, A.ns - s0));

    // DH chain up to the last frame this group needs; the last warp always
    // runs to the end effector for the pose cost.  Each own centre goes to
    // shared memory, and its box over the warp's 32 samples (centre +-
    // radius, warp-wide floating-point min / max, exact) to the sphere
    // boxes; their union is the warp's box.
    Frame F;
#pragma unroll
    for (int k = 0; k < 9; ++k) F.R[k] = S.base[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) F.t[k] = S.base[9 + k];
    float3 lo = make_float3(kInf, kInf, kInf), hi = make_float3(-kInf, -kInf, -kInf);
    int f = 0;
#pragma unroll
    for (int s = 0; s < SPG; ++s) {
        if (s < cnt) {
            const int fs = S.frame[s0 + s];
            while (f < fs) {
                const float2 sc = S.sc[f * 32 + lane];
                frame_step_sc(F, sc.x, sc.y, S.dh[f], S.tw[f]);
                ++f;
            }
            const float4 sp = S.sph[s0 + s];
            const float3 c = sphere_centre(F, sp);
            S.own[(s0 + s) * 32 + lane] = make_float4(c.x, c.y, c.z, sp.w);
            const float4 bl = make_float4(warp_min(c.x - sp.w), warp_min(c.y - sp.w),
                                          warp_min(c.z - sp.w), 0.f);
            const float4 bh = make_float4(warp_max(c.x + sp.w), warp_max(c.y + sp.w),
                                          warp_max(c.z + sp.w), 0.f);
            if (lane == 0) {
                S.sbox[2 * (s0 + s)] = bl;
                S.sbox[2 * (s0 + s) + 1] = bh;
            }
            lo.x = fminf(lo.x, bl.x); lo.y = fminf(lo.y, bl.y); lo.z = fminf(lo.z, bl.z);
            hi.x = fmaxf(hi.x, bh.x); hi.y = fmaxf(hi.y, bh.y); hi.z = fmaxf(hi.z, bh.z);
        }
    }
    if (g == kGroups - 1) {
        while (f < d) {
            const float2 sc = S.sc[f * 32 + lane];
            frame_step_sc(F, sc.x, sc.y, S.dh[f], S.tw[f]);
            ++f;
        }
        *pose_out = pose_cost(F, S.goal, S.goal + 3, P.w_rot);
    }
    // with an arm-pair surrogate, the neighbours this lane needs (the same in
    // every warp) and those no lane needs, decided ahead (pair_bits)
    const unsigned need_nb = A.pair_mask ? S.need[lane] : ~0u;
    const unsigned skip_nb = A.pair_mask ? *S.skip : 0u;
    // the obstacle passes below need only the warp's own spheres and boxes:
    // they run before the barrier that publishes every group's centres to
    // the self pass, so a warp with a short kinematic chain spends the wait
    // for the longest one on its passes
    __syncwarp();
    if (cnt > 0) {
        // world boxes (exact): a box whose gap to the warp's box is at least
        // B_world + 1 mm is skipped (the signed distance of every own sphere
        // to it is at least that gap, outside the ramp); the others are
        // tested one per lane, then against every own sphere
        float mbox = kInf;
        for (int b0 = 0; b0 < n_aabb; b0 += 32) {
            const float tb = P.B_world + 1e-3f;
            bool nr = false;
            if (b0 + lane < n_aabb) {
                const float4 bc = S.aabb[2 * (b0 + lane)], bh = S.aabb[2 * (b0 + lane) + 1];
                const float gx = fmaxf(fmaxf(__fsub_rn(bc.x, bh.x) - hi.x, lo.x - __fadd_rn(bc.x, bh.x)), 0.f);
                const float gy = fmaxf(fmaxf(__fsub_rn(bc.y, bh.y) - hi.y, lo.y - __fadd_rn(bc.y, bh.y)), 0.f);
                const float gz = fmaxf(fmaxf(__fsub_rn(bc.z, bh.z) - hi.z, lo.z - __fadd_rn(bc.z, bh.z)), 0.f);
                nr = gx * gx + gy * gy + gz * gz < tb * tb;
            }
            unsigned box_near = __ballot_sync(0xffffffffu, nr);
            while (box_near) {
                const int b = b0 + __ffs(box_near) - 1;
                box_near &= box_near - 1u;
                const float4 bc = S.aabb[2 * b], bh = S.aabb[2 * b + 1];
#pragma unroll
                for (int s = 0; s < SPG; ++s)
                    if (s < cnt) {
                        const float4 o = S.own[(s0 + s) * 32 + lane];
                        mbox = fminf(mbox, sphere_aabb(make_float3(o.x, o.y, o.z), o.w, bc, bh));
                    }
            }
        }
        if (mbox < P.B_world) atomicMin(&S.red[lane], float_to_ordered(mbox));

        const float tw = __fadd_rn(P.B_world, kCullMargin), tn = __fadd_rn(P.B, kCullMargin);
        obstacle_pairs<SPG>(P, S, lo, hi, n_cl, n_world, tw, tn, skip_nb, s0, cnt, lane, need_nb,
                            S.cand + g * S.cand_cap);
    }

    // every group's centres and sphere boxes, and the block's obstacle pairs,
    // are in shared memory
    __syncthreads();

    // the obstacle pairs of every warp, split evenly over the warps
    {
        const int no = min(*S.opn, kObstaclePairCap);
        for (int i = g; i < no; i += kGroups) {
            const int2 e = S.opairs[i];
            obstacle_pair(P, S, e.x, __int_as_float(e.y), lane, need_nb);
        }
    }
    // self collision: the arm's pair list, split evenly over the 8 warps.  With
    // a learned surrogate, a rollout step whose predicted clearance is at least
    // B_self + margin skips the exact pass (its self term is zero); the warp
    // skips the loop when none of its 32 steps needs it.
    {
        bool need = true;
        if (A.learned)
            need = valid && D.dhat[A.off_kh + (long long)h * K + n] < P.B_self + A.self_margin;
        const int np = (!A.learned || __any_sync(0xffffffffu, need)) ? A.n_self : 0;
        // warp g takes pairs g, g + 8, g + 16, ... (interleaved, so that the
        // pairs near contact, which cluster in the list, spread over the
        // warps); 32 pairs at a time, one per lane, tested on the two spheres' boxes
        // over the sub-batch: a pair whose boxes are at least B_self + 1 mm
        // apart has every sample's spheres that far apart (each ball lies in
        // its box), outside the ramp, and is skipped (no result changes); the
        // exact test runs on the others, for every lane
        float m = kInf;
        const unsigned char *ownb = reinterpret_cast<const unsigned char *>(S.own) + lane * 16;
        const float tb = P.B_self + 1e-3f;
        for (int base = g; base < np; base += 32 * kGroups) {
            bool near = false;
            const int ip = base + kGroups * lane;
            if (ip < np) {
                const int o = S.pairs[ip].x;
                const int a1 = (o & 0xffff) >> 9, a2 = (int)((unsigned)o >> 25);
                const float4 l1 = S.sbox[2 * a1], h1 = S.sbox[2 * a1 + 1];
                const float4 l2 = S.sbox[2 * a2], h2 = S.sbox[2 * a2 + 1];
                const float gx = fmaxf(fmaxf(l2.x - h1.x, l1.x - h2.x), 0.f);
                const float gy = fmaxf(fmaxf(l2.y - h1.y, l1.y - h2.y), 0.f);
                const float gz = fmaxf(fmaxf(l2.z - h1.z, l1.z - h2.z), 0.f);
                near = gx * gx + gy * gy + gz * gz < tb * tb;
            }
            unsigned mk = __ballot_sync(0xffffffffu, near);
            while (mk) {
                const int i = base + kGroups * (__ffs(mk) - 1);
                mk &= mk - 1u;
                const int2 pr = S.pairs[i];
                const float4 c1 = *reinterpret_cast<const float4 *>(ownb + (pr.x & 0xffff));
                const float4 c2 = *reinterpret_cast<const float4 *>(ownb + ((unsigned)pr.x >> 16));
                pair_exact_t2(c1, c2, __int_as_float(pr.y), m);
            }
        }
        if (need && m < P.B_self) atomicMin(&S.red[1 * 32 + lane], float_to_ordered(m));
    }
}

// Per-block shared state read after the barrier that ends a sub-batch (the
// per-lane minima, the end-effector pose cost, the obstacle-pair count) is
// double-buffered by sub-batch parity, and the neighbour weights by
// work-unit parity, so that warp 0's per-sample cost of one sub-batch
// overlaps the other warps' next sub-batch (or the staging of the next
// unit) without a barrier between them; the own centres and the obstacle
// pairs are read only before that barrier and need one buffer.  The joint
// sines and cosines are double-buffered as well: each sub-batch computes the
// next one's behind its passes.  Two block barriers per sub-batch of 32
// samples (own centres and obstacle pairs written; minima complete), one
// more per work unit (inputs staged).  The next work unit's index is
// fetched one unit ahead.
//
// The kernel is built for three register budgets: MB resident blocks per SM
// (MB = 4: 64 registers per thread; MB = 3: 80; MB = 2: up to 128; none
// spills), compiled in separate translation units; the launch shape picks one.
// SIZES is the set of sphere-group sizes the build holds (bit s for size s):
// a build for the sizes the context's arms have (one or two group routines
// instead of eight) keeps the hot instruction footprint small; kAllSizes
// holds every size.
template <int MB, unsigned SIZES>
__global__ void __launch_bounds__(kRolloutThreads, MB) k_rollout(Params P, Dev D,
                                                                const RolloutTile *tiles,
                                                                int n_tiles, int iter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NA = P.n_arms;
    RolloutSmem S;
    const int red_stride = (2 + NA) * 32;
    {
        // the same layout as rollout_smem_bytes
        unsigned char *p = smraw;
        const size_t n_other = (size_t)rollout_other_cap(P, NA);
        const size_t n_cl = (size_t)rollout_cluster_cap(P, NA);
        S.other = (float4 *)p;     p += align16(sizeof(float4) * n_other);
        S.aabb = (float4 *)p;      p += align16(sizeof(float4) * 2 * P.aabb_cap);
        S.sph = (float4 *)p;       p += align16(sizeof(float4) * P.max_ns);
        S.own = (float4 *)p;       p += align16(sizeof(float4) * P.max_ns * 32);
        S.cbox = (float4 *)p;      p += align16(sizeof(float4) * 2 * n_cl);
        S.sbox = (float4 *)p;      p += align16(sizeof(float4) * 2 * P.max_ns);
        S.frame = (int *)p;        p += align16(sizeof(int) * P.max_ns);
        S.pairs = (int2 *)p;       p += align16(sizeof(int2) * P.max_pairs);
        S.cinfo = (int *)p;        p += align16(sizeof(int) * n_cl);
        S.nb_start = (int *)p;     p += align16(sizeof(int) * (MRS_MAX_ARMS + 1));
        S.nb_cstart = (int *)p;    p += align16(sizeof(int) * MRS_MAX_ARMS);
        S.nb_alpha = (float *)p;   p += align16(sizeof(float) * 2 * MRS_MAX_ARMS);
        S.nb_arm = (int *)p;       p += align16(sizeof(int) * MRS_MAX_ARMS);
        S.sc = (float2 *)p;        p += align16(sizeof(float2) * 2 * kMaxDof * 32);
        S.dh = (float4 *)p;        p += align16(sizeof(float4) * kMaxDof);
        S.tw = (float2 *)p;        p += align16(sizeof(float2) * kMaxDof);
        S.base = (float *)p;       p += align16(sizeof(float) * 12);
        S.goal = (float *)p;       p += align16(sizeof(float) * 12);
        S.seg = p;                 p += align16(n_other);
        S.cand = (unsigned short *)p;
        S.cand_cap = rollout_cand_cap(P, NA);
        p += align16(sizeof(unsigned short) * kGroups * S.cand_cap);
        S.opairs = (int2 *)p;      p += align16(sizeof(int2) * kObstaclePairCap);
        S.red = (int *)p;
    }
    float2 *const sc_base = S.sc;   // [2][kMaxDof][32] by sub-batch parity
    __shared__ int s_tile[2];
    __shared__ float s_pose[2][32];
    __shared__ float s_lim[32];   // the sub-batch's joint-limit terms, copied ahead by warp 0
    __shared__ long long s_idx[32];   // and each sample's stage-cost offset
    __shared__ float s_qn[kMaxDof * 32];   // the next sub-batch's joint angles, copied ahead
    __shared__ ArmHdr s_ah[2];    // the unit arm's scalars, by unit parity
    __shared__ int s_opn[2];      // obstacle pairs listed, by sub-batch parity
    __shared__ unsigned s_need[2][32], s_skip[2];   // pair_bits, by sub-batch parity
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_world = D.world_n[0], n_aabb = D.world_n[1];
    const int ncw = (n_world + 7) >> 3;   // world clusters
    const long long cycle = *D.cycle;

    // both minima buffers start at +inf; every sub-batch's cost stage resets
    // the entries it used, so they are +inf again when reused
    for (int k = threadIdx.x; k < 2 * red_stride; k += kRolloutThreads) S.red[k] = float_to_ordered(kInf);
    if (threadIdx.x < 2) {
        s_opn[threadIdx.x] = 0;
        s_skip[threadIdx.x] = 0u;
    }
    if (threadIdx.x < 64) s_need[threadIdx.x >> 5][threadIdx.x & 31] = ~0u;
    __shared__ __align__(8) uint64_t s_bar;   // completion of the plan-slice copies
    uint32_t bar_phase = 0;
    if (threadIdx.x == 0) {
        s_tile[0] = atomicAdd(&D.work[iter], 1);
        tc::mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    int buf = 0;   // sub-batch parity
    for (int it = 0;; ++it) {
        const int tp = it & 1;   // work-unit parity
        const int ti = s_tile[tp];
        if (ti >= n_tiles) break;
        if (threadIdx.x == kRolloutThreads - 1) s_tile[tp ^ 1] = atomicAdd(&D.work[iter], 1);
        const RolloutTile T = tiles[ti];
        const ArmDev &A = D.arms[T.arm];
        const int h = T.h;

        // the world at the step's time, the boxes, the arm's constants and its
        // self pairs, staged by warps 2 to 7 first (their loads overlap the
        // neighbour list below); warp 0 may still be in the previous unit's
        // cost stage and warp 1 issues the plan copies
        if (g >= 2) {
            constexpr int kStage = kRolloutThreads - 64;
            const int tl = (int)threadIdx.x - 64;
            const float t_h = __fmaf_rn((float)(h + 1), P.dt, *D.world_t);
            // the world spheres at the step's time, and the box of each
            // cluster of 8 (aligned groups of 8 lanes: the 192 staging
            // threads keep a sphere's index and its lane congruent mod 32)
            for (int k0 = tl - lane; k0 < n_world; k0 += kStage) {
                const int k = k0 + lane;
                float3 bl = make_float3(kInf, kInf, kInf), bh = make_float3(-kInf, -kInf, -kInf);
                if (k < n_world) {
                    const float4 o = D.world_s[k], v = D.world_vel_s[k];
                    const float4 w = make_float4(__fmaf_rn(v.x, t_h, o.x), __fmaf_rn(v.y, t_h, o.y),
                                                 __fmaf_rn(v.z, t_h, o.z), o.w);
                    S.other[k] = w;
                    bl = make_float3(w.x - w.w, w.y - w.w, w.z - w.w);
                    bh = make_float3(w.x + w.w, w.y + w.w, w.z + w.w);
                }
                cluster_box(bl, bh);
                if ((lane & 7) == 0 && k < n_world) {
                    S.cbox[2 * (k >> 3)] = make_float4(bl.x, bl.y, bl.z, 0.f);
                    S.cbox[2 * (k >> 3) + 1] = make_float4(bh.x, bh.y, bh.z, 0.f);
                    S.cinfo[k >> 3] = k | (min(8, n_world - k) << 16);
                }
            }
            for (int k = (tl + 128) % kStage; k < 2 * n_aabb; k += kStage) S.aabb[k] = D.aabb[k];
            {
                const int k = (tl + 96) % kStage;
                if (k < A.dof) {
                    S.dh[k] = A.dh[k];
                    S.tw[k] = A.twist[k];
                }
                if (k < 9) S.base[k] = A.base_R[k];
                else if (k < 12) S.base[k] = A.base_t[k - 9];
                else if (k < 24) S.goal[k - 12] = D.input[A.off_in + 2 * A.dof + k - 12];
            }
            if (tl == 191) {
                ArmHdr hd;
                hd.dof = A.dof; hd.K = A.K; hd.ns = A.ns; hd.n_self = A.n_self;
                hd.learned = A.learned; hd.H = A.H; hd.pair_mask = A.pair_mask;
                hd.pair_margin = A.pair_margin; hd.self_margin = A.self_margin; hd.spg = A.spg;
                hd.off_kh = A.off_kh; hd.off_khd = A.off_khd;
                s_ah[tp] = hd;
            }
            for (int k = (tl + 64) % kStage; k < A.ns; k += kStage) {
                S.sph[k] = A.sph[k];
                S.frame[k] = A.frame[k];
            }
            // self pairs as byte offsets of both spheres in the own buffer,
            // with their squared ramp bound
            for (int k = tl; k < A.n_self; k += kStage) {
                const int pr = D.self_pairs[A.self_off + k];
                S.pairs[k] = make_int2(((pr & 0xff) << 9) | ((pr >> 8) << 25),
                                       __float_as_int(D.self_t2[A.self_off + k]));
            }
        }

        // neighbour list (published plans whose horizon reaches step h), in
        // every warp: lane i decides for arm i
        bool ok = false;
        int ns_i = 0;
        {
            const int i = lane;
            if (i < NA && i != T.arm && h < D.arms[i].H &&   // min(H_j, H_i)
                plan_usable(P, D.board_valid[i], D.board_stamp[i], cycle)) {
                ok = true;
                ns_i = D.arms[i].ns;
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        const int nnb = __popc(mask);
        const int ncl_i = (ns_i + 7) >> 3;   // clusters of the neighbour's plan slice
        int incl = ns_i, inclc = ncl_i;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            const int vc = __shfl_up_sync(0xffffffffu, inclc, o);
            if (lane >= o) {
                incl += v;
                inclc += vc;
            }
        }
        const int pos = __popc(mask & ((1u << lane) - 1u));   // this lane's neighbour slot
        const int n_cl = ncw + __shfl_sync(0xffffffffu, inclc, 31);
        if (g == 1) {   // warp 0 may still be in the previous unit's cost stage
            if (ok) {
                S.nb_start[pos] = n_world + incl - ns_i;
                S.nb_cstart[pos] = ncw + inclc - ncl_i;
                S.nb_arm[pos] = lane;
            }
            if (lane == 31) S.nb_start[nnb] = n_world + incl;
        }
        // the neighbours' plan spheres at step h (one contiguous 16 N_S-byte
        // run per neighbour on the board, time-major) are copied into their
        // slots of S.other by the bulk-copy engine, issued by one thread of
        // warp 1 against one mbarrier
        const int n_plan = __shfl_sync(0xffffffffu, incl, 31);   // plan spheres of all neighbours
        if (g == 1 && n_plan > 0) {
            if (lane == 0) {
                tc::fence_async_smem();   // the previous unit's generic reads come first
                fused_bar_expect(&s_bar, (uint32_t)n_plan * 16u);
            }
            for (int nb = 0; nb < nnb; ++nb) {
                const int src = __fns(mask, 0, nb + 1);          // lane (= arm) of neighbour nb
                const int start = n_world + __shfl_sync(0xffffffffu, incl - ns_i, src);
                if (lane == 0) {
                    const ArmDev &Ai = D.arms[src];
                    bulk_load(&S.other[start], D.board_sph + (Ai.off_hs >> 2) + (size_t)h * Ai.ns,
                              (uint32_t)Ai.ns * 16u, &s_bar);
                }
            }
        }
        // the first sub-batch's joint sines and cosines (warp j takes joint j)
        // are staged with the unit, so the staging barrier also serves them
        if (it == 0) {     // the sampled trajectories, limit terms and priorities come from
            pdl_wait();    // the sample kernel
            pdl_trigger();
        }
        if (g == 1 && ok) S.nb_alpha[tp * MRS_MAX_ARMS + pos] = D.alpha[T.arm * NA + lane];
        if (A.pair_mask)   // the unit's first sub-batch's neighbour masks
            pair_masks(P, D, A, mask, nnb, h, T.n0 + lane, g, lane, s_need[buf], &s_skip[buf]);
        {
            const int n = T.n0 + lane;
            const bool valid = n < A.K;
            float2 *sc = sc_base + buf * (kMaxDof * 32);
            // joint j on warp (j + 1) mod 8: warp 0, still in the previous
            // unit's cost stage, takes a joint only for 8 or more
            for (int j = (g + kGroups - 1) % kGroups; j < A.dof; j += kGroups) {
                float sn, cs;
                const float qj = D.traj[A.off_khd + ((long long)h * A.dof + j) * A.K + (valid ? n : 0)];
                sincosf(__fadd_rn(qj, A.dh[j].w), &sn, &cs);
                sc[j * 32 + lane] = make_float2(sn, cs);
            }
        }
        if (n_plan > 0) {
            // bounded wait (P.wait_polls polls) for the plan copies, then the
            // derived layouts; if a copy did not land in time the block
            // records the error, waits (bounded, the full default limit) for
            // the copies still in flight and stops
            const bool landed = tc::mbar_wait(&s_bar, bar_phase, P.wait_polls);
            if (__syncthreads_or(!landed)) {
                if (threadIdx.x == 0) atomicExch(D.err, 1);
                tc::mbar_wait(&s_bar, bar_phase);
                return;
            }
            bar_phase ^= 1u;
            // the set of each neighbour's plan spheres and the box of each of
            // its clusters of 8 (counted from the slice's start), one warp per
            // neighbour
            for (int w = g; w < nnb; w += kGroups) {
                const int st = S.nb_start[w], en = S.nb_start[w + 1], cs = S.nb_cstart[w];
                for (int k0 = st; k0 < en; k0 += 32) {
                    const int k = k0 + lane;
                    float3 bl = make_float3(kInf, kInf, kInf), bh = make_float3(-kInf, -kInf, -kInf);
                    if (k < en) {
                        const float4 q = S.other[k];
                        S.seg[k] = (unsigned char)(2 + w);
                        bl = make_float3(q.x - q.w, q.y - q.w, q.z - q.w);
                        bh = make_float3(q.x + q.w, q.y + q.w, q.z + q.w);
                    }
                    cluster_box(bl, bh);
                    if ((lane & 7) == 0 && k < en) {
                        const int c = cs + ((k - st) >> 3);
                        S.cbox[2 * c] = make_float4(bl.x, bl.y, bl.z, 0.f);
                        S.cbox[2 * c + 1] = make_float4(bh.x, bh.y, bh.z, 0.f);
                        S.cinfo[c] = k | (min(8, en - k) << 16) | ((2 + w) << 20);
                    }
                }
            }
        }
        __syncthreads();   // the unit's inputs are staged
        const int n_nb = nnb;
        const ArmHdr &AH = s_ah[tp];   // staged above

        for (int sb = 0; sb < T.nsub; ++sb, buf ^= 1) {
            RolloutSmem Sb = S;
            Sb.red = S.red + buf * red_stride;
            Sb.sc = sc_base + buf * (kMaxDof * 32);
            Sb.opn = s_opn + buf;
            Sb.need = s_need[buf];
            Sb.skip = &s_skip[buf];
            const int n = T.n0 + sb * 32 + lane;
            const bool valid = n < AH.K;
            // warp 0 uses the sub-batch's stop / joint-limit terms in its cost
            // stage: copied to shared memory now, behind the kinematics
            if (g == 0 && valid) {
                const long long idx = AH.off_kh + (long long)h * AH.K + n;
                cp_async4(&s_lim[lane], D.stage_lim + idx);
                s_idx[lane] = idx;
            }
            // the next sub-batch's joint angles (warp j takes joint j), loaded
            // now and turned into sines and cosines after this sub-batch's
            // passes, into the other parity's buffer: the barrier that ends
            // this sub-batch publishes them (the first sub-batch's came with
            // the staging)
            const bool next = sb + 1 < T.nsub;
            if (next) {
                const int n_next = n + 32;
                const bool valid_next = n_next < AH.K;
                for (int j = (g + kGroups - 1) % kGroups; j < AH.dof; j += kGroups)
                    cp_async4(&s_qn[j * 32 + lane],
                              D.traj + AH.off_khd + ((long long)h * AH.dof + j) * AH.K +
                                  (valid_next ? n_next : 0));
            }
            const bool pm = AH.pair_mask != 0u;
            float pose = 0.f;
            // the group routine of the arm's size (only the sizes the build holds)
#define MRS_GROUP(SZ)                                                                          \
    if constexpr ((SIZES >> SZ) & 1u)                                                           \
        rollout_group<SZ>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, n_cl, &pose)
            if constexpr (single_size(SIZES) > 0)
                rollout_group<single_size(SIZES)>(P, D, AH, Sb, h, n, valid, g, lane, n_world,
                                                  n_aabb, n_nb, n_cl, &pose);
            else switch (AH.spg) {
                case 1: MRS_GROUP(1); break;
                case 2: MRS_GROUP(2); break;
                case 3: MRS_GROUP(3); break;
                case 4: MRS_GROUP(4); break;
                case 5: MRS_GROUP(5); break;
                case 6: MRS_GROUP(6); break;
                case 7: MRS_GROUP(7); break;
                default: MRS_GROUP(8); break;
            }
#undef MRS_GROUP
            if (g == kGroups - 1) s_pose[buf][lane] = pose;
            if (pm) {
                // every warp read this sub-batch's masks before the group's
                // first barrier: reset for their next use, two sub-batches on
                if (g == kGroups - 1) {
                    s_need[buf][lane] = ~0u;
                    if (lane == 0) s_skip[buf] = 0u;
                }
                if (next)   // the next sub-batch's masks, behind this one's passes
                    pair_masks(P, D, AH, mask, n_nb, h, n + 32, g, lane, s_need[buf ^ 1],
                               &s_skip[buf ^ 1]);
            }
            if (next) {
                float2 *sc = sc_base + (buf ^ 1) * (kMaxDof * 32);
                cp_async_wait_all();
                for (int j = (g + kGroups - 1) % kGroups; j < AH.dof; j += kGroups) {
                    float sn, cs;
                    sincosf(__fadd_rn(s_qn[j * 32 + lane], S.dh[j].w), &sn, &cs);
                    sc[j * 32 + lane] = make_float2(sn, cs);
                }
            }
            __syncthreads();   // every warp's minima, the pose cost and the next sines are in

            // stage cost of Eq. 5 plus the prioritised coordination term (Eq. 9)
            if (g == 0) {
                cp_async_wait_all();
                if (valid) {
                    const long long idx = s_idx[lane];
                    const float dw = ordered_to_float(Sb.red[0 * 32 + lane]);
                    const float dsf = ordered_to_float(Sb.red[1 * 32 + lane]);
                    float dyn = 0.f;   // neighbours in order; four loads in flight
#pragma unroll 4
                    for (int nb = 0; nb < n_nb; ++nb) {
                        const float rho = fmaxf(ordered_to_float(Sb.red[(2 + nb) * 32 + lane]), 0.f);
                        dyn = __fmaf_rn(S.nb_alpha[tp * MRS_MAX_ARMS + nb], ramp(rho, P.B), dyn);
                    }
                    float c = __fmul_rn(P.w_pose, s_pose[buf][lane]);
                    c = __fadd_rn(c, s_lim[lane]);
                    c = __fmaf_rn(P.w_coll, ramp(dw, P.B_world), c);
                    c = __fmaf_rn(P.w_self, ramp(dsf, P.B_self), c);
                    c = __fmaf_rn(P.w_dyn, dyn, c);
                    D.stage[idx] = c;
                }
                // this lane's minima are read: +inf again for their next use,
                // and the obstacle-pair list of this parity is empty again
                for (int k = lane; k < (2 + n_nb) * 32; k += 32) Sb.red[k] = float_to_ordered(kInf);
                if (lane == 0) *Sb.opn = 0;
            }
        }
    }
}

// Resident blocks per SM of variant MB from the kernel's own limits: shared
// memory (with the 1 KB the driver reserves per block), registers (allocated
// per warp in units of 256), threads.
template <int MB>
int rollout_occupancy_t(size_t smem)
{
    cudaFuncAttributes fa{};
    if (raise_smem_limit((const void *)k_rollout<MB, kAllSizes>, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_rollout<MB, kAllSizes>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_rollout<MB, kAllSizes>) != cudaSuccess)
        return 1;
    const int warps = kRolloutThreads / 32;
    const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int nb = (int)((228u * 1024u) / (smem + fa.sharedSizeBytes + 1024));
    nb = std::min(nb, 65536 / std::max(1, regs_per_warp * warps));
    nb = std::min(nb, 2048 / kRolloutThreads);
    return nb > 0 ? nb : 1;
}

template <int MB, unsigned SIZES>
cudaError_t rollout_configure_t(size_t smem)
{
    const cudaError_t e = raise_smem_limit((const void *)k_rollout<MB, SIZES>, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rollout<MB, SIZES>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
}

template <int MB, unsigned SIZES>
cudaError_t rollout_launch_t(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                             cudaStream_t s, bool pdl)
{
    const int grid = L.n_rollout_tiles < L.rollout_grid ? L.n_rollout_tiles : L.rollout_grid;
    return launch_k(k_rollout<MB, SIZES>, grid, kRolloutThreads, L.smem_rollout, s, pdl, P, D,
                    L.rollout_tiles, L.n_rollout_tiles, iter);
}

// the builds for a few sphere-group sizes (rollout_spg4.cu: 4, rollout_spg5.cu:
// 5, rollout_spg57.cu: 5 and 7), all three register budgets of each, chosen by
// the launch's variant; each build is used when it holds every arm's size
constexpr unsigned kSizes4 = 1u << 4, kSizes5 = 1u << 5, kSizes57 = (1u << 5) | (1u << 7);
cudaError_t rollout_configure_spg4(size_t smem);
cudaError_t rollout_launch_spg4(int variant, const Params &P, const Dev &D, const LaunchPlan &L,
                                int iter, cudaStream_t s, bool pdl);
cudaError_t rollout_configure_spg5(size_t smem);
cudaError_t rollout_launch_spg5(int variant, const Params &P, const Dev &D, const LaunchPlan &L,
                                int iter, cudaStream_t s, bool pdl);
cudaError_t rollout_configure_spg57(size_t smem);
cudaError_t rollout_launch_spg57(int variant, const Params &P, const Dev &D, const LaunchPlan &L,
                                 int iter, cudaStream_t s, bool pdl);

// the two- and four-blocks-per-SM variants (rollout_mb2.cu, rollout_mb4.cu)
int rollout_occupancy_mb2(size_t smem);
cudaError_t rollout_configure_mb2(size_t smem);
cudaError_t rollout_launch_mb2(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                               cudaStream_t s, bool pdl);
int rollout_occupancy_mb4(size_t smem);
cudaError_t rollout_configure_mb4(size_t smem);
cudaError_t rollout_launch_mb4(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                               cudaStream_t s, bool pdl);

}  // namespace mrs
