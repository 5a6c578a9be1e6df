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
// lane; its centres stay in registers.  The samples per tile, the tile order
// and the resident blocks per SM are chosen at run time (mrs_autotune).
//
// Pair test.  A pair (own sphere c, radius r; other sphere p, radius r_p) can
// change a ramp cost max(0, 1 - dist/B) only if |c - p| < r + r_p + B.  With
//   g = |c - p|^2 - (r + B + r_p)^2
//     = [|p|^2 - r_p^2] - 2 c.p - 2 (r + B) r_p + [|c|^2 - (r + B)^2]
// the bracketed per-sphere terms are precomputed, so the inner loop is four
// FMAs and a min per pair, without branches, issued as packed f32x2
// instructions on two own spheres at a time.  An own sphere whose minimum g
// falls below eps_g (the FP32 cancellation margin of this expansion over the
// workspace) gets an exact pass: direct squared distance, and the square root
// only for pairs inside the ramp.  Since the cost is zero outside the ramp,
// the result equals the brute-force minimum of Eq. 6 restricted to the ramp.
#pragma once

#include <algorithm>

#include "kernels.cuh"
#include "tc_gemm.cuh"

// build-time knob of the pre-test loop
#ifndef MRS_PRETEST_UNROLL
#define MRS_PRETEST_UNROLL 1
#endif

namespace mrs {

constexpr int kPretestUnroll = MRS_PRETEST_UNROLL;

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
    float *other_w;    // |p|^2 - r_p^2 of each
    ulonglong2 *pa;    // packed pairs for the f32x2 pre-test: (x, x), (y, y)
    ulonglong2 *pb;    //                                      (z, z), (r, r)
    unsigned long long *pc;   //                               (w, w)
    float4 *aabb;      // [2 * n_aabb] centre, half extents
    float4 *sph;       // [ns] local centre + radius
    int *frame;        // [ns]
    int2 *pairs;       // [n_self] byte offsets of both spheres in own (o1 | o2 << 16),
                       // and (r1 + B_self + r2)^2 as float bits
    float4 *own;       // [ns][32] own sphere centre and radius of each sample
    int *red;          // [(2 + n_nb) * 32] ordered-int minima: world, self, neighbours
    int *nb_start;     // [n_nb + 1] ranges in `other` (after the world spheres)
    float *nb_alpha;   // [n_nb]
    int *nb_arm;       // [n_nb] arm index of each neighbour
    unsigned short *cand;   // [kGroups][cand_cap] per-warp candidate lists
    int cand_cap;
    float4 *sbox;           // [ns][2] per-sphere bounding box over the sub-batch: lo, hi
    float *box;             // [kGroups][8] per-warp bounding box: lo xyz, hi xyz
    float *marg;            // [2] cull margins 1 mm + eps_g / B of the world and plan passes
    float4 *nbbox;          // [2 * n_arms] box of each neighbour's plan spheres at the unit's step
    float2 *sc;             // [dof][32] sin, cos of q_j + theta_j of the sub-batch's samples
    float4 *dh;             // [kMaxDof] the arm's DH rows (a, d, alpha, theta)
    float2 *tw;             // [kMaxDof] sin, cos of the twists
    float *base;            // [12] base rotation (row-major) and translation
    float *goal;            // [12] the arm's goal position and rotation (sensed input)
};

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Capacity of a warp's candidate list: the largest single pass (the world
// spheres, or one neighbour's plan slice), rounded up to 8.
__host__ __device__ inline int rollout_cand_cap(const Params &P)
{
    const int m = P.world_cap > P.max_ns ? P.world_cap : P.max_ns;
    return (m + 7) & ~7;
}

// packed binary32 pairs (Blackwell f32x2 FMA: two lanes, each rounded exactly
// like the scalar instruction)
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// minimum of three (sm_100+ three-input min; exact, like fminf twice)
__device__ __forceinline__ float min3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
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

// store one other sphere (and its |p|^2 - r^2) in every layout the passes read
__device__ __forceinline__ void put_other(const RolloutSmem &S, int k, float4 w)
{
    const float pw = __fmaf_rn(w.z, w.z, __fmaf_rn(w.y, w.y, __fmaf_rn(w.x, w.x,
                                -__fmul_rn(w.w, w.w))));
    S.other[k] = w;
    S.other_w[k] = pw;
    S.pa[k] = make_ulonglong2(pack2(w.x, w.x), pack2(w.y, w.y));
    S.pb[k] = make_ulonglong2(pack2(w.z, w.z), pack2(w.w, w.w));
    S.pc[k] = pack2(pw, pw);
}

// the derived layouts of a sphere already in S.other[k] (a plan sphere
// copied there by the bulk-copy engine)
__device__ __forceinline__ void put_derived(const RolloutSmem &S, int k, float4 w)
{
    const float pw = __fmaf_rn(w.z, w.z, __fmaf_rn(w.y, w.y, __fmaf_rn(w.x, w.x,
                                -__fmul_rn(w.w, w.w))));
    S.other_w[k] = pw;
    S.pa[k] = make_ulonglong2(pack2(w.x, w.x), pack2(w.y, w.y));
    S.pb[k] = make_ulonglong2(pack2(w.z, w.z), pack2(w.w, w.w));
    S.pc[k] = pack2(pw, pw);
}

// exact distance of a candidate pair, as in the oracle: sqrt(d2) - r - r_p
__device__ __forceinline__ void pair_exact(float3 c, float rB, float r, float4 p, float &m)
{
    const float dx = __fsub_rn(p.x, c.x), dy = __fsub_rn(p.y, c.y), dz = __fsub_rn(p.z, c.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    const float t = __fadd_rn(rB, p.w);
    if (d2 < __fmul_rn(t, t)) m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), r), p.w));
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

// The same test for a self pair whose squared ramp bound (r1 + B + r2)^2 was
// computed beforehand with the same sums: sqrt(d2) - r1 - r2 when inside
__device__ __forceinline__ void pair_exact_t2(float4 c1, float4 c2, float t2, float &m)
{
    const float dx = __fsub_rn(c2.x, c1.x), dy = __fsub_rn(c2.y, c1.y), dz = __fsub_rn(c2.z, c1.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (d2 < t2) m = fminf(m, __fsub_rn(__fsub_rn(sqrtf(d2), c1.w), c2.w));
}

// Candidates of one pass: the other spheres in [k0, k1) that come within
// r_p + B + margin of the box bounding the warp's own spheres (each centre
// +- its radius, over the 32 lanes).  A sphere outside is farther than
// r + r_p + B + margin from every own sphere, so its pairs are outside the
// ramp and, with margin >= eps_g / B, also fail the pre-test: dropping them
// changes no result.  Warp-cooperative; returns the count (warp-uniform).
__device__ __forceinline__ int cull(const RolloutSmem &S, int k0, int k1, float B, float margin,
                                    const float *box, int lane, unsigned short *list)
{
    const float3 lo = make_float3(box[0], box[1], box[2]), hi = make_float3(box[3], box[4], box[5]);
    int nc = 0;
    for (int base = k0; base < k1; base += 32) {
        const int k = base + lane;
        bool keep = false;
        if (k < k1) {
            const float4 p = S.other[k];
            const float dx = fmaxf(fmaxf(lo.x - p.x, p.x - hi.x), 0.f);
            const float dy = fmaxf(fmaxf(lo.y - p.y, p.y - hi.y), 0.f);
            const float dz = fmaxf(fmaxf(lo.z - p.z, p.z - hi.z), 0.f);
            const float t = p.w + B + margin;
            keep = dx * dx + dy * dy + dz * dz < t * t;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) list[nc + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
        nc += __popc(m);
    }
    __syncwarp();
    return nc;
}

// Minimum signed distance, inside the ramp of buffer B, between the warp's
// own spheres and the candidates other[list[0 .. nc)).  Returns +inf when no
// pair is in the ramp.
// Own sphere centres arrive packed in pairs as -2c (NP = ceil(SPG / 2)); the
// pre-test runs on both spheres of a pair with one f32x2 FMA chain.
template <int NP>
__device__ __forceinline__ float clearance_pass(const RolloutSmem &S, const unsigned short *list,
                                                int nc, float B, float eps_g, int s0, int cnt,
                                                int lane, const f32x2 (&MX)[NP],
                                                const f32x2 (&MY)[NP], const f32x2 (&MZ)[NP])
{
    f32x2 MR[NP];
    float gmin[2 * NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int a = 2 * q, b = 2 * q + 1;
        const float ra = (a < cnt) ? -2.f * __fadd_rn(S.sph[s0 + a].w, B) : 0.f;
        const float rb = (b < cnt) ? -2.f * __fadd_rn(S.sph[s0 + b].w, B) : 0.f;
        MR[q] = pack2(ra, rb);
        gmin[a] = gmin[b] = kInf;
    }
    // two candidates per step: their values meet the running minimum in one
    // three-input min
    int i = 0;
#pragma unroll kPretestUnroll
    for (; i + 1 < nc; i += 2) {
        const int k = list[i], k1 = list[i + 1];
        const ulonglong2 A0 = S.pa[k], B0 = S.pb[k], A1 = S.pa[k1], B1 = S.pb[k1];
        const f32x2 W0 = S.pc[k], W1 = S.pc[k1];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float g0, g1, h0, h1;
            unpack2(fma2(MX[q], A0.x, fma2(MY[q], A0.y, fma2(MZ[q], B0.x, fma2(MR[q], B0.y, W0)))),
                    g0, g1);
            unpack2(fma2(MX[q], A1.x, fma2(MY[q], A1.y, fma2(MZ[q], B1.x, fma2(MR[q], B1.y, W1)))),
                    h0, h1);
            gmin[2 * q] = min3(gmin[2 * q], g0, h0);
            gmin[2 * q + 1] = min3(gmin[2 * q + 1], g1, h1);
        }
    }
    if (i < nc) {
        const int k = list[i];
        const ulonglong2 A = S.pa[k], Bv = S.pb[k];
        const f32x2 W = S.pc[k];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float g0, g1;
            unpack2(fma2(MX[q], A.x, fma2(MY[q], A.y, fma2(MZ[q], Bv.x, fma2(MR[q], Bv.y, W)))),
                    g0, g1);
            gmin[2 * q] = fminf(gmin[2 * q], g0);
            gmin[2 * q + 1] = fminf(gmin[2 * q + 1], g1);
        }
    }
    // own spheres whose pre-test minimum is within the margin of the ramp
    unsigned flagged = 0u;
#pragma unroll
    for (int s = 0; s < 2 * NP; ++s) {
        if (s < cnt) {
            // g = gmin + |c|^2 - (r + B)^2 with c = -m/2
            float x0, x1, y0, y1, z0, z1;
            unpack2(MX[s / 2], x0, x1);
            unpack2(MY[s / 2], y0, y1);
            unpack2(MZ[s / 2], z0, z1);
            const float cx = -0.5f * ((s & 1) ? x1 : x0), cy = -0.5f * ((s & 1) ? y1 : y0),
                        cz = -0.5f * ((s & 1) ? z1 : z0);
            const float rB = __fadd_rn(S.sph[s0 + s].w, B);
            const float ac = __fmaf_rn(cz, cz, __fmaf_rn(cy, cy, __fmaf_rn(cx, cx, -__fmul_rn(rB, rB))));
            if (__fadd_rn(gmin[s], ac) < eps_g) flagged |= 1u << s;
        }
    }
    // exact pass (rare): one loop for all flagged spheres, centres read back
    // from the warp's shared-memory copy
    float m = kInf;
    unsigned any = __ballot_sync(0xffffffffu, flagged != 0u);
    while (any) {
        unsigned bits = flagged;
        flagged = 0u;
        if (bits) {
            const int s = __ffs(bits) - 1;
            flagged = bits & (bits - 1u);
            const float4 o = S.own[(s0 + s) * 32 + lane];
            const float3 c = make_float3(o.x, o.y, o.z);
            const float r = S.sph[s0 + s].w;
            const float rB = __fadd_rn(r, B);
            for (int j = 0; j < nc; ++j) pair_exact(c, rB, r, S.other[list[j]], m);
        }
        any = __ballot_sync(0xffffffffu, flagged != 0u);
    }
    return m;
}

// centre of own sphere s from the packed -2c registers
template <int NP>
__device__ __forceinline__ float3 own_centre(const f32x2 (&MX)[NP], const f32x2 (&MY)[NP],
                                             const f32x2 (&MZ)[NP], int s)
{
    float x0, x1, y0, y1, z0, z1;
    unpack2(MX[s / 2], x0, x1);
    unpack2(MY[s / 2], y0, y1);
    unpack2(MZ[s / 2], z0, z1);
    return make_float3(-0.5f * ((s & 1) ? x1 : x0), -0.5f * ((s & 1) ? y1 : y0),
                       -0.5f * ((s & 1) ? z1 : z0));
}

// The same minimum for a few candidates: their exact distances to every own
// sphere, the square root only inside the ramp (for few candidates the
// pre-test and the flags of clearance_pass cost more than the exact tests;
// how few is the launch shape's exact_max).
template <int NP>
__device__ __forceinline__ float few_candidates(const RolloutSmem &S, const unsigned short *list,
                                                int nc, float B, int s0, int cnt,
                                                const f32x2 (&MX)[NP], const f32x2 (&MY)[NP],
                                                const f32x2 (&MZ)[NP])
{
    float m = kInf;
    for (int j = 0; j < nc; ++j) {
        const float4 p = S.other[list[j]];
#pragma unroll
        for (int s = 0; s < 2 * NP; ++s)
            if (s < cnt) {
                const float r = S.sph[s0 + s].w, rB = __fadd_rn(r, B);
                pair_exact(own_centre<NP>(MX, MY, MZ, s), rB, r, p, m);
            }
    }
    return m;
}

template <int SPG>
__device__ __forceinline__ void rollout_group(const Params &P, const Dev &D, const ArmHdr &A,
                                              const RolloutSmem &S, int h, int n, bool valid,
                                              int g, int lane, int n_world, int n_aabb, int n_nb,
                                              float *pose_out)
{
    const int d = A.dof, K = A.K;
    const int s0 = g * SPG;
    const int cnt = max(0, min(SPG, A.ns - s0));

    // DH chain up to the last frame this group needs; the last warp always
    // runs to the end effector for the pose cost.  Own centres are kept as
    // packed pairs of -2c (padding far away, never tested).
    constexpr int NP = (SPG + 1) / 2;
    f32x2 MX[NP], MY[NP], MZ[NP];
    Frame F;
#pragma unroll
    for (int k = 0; k < 9; ++k) F.R[k] = S.base[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) F.t[k] = S.base[9 + k];
    int f = 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float cx[2], cy[2], cz[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = 2 * q + u;
            if (s < cnt) {
                const int fs = S.frame[s0 + s];
                while (f < fs) {
                    const float2 sc = S.sc[f * 32 + lane];
                    frame_step_sc(F, sc.x, sc.y, S.dh[f], S.tw[f]);
                    ++f;
                }
                const float3 c = sphere_centre(F, S.sph[s0 + s]);
                cx[u] = -2.f * c.x; cy[u] = -2.f * c.y; cz[u] = -2.f * c.z;
                S.own[(s0 + s) * 32 + lane] = make_float4(c.x, c.y, c.z, S.sph[s0 + s].w);
            } else {
                cx[u] = cy[u] = cz[u] = -2e15f;
            }
        }
        MX[q] = pack2(cx[0], cx[1]);
        MY[q] = pack2(cy[0], cy[1]);
        MZ[q] = pack2(cz[0], cz[1]);
    }
    if (g == kGroups - 1) {
        while (f < d) {
            const float2 sc = S.sc[f * 32 + lane];
            frame_step_sc(F, sc.x, sc.y, S.dh[f], S.tw[f]);
            ++f;
        }
        *pose_out = pose_cost(F, S.goal, S.goal + 3, P.w_rot);
    }

    // box bounding each own sphere (centre +- radius) over the warp's 32
    // samples (warp-wide floating-point min / max), kept for the self pass,
    // and their union: the warp's box
    float3 lo = make_float3(kInf, kInf, kInf), hi = make_float3(-kInf, -kInf, -kInf);
    unsigned short *list = S.cand + g * S.cand_cap;
    float *box = S.box + g * 8;
    if (cnt > 0) {
#pragma unroll
        for (int s = 0; s < SPG; ++s)
            if (s < cnt) {
                const float3 c = own_centre<NP>(MX, MY, MZ, s);
                const float r = S.sph[s0 + s].w;
                const float4 bl = make_float4(warp_min(c.x - r), warp_min(c.y - r), warp_min(c.z - r), 0.f);
                const float4 bh = make_float4(warp_max(c.x + r), warp_max(c.y + r), warp_max(c.z + r), 0.f);
                if (lane == 0) {
                    S.sbox[2 * (s0 + s)] = bl;
                    S.sbox[2 * (s0 + s) + 1] = bh;
                }
                lo.x = fminf(lo.x, bl.x); lo.y = fminf(lo.y, bl.y); lo.z = fminf(lo.z, bl.z);
                hi.x = fmaxf(hi.x, bh.x); hi.y = fmaxf(hi.y, bh.y); hi.z = fmaxf(hi.z, bh.z);
            }
        if (lane == 0) {
            box[0] = lo.x; box[1] = lo.y; box[2] = lo.z;
            box[3] = hi.x; box[4] = hi.y; box[5] = hi.z;
        }
    }
    // the obstacle passes below need only the warp's own spheres and box:
    // they run before the barrier that publishes every group's centres to
    // the self pass, so a warp with a short kinematic chain spends the wait
    // for the longest one on its passes
    __syncwarp();
    if (cnt > 0) {

        // world boxes (exact), then one pre-tested pass per sphere set over its
        // candidates: the world spheres (slot 0, buffer B_world) and each
        // published neighbour plan at this step (slot 2 + nb, buffer B)
        // A box whose gap to the warp's bounding box is at least B_world +
        // 1 mm is skipped: the signed distance of every own sphere to it is
        // at least that gap (the sphere lies inside the warp box by its
        // radius along each separating axis), so it is outside the ramp and
        // changes no result.
        // the world boxes and the neighbours' plan boxes near enough to
        // matter, tested one per lane; the others are skipped
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
                    if (s < cnt)
                        mbox = fminf(mbox, sphere_aabb(own_centre<NP>(MX, MY, MZ, s), S.sph[s0 + s].w,
                                                       bc, bh));
            }
        }
        unsigned nb_near;   // at most 31 neighbours
        {
            const float tn = P.B + S.marg[1];
            bool nr = false;
            if (lane < n_nb) {
                const float4 pl = S.nbbox[2 * lane], ph = S.nbbox[2 * lane + 1];
                const float gx = fmaxf(fmaxf(pl.x - hi.x, lo.x - ph.x), 0.f);
                const float gy = fmaxf(fmaxf(pl.y - hi.y, lo.y - ph.y), 0.f);
                const float gz = fmaxf(fmaxf(pl.z - hi.z, lo.z - ph.z), 0.f);
                nr = gx * gx + gy * gy + gz * gz < tn * tn;
            }
            nb_near = __ballot_sync(0xffffffffu, nr);
        }
        for (int ps = 0; ps <= n_nb; ++ps) {
            const bool world = ps == 0;
            const int k0 = world ? 0 : S.nb_start[ps - 1];
            const int k1 = world ? n_world : S.nb_start[ps];
            const float Bp = world ? P.B_world : P.B;
            // with an arm-pair surrogate, a step whose predicted clearance to
            // this neighbour's plan is at least B + margin skips the exact
            // pass (its coordination term is zero); a plan published without
            // joints always takes the exact pass
            // a neighbour whose plan box is at least B + margin from the warp's
            // box has every plan sphere culled: no candidate, no term
            if (!world && !((nb_near >> (ps - 1)) & 1u)) continue;
            bool need = true;
            if (!world) {
                const int ai = S.nb_arm[ps - 1];
                if ((A.pair_mask >> ai) & 1u)
                    need = valid && (D.board_valid[ai] != 1 ||
                                     D.rhohat[A.off_kh * P.n_arms + (long long)ai * A.H * K +
                                              (long long)h * K + n] < P.B + A.pair_margin);
                if (!__any_sync(0xffffffffu, need)) continue;
            }
            const int nc = cull(S, k0, k1, Bp, world ? S.marg[0] : S.marg[1], box, lane, list);
            // nc is warp-uniform
            float m = nc > P.exact_max
                          ? clearance_pass<NP>(S, list, nc, Bp, P.eps_g, s0, cnt, lane, MX, MY, MZ)
                      : nc > 0 ? few_candidates<NP>(S, list, nc, Bp, s0, cnt, MX, MY, MZ)
                               : kInf;
            if (world) m = fminf(m, mbox);
            if (need && m < Bp)
                atomicMin(&S.red[(world ? 0 : ps + 1) * 32 + lane], float_to_ordered(m));
        }
    }

    // every group's centres and sphere boxes are in shared memory
    __syncthreads();

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
// per-lane minima, the end-effector pose cost) is double-buffered by
// sub-batch parity, and the neighbour weights by work-unit parity, so that
// warp 0's per-sample cost of one sub-batch overlaps the other warps' next
// sub-batch (or the staging of the next unit) without a barrier between
// them; the own centres are read only before that barrier and need one
// buffer.  The joint sines and cosines are double-buffered as well: each
// sub-batch computes the next one's behind its passes.  Two block barriers
// per sub-batch of 32 samples (own centres written; minima complete), one
// more per work unit (inputs staged).  The next work unit's index is
// fetched one unit ahead.
//
// The kernel is built for two register budgets: MB resident blocks per SM
// (MB = 3: 80 registers per thread; MB = 2: up to 128, no spills), compiled
// in separate translation units; the launch shape picks one.
template <int MB>
__global__ void __launch_bounds__(kRolloutThreads, MB) k_rollout(Params P, Dev D,
                                                                const RolloutTile *tiles,
                                                                int n_tiles, int iter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NA = P.n_arms;
    RolloutSmem S;
    const int red_stride = (2 + NA) * 32;
    {
        unsigned char *p = smraw;
        const size_t n_other = (size_t)P.world_cap + (size_t)P.max_ns * NA;
        S.other = (float4 *)p;     p += align16(sizeof(float4) * n_other);
        S.aabb = (float4 *)p;      p += align16(sizeof(float4) * 2 * P.aabb_cap);
        S.sph = (float4 *)p;       p += align16(sizeof(float4) * P.max_ns);
        S.own = (float4 *)p;       p += align16(sizeof(float4) * P.max_ns * 32);
        S.other_w = (float *)p;    p += align16(sizeof(float) * n_other);
        S.pa = (ulonglong2 *)p;    p += align16(sizeof(ulonglong2) * n_other);
        S.pb = (ulonglong2 *)p;    p += align16(sizeof(ulonglong2) * n_other);
        S.pc = (unsigned long long *)p; p += align16(sizeof(unsigned long long) * n_other);
        S.frame = (int *)p;        p += align16(sizeof(int) * P.max_ns);
        S.pairs = (int2 *)p;       p += align16(sizeof(int2) * P.max_pairs);
        S.nb_start = (int *)p;     p += align16(sizeof(int) * (MRS_MAX_ARMS + 1));
        S.nb_alpha = (float *)p;   p += align16(sizeof(float) * 2 * MRS_MAX_ARMS);
        S.nb_arm = (int *)p;       p += align16(sizeof(int) * MRS_MAX_ARMS);
        S.sbox = (float4 *)p;      p += align16(sizeof(float4) * 2 * P.max_ns);
        S.box = (float *)p;        p += align16(sizeof(float) * kGroups * 8);
        S.marg = (float *)p;       p += align16(sizeof(float) * 2);
        S.nbbox = (float4 *)p;     p += align16(sizeof(float4) * 2 * NA);
        S.sc = (float2 *)p;        p += align16(sizeof(float2) * 2 * kMaxDof * 32);
        S.dh = (float4 *)p;        p += align16(sizeof(float4) * kMaxDof);
        S.tw = (float2 *)p;        p += align16(sizeof(float2) * kMaxDof);
        S.base = (float *)p;       p += align16(sizeof(float) * 12);
        S.goal = (float *)p;       p += align16(sizeof(float) * 12);
        S.cand = (unsigned short *)p;
        S.cand_cap = rollout_cand_cap(P);
        p += align16(sizeof(unsigned short) * kGroups * S.cand_cap);
        S.red = (int *)p;
    }
    float2 *const sc_base = S.sc;   // [2][kMaxDof][32] by sub-batch parity
    __shared__ int s_tile[2];
    __shared__ float s_pose[2][32];
    __shared__ float s_lim[32];   // the sub-batch's joint-limit terms, copied ahead by warp 0
    __shared__ long long s_idx[32];   // and each sample's stage-cost offset
    __shared__ float s_qn[kMaxDof * 32];   // the next sub-batch's joint angles, copied ahead
    __shared__ ArmHdr s_ah[2];    // the unit arm's scalars, by unit parity
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_world = D.world_n[0], n_aabb = D.world_n[1];
    const long long cycle = *D.cycle;

    // both minima buffers start at +inf; every sub-batch's cost stage resets
    // the entries it used, so they are +inf again when reused
    for (int k = threadIdx.x; k < 2 * red_stride; k += kRolloutThreads) S.red[k] = float_to_ordered(kInf);
    __shared__ __align__(8) uint64_t s_bar;   // completion of the plan-slice copies
    uint32_t bar_phase = 0;
    if (threadIdx.x == 1) {
        S.marg[0] = 1e-3f + P.eps_g / P.B_world;
        S.marg[1] = 1e-3f + P.eps_g / P.B;
    }
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
            for (int k = tl; k < n_world; k += kStage) {
                const float4 o = D.world[k], v = D.world_vel[k];
                put_other(S, k, make_float4(__fmaf_rn(v.x, t_h, o.x), __fmaf_rn(v.y, t_h, o.y),
                                            __fmaf_rn(v.z, t_h, o.z), o.w));
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
        int incl = ns_i;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int pos = __popc(mask & ((1u << lane) - 1u));   // this lane's neighbour slot
        if (g == 1) {   // warp 0 may still be in the previous unit's cost stage
            if (ok) {
                S.nb_start[pos] = n_world + incl - ns_i;
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
            for (int k = threadIdx.x; k < n_plan; k += blockDim.x)
                put_derived(S, n_world + k, S.other[n_world + k]);
            // box of each neighbour's plan spheres (centre +- radius), one warp
            // per neighbour
            for (int w = g; w < nnb; w += kGroups) {
                float3 bl = make_float3(kInf, kInf, kInf), bh = make_float3(-kInf, -kInf, -kInf);
                for (int k = S.nb_start[w] + lane; k < S.nb_start[w + 1]; k += 32) {
                    const float4 q = S.other[k];
                    bl.x = fminf(bl.x, q.x - q.w); bl.y = fminf(bl.y, q.y - q.w); bl.z = fminf(bl.z, q.z - q.w);
                    bh.x = fmaxf(bh.x, q.x + q.w); bh.y = fmaxf(bh.y, q.y + q.w); bh.z = fmaxf(bh.z, q.z + q.w);
                }
                const float4 l4 = make_float4(warp_min(bl.x), warp_min(bl.y), warp_min(bl.z), 0.f);
                const float4 h4 = make_float4(warp_max(bh.x), warp_max(bh.y), warp_max(bh.z), 0.f);
                if (lane == 0) {
                    S.nbbox[2 * w] = l4;
                    S.nbbox[2 * w + 1] = h4;
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
            float pose = 0.f;
            switch (AH.spg) {
                case 1: rollout_group<1>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 2: rollout_group<2>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 3: rollout_group<3>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 4: rollout_group<4>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 5: rollout_group<5>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 6: rollout_group<6>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                case 7: rollout_group<7>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
                default: rollout_group<8>(P, D, AH, Sb, h, n, valid, g, lane, n_world, n_aabb, n_nb, &pose); break;
            }
            if (g == kGroups - 1) s_pose[buf][lane] = pose;
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
                    float dyn = 0.f;
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
                // this lane's minima are read: +inf again for their next use
                for (int k = lane; k < (2 + n_nb) * 32; k += 32) Sb.red[k] = float_to_ordered(kInf);
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
    if (raise_smem_limit((const void *)k_rollout<MB>, smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_rollout<MB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_rollout<MB>) != cudaSuccess)
        return 1;
    const int warps = kRolloutThreads / 32;
    const int regs_per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int nb = (int)((228u * 1024u) / (smem + fa.sharedSizeBytes + 1024));
    nb = std::min(nb, 65536 / std::max(1, regs_per_warp * warps));
    nb = std::min(nb, 2048 / kRolloutThreads);
    return nb > 0 ? nb : 1;
}

template <int MB>
cudaError_t rollout_configure_t(size_t smem)
{
    return raise_smem_limit((const void *)k_rollout<MB>, smem);
}

template <int MB>
cudaError_t rollout_launch_t(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                             cudaStream_t s, bool pdl)
{
    const int grid = L.n_rollout_tiles < L.rollout_grid ? L.n_rollout_tiles : L.rollout_grid;
    return launch_k(k_rollout<MB>, grid, kRolloutThreads, L.smem_rollout, s, pdl, P, D,
                    L.rollout_tiles, L.n_rollout_tiles, iter);
}

// the two-blocks-per-SM variant (rollout_mb2.cu)
int rollout_occupancy_mb2(size_t smem);
cudaError_t rollout_configure_mb2(size_t smem);
cudaError_t rollout_launch_mb2(const Params &P, const Dev &D, const LaunchPlan &L, int iter,
                               cudaStream_t s, bool pdl);

}  // namespace mrs
