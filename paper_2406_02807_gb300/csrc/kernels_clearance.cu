// Differentiable clearance: nearest-point distance through the CAPT and the hinge cost.
//
// With r_min = 0 every leaf stores all points within r_max of its cell (Alg. 1, Lemma 1
// case 1), so for a centre x in that cell the nearest stored point is the nearest
// cloud point whenever it is within r_max.  The forward pass therefore scans the whole
// set (no early exit), keeping the minimum FP32 squared distance and its slot.
//
// Forward:
//  1. Distances (k_clearance_dist): one block per trajectory, each warp owning a
//     contiguous range of its waypoints (close in space, so the block's warps share set
//     blocks in L1); passes of 128 consecutive spheres (4 per lane, three 16-byte
//     loads): a sphere farther than r_max from the cloud's bounding box is farther than
//     r_max from every point, so it gets d = r_max, argmin = -1 at once (one 16-byte
//     store per output when all four of a lane's spheres are that far); the others are
//     queued.  Rounds of 32 queued spheres: descent and leaf box test against r_max;
//     each set of a sphere that passes is scanned in full by the whole warp in packed
//     FP32x2 arithmetic, every lane keeping a running minimum of (d^2, slot) keys,
//     reduced by two warp-wide 32-bit minimum reductions per set.  With the tree's
//     nearest-candidate lists (LISTS) a queued sphere first looks up its grid cell's
//     list and only the spheres of fallback cells take the descent and the set scan.
//  2. Costs, in a fixed order (lane-strided over the spheres, a butterfly, then the
//     waypoints in order), so the cost is bitwise reproducible whatever the launch
//     configuration: summed by the distance kernel's block after a block barrier (COST,
//     trajectories of at most kFusedCostMaxW waypoints), else by k_clearance_cost, one
//     warp per trajectory.
// Backward: elementwise, one thread per sphere, from the saved distance and argmin.
#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace capt {

constexpr int kClearQueue = 160;

struct ClearScratch {
    float4 nq[kClearQueue];          // queued spheres: centre
    unsigned long long ni[kClearQueue];   // their global sphere index
    // the round's entries (spheres whose leaf box is within r_max): centre, first block
    // and block count of the set
    float4 ec[32];
    uint32_t eb0[32];
    uint32_t enb[32];
};

// Blocks of one set scanned per lane per step: a set of up to 32 x kClearV blocks
// (the common case) takes one step, all its loads in flight together.
constexpr int kClearV = 3;

// Key of cloud point i for centre c on the nearest-candidate lists: the FP32 squared
// distance of the paper's scan (the same expression as block_d2, so the same bits) and
// the point index, so that the smallest key is the lowest-index nearest point.
__device__ __forceinline__ unsigned long long near_key(const float* __restrict__ cloud4, uint32_t i, const float4& c) {
    const float4 p = __ldg(reinterpret_cast<const float4*>(cloud4) + i);
    const float dx = __fsub_rn(p.x, c.x), dy = __fsub_rn(p.y, c.y), dz = __fsub_rn(p.z, c.z);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return ((unsigned long long)__float_as_uint(d2) << 32) | i;
}

// With LISTS, a queued sphere first looks up its grid cell's nearest-candidate list
// (capt_build_near_lists): an empty list answers r_max, -1; a list is scanned by the
// sphere's own lane, four entries per 16-byte load, and gives the paper's answer bit for
// bit (the argument is in dist_grid.cu); only the spheres of fallback cells go on below.
// One round over the first n queued spheres of the trajectory at `tbase` (sphere index
// offset of the trajectory in dist / argmin).  Each lane descends for its sphere and
// applies the leaf box test against r_max; spheres that fail get d = r_max at once, the
// others become entries.  Each entry's set is then scanned by the whole warp (lane l on
// blocks l, l + 32, l + 64 per step) keeping a running minimum of (d^2, slot) keys, and
// two 32-bit warp reductions (d^2, then the slot) give the smallest key, which lane e
// keeps for entry e.  The lowest key is the smallest FP32 squared distance, ties going
// to the lowest slot, i.e. the lowest point index.  Once every entry is scanned, lane e
// turns entry e's key into its distance and point index (the index loads of all entries
// in flight together) and writes them.
template <bool LISTS>
__device__ __forceinline__ void clearance_round(const DevArgs& t, const float* Ts, ClearScratch* ws, uint32_t n,
                                                uint64_t tbase, float rmax, float rmax2, float* __restrict__ dist,
                                                int32_t* __restrict__ argmin, uint32_t lane, uint32_t lt_mask) {
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    const bool live = lane < n;
    bool act = false;
    uint32_t nb = 0, fb = 0;
    uint64_t gi = 0;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    bool paper = live;
    if (live) {
        c = ws->nq[lane];
        gi = ws->ni[lane];
    }
    if constexpr (LISTS) {
        if (live) {
            bool inside;
            const uint2 rec = __ldg(reinterpret_cast<const uint2*>(t.nl_cell) + grid_cell(t.g, c.x, c.y, c.z, inside));
            if (rec.y != kNearFallback) {
                paper = false;
                unsigned long long best = ~0ull;
                const uint4* e = reinterpret_cast<const uint4*>(t.nl_cand + rec.x);
                for (uint32_t j = 0; j < rec.y / 4u; j++) {
                    const uint4 ix = __ldg(e + j);
                    const unsigned long long k0 = near_key(t.nl_cloud, ix.x, c), k1 = near_key(t.nl_cloud, ix.y, c);
                    const unsigned long long k2 = near_key(t.nl_cloud, ix.z, c), k3 = near_key(t.nl_cloud, ix.w, c);
                    const unsigned long long a01 = k0 < k1 ? k0 : k1, a23 = k2 < k3 ? k2 : k3;
                    const unsigned long long a4 = a01 < a23 ? a01 : a23;
                    best = a4 < best ? a4 : best;
                }
                const float dd = rec.y ? __fsqrt_rn(__uint_as_float((uint32_t)(best >> 32))) : rmax;
                if (dd < rmax) {
                    dist[tbase + gi] = dd;
                    argmin[tbase + gi] = (int32_t)(uint32_t)best;
                } else {
                    dist[tbase + gi] = rmax;
                    argmin[tbase + gi] = -1;
                }
            }
        }
    }
    if (paper) {
        const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
        float4 a, b;
        load_leaf(t.leaves, leaf, a, b);
        const uint32_t cnt = __float_as_uint(b.w);
        act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= rmax2;
        nb = act ? (cnt + 3u) >> 2 : 0u;
        fb = __float_as_uint(a.w);
        if (!act) {
            // every stored point is farther than r_max
            dist[tbase + gi] = rmax;
            argmin[tbase + gi] = -1;
        }
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, act);
    if (mask == 0) return;
    const uint32_t n_ent = __popc(mask);
    // entries in lane order; lane e later finishes entry e, so it takes that entry's
    // output index now
    const uint32_t pos = __popc(mask & lt_mask);
    __syncwarp();
    if (act) {
        ws->ec[pos] = c;
        ws->eb0[pos] = fb;
        ws->enb[pos] = nb;
    }
    uint32_t src_lane = 0;
    {
        // lane e < n_ent: the lane holding entry e is the e-th set bit of mask
        uint32_t mm = mask;
        for (uint32_t k = 0; k < lane && mm; k++) mm &= mm - 1;
        src_lane = mm ? (uint32_t)(__ffs(mm) - 1) : 0u;
    }
    const uint64_t my_gi = __shfl_sync(0xffffffffu, gi, src_lane);
    __syncwarp();
    unsigned long long mine = ~0ull;   // lane e: smallest key of entry e
    for (uint32_t e = 0; e < n_ent; e++) {
        const float4 ce = ws->ec[e];
        const uint32_t b0 = ws->eb0[e];
        const uint32_t nbs = ws->enb[e];
        const uint64_t cxx = f2_dup(ce.x), cyy = f2_dup(ce.y), czz = f2_dup(ce.z), z2 = f2_dup(t.nzero);
        unsigned long long best = ~0ull;
        for (uint32_t r = lane; r < nbs; r += 32 * kClearV) {
            uint64_t s01[kClearV], s23[kClearV];
#pragma unroll
            for (int v = 0; v < kClearV; v++) {
                s01[v] = s23[v] = ~0ull;
                if (r + 32u * v < nbs)
                    block_d2(blocks, t.plane, (int64_t)b0 + r + 32u * v, cxx, cyy, czz, z2, s01[v], s23[v]);
            }
#pragma unroll
            for (int v = 0; v < kClearV; v++) {
                if (r + 32u * v < nbs) {
                    const float2 d01 = f2_split(s01[v]), d23 = f2_split(s23[v]);
                    float bd = d01.x;
                    uint32_t bq = 0;
                    if (d01.y < bd) { bd = d01.y; bq = 1; }
                    if (d23.x < bd) { bd = d23.x; bq = 2; }
                    if (d23.y < bd) { bd = d23.y; bq = 3; }
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(bd) << 32) | (4u * (r + 32u * v) + bq);
                    best = key < best ? key : best;
                }
            }
        }
        // minimum key over the warp in two 32-bit reductions: the smallest d^2 (the bits
        // of a non-negative float order as unsigned integers), then the smallest slot
        // among the lanes that hold it
        const uint32_t hi = (uint32_t)(best >> 32);
        const uint32_t mhi = __reduce_min_sync(0xffffffffu, hi);
        const uint32_t mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? (uint32_t)best : 0xffffffffu);
        if (lane == e) mine = ((unsigned long long)mhi << 32) | mlo;
    }
    if (lane < n_ent) {
        const float dd = __fsqrt_rn(__uint_as_float((uint32_t)(mine >> 32)));
        const uint64_t i = tbase + my_gi;
        if (dd < rmax) {
            dist[i] = dd;
            argmin[i] = (int32_t)__ldg(t.ids + 4 * (size_t)ws->eb0[lane] + (uint32_t)(mine & 0xffffffffu));
        } else {
            dist[i] = rmax;
            argmin[i] = -1;
        }
    }
    __syncwarp();
}

// One pass over the spheres [p0, p0 + 128) of [.., s_hi) of the trajectory whose first
// sphere is tbase (4 per lane, three 16-byte loads): a sphere farther than r_max from
// the cloud's bounding box is farther than r_max from every point and gets d = r_max,
// argmin = -1 at once (one 16-byte store per output when all four of a lane's spheres
// are that far); the others are queued (centre and global index).
__device__ __forceinline__ void clearance_pass(const float* __restrict__ centers, uint64_t tbase, uint32_t p0,
                                               uint32_t s_hi, const float4& rlo, const float4& rhi, float rmax,
                                               float rmax2, float* __restrict__ dist, int32_t* __restrict__ argmin,
                                               ClearScratch* ws, uint32_t& n_q, uint32_t lane, uint32_t lt_mask) {
    const uint64_t i0 = tbase + p0 + 4 * lane;
    const uint32_t nv = p0 + 4 * lane < s_hi ? min(4u, s_hi - (p0 + 4 * lane)) : 0u;
    const float* src = centers + 3 * i0;
    float v[12];
    if (nv == 4 && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0)) {
        const float4* q = reinterpret_cast<const float4*>(src);
        const float4 a = __ldg(q), b = __ldg(q + 1), cc = __ldg(q + 2);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        v[8] = cc.x; v[9] = cc.y; v[10] = cc.z; v[11] = cc.w;
    } else {
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = (uint32_t)(k / 3) < nv ? __ldg(src + k) : 0.f;
    }
    bool nr[4];
#pragma unroll
    for (int k = 0; k < 4; k++)
        nr[k] = (uint32_t)k < nv && box_dist2(v[3 * k], v[3 * k + 1], v[3 * k + 2], rlo, rhi) <= rmax2;
    const bool all_far = nv == 4 && !(nr[0] | nr[1] | nr[2] | nr[3]) &&
                         ((reinterpret_cast<uintptr_t>(dist + i0) | reinterpret_cast<uintptr_t>(argmin + i0)) & 15u) == 0;
    if (all_far) {
        *reinterpret_cast<float4*>(dist + i0) = make_float4(rmax, rmax, rmax, rmax);
        *reinterpret_cast<int4*>(argmin + i0) = make_int4(-1, -1, -1, -1);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const bool near = nr[k];
        if ((uint32_t)k < nv && !near && !all_far) {
            dist[i0 + k] = rmax;
            argmin[i0 + k] = -1;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, near);
        if (near) {
            const uint32_t pos = n_q + __popc(mask & lt_mask);
            ws->nq[pos] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], 0.f);
            ws->ni[pos] = i0 + k;
        }
        n_q += __popc(mask);
    }
}

// Rounds of 32 while at least 32 spheres are queued; the rest moves to the front.
template <bool LISTS>
__device__ __forceinline__ void clearance_drain(const DevArgs& t, const float* Ts, ClearScratch* ws, uint32_t& n_q,
                                                float rmax, float rmax2, float* __restrict__ dist,
                                                int32_t* __restrict__ argmin, uint32_t lane, uint32_t lt_mask) {
    __syncwarp();
    uint32_t r0 = 0;
    for (; n_q - r0 >= 32; r0 += 32) {
        if (r0) {
            const float4 cc = ws->nq[r0 + lane];
            const unsigned long long ii = ws->ni[r0 + lane];
            __syncwarp();
            ws->nq[lane] = cc;
            ws->ni[lane] = ii;
            __syncwarp();
        }
        clearance_round<LISTS>(t, Ts, ws, 32, 0, rmax, rmax2, dist, argmin, lane, lt_mask);
    }
    const uint32_t rest = n_q - r0;
    float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned long long ii = 0;
    if (lane < rest) {
        cc = ws->nq[r0 + lane];
        ii = ws->ni[r0 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        ws->nq[lane] = cc;
        ws->ni[lane] = ii;
    }
    n_q = rest;
    __syncwarp();
}

// The cost term of one waypoint: sphere s = lane + 32 m (distances a for s = lane, b
// for s = lane + 32) summed by its lane, then a butterfly (every lane ends with it).
__device__ __forceinline__ float waypoint_term(float a, float b, int S, float rm0, float rm1, uint32_t lane) {
    float term = 0.f;
    if (lane < (uint32_t)S) {
        const float hh = fmaxf(0.f, __fsub_rn(rm0, a));
        term = __fadd_rn(term, __fmul_rn(hh, hh));
    }
    if (lane + 32 < (uint32_t)S) {
        const float hh = fmaxf(0.f, __fsub_rn(rm1, b));
        term = __fadd_rn(term, __fmul_rn(hh, hh));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term = __fadd_rn(term, __shfl_xor_sync(0xffffffffu, term, o));
    return term;
}

// Cost of one trajectory from its distances d[w S + s], in a fixed order: per waypoint,
// sphere s = lane + 32 m summed by its lane, then a butterfly; the waypoints are added
// in order (every lane ends with the same value).  Four waypoints' loads at a time.  NC:
// the distances were written by an earlier launch (read-only path); else by this warp.
template <bool NC>
__device__ __forceinline__ float trajectory_cost(const float* d, int W, int S, float rm0, float rm1, uint32_t lane) {
    float acc = 0.f;
    for (int w0 = 0; w0 < W; w0 += 4) {
        float a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            a[k] = b[k] = 0.f;
            const int w = w0 + k;
            if (w < W) {
                const float* dw = d + (uint64_t)w * (uint64_t)S;
                if (lane < (uint32_t)S) a[k] = NC ? __ldg(dw + lane) : dw[lane];
                if (lane + 32 < (uint32_t)S) b[k] = NC ? __ldg(dw + lane + 32) : dw[lane + 32];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (w0 + k >= W) break;
            acc = __fadd_rn(acc, waypoint_term(a[k], b[k], S, rm0, rm1, lane));
        }
    }
    return acc;
}

// With COST the block also sums its trajectory's cost once every distance is written:
// after a block barrier each warp forms the terms of its waypoints (trajectory_cost's
// per-waypoint arithmetic) into shared memory, and after a second one thread adds them
// in waypoint order, so the cost is bitwise that of k_clearance_cost.
template <bool STAGE, bool LISTS, bool COST>
__global__ void __launch_bounds__(512, 2) k_clearance_dist(DevArgs t, const float* __restrict__ centers, int W,
                                                           int S, float* __restrict__ dist,
                                                           int32_t* __restrict__ argmin, uint32_t pf_blocks,
                                                           const float* __restrict__ radii, float margin,
                                                           float* __restrict__ cost) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    // blocks start in about index order as earlier ones finish, so trajectory
    // blockIdx.x + pf_blocks is one that starts a few block-lifetimes from now: its
    // centres are fetched into L2 meanwhile
    if (pf_blocks && threadIdx.x == 0 && (uint64_t)blockIdx.x + pf_blocks < gridDim.x)
        prefetch_l2(centers + 3 * ((uint64_t)blockIdx.x + pf_blocks) * (uint64_t)W * (uint64_t)S,
                    (uint64_t)W * (uint64_t)S * 12u);
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);   // contains a block barrier
        off = stage_offset(t);
    }
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    ClearScratch* ws = reinterpret_cast<ClearScratch*>(smem_raw + off) + warp;
    const float rmax = t.r_max, rmax2 = __fmul_rn(t.r_max, t.r_max);
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    // one trajectory per block (the grid covers them all, so the hardware hands out
    // blocks as earlier ones finish); warp k owns a contiguous range of waypoints, whose
    // spheres are close in space, so the block's warps share set blocks in L1
    const uint64_t traj = blockIdx.x;
    const uint32_t w_lo = (uint32_t)(((uint64_t)W * warp) / nw), w_hi = (uint32_t)(((uint64_t)W * (warp + 1)) / nw);
    const uint64_t tbase = traj * (uint64_t)W * (uint64_t)S;        // first sphere of the trajectory
    const uint32_t s_lo = w_lo * (uint32_t)S, s_hi = w_hi * (uint32_t)S;   // this warp's spheres
    uint32_t n_q = 0;
    for (uint32_t p0 = s_lo; p0 < s_hi; p0 += 128) {
        clearance_pass(centers, tbase, p0, s_hi, rlo, rhi, rmax, rmax2, dist, argmin, ws, n_q, lane, lt_mask);
        if (n_q >= 32) clearance_drain<LISTS>(t, Ts, ws, n_q, rmax, rmax2, dist, argmin, lane, lt_mask);
    }
    if (n_q) {
        __syncwarp();
        clearance_round<LISTS>(t, Ts, ws, n_q, 0, rmax, rmax2, dist, argmin, lane, lt_mask);
    }
    if constexpr (COST) {
        float* wterm = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(ws - warp) +
                                                sizeof(ClearScratch) * (size_t)nw);
        __syncthreads();   // every distance of the trajectory written and visible to the block
        float rm0 = 0.f, rm1 = 0.f;
        if (lane < (uint32_t)S) rm0 = __fadd_rn(radii[lane], margin);
        if (lane + 32 < (uint32_t)S) rm1 = __fadd_rn(radii[lane + 32], margin);
        for (uint32_t w = w_lo; w < w_hi; w++) {
            const float* dw = dist + tbase + (uint64_t)w * (uint64_t)S;
            const float term = waypoint_term(lane < (uint32_t)S ? dw[lane] : 0.f,
                                             lane + 32 < (uint32_t)S ? dw[lane + 32] : 0.f, S, rm0, rm1, lane);
            if (lane == 0) wterm[w] = term;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.f;
            for (int w = 0; w < W; w++) acc = __fadd_rn(acc, wterm[w]);
            cost[traj] = acc;
        }
    }
}

// Cost per trajectory from the written distances, one warp per trajectory, in the order
// of trajectory_cost.  The result does not depend on the launch configuration.
__global__ void k_clearance_cost(const float* __restrict__ radii, const float* __restrict__ dist, uint64_t T, int W,
                                 int S, float margin, float* __restrict__ cost) {
    const uint32_t lane = lane_id();
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    float rm0 = 0.f, rm1 = 0.f;   // r_s + margin for s = lane, lane + 32
    if (lane < (uint32_t)S) rm0 = __fadd_rn(radii[lane], margin);
    if (lane + 32 < (uint32_t)S) rm1 = __fadd_rn(radii[lane + 32], margin);
    for (uint64_t traj = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); traj < T; traj += nwarps) {
        const float c = trajectory_cost<true>(dist + traj * (uint64_t)W * (uint64_t)S, W, S, rm0, rm1, lane);
        if (lane == 0) cost[traj] = c;
    }
}

__global__ void k_clearance_bwd(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii,
                                const float* __restrict__ dist, const int32_t* __restrict__ argmin,
                                const float* __restrict__ grad_cost, uint64_t T, int W, int S, float margin,
                                float* __restrict__ grad) {
    const uint64_t m = T * (uint64_t)W * (uint64_t)S;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % (uint64_t)S);
        const uint64_t traj = i / ((uint64_t)W * (uint64_t)S);
        const float d = __ldg(dist + i);
        const int32_t a = __ldg(argmin + i);
        const float h = fmaxf(0.f, __fsub_rn(__fadd_rn(__ldg(radii + s), margin), d));
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (h > 0.f && d < t.r_max && d > 0.f && a >= 0) {
            // d cost / d c = g * (-2 h) * (c - p*) / d
            const float k = __fdiv_rn(__fmul_rn(__fmul_rn(-2.f, h), __ldg(grad_cost + traj)), d);
            const float* p = t.cloud + 3 * (size_t)a;
            g0 = __fmul_rn(k, __fsub_rn(__ldg(centers + 3 * i), __ldg(p)));
            g1 = __fmul_rn(k, __fsub_rn(__ldg(centers + 3 * i + 1), __ldg(p + 1)));
            g2 = __fmul_rn(k, __fsub_rn(__ldg(centers + 3 * i + 2), __ldg(p + 2)));
        }
        grad[3 * i] = g0;
        grad[3 * i + 1] = g1;
        grad[3 * i + 2] = g2;
    }
}

// Sequential work count of the clearance forward, one thread per sphere, in the order
// the kernel's method defines it: every sphere gets the box test against the cloud's
// bounding box at r_max; a sphere within r_max of it descends and gets the leaf box
// test at r_max; a sphere passing that scans its whole set (no early exit: the
// nearest point is wanted).  counts += [spheres, spheres near the cloud box, spheres
// passing the leaf box, points scanned, blocks scanned (4 slots each)].  With LISTS the
// near spheres first look up their cell: counts[5] += those answered by a list (an
// empty one included), counts[6] += list entries scanned, counts[7] += those of
// fallback cells, and only these descend (entries 2-4 count their work).
__global__ void k_count_clearance(DevArgs t, const float* __restrict__ centers, uint64_t m, bool lists,
                                  unsigned long long* counts) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const float rmax2 = __fmul_rn(t.r_max, t.r_max);
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    if (i < m) {
        const float x = centers[3 * i], y = centers[3 * i + 1], z = centers[3 * i + 2];
        v[0] = 1;
        if (box_dist2(x, y, z, rlo, rhi) <= rmax2) {
            v[1] = 1;
            bool paper = true;
            if (lists) {
                bool inside;
                const uint2 rec = reinterpret_cast<const uint2*>(t.nl_cell)[grid_cell(t.g, x, y, z, inside)];
                if (rec.y != kNearFallback) {
                    paper = false;
                    v[5] = 1;
                    v[6] = rec.y;
                } else {
                    v[7] = 1;
                }
            }
            if (paper) {
                const uint32_t leaf = descend(x, y, z, t, nullptr);
                float4 a, b;
                load_leaf(t.leaves, leaf, a, b);
                const uint32_t cnt = __float_as_uint(b.w);
                if (cnt > 0 && box_dist2(x, y, z, a, b) <= rmax2) {
                    v[2] = 1;
                    v[3] = cnt;
                    v[4] = (cnt + 3u) / 4u;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0 && v[0]) {
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (v[k]) atomicAdd(counts + k, v[k]);
    }
}

int launch_count_clearance(const DevArgs& t, const float* centers, uint64_t m, bool lists, uint64_t* counts,
                           cudaStream_t st, std::string& err) {
    if (m == 0) return CAPT_OK;
    const unsigned threads = 256;
    k_count_clearance<<<(unsigned)((m + threads - 1) / threads), threads, 0, st>>>(
        t, centers, m, lists && t.nl_cell, reinterpret_cast<unsigned long long*>(counts));
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("clearance count launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

// Trajectories of at most this many waypoints get their cost in the distance kernel.
constexpr int kFusedCostMaxW = 1024;

int launch_clearance_fwd(const DevArgs& t, const float* centers, const float* radii, uint64_t T, int W, int S,
                         float margin, float* cost, float* dist, int32_t* argmin, const capt_launch_cfg& cfg,
                         cudaStream_t st, std::string& err) {
    if (T == 0) return CAPT_OK;
    if (W > 8192) { err = "clearance takes at most 8192 waypoints per trajectory"; return CAPT_E_ARG; }
    if (T > 0x7fffffffull) { err = "too many trajectories for one launch"; return CAPT_E_ARG; }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    const bool lists = cfg.grid && t.nl_cell;
    const bool fused = W <= kFusedCostMaxW;
    using Fn = void (*)(DevArgs, const float*, int, int, float*, int32_t*, uint32_t, const float*, float, float*);
    static const Fn table[8] = {k_clearance_dist<false, false, false>, k_clearance_dist<false, false, true>,
                                k_clearance_dist<false, true, false>,  k_clearance_dist<false, true, true>,
                                k_clearance_dist<true, false, false>,  k_clearance_dist<true, false, true>,
                                k_clearance_dist<true, true, false>,   k_clearance_dist<true, true, true>};
    const Fn fn = table[(stage ? 4 : 0) + (lists ? 2 : 0) + (fused ? 1 : 0)];
    const int warps = std::max(1, std::min(16, std::min((int)cfg.warps_per_block, W)));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(ClearScratch) * (size_t)warps +
                        (fused ? 4 * (size_t)W : 0u);
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    uint32_t pf_blocks = 0;
    if (cfg.prefetch > 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, warps * 32, smem);
        pf_blocks = (uint32_t)std::max(1, occ) * (uint32_t)sm_count() * (uint32_t)cfg.prefetch;
    }
    fn<<<(unsigned)T, warps * 32, smem, st>>>(t, centers, W, S, dist, argmin, pf_blocks, radii, margin, cost);
    if (!fused) {
        const uint64_t cost_blocks = std::min<uint64_t>((T + 7) / 8, (uint64_t)sm_count() * 16);
        k_clearance_cost<<<(unsigned)cost_blocks, 256, 0, st>>>(radii, dist, T, W, S, margin, cost);
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("clearance launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_clearance_bwd(const DevArgs& t, const float* centers, const float* radii, const float* dist,
                         const int32_t* argmin, const float* grad_cost, uint64_t T, int W, int S, float margin,
                         float* grad, cudaStream_t st, std::string& err) {
    const uint64_t m = T * (uint64_t)W * (uint64_t)S;
    if (m == 0) return CAPT_OK;
    const unsigned threads = 256;
    const uint64_t blocks = std::min<uint64_t>((m + threads - 1) / threads, (uint64_t)sm_count() * 16);
    k_clearance_bwd<<<(unsigned)blocks, threads, 0, st>>>(t, centers, radii, dist, argmin, grad_cost, T, W, S, margin,
                                                          grad);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("clearance bwd launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

}  // namespace capt
