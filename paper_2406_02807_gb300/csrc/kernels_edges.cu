// Batched edge validation: the configuration-level early exit of Sec. IV-D applied to
// whole straight-line edges, with the interpolated configurations and their sphere
// centres generated inside the kernel.
//
// A warp validates up to 32 consecutive configurations of one edge per pass, one per
// lane: each lane interpolates its configuration, walks the arm's kinematic chain in
// FP32 and, as each sphere centre appears, applies the root box test (the bounding box
// of the cloud contains every affordance set, so a sphere that misses it misses every
// point).  Spheres that come near the cloud are queued in shared memory and processed
// in rounds of 32 (descent, leaf box test, load-balanced scan, scan.cuh); the first
// hit invalidates the edge and ends the pass.
//
// Persistent mode: work items are (edge, chunk of configurations), enumerated edge by
// edge; the chunks of an edge interleave its configurations (item ci of nci takes every
// nci-th one from ci), so that the first items in flight sample the whole edge.  A
// setup kernel writes the exclusive prefix of the per-edge item counts and resets the
// work counter and the validity flags; the persistent kernel's warps take
// items from the counter with one atomic each and skip items of edges already known to
// collide.  capt_edge_plan_create captures both launches into a CUDA graph.
// Per-edge mode (the baseline): one kernel launch per edge.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace capt {

// The arm as the kernels read it: spheres ordered by the link they hang on, so that a
// lane can place each link's spheres right after rotating that link's frame.
struct ArmPlan {
    int32_t J, S;
    float base[3];
    int32_t axis[CAPT_MAX_JOINTS];
    float link[CAPT_MAX_JOINTS][3];
    int32_t sbeg[CAPT_MAX_JOINTS + 1];   // spheres of link j: [sbeg[j], sbeg[j + 1])
    float off[CAPT_MAX_SPHERES][3];      // offsets in the link frame, in that order
    float r2[CAPT_MAX_SPHERES];          // fl(r * r), in that order
    float rr[CAPT_MAX_SPHERES];          // r, in that order (for the distance-bound grid)
    // per link: a bounding sphere of its spheres (centre offset in the link frame) and
    // the squared box distance beyond which none of them can reach the cloud's box
    float cull_o[CAPT_MAX_JOINTS][3];
    float cull_t[CAPT_MAX_JOINTS];
};


ArmPlan make_plan(const capt_arm& a) {
    ArmPlan p{};
    p.J = a.n_joints;
    p.S = a.n_spheres;
    for (int d = 0; d < 3; d++) p.base[d] = a.base[d];
    for (int j = 0; j < a.n_joints; j++) {
        p.axis[j] = a.axis[j];
        for (int d = 0; d < 3; d++) p.link[j][d] = a.link[j][d];
    }
    int n = 0;
    for (int j = 0; j < a.n_joints; j++) {
        p.sbeg[j] = n;
        for (int s = 0; s < a.n_spheres; s++)
            if (a.sphere_link[s] == j) {
                for (int d = 0; d < 3; d++) p.off[n][d] = a.sphere_offset[s][d];
                p.r2[n] = a.sphere_radius[s] * a.sphere_radius[s];
                p.rr[n] = a.sphere_radius[s];
                n++;
            }
    }
    p.sbeg[a.n_joints] = n;
    // Link culling bound.  The FP32 centre of sphere s lies within |o_s - o_b| of the
    // FP32 centre of the bounding point o_b up to rounding (R is orthonormal to a few
    // ulps after at most 16 rotations), so a sphere whose FP32 box test passes has its
    // bounding point within rho = max_s(|o_s - o_b| + r_s) of the box, plus rounding;
    // delta = 1e-4 (1 + M), with M a bound on every coordinate the chain produces, is
    // orders of magnitude above that rounding.  A lane whose bounding point is farther
    // than rho + delta (squared, with a relative margin) has no sphere of the link near.
    double M = 1.0;
    for (int d = 0; d < 3; d++) M += std::fabs((double)a.base[d]);
    for (int j = 0; j < a.n_joints; j++)
        M += std::fabs((double)a.link[j][0]) + std::fabs((double)a.link[j][1]) + std::fabs((double)a.link[j][2]);
    double omax = 0.0;
    for (int i = 0; i < n; i++)
        omax = std::max(omax, std::fabs((double)p.off[i][0]) + std::fabs((double)p.off[i][1]) +
                                  std::fabs((double)p.off[i][2]) + std::sqrt((double)p.r2[i]));
    M += omax;
    const double delta = 1e-4 * M;
    for (int j = 0; j < a.n_joints; j++) {
        p.cull_t[j] = INFINITY;
        p.cull_o[j][0] = p.cull_o[j][1] = p.cull_o[j][2] = 0.f;
        if (p.sbeg[j + 1] == p.sbeg[j]) continue;
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = p.sbeg[j]; i < p.sbeg[j + 1]; i++)
            for (int d = 0; d < 3; d++) {
                lo[d] = std::min(lo[d], (double)p.off[i][d]);
                hi[d] = std::max(hi[d], (double)p.off[i][d]);
            }
        double ob[3];
        for (int d = 0; d < 3; d++) {
            p.cull_o[j][d] = (float)((lo[d] + hi[d]) / 2);
            ob[d] = p.cull_o[j][d];
        }
        double rho = 0.0;
        for (int i = p.sbeg[j]; i < p.sbeg[j + 1]; i++) {
            const double dx = p.off[i][0] - ob[0], dy = p.off[i][1] - ob[1], dz = p.off[i][2] - ob[2];
            rho = std::max(rho, std::sqrt(dx * dx + dy * dy + dz * dz) + std::sqrt((double)p.r2[i]));
        }
        const double tt = (rho + delta) * (rho + delta) * (1.0 + 1e-5);
        p.cull_t[j] = std::isfinite(tt) ? std::nextafter((float)tt, INFINITY) : INFINITY;
    }
    return p;
}

// sin and cos of x in FP32 by Cody-Waite reduction modulo pi/2 (Cody and Waite,
// "Software Manual for the Elementary Functions", 1980) and Taylor polynomials on
// [-pi/4, pi/4] (sin to degree 9, cos to degree 10), every step rounded separately.
// pi/2 = 1.5703125 + 4.837512969970703125e-4 + 7.549790126404332e-8, the first two
// with 12 significant bits so k * piece is exact for |k| < 2^12.
__device__ __forceinline__ void sincos_cw(float x, float& so, float& co) {
    const float kf = rintf(__fmul_rn(x, 0.636619746685f));
    float r = __fsub_rn(x, __fmul_rn(kf, 1.5703125f));
    r = __fsub_rn(r, __fmul_rn(kf, 4.837512969970703125e-4f));
    r = __fsub_rn(r, __fmul_rn(kf, 7.549790126404332e-8f));
    const float r2 = __fmul_rn(r, r);
    float ps = 2.7557318844628753e-6f;
    ps = __fsub_rn(__fmul_rn(ps, r2), 1.9841270113829523e-4f);
    ps = __fadd_rn(__fmul_rn(ps, r2), 8.333333767950535e-3f);
    ps = __fsub_rn(__fmul_rn(ps, r2), 0.1666666716337204f);
    const float s = __fadd_rn(r, __fmul_rn(__fmul_rn(r, r2), ps));
    float pc = -2.755731998149713e-7f;
    pc = __fadd_rn(__fmul_rn(pc, r2), 2.4801587642286904e-5f);
    pc = __fsub_rn(__fmul_rn(pc, r2), 1.3888889225199819e-3f);
    pc = __fadd_rn(__fmul_rn(pc, r2), 4.16666679084301e-2f);
    pc = __fsub_rn(__fmul_rn(pc, r2), 0.5f);
    const float c = __fadd_rn(1.0f, __fmul_rn(r2, pc));
    const int q = ((int)kf) & 3;
    so = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
    co = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}

// R <- R * Rot(axis, q): columns A and B (in right-handed order around the axis) mix.
template <int A, int B>
__device__ __forceinline__ void rotate_cols(float R[9], float s, float c) {
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const float ca = R[3 * r + A], cb = R[3 * r + B];
        R[3 * r + A] = __fadd_rn(__fmul_rn(c, ca), __fmul_rn(s, cb));
        R[3 * r + B] = __fsub_rn(__fmul_rn(c, cb), __fmul_rn(s, ca));
    }
}

__device__ __forceinline__ void rotate_frame(float R[9], int axis, float s, float c) {
    if (axis == 2) rotate_cols<0, 1>(R, s, c);
    else if (axis == 1) rotate_cols<2, 0>(R, s, c);
    else rotate_cols<1, 2>(R, s, c);
}

__device__ __forceinline__ float row_dot(const float R[9], int r, float v0, float v1, float v2) {
    return __fadd_rn(__fadd_rn(__fmul_rn(R[3 * r], v0), __fmul_rn(R[3 * r + 1], v1)), __fmul_rn(R[3 * r + 2], v2));
}

// Centres p + R o of one link's points: x and y as an FP32x2 pair (each element the
// scalar expression p_r + ((R_r0 o_0 + R_r1 o_1) + R_r2 o_2), rounded the same way: the
// products by f2_mulz, so that none is fused into its sum), z alone.  Set up once per
// link from its frame; nzero is DevArgs::nzero.
struct LinkXform {
    uint64_t c0, c1, c2, p01, z2;   // {R00, R10}, {R01, R11}, {R02, R12}, {p0, p1}, {-0, -0}
    float r20, r21, r22, p2;
    __device__ __forceinline__ void set(const float R[9], const float p[3], float nzero) {
        z2 = f2_dup(nzero);
        asm("mov.b64 %0, {%1, %2};" : "=l"(c0) : "f"(R[0]), "f"(R[3]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(c1) : "f"(R[1]), "f"(R[4]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(c2) : "f"(R[2]), "f"(R[5]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(p01) : "f"(p[0]), "f"(p[1]));
        r20 = R[6];
        r21 = R[7];
        r22 = R[8];
        p2 = p[2];
    }
    __device__ __forceinline__ void apply(float ox, float oy, float oz, float& cx, float& cy, float& cz) const {
        const uint64_t xy = f2_add(
            p01, f2_add(f2_add(f2_mulz(c0, f2_dup(ox), z2), f2_mulz(c1, f2_dup(oy), z2)), f2_mulz(c2, f2_dup(oz), z2)));
        const float2 v = f2_split(xy);
        cx = v.x;
        cy = v.y;
        cz = __fadd_rn(p2, __fadd_rn(__fadd_rn(__fmul_rn(r20, ox), __fmul_rn(r21, oy)), __fmul_rn(r22, oz)));
    }
};

__device__ __forceinline__ void link_point(const float R[9], const float p[3], float ox, float oy, float oz, float& cx,
                                           float& cy, float& cz) {
    cx = __fadd_rn(p[0], row_dot(R, 0, ox, oy, oz));
    cy = __fadd_rn(p[1], row_dot(R, 1, ox, oy, oz));
    cz = __fadd_rn(p[2], row_dot(R, 2, ox, oy, oz));
}

struct EdgeScratch {
    float4 nc[64];   // queued near spheres (< 32 left over + 32 from one sphere step);
                     // with the grid: centre and r, awaiting classification
    float4 rq[64];   // with the grid: the undecided ones, centre and r^2
    RoundEntries re;
};

// With the distance-bound grid: classify the first n queued spheres of an edge pass by
// their cells (dist_grid.cu).  Returns true when one of them certainly collides (the
// edge is invalid); the undecided ones join the rest queue (a round runs once it holds
// 32), the others are dropped; the rest of the queue moves to the front.
template <int MODE>
__device__ __forceinline__ bool edge_grid_step(const DevArgs& t, const float* Ts, EdgeScratch* ws, uint32_t n,
                                               uint32_t& n_near, uint32_t& n_rest, uint32_t lane,
                                               uint32_t lt_mask) {
    const bool live = lane < n;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    int cls = 0;
    if (live) {
        c = ws->nc[lane];
        cls = grid_classify(t, c.x, c.y, c.z, c.w);
    }
    if (__any_sync(0xffffffffu, cls == 1)) return true;
    const uint32_t km = __ballot_sync(0xffffffffu, cls == 2);
    if (cls == 2) ws->rq[n_rest + __popc(km & lt_mask)] = make_float4(c.x, c.y, c.z, __fmul_rn(c.w, c.w));
    n_rest += __popc(km);
    const bool mv = lane + n < n_near;
    const float4 cc = mv ? ws->nc[lane + n] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    if (mv) ws->nc[lane] = cc;
    n_near -= n;
    __syncwarp();
    if (n_rest >= 32) {
        if (sphere_round<true, MODE>(t, Ts, &ws->re, nullptr, ws->rq[lane], 0, true, lane, lt_mask)) return true;
        const bool mr = lane + 32 < n_rest;
        const float4 cr = mr ? ws->rq[lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (mr) ws->rq[lane] = cr;
        n_rest -= 32;
        __syncwarp();
    }
    return false;
}

// One pass: configurations k0 + stride * i, i = 0 .. count - 1 (count <= 32), of the
// edge with n_e configurations from qa_e to qb_e, lane i taking the i-th.  Returns true
// as soon as one of them collides.
template <int MODE, bool GRID>
__device__ bool edge_pass(const DevArgs& t, const ArmPlan& arm, const float* __restrict__ qa_e,
                          const float* __restrict__ qb_e, int n_e, int k0, int stride, int count, const float* Ts,
                          EdgeScratch* ws) {
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const bool live = (int)lane < count;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    // q_k = q_a + (k / (n - 1)) (q_b - q_a)
    const float tk = n_e > 1 ? __fdiv_rn((float)(k0 + stride * (int)lane), (float)(n_e - 1)) : 0.f;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {arm.base[0], arm.base[1], arm.base[2]};
    uint32_t n_near = 0, n_rest = 0;
    for (int j = 0; j < arm.J; j++) {
        const float a = __ldg(qa_e + j), b = __ldg(qb_e + j);
        const float q = __fadd_rn(a, __fmul_rn(tk, __fsub_rn(b, a)));
        float sj, cj;
        sincos_cw(q, sj, cj);
        rotate_frame(R, arm.axis[j], sj, cj);
        int i_end = arm.sbeg[j + 1];
        if (arm.sbeg[j] < i_end) {
            // no lane's bounding sphere of this link reaches the cloud's box: none of the
            // link's spheres can come near it (the configurations of a pass lie on one
            // edge, so their links are near or far together more often than not)
            float bx, by, bz;
            link_point(R, p, arm.cull_o[j][0], arm.cull_o[j][1], arm.cull_o[j][2], bx, by, bz);
            const bool ln = live && box_dist2(bx, by, bz, rlo, rhi) <= arm.cull_t[j];
            if (!__any_sync(0xffffffffu, ln)) i_end = arm.sbeg[j];
        }
        for (int i = arm.sbeg[j]; i < i_end; i++) {
            const float ox = arm.off[i][0], oy = arm.off[i][1], oz = arm.off[i][2];
            float cx, cy, cz;
            link_point(R, p, ox, oy, oz, cx, cy, cz);
            const float r2 = arm.r2[i];
            const bool near = live && box_dist2(cx, cy, cz, rlo, rhi) <= r2;
            const uint32_t mask = __ballot_sync(0xffffffffu, near);
            if (near) ws->nc[n_near + __popc(mask & lt_mask)] = make_float4(cx, cy, cz, GRID ? arm.rr[i] : r2);
            n_near += __popc(mask);
            if (GRID && n_near >= 32) {
                __syncwarp();
                if (edge_grid_step<MODE>(t, Ts, ws, 32, n_near, n_rest, lane, lt_mask)) return true;
            } else if (n_near >= 32) {
                __syncwarp();
                if (sphere_round<true, MODE>(t, Ts, &ws->re, nullptr, ws->nc[lane], 0, true, lane, lt_mask)) return true;
                const uint32_t rest = n_near - 32;
                float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
                if (lane < rest) cc = ws->nc[32 + lane];
                __syncwarp();
                if (lane < rest) ws->nc[lane] = cc;
                __syncwarp();
                n_near = rest;
            }
        }
        const float l0 = arm.link[j][0], l1 = arm.link[j][1], l2 = arm.link[j][2];
        const float tx = row_dot(R, 0, l0, l1, l2);
        const float ty = row_dot(R, 1, l0, l1, l2);
        const float tz = row_dot(R, 2, l0, l1, l2);
        p[0] = __fadd_rn(p[0], tx);
        p[1] = __fadd_rn(p[1], ty);
        p[2] = __fadd_rn(p[2], tz);
    }
    if constexpr (GRID) {
        __syncwarp();
        if (n_near && edge_grid_step<MODE>(t, Ts, ws, n_near, n_near, n_rest, lane, lt_mask)) return true;
        if (n_rest == 0) return false;
        const bool in_rest = lane < n_rest;
        const float4 c = in_rest ? ws->rq[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        return sphere_round<true, MODE>(t, Ts, &ws->re, nullptr, c, 0, in_rest, lane, lt_mask);
    }
    if (n_near == 0) return false;
    __syncwarp();
    const bool in_queue = lane < n_near;
    const float4 c = in_queue ? ws->nc[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    return sphere_round<true, MODE>(t, Ts, &ws->re, nullptr, c, 0, in_queue, lane, lt_mask);
}

__device__ __forceinline__ uint8_t load_volatile_u8(const uint8_t* p) {
    return *reinterpret_cast<const volatile uint8_t*>(p);
}

// Exclusive prefix of per-edge work items; resets validity and the work counter.
// One block; scratch = [E + 1 offsets][counter].  The offsets, the total and the
// counter are 32-bit words, so the prefix is summed in 64 bits and the batch is refused
// on the device when its total exceeds kMaxEdgeItems (2^31 items, 2^36 or more
// configurations): the counter then stays far from wrapping (it ends at most one take
// per warp past the total).  A refused batch does no work, reports every edge as not
// valid (0) and latches kStatusBounds in the status word.
constexpr uint64_t kMaxEdgeItems = 1ull << 31;

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += u;
    }
    return v;
}

__global__ void k_edges_setup(const int32_t* __restrict__ ns, uint32_t E, uint32_t chunk, uint32_t* scratch,
                              uint8_t* __restrict__ valid, int* status) {
    __shared__ unsigned long long warp_sums[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t base = 0; base < E; base += blockDim.x) {
        const uint32_t e = base + threadIdx.x;
        uint32_t items = 0;   // at most 2^26 (n_e < 2^31, chunk >= 32)
        if (e < E) {
            const int n = ns[e];
            items = n > 0 ? (uint32_t)(((uint64_t)n + chunk - 1) / chunk) : 0u;
            valid[e] = 1;
        }
        const unsigned long long incl = warp_incl_scan64(items);
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = lane < nw ? warp_sums[lane] : 0ull;
            v = warp_incl_scan64(v);
            if (lane < nw) warp_sums[lane] = v;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? warp_sums[warp - 1] : 0ull);
        // offsets past the limit are never read: the batch is refused below
        if (e < E) scratch[e] = (uint32_t)min(before + incl - items, (unsigned long long)kMaxEdgeItems);
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[nw - 1];
        __syncthreads();
    }
    const bool refuse = carry > kMaxEdgeItems;
    if (refuse) {
        for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) valid[e] = 0;
    }
    if (threadIdx.x == 0) {
        scratch[E] = refuse ? 0u : (uint32_t)carry;
        scratch[E + 1] = 0;   // work counter
        // configurations evaluated (64 bits, 8-byte aligned, in the scratch's slack)
        *reinterpret_cast<unsigned long long*>(scratch + edge_eval_word(E)) = 0ull;
        if (refuse) atomicOr(status, kStatusBounds);
    }
}

template <bool STAGE, int MODE, bool GRID>
__global__ void __launch_bounds__(512, 2) k_edges_persistent(DevArgs t, const __grid_constant__ ArmPlan arm,
                                                             const float* __restrict__ qa, const float* __restrict__ qb,
                                                             const int32_t* __restrict__ ns, uint32_t E, uint32_t chunk,
                                                             uint32_t* scratch, uint8_t* valid) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);
        off = stage_offset(t);
    }
    const uint32_t lane = lane_id();
    EdgeScratch* ws = reinterpret_cast<EdgeScratch*>(smem_raw + off) + (threadIdx.x >> 5);
    const uint32_t total_items = scratch[E];
    uint32_t* counter = scratch + E + 1;
    unsigned long long evaluated = 0;   // configurations this warp ran (lane 0's count)
    const int J = arm.J;
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total_items) break;
        // edge = last e with scratch[e] <= item (binary search over the prefix)
        uint32_t lo = 0, hi = E;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(scratch + mid) <= item) lo = mid;
            else hi = mid;
        }
        const uint32_t e = lo;
        if (load_volatile_u8(valid + e) == 0) continue;
        const int n_e = __ldg(ns + e);
        // the edge's items interleave its configurations: item ci of nci takes
        // ci, ci + nci, ci + 2 nci, ..., so its first passes sample the whole edge and a
        // colliding stretch is met early wherever it lies
        const int nci = (int)(((int64_t)n_e + chunk - 1) / chunk);
        const int ci = (int)(item - __ldg(scratch + e));
        const int cnt = (int)(((int64_t)n_e - ci + nci - 1) / nci);
        const float* qa_e = qa + (size_t)e * J;
        const float* qb_e = qb + (size_t)e * J;
        for (int j = 0; j < cnt; j += 32) {
            evaluated += (unsigned long long)min(32, cnt - j);
            if (edge_pass<MODE, GRID>(t, arm, qa_e, qb_e, n_e, ci + nci * j, nci, min(32, cnt - j), Ts, ws)) {
                if (lane == 0) valid[e] = 0;
                break;
            }
            if (load_volatile_u8(valid + e) == 0) break;
        }
    }
    if (lane == 0 && evaluated)
        atomicAdd(reinterpret_cast<unsigned long long*>(scratch + edge_eval_word(E)), evaluated);
}

// One edge per launch (the per-edge baseline): warps stride over its configurations.
template <int MODE, bool GRID>
__global__ void __launch_bounds__(512, 2) k_edge_single(DevArgs t, const __grid_constant__ ArmPlan arm,
                                                        const float* __restrict__ qa_e, const float* __restrict__ qb_e,
                                                        int n_e, uint8_t* valid_e) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EdgeScratch* ws = reinterpret_cast<EdgeScratch*>(smem_raw) + (threadIdx.x >> 5);
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    const int gw = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    for (int64_t k = (int64_t)gw * 32; k < n_e; k += (int64_t)warps * 32) {
        if (load_volatile_u8(valid_e) == 0) break;
        if (edge_pass<MODE, GRID>(t, arm, qa_e, qb_e, n_e, (int)k, 1, (int)min((int64_t)32, n_e - k), nullptr, ws)) {
            if (lane_id() == 0) *valid_e = 0;
            break;
        }
    }
}

// ------------------------------------------------------------------------------------
// Configurations given by their joint angles: the kinematics of the edge kernel, one
// lane per configuration, with the per-configuration early exit of Sec. IV-D (a hit
// resolves its own configuration only; the others of the pass go on).
// ------------------------------------------------------------------------------------
struct JointScratch {
    float4 nc[64];     // queued near spheres: centre and r^2 (< 32 left over + 32 new);
                       // with the grid: centre and r, awaiting classification
    uint32_t ng[64];   // their configuration (lane of the pass)
    float4 rq[64];     // with the grid: the undecided ones, centre and r^2
    uint32_t rg[64];   // their configuration
    uint32_t ghit[32]; // per configuration of the pass: 1 once it collides
    RoundEntries re;
};

template <bool STAGE, int MODE, bool GRID>
__global__ void __launch_bounds__(512, 2) k_joint_configs(DevArgs t, const __grid_constant__ ArmPlan arm,
                                                          const float* __restrict__ q, uint64_t C,
                                                          uint8_t* __restrict__ out, unsigned long long* ctr) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);
        off = stage_offset(t);
    }
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = (1u << lane) - 1u;
    JointScratch* ws = reinterpret_cast<JointScratch*>(smem_raw + off) + (threadIdx.x >> 5);
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    const uint64_t passes = (C + 31) / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const int J = arm.J;
    auto run_round = [&](uint32_t n) {
        const bool in_queue = lane < n;
        const float4 c = in_queue ? ws->nc[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t g = in_queue ? ws->ng[lane] : 0u;
        sphere_round<false, MODE>(t, Ts, &ws->re, ws->ghit, c, g, in_queue, lane, lt_mask);
    };
    // with the grid: a round over the first n undecided spheres, the rest to the front
    uint32_t n_rest = 0;
    auto rest_round = [&](uint32_t n) {
        const bool in_queue = lane < n;
        const float4 c = in_queue ? ws->rq[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t g = in_queue ? ws->rg[lane] : 0u;
        sphere_round<false, MODE>(t, Ts, &ws->re, ws->ghit, c, g, in_queue, lane, lt_mask);
        const bool mv = lane + n < n_rest;
        const float4 cc = mv ? ws->rq[lane + n] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t gg = mv ? ws->rg[lane + n] : 0u;
        __syncwarp();
        if (mv) {
            ws->rq[lane] = cc;
            ws->rg[lane] = gg;
        }
        n_rest -= n;
        __syncwarp();
    };
    // with the grid: classify the first n queued spheres by their cells; a certain hit
    // resolves its configuration, a certain miss is dropped, the undecided join the rest
    auto classify = [&](uint32_t n, uint32_t& n_near) {
        const bool live = lane < n;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t g = 0;
        int cls = 0;
        if (live) {
            c = ws->nc[lane];
            g = ws->ng[lane];
            if (!ws->ghit[g]) cls = grid_classify(t, c.x, c.y, c.z, c.w);
        }
        if (cls == 1) ws->ghit[g] = 1;
        const uint32_t km = __ballot_sync(0xffffffffu, cls == 2);
        if (cls == 2) {
            const uint32_t pos = n_rest + __popc(km & lt_mask);
            ws->rq[pos] = make_float4(c.x, c.y, c.z, __fmul_rn(c.w, c.w));
            ws->rg[pos] = g;
        }
        n_rest += __popc(km);
        const bool mv = lane + n < n_near;
        const float4 cc = mv ? ws->nc[lane + n] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t gg = mv ? ws->ng[lane + n] : 0u;
        __syncwarp();
        if (mv) {
            ws->nc[lane] = cc;
            ws->ng[lane] = gg;
        }
        n_near -= n;
        __syncwarp();
        if (n_rest >= 32) rest_round(32);
    };
    const TileSched sched{ctr, nwarps};
    for (uint64_t pass = sched.first((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); pass < passes;
         pass = sched.next(pass)) {
        const uint64_t k = pass * 32 + lane;
        const bool live = k < C;
        const float* qk = q + (live ? k : 0) * (uint64_t)J;
        ws->ghit[lane] = 0;
        __syncwarp();
        bool done = !live;   // this lane's configuration needs no more spheres
        float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
        float p[3] = {arm.base[0], arm.base[1], arm.base[2]};
        uint32_t n_near = 0;
        for (int j = 0; j < J; j++) {
            float sj, cj;
            sincos_cw(live ? __ldg(qk + j) : 0.f, sj, cj);
            rotate_frame(R, arm.axis[j], sj, cj);
            LinkXform X;
            X.set(R, p, t.nzero);
            for (int i = arm.sbeg[j]; i < arm.sbeg[j + 1]; i++) {
                const float ox = arm.off[i][0], oy = arm.off[i][1], oz = arm.off[i][2];
                float cx, cy, cz;
                X.apply(ox, oy, oz, cx, cy, cz);
                const float r2 = arm.r2[i];
                const bool near = !done && box_dist2(cx, cy, cz, rlo, rhi) <= r2;
                const uint32_t mask = __ballot_sync(0xffffffffu, near);
                if (near) {
                    const uint32_t pos = n_near + __popc(mask & lt_mask);
                    ws->nc[pos] = make_float4(cx, cy, cz, GRID ? arm.rr[i] : r2);
                    ws->ng[pos] = lane;
                }
                n_near += __popc(mask);
                if (GRID && n_near >= 32) {
                    __syncwarp();
                    classify(32, n_near);
                    done = done || ws->ghit[lane] != 0;
                } else if (n_near >= 32) {
                    __syncwarp();
                    run_round(32);
                    const uint32_t rest = n_near - 32;
                    float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
                    uint32_t gg = 0;
                    if (lane < rest) {
                        cc = ws->nc[32 + lane];
                        gg = ws->ng[32 + lane];
                    }
                    __syncwarp();
                    if (lane < rest) {
                        ws->nc[lane] = cc;
                        ws->ng[lane] = gg;
                    }
                    __syncwarp();
                    n_near = rest;
                    done = done || ws->ghit[lane] != 0;
                }
            }
            // every configuration of the pass resolved: the rest of the chain is moot
            if (__all_sync(0xffffffffu, done) && n_near == 0 && n_rest == 0) break;
            const float l0 = arm.link[j][0], l1 = arm.link[j][1], l2 = arm.link[j][2];
            const float tx = row_dot(R, 0, l0, l1, l2);
            const float ty = row_dot(R, 1, l0, l1, l2);
            const float tz = row_dot(R, 2, l0, l1, l2);
            p[0] = __fadd_rn(p[0], tx);
            p[1] = __fadd_rn(p[1], ty);
            p[2] = __fadd_rn(p[2], tz);
        }
        if constexpr (GRID) {
            __syncwarp();
            if (n_near) classify(n_near, n_near);
            if (n_rest) rest_round(n_rest);
        } else if (n_near) {
            __syncwarp();
            run_round(n_near);
        }
        __syncwarp();
        if (live) out[k] = (uint8_t)ws->ghit[lane];
        __syncwarp();
    }
}

int launch_joint_configs(const DevArgs& t, const capt_arm& arm, const float* q, uint64_t C, uint8_t* out,
                         const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st, std::string& err) {
    if (C == 0) return CAPT_OK;
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    // the chunked scan, or the compact one once the replicated sets are dropped
    const bool grid = cfg.grid != 0 && t.grid != nullptr;
    auto fn = grid ? (t.blocks ? (stage ? k_joint_configs<true, kScanChunked, true>
                                        : k_joint_configs<false, kScanChunked, true>)
                               : (stage ? k_joint_configs<true, kScanCompact, true>
                                        : k_joint_configs<false, kScanCompact, true>))
                   : (t.blocks ? (stage ? k_joint_configs<true, kScanChunked, false>
                                        : k_joint_configs<false, kScanChunked, false>)
                               : (stage ? k_joint_configs<true, kScanCompact, false>
                                        : k_joint_configs<false, kScanCompact, false>));
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(JointScratch) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, warps * 32, smem);
    occ = std::max(1, occ);
    const uint64_t passes = (C + 31) / 32;
    const uint64_t need = (passes + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    const ArmPlan plan = make_plan(arm);
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, plan, q, C, out, ctr);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("joint configuration launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

size_t edge_scratch_words(size_t E) { return E + 2 + 62; }

namespace {

// configurations per work item: a multiple of 32 (one per lane per pass)
uint32_t item_chunk(const capt_launch_cfg& cfg) {
    const int c = std::max(1, std::min(1024, (int)cfg.chunk));
    return (uint32_t)(((c + 31) / 32) * 32);
}

}  // namespace

int launch_edges_persistent(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                            const int32_t* ns, uint64_t E, uint8_t* valid, uint32_t* scratch,
                            const capt_launch_cfg& cfg, cudaStream_t st, std::string& err) {
    if (E == 0) return CAPT_OK;
    const uint32_t chunk = item_chunk(cfg);
    k_edges_setup<<<1, 1024, 0, st>>>(ns, (uint32_t)E, chunk, scratch, valid, t.status);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("edge setup launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    const bool grid = cfg.grid != 0 && t.grid != nullptr;
    auto fn = grid ? (t.blocks ? (stage ? k_edges_persistent<true, kScanChunked, true>
                                        : k_edges_persistent<false, kScanChunked, true>)
                               : (stage ? k_edges_persistent<true, kScanCompact, true>
                                        : k_edges_persistent<false, kScanCompact, true>))
                   : (t.blocks ? (stage ? k_edges_persistent<true, kScanChunked, false>
                                        : k_edges_persistent<false, kScanChunked, false>)
                               : (stage ? k_edges_persistent<true, kScanCompact, false>
                                        : k_edges_persistent<false, kScanCompact, false>));
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(EdgeScratch) * (size_t)warps;
    ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, warps * 32, smem);
    occ = std::max(1, occ);
    const ArmPlan plan = make_plan(arm);
    fn<<<(unsigned)(sm_count() * occ), warps * 32, smem, st>>>(t, plan, qa, qb, ns, (uint32_t)E, chunk, scratch, valid);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("edge launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_edges_per_edge(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                          const int32_t* h_ns, uint64_t E, uint8_t* valid, const capt_launch_cfg& cfg,
                          cudaStream_t st, std::string& err) {
    cudaError_t ce = cudaMemsetAsync(valid, 1, E, st);
    if (ce != cudaSuccess) { err = std::string("memset: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = sizeof(EdgeScratch) * (size_t)warps;
    const bool grid = cfg.grid != 0 && t.grid != nullptr;
    auto fn = grid ? (t.blocks ? k_edge_single<kScanChunked, true> : k_edge_single<kScanCompact, true>)
                   : (t.blocks ? k_edge_single<kScanChunked, false> : k_edge_single<kScanCompact, false>);
    ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const ArmPlan plan = make_plan(arm);
    const int J = arm.n_joints;
    for (uint64_t e = 0; e < E; e++) {
        const int n = h_ns[e];
        if (n <= 0) continue;
        const int64_t warps_needed = ((int64_t)n + 31) / 32;
        const unsigned blocks = (unsigned)std::min<int64_t>((warps_needed + warps - 1) / warps, (int64_t)sm_count() * 64);
        fn<<<blocks, warps * 32, smem, st>>>(t, plan, qa + e * J, qb + e * J, n, valid + e);
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("per-edge launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

}  // namespace capt
