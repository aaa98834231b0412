// Batched edge validation: the configuration-level early exit of Sec. IV-D applied to
// whole straight-line edges, with the interpolated configurations and their sphere
// centres generated inside the kernel.
//
// Persistent mode: work items are (edge, chunk of `chunk` consecutive configurations),
// enumerated edge by edge.  A setup kernel writes the exclusive prefix of the per-edge
// item counts and resets the work counter and the validity flags; the persistent
// kernel's warps then take items from the counter with one atomic each.  A warp skips
// an item whose edge is already known to collide, and stops its chunk at the first
// colliding configuration, so colliding edges cost little beyond their first hit.
// The three steps are captured once into a CUDA graph by capt_edge_plan_create.
//
// Per-edge mode (the baseline): one kernel launch per edge, each launching just enough
// warps for that edge's configurations.
#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"

namespace capt {

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

// The two sphere slots a lane owns in every configuration (s = lane, lane + 32),
// loaded once from the arm description into registers.
struct LaneSpheres {
    int f[2];          // link index, -1 for an unused slot
    float o[2][3];     // offset in the link frame
    float r2[2];       // fl(r * r)
};

__device__ __forceinline__ LaneSpheres lane_spheres(const capt_arm& arm) {
    LaneSpheres ls;
    const int lane = (int)lane_id();
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int s = lane + 32 * h;
        const bool v = s < arm.n_spheres;
        ls.f[h] = v ? arm.sphere_link[s] : -1;
        const float r = v ? arm.sphere_radius[s] : 0.f;
        ls.r2[h] = __fmul_rn(r, r);
#pragma unroll
        for (int a = 0; a < 3; a++) ls.o[h][a] = v ? arm.sphere_offset[s][a] : 0.f;
    }
    return ls;
}

// Centres of the lane's two sphere slots for one configuration.  The sines and
// cosines of its joints sit in lanes src_lane0 .. src_lane0 + J - 1 (sj, cj); every
// lane walks the whole chain and keeps the frames its spheres hang on.
__device__ __forceinline__ void fk_lane(const capt_arm& arm, const LaneSpheres& ls, float sj, float cj, int src_lane0,
                                        float c0[3], float c1[3]) {
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {arm.base[0], arm.base[1], arm.base[2]};
    for (int j = 0; j < arm.n_joints; j++) {
        const float s = __shfl_sync(0xffffffffu, sj, src_lane0 + j);
        const float c = __shfl_sync(0xffffffffu, cj, src_lane0 + j);
        rotate_frame(R, arm.axis[j], s, c);
        if (j == ls.f[0]) {
#pragma unroll
            for (int r = 0; r < 3; r++) c0[r] = __fadd_rn(p[r], row_dot(R, r, ls.o[0][0], ls.o[0][1], ls.o[0][2]));
        }
        if (j == ls.f[1]) {
#pragma unroll
            for (int r = 0; r < 3; r++) c1[r] = __fadd_rn(p[r], row_dot(R, r, ls.o[1][0], ls.o[1][1], ls.o[1][2]));
        }
        const float l0 = arm.link[j][0], l1 = arm.link[j][1], l2 = arm.link[j][2];
        const float tx = row_dot(R, 0, l0, l1, l2);
        const float ty = row_dot(R, 1, l0, l1, l2);
        const float tz = row_dot(R, 2, l0, l1, l2);
        p[0] = __fadd_rn(p[0], tx);
        p[1] = __fadd_rn(p[1], ty);
        p[2] = __fadd_rn(p[2], tz);
    }
}

// q_k = q_a + (k / (n - 1)) (q_b - q_a), component j.
__device__ __forceinline__ float interp_joint(const float* qa, const float* qb, int j, int k, int n) {
    const float t = n > 1 ? __fdiv_rn((float)k, (float)(n - 1)) : 0.f;
    const float a = __ldg(qa + j), b = __ldg(qb + j);
    return __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
}

template <int SPL>
struct EdgeScratch {
    static constexpr int E = 32 * SPL;
    float cx[E], cy[E], cz[E], r2[E];
    uint32_t blk[E], start[E], end[E];
};

// Check the SPL / 2 consecutive configurations k0, k0 + 1, .. of edge (qa_e, qb_e, n_e)
// that are below `limit` as one warp tile (64 slots per configuration; S <= 64).
// Returns true if any of them collides.
template <int SPL>
__device__ bool check_configs(const DevArgs& t, const capt_arm& arm, const LaneSpheres& ls, const float* qa_e,
                              const float* qb_e, int n_e, int k0, int limit, const float* Ts,
                              EdgeScratch<SPL>* ws) {
    constexpr int CPT = SPL / 2;
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int J = arm.n_joints;
    // lane (c * 16 + j) computes sin/cos of joint j of configuration k0 + c
    float sj = 0.f, cj = 1.f;
    {
        const int c = (int)(lane >> 4), j = (int)(lane & 15u);
        if (c < CPT && j < J && k0 + c < limit) sincos_cw(interp_joint(qa_e, qb_e, j, k0 + c, n_e), sj, cj);
    }
    bool act[SPL];
    uint32_t nb[SPL], fb[SPL];
    float X[SPL], Y[SPL], Z[SPL], R2[SPL];
#pragma unroll
    for (int c = 0; c < CPT; c++) {
        float p0[3] = {0.f, 0.f, 0.f}, p1[3] = {0.f, 0.f, 0.f};
        const bool live = k0 + c < limit;
        fk_lane(arm, ls, sj, cj, c * 16, p0, p1);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int k = 2 * c + h;
            const float* pc = h == 0 ? p0 : p1;
            act[k] = false;
            nb[k] = fb[k] = 0;
            X[k] = pc[0];
            Y[k] = pc[1];
            Z[k] = pc[2];
            R2[k] = ls.r2[h];
            if (live && ls.f[h] >= 0) {
                const uint32_t leaf = descend(X[k], Y[k], Z[k], t, Ts);
                float4 a, b;
                load_leaf(t.leaves, leaf, a, b);
                const uint32_t cnt = __float_as_uint(b.w);
                act[k] = cnt > 0 && box_dist2(X[k], Y[k], Z[k], a, b) <= R2[k];
                nb[k] = act[k] ? (cnt + 3u) >> 2 : 0u;
                fb[k] = __float_as_uint(a.w);
            }
        }
    }
    uint32_t total = 0, n_ent = 0;
#pragma unroll
    for (int k = 0; k < SPL; k++) {
        const uint32_t mask = __ballot_sync(0xffffffffu, act[k]);
        const uint32_t incl = warp_incl_scan(nb[k]);
        if (act[k]) {
            const uint32_t pos = n_ent + __popc(mask & lt_mask);
            ws->cx[pos] = X[k];
            ws->cy[pos] = Y[k];
            ws->cz[pos] = Z[k];
            ws->r2[pos] = R2[k];
            ws->blk[pos] = fb[k];
            ws->start[pos] = total + incl - nb[k];
            ws->end[pos] = total + incl;
        }
        total += __shfl_sync(0xffffffffu, incl, 31);
        n_ent += __popc(mask);
    }
    __syncwarp();
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    bool hit = false;
    uint32_t e = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t p = base + lane;
        bool h = false;
        if (p < total) {
            while (ws->end[e] <= p) e++;
            const uint32_t b = ws->blk[e] + (p - ws->start[e]);
            const float4 px = __ldg(blocks + 3 * (size_t)b);
            const float4 py = __ldg(blocks + 3 * (size_t)b + 1);
            const float4 pz = __ldg(blocks + 3 * (size_t)b + 2);
            const float x = ws->cx[e], y = ws->cy[e], z = ws->cz[e], rr = ws->r2[e];
            h = (sq_dist(x, y, z, px.x, py.x, pz.x) <= rr) | (sq_dist(x, y, z, px.y, py.y, pz.y) <= rr) |
                (sq_dist(x, y, z, px.z, py.z, pz.z) <= rr) | (sq_dist(x, y, z, px.w, py.w, pz.w) <= rr);
        }
        if (__any_sync(0xffffffffu, h)) { hit = true; break; }
    }
    __syncwarp();
    return hit;
}

__device__ __forceinline__ uint8_t load_volatile_u8(const uint8_t* p) {
    return *reinterpret_cast<const volatile uint8_t*>(p);
}

// Exclusive prefix of per-edge work items; resets validity and the work counter.
// One block; scratch = [E + 1 offsets][counter].
__global__ void k_edges_setup(const int32_t* __restrict__ ns, uint32_t E, uint32_t chunk, uint32_t* scratch,
                              uint8_t* __restrict__ valid) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t base = 0; base < E; base += blockDim.x) {
        const uint32_t e = base + threadIdx.x;
        uint32_t items = 0;
        if (e < E) {
            const int n = ns[e];
            items = n > 0 ? ((uint32_t)n + chunk - 1) / chunk : 0u;
            valid[e] = 1;
        }
        const uint32_t incl = warp_incl_scan(items);
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < nw ? warp_sums[lane] : 0u;
            v = warp_incl_scan(v);
            if (lane < nw) warp_sums[lane] = v;
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? warp_sums[warp - 1] : 0u);
        if (e < E) scratch[e] = before + incl - items;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[E] = carry;
        scratch[E + 1] = 0;   // work counter
    }
}

template <int SPL, bool STAGE>
__global__ void __launch_bounds__(512) k_edges_persistent(DevArgs t, const __grid_constant__ capt_arm arm,
                                                          const float* __restrict__ qa,
                                                          const float* __restrict__ qb, const int32_t* __restrict__ ns,
                                                          uint32_t E, uint32_t chunk, uint32_t* scratch,
                                                          uint8_t* valid) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);
        off = stage_offset(t);
    }
    constexpr int CPT = SPL / 2;
    const uint32_t lane = lane_id();
    EdgeScratch<SPL>* ws = reinterpret_cast<EdgeScratch<SPL>*>(smem_raw + off) + (threadIdx.x >> 5);
    const uint32_t total_items = scratch[E];
    uint32_t* counter = scratch + E + 1;
    const int J = arm.n_joints;
    const LaneSpheres ls = lane_spheres(arm);
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total_items) break;
        // edge = last e with scratch[e] <= item (binary search over the prefix)
        uint32_t lo = 0, hi = E;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(scratch + mid) <= item) lo = mid; else hi = mid;
        }
        const uint32_t e = lo;
        if (load_volatile_u8(valid + e) == 0) continue;
        const int n_e = __ldg(ns + e);
        const int k_begin = (int)((item - __ldg(scratch + e)) * chunk);
        const int k_end = min(n_e, k_begin + (int)chunk);
        const float* qa_e = qa + (size_t)e * J;
        const float* qb_e = qb + (size_t)e * J;
        for (int k = k_begin; k < k_end; k += CPT) {
            if (check_configs<SPL>(t, arm, ls, qa_e, qb_e, n_e, k, k_end, Ts, ws)) {
                if (lane == 0) valid[e] = 0;
                break;
            }
            if (load_volatile_u8(valid + e) == 0) break;
        }
    }
}

// One edge per launch (the per-edge baseline): warps stride over its configurations.
template <int SPL>
__global__ void __launch_bounds__(512) k_edge_single(DevArgs t, const __grid_constant__ capt_arm arm,
                                                     const float* __restrict__ qa_e, const float* __restrict__ qb_e,
                                                     int n_e, uint8_t* valid_e) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int CPT = SPL / 2;
    const LaneSpheres ls = lane_spheres(arm);
    EdgeScratch<SPL>* ws = reinterpret_cast<EdgeScratch<SPL>*>(smem_raw) + (threadIdx.x >> 5);
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    const int gw = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    for (int k = gw * CPT; k < n_e; k += warps * CPT) {
        if (load_volatile_u8(valid_e) == 0) break;
        if (check_configs<SPL>(t, arm, ls, qa_e, qb_e, n_e, k, n_e, nullptr, ws)) {
            if (lane_id() == 0) *valid_e = 0;
            break;
        }
    }
}

size_t edge_scratch_words(size_t E) { return E + 2 + 62; }

namespace {

using PersistentKernel = void (*)(DevArgs, const capt_arm, const float*, const float*, const int32_t*, uint32_t,
                                  uint32_t, uint32_t*, uint8_t*);

PersistentKernel pick_persistent(int spl, bool stage) {
    if (spl == 2) return stage ? k_edges_persistent<2, true> : k_edges_persistent<2, false>;
    if (spl == 4) return stage ? k_edges_persistent<4, true> : k_edges_persistent<4, false>;
    return nullptr;
}

}  // namespace

int launch_edges_persistent(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                            const int32_t* ns, uint64_t E, uint8_t* valid, uint32_t* scratch,
                            const capt_launch_cfg& cfg, cudaStream_t st, std::string& err) {
    if (E == 0) return CAPT_OK;
    const uint32_t chunk = (uint32_t)std::max(1, std::min(1024, (int)cfg.chunk));
    k_edges_setup<<<1, 1024, 0, st>>>(ns, (uint32_t)E, chunk, scratch, valid);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("edge setup launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    PersistentKernel fn = pick_persistent(cfg.spheres_per_lane, stage);
    if (!fn) { err = "edges need spheres_per_lane 2 or 4"; return CAPT_E_ARG; }
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t ws = cfg.spheres_per_lane == 2 ? sizeof(EdgeScratch<2>) : sizeof(EdgeScratch<4>);
    const uint32_t sb = stage ? stage_offset(t) : 0u;
    const size_t smem = sb + ws * (size_t)warps;
    ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, warps * 32, smem);
    occ = std::max(1, occ);
    fn<<<(unsigned)(sm_count() * occ), warps * 32, smem, st>>>(t, arm, qa, qb, ns, (uint32_t)E, chunk, scratch, valid);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("edge launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_edges_per_edge(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                          const int32_t* h_ns, uint64_t E, uint8_t* valid, const capt_launch_cfg& cfg,
                          cudaStream_t st, std::string& err) {
    cudaError_t ce = cudaMemsetAsync(valid, 1, E, st);
    if (ce != cudaSuccess) { err = std::string("memset: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int spl = cfg.spheres_per_lane == 4 ? 4 : 2;
    const int cpt = spl / 2;
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (spl == 2 ? sizeof(EdgeScratch<2>) : sizeof(EdgeScratch<4>)) * (size_t)warps;
    auto fn = spl == 2 ? k_edge_single<2> : k_edge_single<4>;
    ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int J = arm.n_joints;
    for (uint64_t e = 0; e < E; e++) {
        const int n = h_ns[e];
        if (n <= 0) continue;
        const int warps_needed = (n + cpt - 1) / cpt;
        const int blocks = (warps_needed + warps - 1) / warps;
        fn<<<blocks, warps * 32, smem, st>>>(t, arm, qa + e * J, qb + e * J, n, valid + e);
    }
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("per-edge launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

}  // namespace capt
