// Differentiable clearance: nearest-point distance through the CAPT and the hinge cost.
//
// With r_min = 0 every leaf stores all points within r_max of its cell (Alg. 1, Lemma 1
// case 1), so for a centre x in that cell the nearest stored point is the nearest
// cloud point whenever it is within r_max.  The forward pass therefore scans the whole
// set (no early exit), keeping the minimum FP32 squared distance and its slot; a set
// whose box lies farther than r_max is skipped (d = r_max).
//
// Forward layout: a block owns one trajectory at a time (persistent over trajectories);
// its warps take the waypoints (one configuration of S <= 64 spheres per warp pass).
// Each warp compacts its live spheres into an entry list and scans the concatenation of
// their blocks 32 at a time; per step, a segmented warp reduction delivers each
// entry's minimum (squared distance, slot) key to the entry's first lane, which folds
// it into the entry's running minimum.  Per-waypoint costs land in shared memory and
// one thread sums them in waypoint order, so the cost is bitwise reproducible.
//
// Backward: elementwise, one thread per sphere, from the saved distance and argmin.
#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"

namespace capt {

constexpr int kMaxWaypoints = 4096;

struct ClearScratch {
    float cx[64], cy[64], cz[64];
    uint32_t blk[64], start[64], end[64];
    unsigned long long minkey[64];
};

template <bool STAGE>
__global__ void __launch_bounds__(512) k_clearance_fwd(DevArgs t, const float* __restrict__ centers,
                                                       const float* __restrict__ radii, uint64_t T, int W, int S,
                                                       float margin, float* __restrict__ cost,
                                                       float* __restrict__ dist, int32_t* __restrict__ argmin) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);
        off = stage_offset(t);
    }
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    ClearScratch* ws = reinterpret_cast<ClearScratch*>(smem_raw + off) + warp;
    float* partial = reinterpret_cast<float*>(smem_raw + off + sizeof(ClearScratch) * nw);
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    const float rmax = t.r_max, rmax2 = __fmul_rn(t.r_max, t.r_max);
    const uint32_t lt_mask = (1u << lane) - 1u;
    // the lane's two sphere slots: radius and hinge offset r + margin
    float rm[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int s = (int)lane + 32 * h;
        rm[h] = s < S ? __fadd_rn(__ldg(radii + s), margin) : 0.f;
    }
    for (uint64_t traj = blockIdx.x; traj < T; traj += gridDim.x) {
        for (int w = (int)warp; w < W; w += (int)nw) {
            const uint64_t cfg = traj * (uint64_t)W + (uint64_t)w;
            bool act[2];
            uint32_t nb[2], fb[2], pos[2];
            float X[2], Y[2], Z[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int s = (int)lane + 32 * h;
                act[h] = false;
                nb[h] = fb[h] = 0;
                X[h] = Y[h] = Z[h] = 0.f;
                if (s < S) {
                    const uint64_t sph = cfg * (uint64_t)S + s;
                    X[h] = __ldg(centers + 3 * sph);
                    Y[h] = __ldg(centers + 3 * sph + 1);
                    Z[h] = __ldg(centers + 3 * sph + 2);
                    const uint32_t leaf = descend(X[h], Y[h], Z[h], t, Ts);
                    float4 a, b;
                    load_leaf(t.leaves, leaf, a, b);
                    const uint32_t cnt = __float_as_uint(b.w);
                    act[h] = cnt > 0 && box_dist2(X[h], Y[h], Z[h], a, b) <= rmax2;
                    nb[h] = act[h] ? (cnt + 3u) >> 2 : 0u;
                    fb[h] = __float_as_uint(a.w);
                }
            }
            uint32_t total = 0, n_ent = 0;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t mask = __ballot_sync(0xffffffffu, act[h]);
                const uint32_t incl = warp_incl_scan(nb[h]);
                pos[h] = n_ent + __popc(mask & lt_mask);
                if (act[h]) {
                    ws->cx[pos[h]] = X[h];
                    ws->cy[pos[h]] = Y[h];
                    ws->cz[pos[h]] = Z[h];
                    ws->blk[pos[h]] = fb[h];
                    ws->start[pos[h]] = total + incl - nb[h];
                    ws->end[pos[h]] = total + incl;
                    ws->minkey[pos[h]] = ~0ull;
                }
                total += __shfl_sync(0xffffffffu, incl, 31);
                n_ent += __popc(mask);
            }
            __syncwarp();
            uint32_t e = 0;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t p = base + lane;
                unsigned long long key = ~0ull;
                uint32_t my_e = 0xffffffffu;
                if (p < total) {
                    while (ws->end[e] <= p) e++;
                    my_e = e;
                    const uint32_t rel = p - ws->start[e];
                    const uint32_t b = ws->blk[e] + rel;
                    const float4 px = __ldg(blocks + 3 * (size_t)b);
                    const float4 py = __ldg(blocks + 3 * (size_t)b + 1);
                    const float4 pz = __ldg(blocks + 3 * (size_t)b + 2);
                    const float x = ws->cx[e], y = ws->cy[e], z = ws->cz[e];
                    const float d0 = sq_dist(x, y, z, px.x, py.x, pz.x);
                    const float d1 = sq_dist(x, y, z, px.y, py.y, pz.y);
                    const float d2 = sq_dist(x, y, z, px.z, py.z, pz.z);
                    const float d3 = sq_dist(x, y, z, px.w, py.w, pz.w);
                    // lowest slot wins ties (slots are in ascending point index)
                    float bd = d0;
                    uint32_t bq = 0;
                    if (d1 < bd) { bd = d1; bq = 1; }
                    if (d2 < bd) { bd = d2; bq = 2; }
                    if (d3 < bd) { bd = d3; bq = 3; }
                    key = ((unsigned long long)__float_as_uint(bd) << 32) | (unsigned long long)(rel * 4u + bq);
                }
                // segmented minimum over lanes that share an entry (runs are contiguous)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long ok = __shfl_down_sync(0xffffffffu, key, o);
                    const uint32_t oe = __shfl_down_sync(0xffffffffu, my_e, o);
                    if (lane + (uint32_t)o < 32u && oe == my_e && ok < key) key = ok;
                }
                const uint32_t prev_e = __shfl_up_sync(0xffffffffu, my_e, 1);
                if (my_e != 0xffffffffu && (lane == 0 || prev_e != my_e)) {
                    if (key < ws->minkey[my_e]) ws->minkey[my_e] = key;
                }
                __syncwarp();
            }
            __syncwarp();
            float term = 0.f;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int s = (int)lane + 32 * h;
                if (s >= S) continue;
                const uint64_t sph = cfg * (uint64_t)S + s;
                float d = rmax;
                int32_t am = -1;
                if (act[h]) {
                    const unsigned long long k = ws->minkey[pos[h]];
                    const float dd = __fsqrt_rn(__uint_as_float((uint32_t)(k >> 32)));
                    if (dd < rmax) {
                        d = dd;
                        am = (int32_t)__ldg(t.ids + 4 * (size_t)fb[h] + (uint32_t)(k & 0xffffffffu));
                    }
                }
                dist[sph] = d;
                argmin[sph] = am;
                const float hh = fmaxf(0.f, __fsub_rn(rm[h], d));
                term = __fadd_rn(term, __fmul_rn(hh, hh));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) term = __fadd_rn(term, __shfl_xor_sync(0xffffffffu, term, o));
            if (lane == 0) partial[w] = term;
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.f;
            for (int w = 0; w < W; w++) acc = __fadd_rn(acc, partial[w]);
            cost[traj] = acc;
        }
        __syncthreads();
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

int launch_clearance_fwd(const DevArgs& t, const float* centers, const float* radii, uint64_t T, int W, int S,
                         float margin, float* cost, float* dist, int32_t* argmin, const capt_launch_cfg& cfg,
                         cudaStream_t st, std::string& err) {
    if (T == 0) return CAPT_OK;
    if (W > kMaxWaypoints) { err = "clearance supports at most 4096 waypoints per trajectory"; return CAPT_E_ARG; }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    auto fn = stage ? k_clearance_fwd<true> : k_clearance_fwd<false>;
    const int warps = std::max(1, std::min(16, std::min((int)cfg.warps_per_block, W)));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(ClearScratch) * (size_t)warps +
                        sizeof(float) * (size_t)W;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, warps * 32, smem);
    occ = std::max(1, occ);
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, T));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, T, W, S, margin, cost, dist, argmin);
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
