// Sphere and configuration queries (Alg. 3 with the early exit of Sec. IV-D).
//
// Design (GB300): a persistent grid, one warp per tile of 32 x SPL sphere slots.
//  1. Each lane descends its slots (fixed L steps; top levels of T from shared memory
//     when staged), loads the leaf's 32-byte record and applies the box test.
//  2. The warp compacts the surviving slots into a list of "entries" in shared
//     memory (centre, r^2, first block, prefix of block counts), in slot order.
//  3. The affordance scan walks the concatenation of all entries' 4-point blocks, 32
//     blocks per warp step: every lane tests one block (3 float4 loads, 4 FP32
//     distance tests), so lanes stay busy whatever the set sizes are.  The paper
//     vectorises the scan across the points of one set; this spreads it across the
//     points of every live set of the tile.
//  4. A hit resolves its group (sphere, or configuration): later blocks of a resolved
//     group are skipped, and the warp leaves the scan once every group with entries is
//     resolved (for a configuration, at its first colliding sphere).
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "device_common.cuh"
#include "kernels.h"

namespace capt {

template <int SPL>
struct WarpScratch {
    static constexpr int E = 32 * SPL;
    float4 c[E];          // centre and r^2 of each entry
    int32_t boff[E];      // first block of the entry minus its start in the block list
    uint32_t end[E];      // exclusive end of the entry in the block list
    uint32_t grp[E];      // group (sphere slot or configuration) of the entry
    uint32_t ghit[E];     // per group: 1 once it collides
};

// 4 FP32 sphere tests against one 4-point block (3 x 16-byte loads).
__device__ __forceinline__ bool block_hit(const float4* __restrict__ blocks, int32_t b, const float4& c) {
    const float4 px = __ldg(blocks + 3 * (size_t)b);
    const float4 py = __ldg(blocks + 3 * (size_t)b + 1);
    const float4 pz = __ldg(blocks + 3 * (size_t)b + 2);
    return (sq_dist(c.x, c.y, c.z, px.x, py.x, pz.x) <= c.w) | (sq_dist(c.x, c.y, c.z, px.y, py.y, pz.y) <= c.w) |
           (sq_dist(c.x, c.y, c.z, px.z, py.z, pz.z) <= c.w) | (sq_dist(c.x, c.y, c.z, px.w, py.w, pz.w) <= c.w);
}

template <int SPL, bool STAGE, int MODE>
__global__ void __launch_bounds__(512) k_query(DevArgs t, const float* __restrict__ centers,
                                               const float* __restrict__ radii, uint64_t n_items, int S, int rows,
                                               int cpt, uint8_t* __restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);
        off = stage_offset(t);
    }
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    WarpScratch<SPL>* ws = reinterpret_cast<WarpScratch<SPL>*>(smem_raw + off) + warp;
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    const uint64_t per_tile = MODE == kModeSpheres ? 32ull * SPL : (uint64_t)cpt;
    const uint64_t n_tiles = (n_items + per_tile - 1) / per_tile;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t span = 32u * (uint32_t)rows;
    // one configuration per tile: its first hit ends the tile, no per-group bookkeeping
    const bool single = MODE == kModeConfigs && cpt == 1;

    for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < n_tiles; tile += nwarps) {
        // ---- 1. descent and box test per slot ----
        bool act[SPL];
        uint32_t nb[SPL], fb[SPL];
        float4 C[SPL];
        bool any = false;
#pragma unroll
        for (int k = 0; k < SPL; k++) {
            const uint32_t j = (uint32_t)k * 32u + lane;
            bool valid;
            uint64_t sph;
            float r;
            if constexpr (MODE == kModeSpheres) {
                sph = tile * per_tile + j;
                valid = sph < n_items;
                r = valid ? __ldg(radii + sph) : 0.f;
            } else {
                const uint32_t g = j / span, s = j - g * span;
                const uint64_t cfg = tile * per_tile + g;
                valid = g < (uint32_t)cpt && s < (uint32_t)S && cfg < n_items;
                sph = cfg * (uint64_t)S + s;
                r = valid ? __ldg(radii + s) : 0.f;
            }
            act[k] = false;
            nb[k] = 0;
            fb[k] = 0;
            C[k] = make_float4(0.f, 0.f, 0.f, __fmul_rn(r, r));
            if (valid) {
                C[k].x = __ldg(centers + 3 * sph);
                C[k].y = __ldg(centers + 3 * sph + 1);
                C[k].z = __ldg(centers + 3 * sph + 2);
                const uint32_t leaf = descend(C[k].x, C[k].y, C[k].z, t, Ts);
                float4 a, b;
                load_leaf(t.leaves, leaf, a, b);
                const uint32_t cnt = __float_as_uint(b.w);
                act[k] = cnt > 0 && box_dist2(C[k].x, C[k].y, C[k].z, a, b) <= C[k].w;
                nb[k] = act[k] ? (cnt + 3u) >> 2 : 0u;
                fb[k] = __float_as_uint(a.w);
            }
            any |= act[k];
        }
        if (!__any_sync(0xffffffffu, any)) {
            // no sphere of the tile reaches a point's box: every flag is 0
            if constexpr (MODE == kModeSpheres) {
#pragma unroll
                for (int k = 0; k < SPL; k++) {
                    const uint64_t sph = tile * per_tile + (uint64_t)k * 32u + lane;
                    if (sph < n_items) out[sph] = 0;
                }
            } else {
                const uint64_t cfg = tile * per_tile + lane;
                if (lane < (uint32_t)cpt && cfg < n_items) out[cfg] = 0;
            }
            continue;
        }
        // ---- 2. compaction into the warp's entry list (slot order) ----
        if (!single)
            for (uint32_t g = lane; g < (uint32_t)(32 * SPL); g += 32) ws->ghit[g] = 0;
        uint32_t total = 0, n_ent = 0;
#pragma unroll
        for (int k = 0; k < SPL; k++) {
            const uint32_t mask = __ballot_sync(0xffffffffu, act[k]);
            if (mask == 0) continue;
            const uint32_t incl = warp_incl_scan(nb[k]);
            if (act[k]) {
                const uint32_t pos = n_ent + __popc(mask & lt_mask);
                const uint32_t start = total + incl - nb[k];
                ws->c[pos] = C[k];
                ws->boff[pos] = (int32_t)fb[k] - (int32_t)start;
                ws->end[pos] = total + incl;
                if constexpr (MODE == kModeSpheres) ws->grp[pos] = (uint32_t)k * 32u + lane;
                else ws->grp[pos] = ((uint32_t)k * 32u + lane) / span;
            }
            total += __shfl_sync(0xffffffffu, incl, 31);
            n_ent += __popc(mask);
        }
        __syncwarp();
        // ---- 3. load-balanced scan over all live blocks ----
        uint32_t e = 0;
        bool tile_hit = false;
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t p = base + lane;
            bool h = false;
            if (p < total) {
                while (ws->end[e] <= p) e++;
                if (single) {
                    h = block_hit(blocks, ws->boff[e] + (int32_t)p, ws->c[e]);
                } else {
                    const uint32_t g = ws->grp[e];
                    if (!ws->ghit[g]) {
                        h = block_hit(blocks, ws->boff[e] + (int32_t)p, ws->c[e]);
                        if (h) ws->ghit[g] = 1;
                    }
                }
            }
            if (single) {
                if (__any_sync(0xffffffffu, h)) { tile_hit = true; break; }
                continue;
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, h)) {
                // leave once every group that still has blocks ahead is resolved
                bool open = false;
                for (uint32_t q = lane; q < n_ent; q += 32)
                    open |= (ws->end[q] > base + 32) && !ws->ghit[ws->grp[q]];
                if (!__any_sync(0xffffffffu, open)) break;
            }
        }
        __syncwarp();
        // ---- 4. results ----
        if constexpr (MODE == kModeSpheres) {
#pragma unroll
            for (int k = 0; k < SPL; k++) {
                const uint64_t sph = tile * per_tile + (uint64_t)k * 32u + lane;
                if (sph < n_items) out[sph] = act[k] ? (uint8_t)ws->ghit[k * 32 + lane] : (uint8_t)0;
            }
        } else {
            const uint64_t cfg = tile * per_tile + lane;
            if (lane < (uint32_t)cpt && cfg < n_items) out[cfg] = single ? (uint8_t)tile_hit : (uint8_t)ws->ghit[lane];
        }
        __syncwarp();
    }
}

// Sequential Alg. 3 per configuration (one thread each), counting the method's own
// work: spheres examined up to the first hit, spheres whose box test passed, and
// affordance points scanned up to the first hit in stored order.
__global__ void k_count_configs(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii,
                                uint64_t C, int S, unsigned long long* counts) {
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nsph = 0, npass = 0, npts = 0;
    if (c < C) {
        for (int s = 0; s < S; s++) {
            const float* x = centers + 3 * (c * (uint64_t)S + s);
            const float r = radii[s], r2 = __fmul_rn(r, r);
            const uint32_t leaf = descend(x[0], x[1], x[2], t, nullptr);
            float4 a, b;
            load_leaf(t.leaves, leaf, a, b);
            nsph++;
            const uint32_t cnt = __float_as_uint(b.w);
            if (cnt == 0 || !(box_dist2(x[0], x[1], x[2], a, b) <= r2)) continue;
            npass++;
            const uint32_t b0 = __float_as_uint(a.w);
            bool hit = false;
            for (uint32_t j = 0; j < cnt && !hit; j++) {
                const float* blk = t.blocks + 12 * (size_t)(b0 + j / 4);
                const uint32_t q = j & 3u;
                npts++;
                hit = sq_dist(x[0], x[1], x[2], blk[q], blk[4 + q], blk[8 + q]) <= r2;
            }
            if (hit) break;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nsph += __shfl_xor_sync(0xffffffffu, nsph, o);
        npass += __shfl_xor_sync(0xffffffffu, npass, o);
        npts += __shfl_xor_sync(0xffffffffu, npts, o);
    }
    if ((threadIdx.x & 31) == 0 && nsph) {
        atomicAdd(counts, nsph);
        atomicAdd(counts + 1, npass);
        atomicAdd(counts + 2, npts);
    }
}

__global__ void k_leaves(DevArgs t, const float* __restrict__ centers, uint64_t m, uint32_t* __restrict__ leaves) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) leaves[i] = descend(centers[3 * i], centers[3 * i + 1], centers[3 * i + 2], t, nullptr);
}

// ------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------
int sm_count() {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
    return cache[dev];
}

namespace {

using QueryKernel = void (*)(DevArgs, const float*, const float*, uint64_t, int, int, int, uint8_t*);

template <int MODE>
QueryKernel pick_query(int spl, bool stage) {
    switch (spl * 2 + (stage ? 1 : 0)) {
        case 2: return k_query<1, false, MODE>;
        case 3: return k_query<1, true, MODE>;
        case 4: return k_query<2, false, MODE>;
        case 5: return k_query<2, true, MODE>;
        case 8: return k_query<4, false, MODE>;
        case 9: return k_query<4, true, MODE>;
        default: return nullptr;
    }
}

size_t scratch_bytes(int spl) {
    switch (spl) {
        case 1: return sizeof(WarpScratch<1>);
        case 2: return sizeof(WarpScratch<2>);
        default: return sizeof(WarpScratch<4>);
    }
}

// Blocks per SM the kernel can keep resident (cached per kernel, block size, smem).
int occupancy(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<std::string, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string key = std::to_string((uintptr_t)fn) + ":" + std::to_string(threads) + ":" + std::to_string(smem) +
                      ":" + std::to_string(dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
    cache[key] = nb;
    return nb;
}

}  // namespace

int launch_query(const DevArgs& t, int mode, const float* centers, const float* radii, uint64_t n_items, int S,
                 uint8_t* out, const capt_launch_cfg& cfg, cudaStream_t st, std::string& err) {
    if (n_items == 0) return CAPT_OK;
    int spl = cfg.spheres_per_lane;
    int rows = 1, cpt = 1;
    if (mode == kModeConfigs) {
        rows = (S + 31) / 32;
        if (spl < rows) spl = rows;
        if (spl % rows) spl = rows * ((spl + rows - 1) / rows);
        if (spl > 4) { err = "configurations of more than 64 spheres need more slots than a warp holds"; return CAPT_E_ARG; }
        cpt = spl / rows;
    }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    QueryKernel fn = mode == kModeSpheres ? pick_query<kModeSpheres>(spl, stage) : pick_query<kModeConfigs>(spl, stage);
    if (!fn) { err = "unsupported spheres_per_lane"; return CAPT_E_ARG; }
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + scratch_bytes(spl) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int occ = std::max(1, occupancy((const void*)fn, warps * 32, smem));
    const uint64_t per_tile = mode == kModeSpheres ? 32ull * spl : (uint64_t)cpt;
    const uint64_t tiles = (n_items + per_tile - 1) / per_tile;
    const uint64_t need = (tiles + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, n_items, S, rows, cpt, out);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("query launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_count_configs(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S,
                         uint64_t* counts, cudaStream_t st, std::string& err) {
    if (C == 0) return CAPT_OK;
    const unsigned threads = 256;
    k_count_configs<<<(unsigned)((C + threads - 1) / threads), threads, 0, st>>>(
        t, centers, radii, C, S, reinterpret_cast<unsigned long long*>(counts));
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("count launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_leaves(const DevArgs& t, const float* centers, uint64_t m, uint32_t* leaves, cudaStream_t st,
                  std::string& err) {
    if (m == 0) return CAPT_OK;
    const unsigned threads = 256;
    k_leaves<<<(unsigned)((m + threads - 1) / threads), threads, 0, st>>>(t, centers, m, leaves);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("leaves launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

}  // namespace capt
