// Sphere and configuration queries (Alg. 3 with the early exit of Sec. IV-D).
//
// Design (GB300): a persistent grid, one warp per tile of 32 x SPL sphere slots.
//  1. Root box test: every lane loads its slots' centres and tests them against the
//     bounding box of the whole cloud.  That box contains every affordance set, so a
//     sphere that misses it misses every point (the same FP32 argument as the leaf box
//     test of Alg. 3: clamping to a box that contains p never moves farther than p).
//     The surviving ("near") spheres are compacted into a per-warp list; a tile with
//     none is answered without any descent.
//  2. Near spheres are processed 32 at a time: one lane each descends (fixed L steps,
//     3 levels per step on the blocked split array), loads its leaf's 32-byte record
//     and applies the leaf box test of Alg. 3.
//  3. Spheres that pass become "entries" (centre, r^2, first block, prefix of block
//     counts); the affordance scan walks the concatenation of all entries' 4-point
//     blocks 32 at a time, every lane testing one block (3 float4 loads, 4 FP32
//     distance tests).  The paper vectorises the scan across the points of one set;
//     this spreads it across the points of every live set of the round, so lanes stay
//     busy whatever the set sizes are.
//  4. A hit resolves its group (a sphere, or a configuration): later spheres and
//     blocks of a resolved group are skipped; with one configuration per tile the
//     first hit ends the tile (Sec. IV-D early termination).
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "device_common.cuh"
#include "kernels.h"

namespace capt {

template <int SPL, int MODE>
struct WarpScratch {
    static constexpr int E = 32 * SPL;
    static constexpr int IN = MODE == kModeSpheres ? 4 * E : 3 * E;
    float in[2][IN];      // double-buffered tile inputs: centres, then radii (sphere mode)
    uint64_t bar[2];      // completion of the bulk copy into in[0] / in[1]
    uint32_t nslot[E];    // near spheres of the tile (slot numbers, slot order)
    uint32_t ghit[E];     // per group: 1 once it collides
    float4 c[32];         // entries of the current round: centre and r^2
    int32_t boff[32];     // first block of the entry minus its start in the block list
    uint32_t end[32];     // exclusive end of the entry in the block list
    uint32_t grp[32];     // group of the entry
};

// Where a tile's inputs live: centres (and, per sphere, radii) are contiguous runs that
// one bulk copy each can move when they are 16-byte aligned and sized.
struct TileSrc {
    const float* c;
    const float* r;
    uint32_t c_bytes, r_bytes;
    bool bulk;
};

__device__ __forceinline__ bool aligned16(const void* p, uint32_t bytes) {
    return ((reinterpret_cast<uintptr_t>(p) | bytes) & 15u) == 0;
}

__device__ __forceinline__ void bulk_copy(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Packed FP32x2 arithmetic (two IEEE-rounded FP32 operations per instruction; the
// element results are bitwise those of the scalar __fsub_rn / __fmul_rn / __fadd_rn).
__device__ __forceinline__ uint64_t f2_dup(float a) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ bool f2_le(uint64_t v, float r2) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return (a <= r2) | (b <= r2);
}

// 4 FP32 sphere tests against one 4-point block (3 x 16-byte loads).  Per point the
// squared distance is ((p_x - c_x)^2 + (p_y - c_y)^2) + (p_z - c_z)^2, each operation
// rounded: p - c is the exact negation of c - p, so the squares equal those of the
// defining expression.  cxx, cyy, czz hold the centre coordinate twice.
__device__ __forceinline__ bool block_hit2(const float4* __restrict__ blocks, int32_t b, uint64_t cxx, uint64_t cyy,
                                           uint64_t czz, float r2) {
    const ulonglong2 px = __ldg(reinterpret_cast<const ulonglong2*>(blocks + 3 * (size_t)b));
    const ulonglong2 py = __ldg(reinterpret_cast<const ulonglong2*>(blocks + 3 * (size_t)b + 1));
    const ulonglong2 pz = __ldg(reinterpret_cast<const ulonglong2*>(blocks + 3 * (size_t)b + 2));
    const uint64_t x01 = f2_sub(px.x, cxx), x23 = f2_sub(px.y, cxx);
    const uint64_t y01 = f2_sub(py.x, cyy), y23 = f2_sub(py.y, cyy);
    const uint64_t z01 = f2_sub(pz.x, czz), z23 = f2_sub(pz.y, czz);
    const uint64_t s01 = f2_add(f2_add(f2_mul(x01, x01), f2_mul(y01, y01)), f2_mul(z01, z01));
    const uint64_t s23 = f2_add(f2_add(f2_mul(x23, x23), f2_mul(y23, y23)), f2_mul(z23, z23));
    return f2_le(s01, r2) | f2_le(s23, r2);
}

__device__ __forceinline__ bool block_hit(const float4* __restrict__ blocks, int32_t b, const float4& c) {
    return block_hit2(blocks, b, f2_dup(c.x), f2_dup(c.y), f2_dup(c.z), c.w);
}

template <int SPL, bool STAGE, int MODE>
__global__ void __launch_bounds__(512, SPL <= 2 ? 3 : 2)
    k_query(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii, uint64_t n_items, int S,
            int rows, int cpt, uint8_t* __restrict__ out) {
    using WS = WarpScratch<SPL, MODE>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ float r2s[64];   // configuration mode: fl(r_s^2) per sphere index
    if (MODE == kModeConfigs)
        for (int i = (int)threadIdx.x; i < S; i += (int)blockDim.x) r2s[i] = __fmul_rn(radii[i], radii[i]);
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);   // contains a block barrier
        off = stage_offset(t);
    } else {
        __syncthreads();
    }
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    WS* ws = reinterpret_cast<WS*>(smem_raw + off) + warp;
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    const uint64_t per_tile = MODE == kModeSpheres ? 32ull * SPL : (uint64_t)cpt;
    const uint64_t n_tiles = (n_items + per_tile - 1) / per_tile;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t lt_mask = (1u << lane) - 1u;
    // a configuration occupies span = 32 * rows slots (rows = 1 or 2, S <= 64)
    const uint32_t lg_span = rows == 2 ? 6u : 5u;
    const uint32_t span_mask = (1u << lg_span) - 1u;
    const uint32_t n_groups = MODE == kModeSpheres ? 32u * SPL : (uint32_t)cpt;
    // one configuration per tile: its first hit ends the tile, no per-group bookkeeping
    const bool single = MODE == kModeConfigs && cpt == 1;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);

    // Slot j of a tile: its group and its index within the tile's input run.
    auto slot_group = [&](uint32_t j) -> uint32_t {
        if constexpr (MODE == kModeSpheres) return j;
        else return j >> lg_span;
    };
    auto slot_local = [&](uint32_t j) -> uint32_t {
        if constexpr (MODE == kModeSpheres) return j;
        else return (j >> lg_span) * (uint32_t)S + (j & span_mask);
    };

    // Tile inputs are staged per warp by the bulk copy engine, double-buffered: while the
    // warp works on one tile, the copy of its next tile is in flight.  Ragged or
    // misaligned tiles (and every tile after a copy that did not complete) are loaded
    // directly into the same buffer instead.
    auto tile_src = [&](uint64_t tl) {
        TileSrc ts;
        const uint64_t first = tl * per_tile;
        const uint64_t cnt = min(per_tile, n_items - first);
        if constexpr (MODE == kModeSpheres) {
            ts.c = centers + 3 * first;
            ts.r = radii + first;
            ts.c_bytes = (uint32_t)(cnt * 12);
            ts.r_bytes = (uint32_t)(cnt * 4);
            ts.bulk = aligned16(ts.c, ts.c_bytes) && aligned16(ts.r, ts.r_bytes);
        } else {
            ts.c = centers + 3 * first * (uint64_t)S;
            ts.r = nullptr;
            ts.c_bytes = (uint32_t)(cnt * (uint64_t)S * 12);
            ts.r_bytes = 0;
            ts.bulk = aligned16(ts.c, ts.c_bytes);
        }
        return ts;
    };
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ws->bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ws->bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    bool bulk_ok = true;        // cleared for good if a copy ever fails to complete
    uint32_t uses0 = 0, uses1 = 0;  // completed phases of bar[0] / bar[1]
    auto issue = [&](uint64_t tl, int b) -> bool {
        if (tl >= n_tiles || !bulk_ok) return false;
        const TileSrc ts = tile_src(tl);
        if (!ts.bulk) return false;
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile(
                "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                    smem_u32(&ws->bar[b])),
                "r"(ts.c_bytes + ts.r_bytes)
                : "memory");
            bulk_copy(ws->in[b], ts.c, ts.c_bytes, &ws->bar[b]);
            if (ts.r_bytes) bulk_copy(ws->in[b] + 3 * 32 * SPL, ts.r, ts.r_bytes, &ws->bar[b]);
        }
        return true;
    };

    uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int buf = 0;
    bool staged = issue(tile, 0);
    for (; tile < n_tiles; tile += nwarps, buf ^= 1) {
        const bool next_staged = issue(tile + nwarps, buf ^ 1);
        float* in = ws->in[buf];
        bool from_smem = false;
        if (staged) {
            const uint32_t parity = (buf ? uses1 : uses0) & 1u;
            bool done = false;
            for (uint32_t it = 0; it < (1u << 22) && !done; it++) done = mbar_try_wait(smem_u32(&ws->bar[buf]), parity);
            done = __all_sync(0xffffffffu, done);
            if (buf) uses1++;
            else uses0++;
            if (done) {
                from_smem = true;
            } else {
                if (lane == 0) atomicOr(t.status, kStatusTimeout);
                bulk_ok = false;
            }
        }
        staged = next_staged && bulk_ok;
        // ---- 1. root box test; near spheres compacted in slot order ----
        uint32_t n_near = 0;
        const uint64_t first = tile * per_tile;                        // first item of the tile
        const uint32_t n_here = (uint32_t)min(per_tile, n_items - first);
        const float* cbase = centers + 3 * first * (MODE == kModeSpheres ? 1ull : (uint64_t)S);
#pragma unroll
        for (int k = 0; k < SPL; k++) {
            const uint32_t j = (uint32_t)k * 32u + lane;
            bool valid;
            if constexpr (MODE == kModeSpheres) {
                valid = j < n_here;
            } else {
                valid = (j >> lg_span) < n_here && (j & span_mask) < (uint32_t)S;
            }
            const uint32_t local = slot_local(j);
            bool near = false;
            if (valid) {
                float x, y, z, r2;
                if (from_smem) {
                    x = in[3 * local];
                    y = in[3 * local + 1];
                    z = in[3 * local + 2];
                } else {
                    x = __ldg(cbase + 3 * local);
                    y = __ldg(cbase + 3 * local + 1);
                    z = __ldg(cbase + 3 * local + 2);
                    in[3 * local] = x;
                    in[3 * local + 1] = y;
                    in[3 * local + 2] = z;
                }
                if constexpr (MODE == kModeSpheres) {
                    float r;
                    if (from_smem) {
                        r = in[3 * 32 * SPL + local];
                    } else {
                        r = __ldg(radii + first + local);
                        in[3 * 32 * SPL + local] = r;
                    }
                    r2 = __fmul_rn(r, r);
                } else {
                    r2 = r2s[j & span_mask];
                }
                near = box_dist2(x, y, z, rlo, rhi) <= r2;
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, near);
            if (near) ws->nslot[n_near + __popc(mask & lt_mask)] = j;
            n_near += __popc(mask);
        }
        if (n_near == 0) {
            // no sphere of the tile comes near the cloud: every flag is 0
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
            __syncwarp();
            continue;
        }
        if (!single)
            for (uint32_t g = lane; g < n_groups; g += 32) ws->ghit[g] = 0;
        __syncwarp();
        bool tile_hit = false;
        for (uint32_t r0 = 0; r0 < n_near; r0 += 32) {
            // ---- 2. descent and leaf box test, one near sphere per lane ----
            const uint32_t q = r0 + lane;
            bool act = false;
            uint32_t nb = 0, fb = 0, g = 0;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < n_near) {
                const uint32_t j = ws->nslot[q];
                const uint32_t local = slot_local(j);
                g = slot_group(j);
                c.x = in[3 * local];
                c.y = in[3 * local + 1];
                c.z = in[3 * local + 2];
                if constexpr (MODE == kModeSpheres) c.w = __fmul_rn(in[3 * 32 * SPL + local], in[3 * 32 * SPL + local]);
                else c.w = r2s[j & span_mask];
                if (single || !ws->ghit[g]) {
                    const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
                    float4 a, b;
                    load_leaf(t.leaves, leaf, a, b);
                    const uint32_t cnt = __float_as_uint(b.w);
                    act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= c.w;
                    nb = act ? (cnt + 3u) >> 2 : 0u;
                    fb = __float_as_uint(a.w);
                }
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, act);
            if (mask == 0) continue;
            // ---- 3. entries of this round and the load-balanced scan ----
            const uint32_t incl = warp_incl_scan(nb);
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t n_ent = __popc(mask);
            if (act) {
                const uint32_t pos = __popc(mask & lt_mask);
                ws->c[pos] = c;
                ws->boff[pos] = (int32_t)fb - (int32_t)(incl - nb);
                ws->end[pos] = incl;
                ws->grp[pos] = g;
            }
            __syncwarp();
            uint32_t e = 0;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t p = base + lane;
                bool h = false;
                if (p < total) {
                    while (ws->end[e] <= p) e++;
                    if (single) {
                        h = block_hit(blocks, ws->boff[e] + (int32_t)p, ws->c[e]);
                    } else {
                        const uint32_t ge = ws->grp[e];
                        if (!ws->ghit[ge]) {
                            h = block_hit(blocks, ws->boff[e] + (int32_t)p, ws->c[e]);
                            if (h) ws->ghit[ge] = 1;
                        }
                    }
                }
                if (single) {
                    if (__any_sync(0xffffffffu, h)) { tile_hit = true; break; }
                    continue;
                }
                __syncwarp();
                if (__any_sync(0xffffffffu, h)) {
                    // leave once every entry that still has blocks ahead is resolved
                    const bool open = lane < n_ent && ws->end[lane] > base + 32 && !ws->ghit[ws->grp[lane]];
                    if (!__any_sync(0xffffffffu, open)) break;
                }
            }
            __syncwarp();
            if (tile_hit) break;
        }
        // ---- 4. results ----
        if constexpr (MODE == kModeSpheres) {
#pragma unroll
            for (int k = 0; k < SPL; k++) {
                const uint64_t sph = tile * per_tile + (uint64_t)k * 32u + lane;
                if (sph < n_items) out[sph] = (uint8_t)ws->ghit[k * 32 + lane];
            }
        } else {
            const uint64_t cfg = tile * per_tile + lane;
            if (lane < (uint32_t)cpt && cfg < n_items) out[cfg] = single ? (uint8_t)tile_hit : (uint8_t)ws->ghit[lane];
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------
// Configuration queries: a warp owns a tile of CPT configurations, their S spheres
// packed densely (sphere i of the tile is sphere i mod S of configuration i / S).
//  1. Each pass covers 128 consecutive spheres: every lane reads 4 of them with three
//     16-byte loads (12 floats = 4 centres) and applies the root box test; spheres of a
//     configuration already known to collide are skipped.  Near spheres are queued in
//     shared memory.
//  2. Whenever 32 are queued, and once at the end of the tile, a round processes 32 of
//     them: descent, leaf box test, then the load-balanced scan of their affordance
//     sets with packed FP32x2 arithmetic; a hit resolves its configuration.
// ------------------------------------------------------------------------------------
constexpr int kQueue = 160;   // near-sphere queue: < 32 left over + 128 from one pass

struct CfgScratch {
    float4 nc[kQueue];     // queued near spheres: centre and r^2
    uint32_t ng[kQueue];   // their configuration within the tile
    uint32_t ghit[16];     // per configuration of the tile: 1 once it collides
    float4 c[32];          // entries of the current round
    int32_t boff[32];
    uint32_t end[32];
    uint32_t grp[32];
};

// One round: the first n (<= 32) queued spheres.  Returns after marking hits.
__device__ __forceinline__ void config_round(const DevArgs& t, const float* Ts, CfgScratch* ws, uint32_t n,
                                             uint32_t lane, uint32_t lt_mask) {
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    bool act = false;
    uint32_t nb = 0, fb = 0, g = 0;
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < n) {
        c = ws->nc[lane];
        g = ws->ng[lane];
        if (!ws->ghit[g]) {
            const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
            float4 a, b;
            load_leaf(t.leaves, leaf, a, b);
            const uint32_t cnt = __float_as_uint(b.w);
            act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= c.w;
            nb = act ? (cnt + 3u) >> 2 : 0u;
            fb = __float_as_uint(a.w);
        }
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, act);
    if (mask == 0) return;
    const uint32_t incl = warp_incl_scan(nb);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t n_ent = __popc(mask);
    __syncwarp();
    if (act) {
        const uint32_t pos = __popc(mask & lt_mask);
        ws->c[pos] = c;
        ws->boff[pos] = (int32_t)fb - (int32_t)(incl - nb);
        ws->end[pos] = incl;
        ws->grp[pos] = g;
    }
    __syncwarp();
    uint32_t e = 0, e_loaded = 0xffffffffu;
    uint64_t cxx = 0, cyy = 0, czz = 0;
    float r2 = 0.f;
    int32_t boff = 0;
    uint32_t ge = 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t p = base + lane;
        bool h = false;
        if (p < total) {
            while (ws->end[e] <= p) e++;
            if (e != e_loaded) {
                const float4 ce = ws->c[e];
                cxx = f2_dup(ce.x);
                cyy = f2_dup(ce.y);
                czz = f2_dup(ce.z);
                r2 = ce.w;
                boff = ws->boff[e];
                ge = ws->grp[e];
                e_loaded = e;
            }
            if (!ws->ghit[ge]) {
                h = block_hit2(blocks, boff + (int32_t)p, cxx, cyy, czz, r2);
                if (h) ws->ghit[ge] = 1;
            }
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, h)) {
            // leave once every entry that still has blocks ahead is resolved
            const bool open = lane < n_ent && ws->end[lane] > base + 32 && !ws->ghit[ws->grp[lane]];
            if (!__any_sync(0xffffffffu, open)) break;
        }
    }
    __syncwarp();
}

#ifndef CFG_MIN_BLOCKS
#define CFG_MIN_BLOCKS 2
#endif

template <int CPT, bool STAGE>
__global__ void __launch_bounds__(512, CFG_MIN_BLOCKS) k_configs(DevArgs t, const float* __restrict__ centers,
                                                    const float* __restrict__ radii, uint64_t C, int S,
                                                    uint8_t* __restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ float r2s[64];
    for (int i = (int)threadIdx.x; i < S; i += (int)blockDim.x) r2s[i] = __fmul_rn(radii[i], radii[i]);
    const float* Ts = nullptr;
    uint32_t off = 0;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);   // contains a block barrier
        off = stage_offset(t);
    } else {
        __syncthreads();
    }
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    CfgScratch* ws = reinterpret_cast<CfgScratch*>(smem_raw + off) + warp;
    const uint64_t n_tiles = (C + CPT - 1) / CPT;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    const uint32_t inv_s = (1u << 20) / (uint32_t)S + 1u;   // i / S = (i * inv_s) >> 20 for i < 4096

    for (uint64_t tile = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < n_tiles; tile += nwarps) {
        const uint64_t first = tile * CPT;
        const uint32_t ncfg = (uint32_t)min((uint64_t)CPT, C - first);
        const uint32_t nsph = ncfg * (uint32_t)S;
        const float* base = centers + 3 * first * (uint64_t)S;
        const bool vec = (reinterpret_cast<uintptr_t>(base) & 15u) == 0;
        if (lane < CPT) ws->ghit[lane] = 0;
        __syncwarp();
        uint32_t n_near = 0;
        for (uint32_t p0 = 0; p0 < nsph; p0 += 128) {
            // ---- root box test of 4 consecutive spheres per lane ----
            const uint32_t i0 = p0 + 4 * lane;
            const uint32_t nv = i0 < nsph ? min(4u, nsph - i0) : 0u;
            float v[12];
            if (vec && nv == 4) {
                const float4* q = reinterpret_cast<const float4*>(base + 3 * (size_t)i0);
                const float4 a = __ldg(q), b = __ldg(q + 1), cc = __ldg(q + 2);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                v[8] = cc.x; v[9] = cc.y; v[10] = cc.z; v[11] = cc.w;
            } else {
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = (uint32_t)(k / 3) < nv ? __ldg(base + 3 * (size_t)i0 + k) : 0.f;
            }
            uint32_t g = (i0 * inv_s) >> 20;
            uint32_t sidx = i0 - g * (uint32_t)S;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float x = v[3 * k], y = v[3 * k + 1], z = v[3 * k + 2];
                const float r2 = r2s[sidx];
                const bool near = (uint32_t)k < nv && !ws->ghit[g] && box_dist2(x, y, z, rlo, rhi) <= r2;
                const uint32_t mask = __ballot_sync(0xffffffffu, near);
                if (near) {
                    const uint32_t pos = n_near + __popc(mask & lt_mask);
                    ws->nc[pos] = make_float4(x, y, z, r2);
                    ws->ng[pos] = g;
                }
                n_near += __popc(mask);
                if (++sidx == (uint32_t)S) { sidx = 0; g++; }
            }
            // ---- rounds of 32 queued near spheres ----
            if (n_near >= 32) {
                __syncwarp();
                uint32_t r0 = 0;
                for (; n_near - r0 >= 32; r0 += 32) {
                    if (r0) {
                        // bring the next 32 to the front of the queue
                        const float4 cc = ws->nc[r0 + lane];
                        const uint32_t gg = ws->ng[r0 + lane];
                        __syncwarp();
                        ws->nc[lane] = cc;
                        ws->ng[lane] = gg;
                        __syncwarp();
                    }
                    config_round(t, Ts, ws, 32, lane, lt_mask);
                }
                // keep the remainder (< 32) at the front
                const uint32_t rest = n_near - r0;
                float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t gg = 0;
                if (lane < rest) {
                    cc = ws->nc[r0 + lane];
                    gg = ws->ng[r0 + lane];
                }
                __syncwarp();
                if (lane < rest) {
                    ws->nc[lane] = cc;
                    ws->ng[lane] = gg;
                }
                n_near = rest;
                __syncwarp();
                // every configuration of the tile resolved: nothing left to learn
                if (__all_sync(0xffffffffu, lane >= ncfg || ws->ghit[lane])) { n_near = 0; break; }
            }
        }
        if (n_near) {
            __syncwarp();
            config_round(t, Ts, ws, n_near, lane, lt_mask);
        }
        __syncwarp();
        if (lane < ncfg) out[first + lane] = (uint8_t)ws->ghit[lane];
        __syncwarp();
    }
}

// Sequential work count per configuration (one thread each), in the order the query
// kernel's method defines it: every sphere up to the configuration's first hit gets the
// root box test; a sphere within reach of the cloud's box descends and gets the leaf box
// test of Alg. 3; a sphere passing that scans its set in stored order up to its first hit.
// counts += [spheres examined, spheres near the cloud box, spheres passing the leaf box,
// points scanned].
__global__ void k_count_configs(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii,
                                uint64_t C, int S, unsigned long long* counts) {
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nsph = 0, nnear = 0, npass = 0, npts = 0;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    if (c < C) {
        for (int s = 0; s < S; s++) {
            const float* x = centers + 3 * (c * (uint64_t)S + s);
            const float r = radii[s], r2 = __fmul_rn(r, r);
            nsph++;
            if (!(box_dist2(x[0], x[1], x[2], rlo, rhi) <= r2)) continue;
            nnear++;
            const uint32_t leaf = descend(x[0], x[1], x[2], t, nullptr);
            float4 a, b;
            load_leaf(t.leaves, leaf, a, b);
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
        nnear += __shfl_xor_sync(0xffffffffu, nnear, o);
        npass += __shfl_xor_sync(0xffffffffu, npass, o);
        npts += __shfl_xor_sync(0xffffffffu, npts, o);
    }
    if ((threadIdx.x & 31) == 0 && nsph) {
        atomicAdd(counts, nsph);
        atomicAdd(counts + 1, nnear);
        atomicAdd(counts + 2, npass);
        atomicAdd(counts + 3, npts);
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
        case 16: return k_query<8, false, MODE>;
        case 17: return k_query<8, true, MODE>;
        default: return nullptr;
    }
}

size_t scratch_bytes(int spl, int mode) {
    if (mode == kModeSpheres) {
        switch (spl) {
            case 1: return sizeof(WarpScratch<1, kModeSpheres>);
            case 2: return sizeof(WarpScratch<2, kModeSpheres>);
            case 4: return sizeof(WarpScratch<4, kModeSpheres>);
            default: return sizeof(WarpScratch<8, kModeSpheres>);
        }
    }
    switch (spl) {
        case 1: return sizeof(WarpScratch<1, kModeConfigs>);
        case 2: return sizeof(WarpScratch<2, kModeConfigs>);
        case 4: return sizeof(WarpScratch<4, kModeConfigs>);
        default: return sizeof(WarpScratch<8, kModeConfigs>);
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

using ConfigKernel = void (*)(DevArgs, const float*, const float*, uint64_t, int, uint8_t*);

ConfigKernel pick_configs(int spl, bool stage) {
    switch (spl * 2 + (stage ? 1 : 0)) {
        case 4: return k_configs<4, false>;
        case 5: return k_configs<4, true>;
        case 8: return k_configs<8, false>;
        case 9: return k_configs<8, true>;
        case 16: return k_configs<16, false>;
        case 17: return k_configs<16, true>;
        default: return nullptr;
    }
}

int launch_configs(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S, uint8_t* out,
                   const capt_launch_cfg& cfg, cudaStream_t st, std::string& err) {
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    ConfigKernel fn = pick_configs(cfg.spheres_per_lane, stage);
    if (!fn) { err = "configuration queries take spheres_per_lane 2, 4 or 8"; return CAPT_E_ARG; }
    const int cpt = 2 * cfg.spheres_per_lane;
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(CfgScratch) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int occ = std::max(1, occupancy((const void*)fn, warps * 32, smem));
    const uint64_t tiles = (C + cpt - 1) / cpt;
    const uint64_t need = (tiles + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, C, S, out);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("configuration launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_query(const DevArgs& t, int mode, const float* centers, const float* radii, uint64_t n_items, int S,
                 uint8_t* out, const capt_launch_cfg& cfg, cudaStream_t st, std::string& err) {
    if (n_items == 0) return CAPT_OK;
    if (mode == kModeConfigs) return launch_configs(t, centers, radii, n_items, S, out, cfg, st, err);
    int spl = cfg.spheres_per_lane;
    int rows = 1, cpt = 1;
    if (mode == kModeConfigs) {
        rows = (S + 31) / 32;
        if (spl < rows) spl = rows;
        if (spl % rows) spl = rows * ((spl + rows - 1) / rows);
        if (spl > 8) { err = "configurations of more than 64 spheres need more slots than a warp holds"; return CAPT_E_ARG; }
        cpt = spl / rows;
    }
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    QueryKernel fn = pick_query<kModeSpheres>(spl, stage);
    if (!fn) { err = "unsupported spheres_per_lane"; return CAPT_E_ARG; }
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + scratch_bytes(spl, mode) * (size_t)warps;
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
