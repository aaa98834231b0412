// Sphere and configuration queries (Alg. 3 with the early exit of Sec. IV-D).
//
// Design (GB300): persistent grids, one warp per tile of spheres or configurations,
// the tiles handed out by a work counter (TileSched) so that no warp is left with the
// expensive tiles at the end.
//  1. Root box test: every sphere is first tested against the bounding box of the
//     whole cloud.  That box contains every affordance set, so a sphere that misses it
//     misses every point (the same FP32 argument as the leaf box test of Alg. 3:
//     clamping to a box that contains p never moves farther than p).  Surviving
//     ("near") spheres are queued per warp; a tile with none needs no descent at all.
//  2. Queued spheres are processed 32 at a time (sphere_round, scan.cuh): one lane
//     each descends (fixed L steps, 3 levels per step on the blocked split array),
//     loads its leaf's 32-byte record and applies the leaf box test; the sets of the
//     spheres that pass are then scanned by the whole warp, in the launch's scan mode:
//     by chunks of 32 points whose boxes the sphere reaches (the default), by whole
//     sets, or over the compact sets.  The paper vectorises the scan across the points
//     of one set; this spreads it across the points of every live set of the round, so
//     lanes stay busy whatever the sizes.
//  3. A hit resolves its group (a sphere, or a configuration): later spheres and
//     blocks of a resolved group are skipped (Sec. IV-D early termination).
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "device_common.cuh"
#include "kernels.h"
#include "scan.cuh"

namespace capt {

// ------------------------------------------------------------------------------------
// Sphere queries: a warp owns a tile of 32 x SPL consecutive spheres.
// ------------------------------------------------------------------------------------
template <int SPL>
struct SphereScratch {
    static constexpr int E = 32 * SPL;
    float in[2][4 * E];   // double-buffered tile inputs: centres, then radii
    uint64_t bar[2];      // completion of the bulk copy into in[0] / in[1]
    uint32_t nslot[E];    // near spheres of the tile (slot numbers, slot order)
    uint32_t ghit[E];     // per sphere of the tile: 1 once it collides
    RoundEntries re;
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

template <int SPL, bool STAGE, int MODE>
__global__ void __launch_bounds__(512, 2)
    k_spheres(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii, uint64_t m,
              uint8_t* __restrict__ out, unsigned long long* ctr, bool use_grid) {
    using WS = SphereScratch<SPL>;
    constexpr uint32_t E = 32 * SPL;
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
    WS* ws = reinterpret_cast<WS*>(smem_raw + off) + warp;
    const uint64_t n_tiles = (m + E - 1) / E;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);

    // Tile inputs (centres, radii) are staged per warp by the bulk copy engine,
    // double-buffered: while the warp works on one tile, the copy of its next tile is in
    // flight.  Ragged or misaligned tiles are loaded directly into the same buffer
    // instead (no copy is in flight into it then).  If a wait gives up (kStagePolls), the
    // warp latches kStatusTimeout, issues no further copies and reads every later tile
    // straight from global memory without writing either buffer, so a copy that is still
    // landing cannot race with it; before the warp exits it waits (kDrainPolls) for every
    // copy it issued that it has not seen complete.
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ws->bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&ws->bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    bool bulk_ok = true;
    bool pend0 = false, pend1 = false;   // a copy into in[0] / in[1] not yet seen complete
    uint32_t ph0 = 0, ph1 = 0;           // parity of the phase that copy completes
    auto issue = [&](uint64_t tl, int b) -> bool {
        if (tl >= n_tiles || !bulk_ok) return false;
        const uint64_t first = tl * E;
        const uint32_t cnt = (uint32_t)min((uint64_t)E, m - first);
        const float* c = centers + 3 * first;
        const float* r = radii + first;
        if (!aligned16(c, cnt * 12u) || !aligned16(r, cnt * 4u)) return false;
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile(
                "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                    smem_u32(&ws->bar[b])),
                "r"(cnt * 16u)
                : "memory");
            bulk_copy(ws->in[b], c, cnt * 12u, &ws->bar[b]);
            bulk_copy(ws->in[b] + 3 * E, r, cnt * 4u, &ws->bar[b]);
        }
        if (b) pend1 = true;
        else pend0 = true;
        return true;
    };
    // bounded wait for the outstanding copy into in[b]; true once it has landed
    auto wait_buf = [&](int b, uint32_t polls) -> bool {
        const uint32_t bar = smem_u32(&ws->bar[b]);
        const uint32_t parity = b ? ph1 : ph0;
        bool done = false;
        for (uint32_t it = 0; it < polls && !done; it++) done = mbar_try_wait(bar, parity);
        done = __all_sync(0xffffffffu, done);
        if (done) {
            if (b) { pend1 = false; ph1 ^= 1u; }
            else { pend0 = false; ph0 ^= 1u; }
        }
        return done;
    };

    const TileSched sched{ctr, nwarps};
    uint64_t tile = sched.first((uint64_t)blockIdx.x * (blockDim.x >> 5) + warp);
    int buf = 0;
    bool staged = issue(tile, 0);
    for (uint64_t nxt; tile < n_tiles; tile = nxt, buf ^= 1) {
        nxt = sched.next(tile);
        const bool next_staged = issue(nxt, buf ^ 1);
        float* in = ws->in[buf];
        bool from_smem = false;
        if (staged) {
            if (wait_buf(buf, kStagePolls)) {
                from_smem = true;
            } else {
                if (lane == 0) atomicOr(t.status, kStatusTimeout);
                bulk_ok = false;
            }
        }
        // after a timeout no buffer is written again: inputs come from global memory
        const bool direct_to_smem = !from_smem && bulk_ok;
        const bool in_smem = from_smem || direct_to_smem;
        staged = next_staged && bulk_ok;
        const uint64_t first = tile * E;
        const uint32_t n_here = (uint32_t)min((uint64_t)E, m - first);
        // ---- root box test; near spheres compacted in slot order ----
        uint32_t n_near = 0;
#pragma unroll
        for (int k = 0; k < SPL; k++) {
            const uint32_t j = (uint32_t)k * 32u + lane;
            bool near = false;
            if (j < n_here) {
                float x, y, z, r;
                if (from_smem) {
                    x = in[3 * j];
                    y = in[3 * j + 1];
                    z = in[3 * j + 2];
                    r = in[3 * E + j];
                } else {
                    x = __ldg(centers + 3 * (first + j));
                    y = __ldg(centers + 3 * (first + j) + 1);
                    z = __ldg(centers + 3 * (first + j) + 2);
                    r = __ldg(radii + first + j);
                    if (direct_to_smem) {
                        in[3 * j] = x;
                        in[3 * j + 1] = y;
                        in[3 * j + 2] = z;
                        in[3 * E + j] = r;
                    }
                }
                near = box_dist2(x, y, z, rlo, rhi) <= __fmul_rn(r, r);
            }
            ws->ghit[j] = 0;
            const uint32_t mask = __ballot_sync(0xffffffffu, near);
            if (near) ws->nslot[n_near + __popc(mask & lt_mask)] = j;
            n_near += __popc(mask);
        }
        __syncwarp();
        // ---- with the distance-bound grid: near spheres it can decide are decided (a
        // certain hit is recorded at once), the undecided ones are compacted in place ----
        if (use_grid) {
            uint32_t n_rest = 0;
            for (uint32_t r0 = 0; r0 < n_near; r0 += 32) {
                const uint32_t q = r0 + lane;
                int cls = 0;
                uint32_t j = 0;
                if (q < n_near) {
                    j = ws->nslot[q];
                    float x, y, z, r;
                    if (in_smem) {
                        x = in[3 * j];
                        y = in[3 * j + 1];
                        z = in[3 * j + 2];
                        r = in[3 * E + j];
                    } else {
                        x = __ldg(centers + 3 * (first + j));
                        y = __ldg(centers + 3 * (first + j) + 1);
                        z = __ldg(centers + 3 * (first + j) + 2);
                        r = __ldg(radii + first + j);
                    }
                    cls = grid_classify(t, x, y, z, r);
                    if (cls == 1) ws->ghit[j] = 1;
                }
                const uint32_t km = __ballot_sync(0xffffffffu, cls == 2);
                __syncwarp();   // every read of this group precedes the writes below
                if (cls == 2) ws->nslot[n_rest + __popc(km & lt_mask)] = j;
                n_rest += __popc(km);
                __syncwarp();
            }
            n_near = n_rest;
        }
        // ---- rounds of 32 near spheres: descent, leaf box, scan ----
        for (uint32_t r0 = 0; r0 < n_near; r0 += 32) {
            const uint32_t q = r0 + lane;
            const bool live = q < n_near;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t j = 0;
            if (live) {
                j = ws->nslot[q];
                float x, y, z, r;
                if (in_smem) {
                    x = in[3 * j];
                    y = in[3 * j + 1];
                    z = in[3 * j + 2];
                    r = in[3 * E + j];
                } else {
                    x = __ldg(centers + 3 * (first + j));
                    y = __ldg(centers + 3 * (first + j) + 1);
                    z = __ldg(centers + 3 * (first + j) + 2);
                    r = __ldg(radii + first + j);
                }
                c = make_float4(x, y, z, __fmul_rn(r, r));
            }
            sphere_round<false, MODE>(t, Ts, &ws->re, ws->ghit, c, j, live, lane, lt_mask);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < SPL; k++) {
            const uint32_t j = (uint32_t)k * 32u + lane;
            if (j < n_here) out[first + j] = (uint8_t)ws->ghit[j];
        }
        __syncwarp();
    }
    // every copy this warp issued has landed before its shared memory can be handed on
    if (pend0) wait_buf(0, kDrainPolls);
    if (pend1) wait_buf(1, kDrainPolls);
}

// ------------------------------------------------------------------------------------
// Configuration queries: a warp owns a tile of CPT configurations, their S spheres
// packed densely (sphere i of the tile is sphere i mod S of configuration i / S).
//  1. Each pass covers 128 consecutive spheres: every lane reads 4 of them with three
//     16-byte loads (12 floats = 4 centres) and applies the root box test; spheres of a
//     configuration already known to collide are skipped.  Near spheres are queued in
//     shared memory.
//  2. Whenever 32 are queued, and once at the end of the tile, a round processes 32 of
//     them (sphere_round); a hit resolves its configuration.
// ------------------------------------------------------------------------------------
constexpr int kQueue = 160;   // near-sphere queue: < 32 left over + 128 from one pass

struct CfgScratch {
    float4 nc[kQueue];     // queued near spheres: centre and r^2
    uint32_t ng[kQueue];   // their configuration within the tile
    uint32_t ghit[32];     // per configuration of the tile: 1 once it collides
    RoundEntries re;
};

#ifndef CFG_MIN_BLOCKS
#define CFG_MIN_BLOCKS 2
#endif

template <int CPT, bool STAGE, int MODE>
__global__ void __launch_bounds__(512, CFG_MIN_BLOCKS) k_configs(DevArgs t, const float* __restrict__ centers,
                                                                 const float* __restrict__ radii, uint64_t C, int S,
                                                                 uint8_t* __restrict__ out, unsigned long long* ctr,
                                                                 uint32_t pf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ __align__(16) float r2s[64];
    for (int i = (int)threadIdx.x; i < S; i += (int)blockDim.x) r2s[i] = __fmul_rn(radii[i], radii[i]);
    uint32_t off = 0;
    if constexpr (STAGE) off = stage_offset(t);
    const float* Ts = nullptr;
    if constexpr (STAGE) {
        Ts = stage_splits(t, smem_raw, &bar);   // contains a block barrier
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
    const BoxPairs bp(rlo, rhi, t.nzero);
    const uint32_t inv_s = (1u << 20) / (uint32_t)S + 1u;   // i / S = (i * inv_s) >> 20 for i < 4096
    const bool s4 = (S & 3) == 0;

    auto run_round = [&](uint32_t n) {
        const bool live = lane < n;
        const float4 c = live ? ws->nc[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t g = live ? ws->ng[lane] : 0u;
        sphere_round<false, MODE>(t, Ts, &ws->re, ws->ghit, c, g, live, lane, lt_mask);
    };

    // L2 lookahead of the centre stream (pf passes of 128 spheres): tiles are taken in
    // increasing order across the grid (from the counter, or w, w + warps, ... without
    // one), so tile + warps is the one some warp starts about one tile-time from now
    const TileSched sched{ctr, nwarps};
    for (uint64_t tile = sched.first((uint64_t)blockIdx.x * (blockDim.x >> 5) + warp); tile < n_tiles;
         tile = sched.next(tile)) {
        const uint64_t first = tile * CPT;
        const uint32_t ncfg = (uint32_t)min((uint64_t)CPT, C - first);
        const uint32_t nsph = ncfg * (uint32_t)S;
        const float* base = centers + 3 * first * (uint64_t)S;
        const bool vec = (reinterpret_cast<uintptr_t>(base) & 15u) == 0;
        if (lane < CPT) ws->ghit[lane] = 0;
        __syncwarp();
        // bit g: configuration g of the tile is known to collide (warp-uniform; refreshed
        // from ghit after every round)
        uint32_t resolved = 0;
        const uint32_t all_cfg = ncfg >= 32u ? 0xffffffffu : ((1u << ncfg) - 1u);
        uint32_t n_near = 0;
        for (uint32_t p0 = 0; p0 < nsph; p0 += 128) {
            // ---- root box test of 4 consecutive spheres per lane ----
            const uint32_t i0 = p0 + 4 * lane;
            // the lane's centres pf passes ahead in this tile, asked of L2 while this pass
            // is tested (each lane's 48 bytes start in a different 128-byte line or share
            // one with a neighbour, so the lanes together cover the whole pass)
            if (pf && i0 + 128 * pf < nsph) prefetch_l2_line(base + 3 * (size_t)(i0 + 128 * pf));
            const uint32_t nv = i0 < nsph ? min(4u, nsph - i0) : 0u;
            float v[12];
            // every lane with four aligned centres (all passes but a tile's ragged last):
            // a warp-uniform branch, so the per-element path costs the others nothing
            if (__all_sync(0xffffffffu, vec && nv == 4)) {
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
            if (s4) {
                // S a multiple of 4: the lane's four spheres are slots sidx .. sidx + 3 of
                // configuration g, their radii one 16-byte load each
                const float4 q2 = reinterpret_cast<const float4*>(r2s)[sidx >> 2];
                const float r2k[4] = {q2.x, q2.y, q2.z, q2.w};
                const bool open = nv > 0 && !((resolved >> (g & 31u)) & 1u);
                float bd2[4];
                box_dist2_x4(v, bp, bd2);
                bool nk[4];
#pragma unroll
                for (int k = 0; k < 4; k++) nk[k] = open && (uint32_t)k < nv && bd2[k] <= r2k[k];
                // most passes have no sphere near the cloud's box at all: one vote skips
                // the four queue appends
                if (__any_sync(0xffffffffu, nk[0] | nk[1] | nk[2] | nk[3])) {
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const bool near = nk[k];
                        const uint32_t mask = __ballot_sync(0xffffffffu, near);
                        if (near) {
                            const uint32_t pos = n_near + __popc(mask & lt_mask);
                            ws->nc[pos] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], r2k[k]);
                            ws->ng[pos] = g;
                        }
                        n_near += __popc(mask);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float x = v[3 * k], y = v[3 * k + 1], z = v[3 * k + 2];
                    const float r2 = r2s[sidx];
                    const bool near = (uint32_t)k < nv && !((resolved >> (g & 31u)) & 1u) &&
                                      box_dist2(x, y, z, rlo, rhi) <= r2;
                    const uint32_t mask = __ballot_sync(0xffffffffu, near);
                    if (near) {
                        const uint32_t pos = n_near + __popc(mask & lt_mask);
                        ws->nc[pos] = make_float4(x, y, z, r2);
                        ws->ng[pos] = g;
                    }
                    n_near += __popc(mask);
                    if (++sidx == (uint32_t)S) { sidx = 0; g++; }
                }
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
                    run_round(32);
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
                resolved = __ballot_sync(0xffffffffu, lane < ncfg && ws->ghit[lane]);
                // every configuration of the tile resolved: nothing left to learn
                if ((resolved & all_cfg) == all_cfg) { n_near = 0; break; }
            }
        }
        if (n_near) {
            __syncwarp();
            run_round(n_near);
        }
        __syncwarp();
        if (lane < ncfg) out[first + lane] = (uint8_t)ws->ghit[lane];
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------
// Configuration queries with the distance-bound grid (dist_grid.cu).  The stream and
// its root box test are those of k_configs; the spheres that reach the cloud's box are
// then classified 32 at a time by their grid cell (one lookup per lane): a sphere the
// grid proves clear is dropped, one it proves colliding resolves its configuration at
// once, and only the undecided rest go on to the descent.  Those are few (a sphere is
// undecided only within about a cell of the distance r from the cloud), so they are
// carried across the warp's tiles with their global configuration index and processed
// in full rounds of 32; a hit there sets the configuration's flag directly (after the
// tile's own write, in the warp's program order).  Whatever is left when the warp runs
// out of tiles makes one last round.
// ------------------------------------------------------------------------------------
struct CfgGridScratch {
    float4 nc[kQueue];     // spheres that reach the cloud's box, awaiting classification: centre, r
    uint8_t ng[kQueue];    // their configuration within the tile
    float4 c2[64];         // undecided spheres carried to a round: centre, r^2
    uint32_t g2[64];       // their configuration (index into the flags)
    uint32_t ghit[32];     // per configuration of the tile: 1 once it collides
    uint32_t ghit2[32];    // per entry of a carried round: 1 once it collides
    RoundEntries re;
};

template <int CPT, int MODE>
__global__ void __launch_bounds__(512, CFG_MIN_BLOCKS) k_configs_grid(DevArgs t, const float* __restrict__ centers,
                                                                      const float* __restrict__ radii, uint64_t C,
                                                                      int S, uint8_t* __restrict__ out,
                                                                      unsigned long long* ctr, uint32_t pf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(16) float r2s[64];
    __shared__ __align__(16) float rs[64];
    for (int i = (int)threadIdx.x; i < S; i += (int)blockDim.x) {
        rs[i] = radii[i];
        r2s[i] = __fmul_rn(radii[i], radii[i]);
    }
    __syncthreads();
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    CfgGridScratch* ws = reinterpret_cast<CfgGridScratch*>(smem_raw) + warp;
    const uint64_t n_tiles = (C + CPT - 1) / CPT;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    const BoxPairs bp(rlo, rhi, t.nzero);
    const uint32_t inv_s = (1u << 20) / (uint32_t)S + 1u;   // i / S = (i * inv_s) >> 20 for i < 4096
    const bool s4 = (S & 3) == 0;

    uint32_t n2 = 0;   // carried undecided spheres (warp-uniform)
    uint64_t first = 0;
    uint32_t ncfg = 0;   // configurations of the current tile (0: none)

    // A round over the first n carried spheres; hits set their flags (and the current
    // tile's resolution); the rest of the carried queue moves to the front.
    auto carried_round = [&](uint32_t n) {
        const bool live = lane < n;
        const float4 c = live ? ws->c2[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t gg = live ? ws->g2[lane] : 0u;
        // an entry of the current tile whose configuration is already decided is skipped
        const uint64_t rel = (uint64_t)gg - first;
        ws->ghit2[lane] = (live && rel < ncfg && ws->ghit[rel]) ? 1u : 0u;
        __syncwarp();
        sphere_round<false, MODE>(t, nullptr, &ws->re, ws->ghit2, c, lane, live, lane, lt_mask);
        __syncwarp();
        if (live && ws->ghit2[lane]) {
            out[gg] = 1;
            if (rel < ncfg) ws->ghit[rel] = 1;
        }
        float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t g3 = 0;
        const bool mv = lane + n < n2;
        if (mv) {
            cc = ws->c2[lane + n];
            g3 = ws->g2[lane + n];
        }
        __syncwarp();
        if (mv) {
            ws->c2[lane] = cc;
            ws->g2[lane] = g3;
        }
        n2 -= n;
        __syncwarp();
    };

    uint32_t resolved = 0;
    uint32_t n1 = 0;
    // Classify the first n queued spheres by their grid cell; the rest of the queue
    // moves to the front.
    auto classify = [&](uint32_t n) {
        const bool live = lane < n;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t g = 0;
        int cls = 0;
        if (live) {
            c = ws->nc[lane];
            g = ws->ng[lane];
            if (!((resolved >> (g & 31u)) & 1u)) cls = grid_classify(t, c.x, c.y, c.z, c.w);
        }
        if (cls == 1) ws->ghit[g] = 1;
        const bool keep = cls == 2;
        const uint32_t km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t pos = n2 + __popc(km & lt_mask);
            ws->c2[pos] = make_float4(c.x, c.y, c.z, __fmul_rn(c.w, c.w));
            ws->g2[pos] = (uint32_t)(first + g);
        }
        n2 += __popc(km);
        // the rest of the queue (< 160 - n) to the front, 32 at a time in order
        for (uint32_t b = 0; b < n1 - n; b += 32) {
            const bool mv = b + lane < n1 - n;
            float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
            uint8_t gq = 0;
            if (mv) {
                cc = ws->nc[n + b + lane];
                gq = ws->ng[n + b + lane];
            }
            __syncwarp();
            if (mv) {
                ws->nc[b + lane] = cc;
                ws->ng[b + lane] = gq;
            }
            __syncwarp();
        }
        n1 -= n;
        __syncwarp();
        resolved = __ballot_sync(0xffffffffu, lane < ncfg && ws->ghit[lane]);
        if (n2 >= 32) carried_round(32);
        resolved = __ballot_sync(0xffffffffu, lane < ncfg && ws->ghit[lane]);
    };

    const TileSched sched{ctr, nwarps};
    for (uint64_t tile = sched.first((uint64_t)blockIdx.x * (blockDim.x >> 5) + warp); tile < n_tiles;
         tile = sched.next(tile)) {
        first = tile * CPT;
        ncfg = (uint32_t)min((uint64_t)CPT, C - first);
        const uint32_t nsph = ncfg * (uint32_t)S;
        const float* base = centers + 3 * first * (uint64_t)S;
        const bool vec = (reinterpret_cast<uintptr_t>(base) & 15u) == 0;
        if (lane < CPT) ws->ghit[lane] = 0;
        __syncwarp();
        resolved = 0;
        const uint32_t all_cfg = ncfg >= 32u ? 0xffffffffu : ((1u << ncfg) - 1u);
        n1 = 0;
        for (uint32_t p0 = 0; p0 < nsph; p0 += 128) {
            // ---- root box test of 4 consecutive spheres per lane ----
            const uint32_t i0 = p0 + 4 * lane;
            // the lane's centres pf passes ahead in this tile, asked of L2 while this pass
            // is tested (each lane's 48 bytes start in a different 128-byte line or share
            // one with a neighbour, so the lanes together cover the whole pass)
            if (pf && i0 + 128 * pf < nsph) prefetch_l2_line(base + 3 * (size_t)(i0 + 128 * pf));
            const uint32_t nv = i0 < nsph ? min(4u, nsph - i0) : 0u;
            float v[12];
            // every lane with four aligned centres (all passes but a tile's ragged last):
            // a warp-uniform branch, so the per-element path costs the others nothing
            if (__all_sync(0xffffffffu, vec && nv == 4)) {
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
            if (s4) {
                const float4 q2 = reinterpret_cast<const float4*>(r2s)[sidx >> 2];
                const float4 qr = reinterpret_cast<const float4*>(rs)[sidx >> 2];
                const float r2k[4] = {q2.x, q2.y, q2.z, q2.w};
                const float rk[4] = {qr.x, qr.y, qr.z, qr.w};
                const bool open = nv > 0 && !((resolved >> (g & 31u)) & 1u);
                float bd2[4];
                box_dist2_x4(v, bp, bd2);
                bool nk[4];
#pragma unroll
                for (int k = 0; k < 4; k++) nk[k] = open && (uint32_t)k < nv && bd2[k] <= r2k[k];
                // most passes have no sphere near the cloud's box at all: one vote skips
                // the four queue appends
                if (__any_sync(0xffffffffu, nk[0] | nk[1] | nk[2] | nk[3])) {
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const bool near = nk[k];
                        const uint32_t mask = __ballot_sync(0xffffffffu, near);
                        if (near) {
                            const uint32_t pos = n1 + __popc(mask & lt_mask);
                            ws->nc[pos] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], rk[k]);
                            ws->ng[pos] = (uint8_t)g;
                        }
                        n1 += __popc(mask);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float x = v[3 * k], y = v[3 * k + 1], z = v[3 * k + 2];
                    const bool near = (uint32_t)k < nv && !((resolved >> (g & 31u)) & 1u) &&
                                      box_dist2(x, y, z, rlo, rhi) <= r2s[sidx];
                    const uint32_t mask = __ballot_sync(0xffffffffu, near);
                    if (near) {
                        const uint32_t pos = n1 + __popc(mask & lt_mask);
                        ws->nc[pos] = make_float4(x, y, z, rs[sidx]);
                        ws->ng[pos] = (uint8_t)g;
                    }
                    n1 += __popc(mask);
                    if (++sidx == (uint32_t)S) { sidx = 0; g++; }
                }
            }
            __syncwarp();
            while (n1 >= 32) classify(32);
            // every configuration of the tile resolved: nothing left to learn
            if ((resolved & all_cfg) == all_cfg) { n1 = 0; break; }
        }
        if (n1) classify(n1);
        __syncwarp();
        if (lane < ncfg) out[first + lane] = (uint8_t)ws->ghit[lane];
        __syncwarp();
    }
    ncfg = 0;
    while (n2) carried_round(min(n2, 32u));
}

// Sequential work count per configuration (one thread each), in the order the query
// kernel's method defines it: every sphere up to the configuration's first hit gets the
// root box test; a sphere within reach of the cloud's box descends and gets the leaf box
// test of Alg. 3; a sphere passing that scans its set in stored order up to its first hit.
// counts += [spheres examined, spheres near the cloud box, spheres passing the leaf box,
// points scanned (Alg. 3 alone), chunk boxes tested, points scanned in the chunks whose
// box the sphere reaches (up to the first hit)].  The first four are the plain method's
// work; the query kernels do the first three, then the last two instead of the fourth.
// With per_sphere, radii holds one radius per sphere (C x S of them) instead of one per
// sphere slot of a configuration (S); sphere queries are counted as configurations of
// one sphere with their own radii.
// With use_grid, a sphere that reaches the cloud's box is first classified by the
// distance-bound grid (counts[6] lookups, counts[7] decided there: a certain miss needs
// nothing more, a certain hit ends its configuration); only the undecided descend.
__global__ void k_count_configs(DevArgs t, const float* __restrict__ centers, const float* __restrict__ radii,
                                uint64_t C, int S, bool per_sphere, bool use_grid, unsigned long long* counts) {
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nsph = 0, nnear = 0, npass = 0, npts = 0, nbox = 0, ncpts = 0, ngl = 0, ngd = 0;
    const float4* cbox = reinterpret_cast<const float4*>(t.cbox);
    const float4 rlo = make_float4(t.lo[0], t.lo[1], t.lo[2], 0.f);
    const float4 rhi = make_float4(t.hi[0], t.hi[1], t.hi[2], 0.f);
    if (c < C) {
        for (int s = 0; s < S; s++) {
            const float* x = centers + 3 * (c * (uint64_t)S + s);
            const float r = radii[per_sphere ? c * (uint64_t)S + s : (uint64_t)s], r2 = __fmul_rn(r, r);
            nsph++;
            if (!(box_dist2(x[0], x[1], x[2], rlo, rhi) <= r2)) continue;
            nnear++;
            if (use_grid) {
                ngl++;
                const int cls = grid_classify(t, x[0], x[1], x[2], r);
                if (cls != 2) ngd++;
                if (cls == 0) continue;
                if (cls == 1) break;
            }
            const uint32_t leaf = descend(x[0], x[1], x[2], t, nullptr);
            float4 a, b;
            load_leaf(t.leaves, leaf, a, b);
            const uint32_t cnt = __float_as_uint(b.w);
            if (cnt == 0 || !(box_dist2(x[0], x[1], x[2], a, b) <= r2)) continue;
            npass++;
            const uint32_t b0 = __float_as_uint(a.w);
            const size_t pl = 4 * (size_t)t.plane;
            bool hit = false;
            for (uint32_t j = 0; j < cnt && !hit; j++) {
                const float* bx = t.blocks + 4 * (size_t)(b0 + j / 4) + (j & 3u);
                npts++;
                hit = sq_dist(x[0], x[1], x[2], bx[0], bx[pl], bx[2 * pl]) <= r2;
            }
            // the same set walked chunk by chunk, points only in chunks whose box passes
            const uint32_t b1 = b0 + (cnt + 3u) / 4u;
            bool chit = false;
            for (uint32_t k = b0 / kChunkBlocks; k <= (b1 - 1u) / kChunkBlocks && !chit; k++) {
                nbox++;
                if (!(box_dist2(x[0], x[1], x[2], cbox[2 * k], cbox[2 * k + 1]) <= r2)) continue;
                const uint32_t j0 = max(b0, k * kChunkBlocks) * 4u - 4u * b0;
                const uint32_t j1 = min(b1 * 4u, (k + 1u) * kChunkBlocks * 4u) - 4u * b0;
                for (uint32_t j = j0; j < j1 && j < cnt && !chit; j++) {
                    const float* bx = t.blocks + 4 * (size_t)(b0 + j / 4) + (j & 3u);
                    ncpts++;
                    chit = sq_dist(x[0], x[1], x[2], bx[0], bx[pl], bx[2 * pl]) <= r2;
                }
            }
            if (chit != hit) atomicOr(t.status, kStatusBounds);   // the two walks must agree
            if (hit) break;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nsph += __shfl_xor_sync(0xffffffffu, nsph, o);
        nnear += __shfl_xor_sync(0xffffffffu, nnear, o);
        npass += __shfl_xor_sync(0xffffffffu, npass, o);
        npts += __shfl_xor_sync(0xffffffffu, npts, o);
        nbox += __shfl_xor_sync(0xffffffffu, nbox, o);
        ncpts += __shfl_xor_sync(0xffffffffu, ncpts, o);
        ngl += __shfl_xor_sync(0xffffffffu, ngl, o);
        ngd += __shfl_xor_sync(0xffffffffu, ngd, o);
    }
    if ((threadIdx.x & 31) == 0 && nsph) {
        atomicAdd(counts, nsph);
        atomicAdd(counts + 1, nnear);
        atomicAdd(counts + 2, npass);
        atomicAdd(counts + 3, npts);
        atomicAdd(counts + 4, nbox);
        atomicAdd(counts + 5, ncpts);
        atomicAdd(counts + 6, ngl);
        atomicAdd(counts + 7, ngd);
    }
}

// Chunk boxes: chunk k covers blocks [8k, 8k + 8); its box is the min / max of the
// finite coordinates there (unused slots hold +inf and are left out; a chunk with none
// gets the empty box lo = +inf, hi = -inf, which no sphere reaches).
__global__ void k_chunk_boxes(const float4* __restrict__ blocks, uint64_t plane, uint64_t total_blocks,
                              uint64_t n_chunks, float4* __restrict__ cbox) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_chunks) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const uint64_t b_end = min(total_blocks, (k + 1) * kChunkBlocks);
    for (uint64_t b = k * kChunkBlocks; b < b_end; b++)
        for (int d = 0; d < 3; d++) {
            const float4 q = blocks[d * plane + b];
            const float v[4] = {q.x, q.y, q.z, q.w};
            for (int u = 0; u < 4; u++)
                if (isfinite(v[u])) {
                    lo[d] = fminf(lo[d], v[u]);
                    hi[d] = fmaxf(hi[d], v[u]);
                }
        }
    cbox[2 * k] = make_float4(lo[0], lo[1], lo[2], 0.f);
    cbox[2 * k + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
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

using SphereKernel = void (*)(DevArgs, const float*, const float*, uint64_t, uint8_t*, unsigned long long*, bool);

template <int SPL, bool STAGE>
SphereKernel pick_spheres_mode(int mode) {
    switch (mode) {
        case kScanPlain: return k_spheres<SPL, STAGE, kScanPlain>;
        case kScanChunked: return k_spheres<SPL, STAGE, kScanChunked>;
        case kScanCompact: return k_spheres<SPL, STAGE, kScanCompact>;
        default: return nullptr;
    }
}

SphereKernel pick_spheres(int spl, bool stage, int mode) {
    switch (spl) {
        case 1: return stage ? pick_spheres_mode<1, true>(mode) : pick_spheres_mode<1, false>(mode);
        case 2: return stage ? pick_spheres_mode<2, true>(mode) : pick_spheres_mode<2, false>(mode);
        case 4: return stage ? pick_spheres_mode<4, true>(mode) : pick_spheres_mode<4, false>(mode);
        case 8: return stage ? pick_spheres_mode<8, true>(mode) : pick_spheres_mode<8, false>(mode);
        default: return nullptr;
    }
}

size_t sphere_scratch_bytes(int spl) {
    switch (spl) {
        case 1: return sizeof(SphereScratch<1>);
        case 2: return sizeof(SphereScratch<2>);
        case 4: return sizeof(SphereScratch<4>);
        default: return sizeof(SphereScratch<8>);
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

using ConfigKernel = void (*)(DevArgs, const float*, const float*, uint64_t, int, uint8_t*, unsigned long long*,
                              uint32_t);

template <int CPT, bool STAGE>
ConfigKernel pick_configs_mode(int mode) {
    switch (mode) {
        case kScanPlain: return k_configs<CPT, STAGE, kScanPlain>;
        case kScanChunked: return k_configs<CPT, STAGE, kScanChunked>;
        case kScanCompact: return k_configs<CPT, STAGE, kScanCompact>;
        default: return nullptr;
    }
}

ConfigKernel pick_configs(int spl, bool stage, int mode) {
    switch (spl) {
        case 2: return stage ? pick_configs_mode<4, true>(mode) : pick_configs_mode<4, false>(mode);
        case 4: return stage ? pick_configs_mode<8, true>(mode) : pick_configs_mode<8, false>(mode);
        case 8: return stage ? pick_configs_mode<16, true>(mode) : pick_configs_mode<16, false>(mode);
        case 16: return stage ? pick_configs_mode<32, true>(mode) : pick_configs_mode<32, false>(mode);
        default: return nullptr;
    }
}

using ConfigGridKernel = void (*)(DevArgs, const float*, const float*, uint64_t, int, uint8_t*, unsigned long long*,
                                  uint32_t);

template <int CPT>
ConfigGridKernel pick_configs_grid_mode(int mode) {
    switch (mode) {
        case kScanPlain: return k_configs_grid<CPT, kScanPlain>;
        case kScanChunked: return k_configs_grid<CPT, kScanChunked>;
        case kScanCompact: return k_configs_grid<CPT, kScanCompact>;
        default: return nullptr;
    }
}

ConfigGridKernel pick_configs_grid(int spl, int mode) {
    switch (spl) {
        case 2: return pick_configs_grid_mode<4>(mode);
        case 4: return pick_configs_grid_mode<8>(mode);
        case 8: return pick_configs_grid_mode<16>(mode);
        case 16: return pick_configs_grid_mode<32>(mode);
        default: return nullptr;
    }
}

// The configuration query with the distance-bound grid (k_configs_grid).
int launch_configs_grid(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S, uint8_t* out,
                        const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st, std::string& err) {
    ConfigGridKernel fn = pick_configs_grid(cfg.spheres_per_lane, cfg.chunk);
    if (!fn) { err = "configuration queries take spheres_per_lane 2, 4, 8 or 16"; return CAPT_E_ARG; }
    const int cpt = 2 * cfg.spheres_per_lane;
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = sizeof(CfgGridScratch) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int occ = std::max(1, occupancy((const void*)fn, warps * 32, smem));
    const uint64_t tiles = (C + cpt - 1) / cpt;
    const uint64_t need = (tiles + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    const uint32_t pf = (uint32_t)std::max(0, std::min(CAPT_MAX_PREFETCH, (int)cfg.prefetch));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, C, S, out, ctr, pf);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("configuration launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_configs(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S, uint8_t* out,
                   const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st, std::string& err) {
    // the grid path carries configuration indices in 32 bits
    if (cfg.grid && t.grid && C < (1ull << 32))
        return launch_configs_grid(t, centers, radii, C, S, out, cfg, ctr, st, err);
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    ConfigKernel fn = pick_configs(cfg.spheres_per_lane, stage, cfg.chunk);
    if (!fn) { err = "configuration queries take spheres_per_lane 2, 4, 8 or 16"; return CAPT_E_ARG; }
    const int cpt = 2 * cfg.spheres_per_lane;
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sizeof(CfgScratch) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int occ = std::max(1, occupancy((const void*)fn, warps * 32, smem));
    const uint64_t tiles = (C + cpt - 1) / cpt;
    const uint64_t need = (tiles + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    const uint32_t pf = (uint32_t)std::max(0, std::min(CAPT_MAX_PREFETCH, (int)cfg.prefetch));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, C, S, out, ctr, pf);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("configuration launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_query(const DevArgs& t, int mode, const float* centers, const float* radii, uint64_t n_items, int S,
                 uint8_t* out, const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st,
                 std::string& err) {
    if (n_items == 0) return CAPT_OK;
    if (mode == kModeConfigs) return launch_configs(t, centers, radii, n_items, S, out, cfg, ctr, st, err);
    const int spl = cfg.spheres_per_lane;
    const bool stage = cfg.staging == CAPT_STAGE_SMEM && t.stage_floats > 0;
    SphereKernel fn = pick_spheres(spl, stage, cfg.chunk);
    if (!fn) { err = "sphere queries take spheres_per_lane 1, 2, 4 or 8"; return CAPT_E_ARG; }
    const int warps = std::max(1, std::min(16, (int)cfg.warps_per_block));
    const size_t smem = (stage ? stage_offset(t) : 0u) + sphere_scratch_bytes(spl) * (size_t)warps;
    cudaError_t ce = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    const int occ = std::max(1, occupancy((const void*)fn, warps * 32, smem));
    const uint64_t per_tile = 32ull * spl;
    const uint64_t tiles = (n_items + per_tile - 1) / per_tile;
    const uint64_t need = (tiles + warps - 1) / warps;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count() * occ, need));
    fn<<<(unsigned)blocks, warps * 32, smem, st>>>(t, centers, radii, n_items, out, ctr, cfg.grid != 0 && t.grid);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("query launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_count_configs(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S,
                         bool per_sphere, bool use_grid, uint64_t* counts, cudaStream_t st, std::string& err) {
    if (C == 0) return CAPT_OK;
    const unsigned threads = 256;
    k_count_configs<<<(unsigned)((C + threads - 1) / threads), threads, 0, st>>>(
        t, centers, radii, C, S, per_sphere, use_grid && t.grid, reinterpret_cast<unsigned long long*>(counts));
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("count launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_chunk_boxes(const float* blocks, uint64_t total_blocks, float* cbox, cudaStream_t st, std::string& err) {
    const uint64_t n = chunk_count(total_blocks);
    const uint64_t plane = total_blocks > 0 ? total_blocks : 1;
    const unsigned threads = 256;
    k_chunk_boxes<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        reinterpret_cast<const float4*>(blocks), plane, total_blocks, n, reinterpret_cast<float4*>(cbox));
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("chunk box launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
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
