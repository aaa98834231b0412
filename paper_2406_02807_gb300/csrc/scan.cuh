// The affordance scan shared by the query and edge kernels.
//
// A "round" takes up to 32 queued spheres (centre and r^2, one per lane): each lane
// descends the tree, loads its leaf record and applies the leaf box test of Alg. 3;
// the spheres that pass become entries.  Their sets are then walked chunk by chunk
// (kChunkBlocks blocks of 4 points): every chunk first meets its FP32 bounding box,
// one chunk per lane, and only the chunks whose box the sphere reaches are scanned,
// 64 blocks per warp step.  Every lane test is three 16-byte loads and four FP32
// distance tests in packed FP32x2 arithmetic.
// The blocks are stored as three planes of float4 (x quads, y quads, z quads), so the
// loads of consecutive blocks by consecutive lanes are contiguous in each plane.
#pragma once

#include "device_common.cuh"


namespace capt {

// Packed FP32x2 arithmetic: two IEEE-rounded FP32 operations per instruction; the
// element results are bitwise those of the scalar __fsub_rn / __fmul_rn / __fadd_rn.
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
__device__ __forceinline__ float2 f2_split(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// Squared distances from a centre (each coordinate duplicated) to the four points of
// block b: ((p_x - c_x)^2 + (p_y - c_y)^2) + (p_z - c_z)^2 per point, each operation
// rounded; p - c is the exact negation of c - p, so the squares are those of the
// defining expression.  Returns the pairs (points 0,1) and (points 2,3).
// The block's quads live in three planes `plane` float4s apart.
__device__ __forceinline__ void block_d2(const float4* __restrict__ blocks, uint64_t plane, int64_t b, uint64_t cxx,
                                         uint64_t cyy, uint64_t czz, uint64_t& s01, uint64_t& s23) {
    const ulonglong2 px = __ldg(reinterpret_cast<const ulonglong2*>(blocks + b));
    const ulonglong2 py = __ldg(reinterpret_cast<const ulonglong2*>(blocks + plane + b));
    const ulonglong2 pz = __ldg(reinterpret_cast<const ulonglong2*>(blocks + 2 * plane + b));
    const uint64_t x01 = f2_sub(px.x, cxx), x23 = f2_sub(px.y, cxx);
    const uint64_t y01 = f2_sub(py.x, cyy), y23 = f2_sub(py.y, cyy);
    const uint64_t z01 = f2_sub(pz.x, czz), z23 = f2_sub(pz.y, czz);
    s01 = f2_add(f2_add(f2_mul(x01, x01), f2_mul(y01, y01)), f2_mul(z01, z01));
    s23 = f2_add(f2_add(f2_mul(x23, x23), f2_mul(y23, y23)), f2_mul(z23, z23));
}

// Does any of the four points of block b lie within r2 of the centre?
__device__ __forceinline__ bool block_hit2(const float4* __restrict__ blocks, uint64_t plane, int64_t b, uint64_t cxx,
                                           uint64_t cyy, uint64_t czz, float r2) {
    uint64_t s01, s23;
    block_d2(blocks, plane, b, cxx, cyy, czz, s01, s23);
    const float2 a = f2_split(s01), c = f2_split(s23);
    return (a.x <= r2) | (a.y <= r2) | (c.x <= r2) | (c.y <= r2);
}

// Per-warp storage of one round.
struct RoundEntries {
    float4 c[32];       // entry: centre and r^2
    uint32_t b0[32];    // its set's first block
    uint32_t b1[32];    // its set's end block
    uint32_t grp[32];   // its group (configuration of the tile)
    uint32_t cend[32];  // exclusive end of its chunks in the round's list of chunks
    uint2 q[64];        // chunks whose box the sphere reaches: {entry, chunk}
};

// One round over the spheres (c, g) held by lanes < n.  Groups already marked in
// ghit are skipped; a hit marks its group.  With SINGLE there is one group and the
// first hit ends the round (return value: whether a hit was found).
//  1. Each lane descends, loads its leaf record and applies the leaf box test of
//     Alg. 3; the spheres that pass are the round's entries.
//  2. Chunk boxes: the blocks are grouped in chunks of kChunkBlocks consecutive blocks
//     (32 points), each with the FP32 box of its points (t.cbox).  The entries' chunks
//     are tested 32 at a time, one per lane, against the sphere (the box test of
//     Alg. 3 at a finer grain: a box that holds p is never farther than p, so a sphere
//     that misses the box misses every point of the chunk).  Chunks that pass are
//     queued.
//  3. Queued chunks are scanned 8 at a time: lane l takes block l % 8 of chunks l / 8
//     and 4 + l / 8, within the entry's set; a hit resolves the entry's group.
template <bool SINGLE>
__device__ __forceinline__ bool sphere_round(const DevArgs& t, const float* Ts, RoundEntries* re, uint32_t* ghit,
                                             float4 c, uint32_t g, bool live, uint32_t lane, uint32_t lt_mask) {
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    const float4* cbox = reinterpret_cast<const float4*>(t.cbox);
    bool act = false;
    uint32_t b0 = 0, b1 = 0, nch = 0;
    if (live && (SINGLE || !ghit[g])) {
        const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
        float4 a, b;
        load_leaf(t.leaves, leaf, a, b);
        const uint32_t cnt = __float_as_uint(b.w);
        act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= c.w;
        if (act) {
            b0 = __float_as_uint(a.w);
            b1 = b0 + ((cnt + 3u) >> 2);
            nch = (b1 - 1u) / kChunkBlocks - b0 / kChunkBlocks + 1u;
        }
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, act);
    if (mask == 0) return false;
    const uint32_t incl = warp_incl_scan(nch);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t n_ent = __popc(mask);
    __syncwarp();
    if (act) {
        const uint32_t pos = __popc(mask & lt_mask);
        re->c[pos] = c;
        re->b0[pos] = b0;
        re->b1[pos] = b1;
        re->grp[pos] = g;
        re->cend[pos] = incl;
    }
    __syncwarp();
    bool found = false;
    uint32_t nq = 0;   // queued chunks (warp-uniform)
    uint32_t ei = 0;   // this lane's entry in the chunk walk (monotone)
    for (uint32_t base = 0; base < total; base += 32) {
        // ---- 2. one chunk box per lane ----
        const uint32_t p = base + lane;
        bool pass = false;
        uint2 item = make_uint2(0u, 0u);
        if (p < total) {
            while (re->cend[ei] <= p) ei++;
            if (SINGLE || !ghit[re->grp[ei]]) {
                const float4 ce = re->c[ei];
                const uint32_t k = re->b0[ei] / kChunkBlocks + (p - (ei ? re->cend[ei - 1] : 0u));
                const float4 lo = __ldg(cbox + 2 * (size_t)k), hi = __ldg(cbox + 2 * (size_t)k + 1);
                pass = box_dist2(ce.x, ce.y, ce.z, lo, hi) <= ce.w;
                item = make_uint2(ei, k);
            }
        }
        const uint32_t pm = __ballot_sync(0xffffffffu, pass);
        if (pass) re->q[nq + __popc(pm & lt_mask)] = item;
        nq += __popc(pm);
        __syncwarp();
        // ---- 3. scan queued chunks, 8 per step (all that are left after the last box step) ----
        const bool last = base + 32 >= total;
        while (nq >= 8 || (last && nq > 0)) {
            bool h = false;
            uint64_t s01[2], s23[2];
            float r2v[2];
            uint32_t gv[2];
            bool v_ok[2];
#pragma unroll
            for (int v = 0; v < 2; v++) {
                const uint32_t j = (lane >> 3) + 4u * v;
                v_ok[v] = false;
                s01[v] = s23[v] = 0;
                r2v[v] = 0.f;
                gv[v] = 0;
                if (j < nq) {
                    const uint2 it = re->q[j];
                    const uint32_t b = it.y * kChunkBlocks + (lane & 7u);
                    gv[v] = re->grp[it.x];
                    if (b >= re->b0[it.x] && b < re->b1[it.x] && (SINGLE || !ghit[gv[v]])) {
                        const float4 ce = re->c[it.x];
                        block_d2(blocks, t.plane, (int64_t)b, f2_dup(ce.x), f2_dup(ce.y), f2_dup(ce.z), s01[v], s23[v]);
                        r2v[v] = ce.w;
                        v_ok[v] = true;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < 2; v++) {
                if (v_ok[v]) {
                    const float2 x = f2_split(s01[v]), y = f2_split(s23[v]);
                    const bool hv = (x.x <= r2v[v]) | (x.y <= r2v[v]) | (y.x <= r2v[v]) | (y.y <= r2v[v]);
                    if (!SINGLE && hv) ghit[gv[v]] = 1;
                    h |= hv;
                }
            }
            if (SINGLE && __any_sync(0xffffffffu, h)) { found = true; break; }
            // drop the (up to) 8 chunks just scanned
            const uint32_t done = nq < 8u ? nq : 8u;
            uint2 keep = make_uint2(0u, 0u);
            if (lane + done < nq) keep = re->q[lane + done];
            __syncwarp();
            if (lane + done < nq) re->q[lane] = keep;
            nq -= done;
            __syncwarp();
        }
        if (found) break;
        if (!SINGLE) {
            // leave once every entry is resolved
            const bool open = lane < n_ent && !ghit[re->grp[lane]];
            if (!__any_sync(0xffffffffu, open)) break;
        }
    }
    __syncwarp();
    return found;
}

}  // namespace capt
