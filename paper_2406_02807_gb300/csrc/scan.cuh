// The affordance scan shared by the query and edge kernels.
//
// A "round" takes up to 32 queued spheres (centre and r^2, one per lane): each lane
// descends the tree, loads its leaf record and applies the leaf box test of Alg. 3;
// the spheres that pass become entries.  In the chunked form their sets are then
// walked chunk by chunk (kChunkBlocks blocks of 4 points): every chunk first meets its
// FP32 bounding box, one chunk per lane, and only the chunks whose box the sphere
// reaches are scanned, 64 blocks per warp step; the compact form walks the chunks of
// the Z-ordered cloud that a leaf lists.  The plain form scans whole sets.  Every lane
// test is three 16-byte loads and four FP32 distance tests in packed FP32x2 arithmetic.
// The blocks are stored as three planes of float4 (x quads, y quads, z quads), so the
// loads of consecutive blocks by consecutive lanes are contiguous in each plane.
#pragma once

#include "device_common.cuh"


namespace capt {

// Packed FP32x2 arithmetic: two IEEE-rounded FP32 operations per instruction; the
// element results are bitwise those of the scalar __fsub_rn / __fmul_rn / __fadd_rn.
// One trap: the code generator fuses a packed multiply whose product has a single use
// into the packed add (or sub, or fma) that consumes it, whatever rounding modifier
// either carries, and a fused multiply-add rounds the sum of products once instead of
// twice (measured on sm_103a: about a fifth of the squared distances changed).  So a
// product that feeds a sum is formed by f2_mulz, an fma with a zero addend that only
// the kernel's arguments know (DevArgs::nzero = -0): fl(a * b + (-0)) = fl(a * b)
// exactly, and an fma is never fused into the add after it.
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
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a * b rounded, element by element; z = f2_dup(t.nzero)
__device__ __forceinline__ uint64_t f2_mulz(uint64_t a, uint64_t b, uint64_t z) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(z));
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
// The block's quads live in three planes `plane` float4s apart; z = f2_dup(t.nzero).
__device__ __forceinline__ void block_d2(const float4* __restrict__ blocks, uint64_t plane, int64_t b, uint64_t cxx,
                                         uint64_t cyy, uint64_t czz, uint64_t z, uint64_t& s01, uint64_t& s23) {
    const ulonglong2 px = __ldg(reinterpret_cast<const ulonglong2*>(blocks + b));
    const ulonglong2 py = __ldg(reinterpret_cast<const ulonglong2*>(blocks + plane + b));
    const ulonglong2 pz = __ldg(reinterpret_cast<const ulonglong2*>(blocks + 2 * plane + b));
    const uint64_t x01 = f2_sub(px.x, cxx), x23 = f2_sub(px.y, cxx);
    const uint64_t y01 = f2_sub(py.x, cyy), y23 = f2_sub(py.y, cyy);
    const uint64_t z01 = f2_sub(pz.x, czz), z23 = f2_sub(pz.y, czz);
    s01 = f2_add(f2_add(f2_mulz(x01, x01, z), f2_mulz(y01, y01, z)), f2_mulz(z01, z01, z));
    s23 = f2_add(f2_add(f2_mulz(x23, x23, z), f2_mulz(y23, y23, z)), f2_mulz(z23, z23, z));
}

// max(a, b, c), NaN if any input is NaN (one instruction on sm_100 and later).
__device__ __forceinline__ float max3_nan(float a, float b, float c) {
    float d;
    asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The bounds of a box arranged for the interleaved coordinates of four consecutive
// centres, loaded as three float4 {x0 y0 z0 x1} {y1 z1 x2 y2} {z2 x3 y3 z3}: as register
// pairs these are (x, y), (z, x), (y, z) twice, so the box's lower and upper corners
// come in those three orders.
struct BoxPairs {
    uint64_t lxy, lzx, lyz, hxy, hzx, hyz, z;   // z: f2_dup(t.nzero)
    __device__ __forceinline__ BoxPairs(const float4& lo, const float4& hi, float nzero) {
        asm("mov.b64 %0, {%1, %2};" : "=l"(lxy) : "f"(lo.x), "f"(lo.y));
        asm("mov.b64 %0, {%1, %2};" : "=l"(lzx) : "f"(lo.z), "f"(lo.x));
        asm("mov.b64 %0, {%1, %2};" : "=l"(lyz) : "f"(lo.y), "f"(lo.z));
        asm("mov.b64 %0, {%1, %2};" : "=l"(hxy) : "f"(hi.x), "f"(hi.y));
        asm("mov.b64 %0, {%1, %2};" : "=l"(hzx) : "f"(hi.z), "f"(hi.x));
        asm("mov.b64 %0, {%1, %2};" : "=l"(hyz) : "f"(hi.y), "f"(hi.z));
        z = f2_dup(nzero);
    }
};

// Squared gaps of one coordinate pair to the box: per element max(lo - x, x - hi, 0)
// (the magnitude of x - clamp(x, lo, hi), the same bits once squared; NaN stays NaN),
// squared exactly.
__device__ __forceinline__ float2 box_gap2(float x0, float x1, uint64_t lo, uint64_t hi, uint64_t z) {
    uint64_t x;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
    const float2 a = f2_split(f2_sub(lo, x)), b = f2_split(f2_sub(x, hi));
    uint64_t g;
    asm("mov.b64 %0, {%1, %2};" : "=l"(g) : "f"(max3_nan(a.x, b.x, 0.f)), "f"(max3_nan(a.y, b.y, 0.f)));
    return f2_split(f2_mulz(g, g, z));
}

// box_dist2 of four consecutive centres v[0..11] (x0 y0 z0 x1 y1 z1 ...), bit for bit:
// ((gx^2 + gy^2) + gz^2) per centre, the differences and squares two at a time.
__device__ __forceinline__ void box_dist2_x4(const float v[12], const BoxPairs& bp, float d2[4]) {
    const float2 p0 = box_gap2(v[0], v[1], bp.lxy, bp.hxy, bp.z);    // x0 y0
    const float2 p1 = box_gap2(v[2], v[3], bp.lzx, bp.hzx, bp.z);    // z0 x1
    const float2 p2 = box_gap2(v[4], v[5], bp.lyz, bp.hyz, bp.z);    // y1 z1
    const float2 p3 = box_gap2(v[6], v[7], bp.lxy, bp.hxy, bp.z);    // x2 y2
    const float2 p4 = box_gap2(v[8], v[9], bp.lzx, bp.hzx, bp.z);    // z2 x3
    const float2 p5 = box_gap2(v[10], v[11], bp.lyz, bp.hyz, bp.z);  // y3 z3
    d2[0] = __fadd_rn(__fadd_rn(p0.x, p0.y), p1.x);
    d2[1] = __fadd_rn(__fadd_rn(p1.y, p2.x), p2.y);
    d2[2] = __fadd_rn(__fadd_rn(p3.x, p3.y), p4.x);
    d2[3] = __fadd_rn(__fadd_rn(p4.y, p5.x), p5.y);
}

// Per-warp storage of one round.
struct RoundEntries {
    float4 c[32];       // entry: centre and r^2
    uint32_t grp[32];   // its group (configuration of the tile)
    // chunked form
    uint32_t b0[32];    // its set's first block
    uint32_t b1[32];    // its set's end block
    uint32_t cend[32];  // exclusive end of its chunks in the round's list of chunks
    uint2 q[64];        // chunks whose box the sphere reaches: {entry, chunk}
    // plain form
    int32_t boff[32];   // first block minus the entry's start in the concatenated list
    uint32_t end[32];   // exclusive end of the entry in the concatenated list
};

// One round over the spheres (c, g) held by lanes < n, chunked form.  Groups already
// marked in ghit are skipped; a hit marks its group.  With SINGLE there is one group
// and the first hit ends the round (return value: whether a hit was found).
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
// With COMPACT the sets are the de-duplicated form (t.cleaves, t.clist): a leaf lists
// the chunks of the Z-ordered cloud that hold a point of its set, and the walk visits
// those chunks (whole, 32 points each; the union is a superset of the set inside the
// cloud, so the flags are the same).
template <bool SINGLE, bool COMPACT>
__device__ __forceinline__ bool round_chunked(const DevArgs& t, const float* Ts, RoundEntries* re, uint32_t* ghit,
                                              float4 c, uint32_t g, bool live, uint32_t lane, uint32_t lt_mask) {
    const float4* blocks = reinterpret_cast<const float4*>(COMPACT ? t.cblocks : t.blocks);
    const uint64_t plane = COMPACT ? t.cplane : t.plane;
    const float4* cbox = reinterpret_cast<const float4*>(COMPACT ? t.ccbox : t.cbox);
    bool act = false;
    uint32_t b0 = 0, b1 = 0, nch = 0;
    if (live && (SINGLE || !ghit[g])) {
        const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
        float4 a, b;
        load_leaf(COMPACT ? t.cleaves : t.leaves, leaf, a, b);
        const uint32_t cnt = __float_as_uint(b.w);
        act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= c.w;
        if (act) {
            b0 = __float_as_uint(a.w);
            if (COMPACT) {
                nch = cnt;   // b0: first entry of the leaf's chunk list
            } else {
                b1 = b0 + ((cnt + 3u) >> 2);
                nch = (b1 - 1u) / kChunkBlocks - b0 / kChunkBlocks + 1u;
            }
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
    // This lane's (entry, chunk) at position p of the walk.  In the compact form the
    // position one step ahead is looked up before the current box is tested, so that
    // its list load overlaps the box load.
    uint32_t ei = 0, k = 0;
    auto locate = [&](uint32_t p) {
        while (re->cend[ei] <= p) ei++;
        const uint32_t j = p - (ei ? re->cend[ei - 1] : 0u);
        k = COMPACT ? __ldg(t.clist + re->b0[ei] + j) : re->b0[ei] / kChunkBlocks + j;
    };
    if (COMPACT && lane < total) locate(lane);
    for (uint32_t base = 0; base < total; base += 32) {
        // ---- 2. one chunk box per lane ----
        const uint32_t p = base + lane;
        if (!COMPACT && p < total) locate(p);
        const uint32_t ec = ei, kc = k;
        if (COMPACT && p + 32 < total) locate(p + 32);
        bool pass = false;
        uint2 item = make_uint2(0u, 0u);
        if (p < total && (SINGLE || !ghit[re->grp[ec]])) {
            const float4 ce = re->c[ec];
            const float4 lo = __ldg(cbox + 2 * (size_t)kc), hi = __ldg(cbox + 2 * (size_t)kc + 1);
            pass = box_dist2(ce.x, ce.y, ce.z, lo, hi) <= ce.w;
            item = make_uint2(ec, kc);
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
                    if ((COMPACT || (b >= re->b0[it.x] && b < re->b1[it.x])) && (SINGLE || !ghit[gv[v]])) {
                        const float4 ce = re->c[it.x];
                        block_d2(blocks, plane, (int64_t)b, f2_dup(ce.x), f2_dup(ce.y), f2_dup(ce.z), f2_dup(t.nzero), s01[v],
                                 s23[v]);
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

// The plain form of a round (Alg. 3's scan of each whole set, no chunk boxes): when
// the sets are large (at least 32 blocks each on average) the warp scans one set at a
// time with all lanes (lane l on blocks l, l + 32, ..., two per step); otherwise it
// walks the concatenation of all the sets 32 blocks at a time.  It wins where chunk
// boxes are loose (point indices with no spatial order) or sets are a chunk or two.
template <bool SINGLE>
__device__ __forceinline__ bool round_plain(const DevArgs& t, const float* Ts, RoundEntries* re, uint32_t* ghit,
                                             float4 c, uint32_t g, bool live, uint32_t lane, uint32_t lt_mask) {
    const float4* blocks = reinterpret_cast<const float4*>(t.blocks);
    bool act = false;
    uint32_t nb = 0, fb = 0;
    if (live && (SINGLE || !ghit[g])) {
        const uint32_t leaf = descend(c.x, c.y, c.z, t, Ts);
        float4 a, b;
        load_leaf(t.leaves, leaf, a, b);
        const uint32_t cnt = __float_as_uint(b.w);
        act = cnt > 0 && box_dist2(c.x, c.y, c.z, a, b) <= c.w;
        nb = act ? (cnt + 3u) >> 2 : 0u;
        fb = __float_as_uint(a.w);
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, act);
    if (mask == 0) return false;
    const uint32_t incl = warp_incl_scan(nb);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t n_ent = __popc(mask);
    __syncwarp();
    if (act) {
        const uint32_t pos = __popc(mask & lt_mask);
        re->c[pos] = c;
        re->boff[pos] = (int32_t)fb - (int32_t)(incl - nb);
        re->end[pos] = incl;
        re->grp[pos] = g;
    }
    __syncwarp();
    bool found = false;
    if (total >= 32u * n_ent) {
    // Large sets: one entry at a time, the whole warp on its blocks (lane l takes blocks
    // fb + l + 32 k, V per step), so block addresses need no per-lane lookup; a hit
    // resolves the entry's group.
    constexpr int V = 2;
    for (uint32_t e = 0; e < n_ent; e++) {
        const uint32_t ge = re->grp[e];
        if (!SINGLE && ghit[ge]) continue;
        const float4 ce = re->c[e];
        const uint32_t b_end = re->end[e];
        const uint32_t b_beg = e ? re->end[e - 1] : 0u;
        const int64_t o = (int64_t)re->boff[e];
        const uint64_t cxx = f2_dup(ce.x), cyy = f2_dup(ce.y), czz = f2_dup(ce.z), z2 = f2_dup(t.nzero);
        bool hit = false;
        for (uint32_t p = b_beg + lane; __any_sync(0xffffffffu, p < b_end); p += 32 * V) {
            uint64_t s01[V], s23[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                s01[v] = s23[v] = 0;
                if (p + 32 * v < b_end) block_d2(blocks, t.plane, o + p + 32 * v, cxx, cyy, czz, z2, s01[v], s23[v]);
            }
            bool h = false;
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (p + 32 * v < b_end) {
                    const float2 x = f2_split(s01[v]), y = f2_split(s23[v]);
                    h |= (x.x <= ce.w) | (x.y <= ce.w) | (y.x <= ce.w) | (y.y <= ce.w);
                }
            }
            if (__any_sync(0xffffffffu, h)) { hit = true; break; }
        }
        if (hit) {
            if (SINGLE) { found = true; break; }
            if (lane == 0) ghit[ge] = 1;
            __syncwarp();
        }
    }
    } else {
    // Small sets: the concatenated blocks of all entries, U per lane per step (32 U per
    // warp step), lane l taking blocks base + l + 32 u; each lane keeps the fields of the
    // entries it is in, reloading them only when it moves on.
    constexpr int U = 1;
    uint32_t ei[U], ce[U];
    float4 cc[U];
    int32_t oo[U];
    uint32_t gg[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        ei[u] = 0;
        ce[u] = 0xffffffffu;
        cc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        oo[u] = 0;
        gg[u] = 0;
    }
    for (uint32_t base = 0; base < total; base += 32 * U) {
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t p = base + lane + 32u * u;
            live[u] = p < total;
            if (live[u]) {
                if (u > 0 && ei[u] < ei[u - 1]) ei[u] = ei[u - 1];
                while (re->end[ei[u]] <= p) ei[u]++;
                if (ei[u] != ce[u]) {
                    cc[u] = re->c[ei[u]];
                    oo[u] = re->boff[ei[u]];
                    gg[u] = re->grp[ei[u]];
                    ce[u] = ei[u];
                }
                live[u] = SINGLE || !ghit[gg[u]];
            }
        }
        uint64_t s01[U], s23[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            s01[u] = s23[u] = 0;
            if (live[u])
                block_d2(blocks, t.plane, (int64_t)oo[u] + base + lane + 32u * u, f2_dup(cc[u].x), f2_dup(cc[u].y),
                         f2_dup(cc[u].z), f2_dup(t.nzero), s01[u], s23[u]);
        }
        bool h = false;
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (!live[u]) continue;
            const float2 x = f2_split(s01[u]), y = f2_split(s23[u]);
            const bool hu = (x.x <= cc[u].w) | (x.y <= cc[u].w) | (y.x <= cc[u].w) | (y.y <= cc[u].w);
            if (!SINGLE && hu) ghit[gg[u]] = 1;
            h |= hu;
        }
        if (SINGLE) {
            if (__any_sync(0xffffffffu, h)) { found = true; break; }
            continue;
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, h)) {
            // leave once every entry that still has blocks ahead is resolved
            const bool open = lane < n_ent && re->end[lane] > base + 32 * U && !ghit[re->grp[lane]];
            if (!__any_sync(0xffffffffu, open)) break;
        }
    }
    }
    __syncwarp();
    return found;
}

// Scan modes of a round: whole sets, chunk boxes over the sets, or the compact
// (de-duplicated) sets.
enum ScanMode : int { kScanPlain = 0, kScanChunked = 1, kScanCompact = 2 };

// One round over the spheres (c, g) held by lanes < n in the given scan mode.
template <bool SINGLE, int MODE = kScanChunked>
__device__ __forceinline__ bool sphere_round(const DevArgs& t, const float* Ts, RoundEntries* re, uint32_t* ghit,
                                             float4 c, uint32_t g, bool live, uint32_t lane, uint32_t lt_mask) {
    if constexpr (MODE == kScanPlain) return round_plain<SINGLE>(t, Ts, re, ghit, c, g, live, lane, lt_mask);
    else return round_chunked<SINGLE, MODE == kScanCompact>(t, Ts, re, ghit, c, g, live, lane, lt_mask);
}

}  // namespace capt
