// CAPT construction on the GPU (Alg. 1, Sec. IV-A/B).  The result is the host
// builder's tree bit for bit: the same split values, the same affordance sets in
// ascending point index, the same FP32 boxes and prune decisions.
//
// 1. Medians.  The points (padded to N = 2^L with +inf) are sorted once per axis by
//    (coordinate, index) with a stable LSD radix sort.  Level by level, every node's
//    points occupy the same aligned segment of length m = N >> l in all three orders.
//    In the order of the level's axis the segment is sorted, so its first half is B1
//    and T_i is the coordinate of its last element; the other two orders are stably
//    partitioned into (B1, B2), which keeps them sorted inside both children.  After L
//    levels each segment holds one point, the leaf's representative t.
// 2. Affordance sets.  In Alg. 1 the set z reaching a node is every point outside the
//    node's subtree that the node's closed cell affords: the FP64 distance to a cell
//    can only grow when the cell shrinks (each rounded step is monotone), so testing
//    z u B2 against the child cell c1 keeps exactly the points that a direct test
//    against c1 keeps.  A leaf's set is therefore {p : cell affords p}, which already
//    holds t (distance 0), or {t} when the r_min test prunes it.  It is computed per
//    leaf over the points that a uniform grid of the cloud places within reach of the
//    cell, with the host builder's FP64 predicate; an FP32 evaluation decides first
//    when it is farther than its error bound from the threshold.
// 3. Each set is sorted by point index (per-warp stable radix sort) and written in the
//    device layout (three planes of 4-point blocks, ids, 32-byte leaf records).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/capt.h"
#include "capt_internal.h"
#include "device_build.h"
#include "device_common.cuh"
#include "kernels.h"

namespace capt {
namespace {


__device__ __forceinline__ float coord(const float* __restrict__ pts, uint32_t n, uint32_t i, int d) {
    return i < n ? pts[3 * (size_t)i + d] : INFINITY;
}

__global__ void k_fill_f32(float* __restrict__ p, uint64_t count, float v) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs: 8-bit digits, one element per thread.
// ---------------------------------------------------------------------------------
constexpr int kSortThreads = 256;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift, uint32_t* __restrict__ hist,
                             uint32_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Exclusive scan of len values in place by one block (chunks of blockDim with a carry).
__global__ void k_scan_exclusive(uint32_t* __restrict__ v, uint32_t len) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t base = 0; base < len; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < len ? v[i] : 0u;
        const uint32_t incl = warp_incl_scan(x);
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t y = lane < nw ? ws[lane] : 0u;
            y = warp_incl_scan(y);
            if (lane < nw) ws[lane] = y;
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? ws[warp - 1] : 0u);
        if (i < len) v[i] = before + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[nw - 1];
        __syncthreads();
    }
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t n,
                                int shift, const uint32_t* __restrict__ off, uint32_t nblocks,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    for (uint32_t j = threadIdx.x; j < (kSortThreads / 32) * 256; j += kSortThreads) (&cnt[0][0])[j] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * kSortThreads + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
        uint32_t before = 0;
        for (uint32_t w = 0; w < warp; w++) before += cnt[w][d];
        const uint32_t pos = off[d * nblocks + blockIdx.x] + before + rank;
        kout[pos] = k;
        vout[pos] = vin[i];
    }
}

// ---------------------------------------------------------------------------------
// Medians level by level
// ---------------------------------------------------------------------------------
__global__ void k_init_keys(const float* __restrict__ pts, uint32_t n, uint32_t N, int d, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        keys[i] = fkey(coord(pts, n, i, d));
        vals[i] = i;
    }
}

// Level l along axis d (segments of m = 2^lg_m): split value per segment and the side
// of every point.
__global__ void k_level_split(const float* __restrict__ pts, uint32_t n, uint32_t N, int lg_m, int d,
                              const uint32_t* __restrict__ ord_d, uint32_t level_base, float* __restrict__ T,
                              uint8_t* __restrict__ left) {
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const uint32_t m = 1u << lg_m, r = pos & (m - 1u);
    const uint32_t p = ord_d[pos];
    left[p] = r < (m >> 1) ? 1 : 0;
    if (r == (m >> 1) - 1u) T[level_base + (pos >> lg_m)] = coord(pts, n, p, d);
}

// Stable partition of every aligned segment of length m = 2^lg_m by side.  Tiles of
// 1024 positions give each position its exclusive count of left points before it in
// its segment and tile; segments longer than a tile add the left counts of their
// earlier tiles (k_part_segments).
constexpr uint32_t kTile = 1024;

__global__ void __launch_bounds__(kTile) k_part_tiles(const uint32_t* __restrict__ ord, uint32_t N, int lg_m,
                                                      const uint8_t* __restrict__ left,
                                                      uint32_t* __restrict__ rank_left,
                                                      uint32_t* __restrict__ tile_left) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t incl_s[kTile];
    const uint32_t pos = blockIdx.x * kTile + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t f = pos < N ? left[ord[pos]] : 0u;
    const uint32_t incl = warp_incl_scan(f);
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) ws[lane] = warp_incl_scan(ws[lane]);
    __syncthreads();
    uint32_t v = incl + (warp ? ws[warp - 1] : 0u);   // inclusive count over the tile
    const uint32_t m = 1u << lg_m;
    if (m < kTile) {                                  // restart at every segment start
        incl_s[threadIdx.x] = v;
        __syncthreads();
        const uint32_t seg_start = threadIdx.x & ~(m - 1u);
        if (seg_start) v -= incl_s[seg_start - 1u];
    }
    if (pos < N) rank_left[pos] = v - f;
    if (threadIdx.x == kTile - 1) tile_left[blockIdx.x] = ws[31];
}

__global__ void k_part_segments(uint32_t* __restrict__ tile_left, uint32_t n_seg, uint32_t tiles_per_seg) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < tiles_per_seg; k++) {
        const uint32_t v = tile_left[s * tiles_per_seg + k];
        tile_left[s * tiles_per_seg + k] = acc;
        acc += v;
    }
}

__global__ void k_part_scatter(const uint32_t* __restrict__ ord, uint32_t N, int lg_m, const uint8_t* __restrict__ left,
                               const uint32_t* __restrict__ rank_left, const uint32_t* __restrict__ tile_left,
                               uint32_t* __restrict__ out) {
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;
    const uint32_t m = 1u << lg_m, half = m >> 1;
    const uint32_t seg0 = pos & ~(m - 1u), r = pos - seg0;
    const uint32_t p = ord[pos];
    uint32_t lb = rank_left[pos];   // left points before pos in its segment
    if (m > kTile) lb += tile_left[pos / kTile];
    out[left[p] ? seg0 + lb : seg0 + half + (r - lb)] = p;
}

// ---------------------------------------------------------------------------------
// Bounding box, grid, sets and layout
// ---------------------------------------------------------------------------------
// box: six order keys (atomicMin on lo, atomicMax on hi), then a non-finite flag (the
// eighth word is the set pass check of k_leaf_sets).
__global__ void k_bbox(const float* __restrict__ pts, uint32_t n, uint32_t* __restrict__ box) {
    __shared__ uint32_t s[6][256];
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    uint32_t nonfinite = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < 3; d++) {
            const float v = pts[3 * (size_t)i + d];
            nonfinite |= isfinite(v) ? 0u : 1u;
            const uint32_t k = fkey(v);
            lo[d] = min(lo[d], k);
            hi[d] = max(hi[d], k);
        }
    for (int d = 0; d < 3; d++) {
        s[d][threadIdx.x] = lo[d];
        s[3 + d][threadIdx.x] = hi[d];
    }
    if (nonfinite) atomicOr(box + 6, 1u);
    __syncthreads();
    for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; d++) {
                s[d][threadIdx.x] = min(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = max(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; d++) {
            atomicMin(box + d, s[d][0]);
            atomicMax(box + 3 + d, s[3 + d][0]);
        }
}

struct GridDesc {
    double origin[3];
    double g;   // cell edge
    int dims[3];
};

// Grid coordinate of v along one axis, clamped to the grid (monotone in v).
__device__ __forceinline__ int grid_coord(double v, double o, double g, int dim) {
    const double f = floor(__ddiv_rn(__dsub_rn(v, o), g));
    return f < 0.0 ? 0 : (f >= (double)dim ? dim - 1 : (int)f);
}

__device__ __forceinline__ uint32_t grid_cell_of(const GridDesc& gd, const float* p) {
    const int cx = grid_coord(p[0], gd.origin[0], gd.g, gd.dims[0]);
    const int cy = grid_coord(p[1], gd.origin[1], gd.g, gd.dims[1]);
    const int cz = grid_coord(p[2], gd.origin[2], gd.g, gd.dims[2]);
    return ((uint32_t)cz * gd.dims[1] + cy) * gd.dims[0] + cx;
}

__global__ void k_grid_count(const float* __restrict__ pts, uint32_t n, GridDesc gd, uint32_t* __restrict__ cell_of,
                             uint32_t* __restrict__ cnt) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = grid_cell_of(gd, pts + 3 * (size_t)i);
    cell_of[i] = c;
    atomicAdd(cnt + c, 1u);
}

__global__ void k_grid_fill(uint32_t n, const uint32_t* __restrict__ cell_of, uint32_t* __restrict__ cursor,
                            uint32_t* __restrict__ items) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) items[atomicAdd(cursor + cell_of[i], 1u)] = i;
}

struct SetArgs {
    const float* pts;
    uint32_t n, N;
    int L;
    const float* T;       // plain Eytzinger split values
    const uint32_t* rep;  // representative per leaf (>= n: pad)
    double thr_afford, thr_prune;   // squared FP64 thresholds of the host builder
    double reach;                   // linear reach of the grid walk (>= sqrt(thr_afford))
    float f32_in, f32_out;          // FP32 decision bounds (f32_in < 0: FP64 always)
    GridDesc gd;
    const uint32_t* cell_start;     // [cells + 1]
    const uint32_t* items;          // point indices grouped by cell
};

// Closed cell of leaf l from the splits on its path (+-inf where none bounds it).
__device__ __forceinline__ void leaf_cell(const SetArgs& a, uint32_t l, double lo[3], double hi[3]) {
    for (int d = 0; d < 3; d++) {
        lo[d] = -INFINITY;
        hi[d] = INFINITY;
    }
    uint32_t i = 0;
    for (int k = 0; k < a.L; k++) {
        const uint32_t bit = (l >> (a.L - 1 - k)) & 1u;
        const double t = a.T[i];
        if (bit) lo[k % 3] = t;
        else hi[k % 3] = t;
        i = 2 * i + 1 + bit;
    }
}

// The host builder's FP64 affordance predicate, one rounded operation at a time.
__device__ __forceinline__ bool affords64(const double lo[3], const double hi[3], const float p[3], double thr) {
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double v = p[d];
        double q = v;
        if (q < lo[d]) q = lo[d];
        if (q > hi[d]) q = hi[d];
        const double e = __dsub_rn(v, q);
        s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return s <= thr;
}

// The same predicate, decided in FP32 where that is safe.  Each clamp is exact and
// each of the FP32 steps has relative error <= 2^-24, so the FP32 sum lies within a
// factor (1 +- 2^-21) of the FP64 one (for thresholds in [1e-30, 1e30], away from
// under- and overflow); f32_in / f32_out sit 1e-5 (relative) inside / outside the
// threshold and only the values between them are decided in FP64.
__device__ __forceinline__ bool affords(const SetArgs& a, const float flo[3], const float fhi[3], const double lo[3],
                                        const double hi[3], const float p[3]) {
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float q = fminf(fmaxf(p[d], flo[d]), fhi[d]);
        const float e = __fsub_rn(p[d], q);
        s = __fadd_rn(s, __fmul_rn(e, e));
    }
    if (s <= a.f32_in) return true;
    if (s > a.f32_out) return false;
    return affords64(lo, hi, p, a.thr_afford);
}

// The host builder's r_min test: every point of the closed cell within r_min of p.
__device__ __forceinline__ bool within_rmin(const double lo[3], const double hi[3], const float* p, double thr) {
    double s = 0.0;
    for (int d = 0; d < 3; d++) {
        if (!isfinite(lo[d]) || !isfinite(hi[d])) return false;
        const double v = p[d];
        const double x = fabs(__dsub_rn(v, lo[d])), y = fabs(__dsub_rn(hi[d], v));
        const double e = x > y ? x : y;
        s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return s <= thr;
}

// Grid range [c0, c1] along one axis covering [lo - reach, hi + reach], rounded
// outwards so that every point within reach of the cell is inside it.  Empty (c0 > c1)
// when lo = +inf (a cell beyond every point).
__device__ __forceinline__ void grid_range(const SetArgs& a, int d, double lo, double hi, int& c0, int& c1) {
    const int dim = a.gd.dims[d];
    if (lo == INFINITY) {
        c0 = 1;
        c1 = 0;
        return;
    }
    const double e0 = __dsub_rd(lo, a.reach), e1 = __dadd_ru(hi, a.reach);
    c0 = e0 == -INFINITY ? 0 : grid_coord(e0, a.gd.origin[d], a.gd.g, dim);
    c1 = e1 == INFINITY ? dim - 1 : grid_coord(e1, a.gd.origin[d], a.gd.g, dim);
}

// Warp per leaf.  COUNT: sizes[l] = |P_l| and pruned[l].  FILL: the members of P_l (in
// grid order) at set_idx[set_begin[l] ...]; the same deterministic walk finds the same
// members, and a write past the counted size is dropped and flagged in *bad.
template <bool FILL>
__global__ void __launch_bounds__(256) k_leaf_sets(SetArgs a, uint32_t* __restrict__ sizes, uint8_t* __restrict__ pruned,
                                                   const unsigned long long* __restrict__ set_begin,
                                                   uint32_t* __restrict__ set_idx, uint32_t* __restrict__ bad) {
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < a.N; l += warps) {
        double lo[3], hi[3];
        leaf_cell(a, l, lo, hi);
        const uint32_t t = a.rep[l];
        const bool pr = t < a.n && within_rmin(lo, hi, a.pts + 3 * (size_t)t, a.thr_prune);
        if (pr) {
            if (lane == 0) {
                if (FILL) set_idx[set_begin[l]] = t;
                else {
                    sizes[l] = 1;
                    pruned[l] = 1;
                }
            }
            continue;
        }
        float flo[3], fhi[3];
        int c0[3], c1[3];
        for (int d = 0; d < 3; d++) {
            flo[d] = (float)lo[d];   // split values are floats: exact
            fhi[d] = (float)hi[d];
            grid_range(a, d, lo[d], hi[d], c0[d], c1[d]);
        }
        uint32_t count = 0;
        const unsigned long long base = FILL ? set_begin[l] : 0ull;
        const uint32_t limit = FILL ? sizes[l] : 0u;
        if (c0[0] <= c1[0])
            for (int z = c0[2]; z <= c1[2]; z++)
                for (int y = c0[1]; y <= c1[1]; y++) {
                    // the cells x = c0..c1 of one row are contiguous in the item list
                    const uint32_t row = ((uint32_t)z * a.gd.dims[1] + y) * a.gd.dims[0];
                    const uint32_t b = a.cell_start[row + c0[0]], e = a.cell_start[row + c1[0] + 1];
                    for (uint32_t j = b; j < e; j += 32) {
                        const uint32_t jj = j + lane;
                        uint32_t p = 0;
                        bool in = false;
                        if (jj < e) {
                            p = a.items[jj];
                            const float* q = a.pts + 3 * (size_t)p;
                            const float pc[3] = {q[0], q[1], q[2]};
                            in = affords(a, flo, fhi, lo, hi, pc);
                        }
                        const uint32_t mask = __ballot_sync(0xffffffffu, in);
                        if (FILL && in) {
                            const uint32_t pos = count + __popc(mask & ((1u << lane) - 1u));
                            if (pos < limit) set_idx[base + pos] = p;
                            else atomicOr(bad, 1u);
                        }
                        count += __popc(mask);
                    }
                }
        if (!FILL && lane == 0) {
            sizes[l] = count;
            pruned[l] = 0;
        }
        if (FILL && lane == 0 && count != limit) atomicOr(bad, 1u);
    }
}

__global__ void k_blocks_of(const uint32_t* __restrict__ sizes, uint32_t N, uint32_t* __restrict__ nb) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < N) nb[l] = (sizes[l] + 3) / 4;
}

// Exclusive scan of 32-bit values into 64-bit offsets by one block; out[len] = total.
__global__ void k_scan64(const uint32_t* __restrict__ v, uint32_t len, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t base = 0; base < len; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long x = i < len ? v[i] : 0ull;
        unsigned long long incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long y = lane < nw ? ws[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= (uint32_t)o) y += u;
            }
            if (lane < nw) ws[lane] = y;
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? ws[warp - 1] : 0ull);
        if (i < len) out[i] = before + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[len] = carry;
}

// Warp per leaf: sort the set by point index (stable LSD radix on 8-bit digits through
// tmp), then write its 4-point blocks (three planes, +inf in unused slots), ids
// (0xffffffff in unused slots) and the 32-byte record.  The box is the host builder's:
// per axis the first (in index order) of the smallest / largest coordinates.
__global__ void __launch_bounds__(256) k_leaf_layout(uint32_t N, const float* __restrict__ pts,
                                                     const uint32_t* __restrict__ sizes,
                                                     const unsigned long long* __restrict__ set_begin,
                                                     const unsigned long long* __restrict__ blk_begin,
                                                     uint32_t* __restrict__ set_idx, uint32_t* __restrict__ tmp,
                                                     int passes, uint64_t plane, float* __restrict__ blocks,
                                                     uint32_t* __restrict__ ids, LeafRec* __restrict__ leaves) {
    __shared__ uint32_t bins_all[8][256];
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* bins = bins_all[threadIdx.x >> 5];
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < N; l += warps) {
        const uint32_t k = sizes[l];
        uint32_t* src = set_idx + set_begin[l];
        uint32_t* dst = tmp + set_begin[l];
        for (int ps = 0; ps < passes && k > 1; ps++) {
            const int shift = 8 * ps;
            for (uint32_t j = lane; j < 256; j += 32) bins[j] = 0;
            __syncwarp();
            for (uint32_t j = lane; j < k; j += 32) atomicAdd(&bins[(src[j] >> shift) & 255u], 1u);
            __syncwarp();
            uint32_t v[8], sum = 0;   // exclusive scan of the 256 bins, 8 per lane
            for (int q = 0; q < 8; q++) {
                v[q] = bins[lane * 8 + q];
                sum += v[q];
            }
            uint32_t run = warp_incl_scan(sum) - sum;
            for (int q = 0; q < 8; q++) {
                bins[lane * 8 + q] = run;
                run += v[q];
            }
            __syncwarp();
            for (uint32_t j0 = 0; j0 < k; j0 += 32) {
                const uint32_t j = j0 + lane;
                const bool valid = j < k;
                const uint32_t key = valid ? src[j] : 0u;
                const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                const uint32_t rank = __popc(peers & lt);
                const uint32_t base = valid ? bins[d] : 0u;
                __syncwarp();
                if (valid) dst[base + rank] = key;
                if (valid && rank == 0) bins[d] = base + __popc(peers);
                __syncwarp();
            }
            uint32_t* sw = src;
            src = dst;
            dst = sw;
            __syncwarp();
        }
        // src holds the sorted set (passes is even, so it is set_idx again)
        const uint64_t b0 = blk_begin[l];
        const uint32_t nb = (k + 3) / 4;
        unsigned long long kmin[3] = {~0ull, ~0ull, ~0ull}, kmax[3] = {0ull, 0ull, 0ull};
        for (uint32_t j = lane; j < 4 * nb; j += 32) {
            const uint64_t b = b0 + j / 4;
            const uint32_t q = j & 3u;
            uint32_t id = 0xffffffffu;
            float c[3] = {INFINITY, INFINITY, INFINITY};
            if (j < k) {
                id = src[j];
                for (int d = 0; d < 3; d++) {
                    c[d] = pts[3 * (size_t)id + d];
                    const unsigned long long key = (unsigned long long)fkey(c[d]) << 32;
                    kmin[d] = min(kmin[d], key | j);
                    kmax[d] = max(kmax[d], key | (0xffffffffu - j));
                }
            }
            blocks[4 * b + q] = c[0];
            blocks[4 * (plane + b) + q] = c[1];
            blocks[4 * (2 * plane + b) + q] = c[2];
            ids[4 * b + q] = id;
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int d = 0; d < 3; d++) {
                kmin[d] = min(kmin[d], __shfl_xor_sync(0xffffffffu, kmin[d], o));
                kmax[d] = max(kmax[d], __shfl_xor_sync(0xffffffffu, kmax[d], o));
            }
        if (lane == 0) {
            LeafRec r;
            for (int d = 0; d < 3; d++) {
                r.lo[d] = k ? pts[3 * (size_t)src[(uint32_t)kmin[d]] + d] : INFINITY;
                r.hi[d] = k ? pts[3 * (size_t)src[0xffffffffu - (uint32_t)kmax[d]] + d] : -INFINITY;
            }
            r.block = (uint32_t)b0;
            r.count = k;
            leaves[l] = r;
        }
        __syncwarp();
    }
}

// Blocked split array of the descent from the plain Eytzinger T (the layout of the
// host's blocked_splits: 8-float blocks of 3-level subtrees in 8-ary heap order, then
// 4-float tail blocks); every other float was set to +inf beforehand.
__global__ void k_blocked_splits(const float* __restrict__ T, int K, int R, uint32_t tail_off, float* __restrict__ out) {
    const uint64_t nblk = tail_off / 8;
    const uint64_t ntail = R ? (1ull << (3 * K)) : 0ull;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nblk) {
        uint64_t u = i, width = 1;
        int k = 0;
        while (u >= width) {   // block i is the u-th of super-level k
            u -= width;
            width *= 8;
            k++;
        }
        const uint64_t e = (1ull << (3 * k)) - 1 + u;   // Eytzinger index of its root
        float* b = out + 8 * i;
        b[0] = T[e];
        b[1] = T[2 * e + 1];
        b[2] = T[2 * e + 2];
        b[3] = T[4 * e + 3];
        b[4] = T[4 * e + 4];
        b[5] = T[4 * e + 5];
        b[6] = T[4 * e + 6];
    } else if (i < nblk + ntail) {
        const uint64_t s = i - nblk, e = ntail - 1 + s;
        float* b = out + tail_off + 4 * s;
        b[0] = T[e];
        if (R == 2) {
            b[1] = T[2 * e + 1];
            b[2] = T[2 * e + 2];
        }
    }
}

// Temporary device buffers of one build, released when the build returns.
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    T* get(size_t count) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    void keep(void* p) { ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end()); }
};

float key_float(uint32_t k) {
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

unsigned grid_of(uint64_t work, unsigned block) {
    return (unsigned)std::max<uint64_t>(1, (work + block - 1) / block);
}

}  // namespace

void DeviceTree::release() {
    for (void* p : {(void*)Tb, (void*)Tplain, (void*)leaves, (void*)blocks, (void*)ids, (void*)cloud, (void*)set_idx,
                    (void*)set_begin, (void*)pruned})
        if (p) cudaFree(p);
    *this = DeviceTree();
}

#define DB_CUDA(call, what)                                              \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) {                                         \
            err = std::string(what) + ": " + cudaGetErrorString(_e);     \
            return CAPT_E_CUDA;                                          \
        }                                                                \
    } while (0)

#define DB_ALLOC(var, T, count)                                          \
    T* var = scratch.get<T>(count);                                      \
    if (!var) {                                                          \
        err = "device allocation failed while building";                 \
        return CAPT_E_NOMEM;                                             \
    }

int launch_sort_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t n, int passes, uint32_t* hist,
                      cudaStream_t st, std::string& err) {
    const uint32_t nsb = grid_of(n, kSortThreads);
    for (int pass = 0; pass < passes; pass++) {
        k_radix_hist<<<nsb, kSortThreads, 0, st>>>(ka, n, 8 * pass, hist, nsb);
        k_scan_exclusive<<<1, 1024, 0, st>>>(hist, 256 * nsb);
        k_radix_scatter<<<nsb, kSortThreads, 0, st>>>(ka, va, n, 8 * pass, hist, nsb, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("sort launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int launch_scan64(const uint32_t* v, uint32_t len, unsigned long long* out, cudaStream_t st, std::string& err) {
    k_scan64<<<1, 1024, 0, st>>>(v, len, out);
    const cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("scan launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

int device_build(const float* d_points, size_t n, float r_min, float r_max, cudaStream_t st, DeviceTree& out,
                 std::string& err) {
    out = DeviceTree();
    if (n && !d_points) { err = "points is NULL"; return CAPT_E_ARG; }
    if (n >= (size_t(1) << 30)) { err = "the device builder takes fewer than 2^30 points"; return CAPT_E_ARG; }
    if (!(r_min >= 0.f) || !(r_max >= r_min) || !std::isfinite(r_max)) {
        err = "need 0 <= r_min <= r_max < inf";
        return CAPT_E_RANGE;
    }
    Scratch scratch;
    uint32_t N = 1;
    int L = 0;
    while (N < n) { N *= 2; L++; }
    const uint32_t un = (uint32_t)n;
    out.n = n;
    out.N = N;
    out.L = L;

    // --- copy of the points, bounding box, finite check ---
    DB_ALLOC(cloud, float, 3 * std::max<size_t>(n, 1));
    if (n) DB_CUDA(cudaMemcpyAsync(cloud, d_points, 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy points");
    DB_ALLOC(box, uint32_t, 8);
    const uint32_t box0[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
    DB_CUDA(cudaMemcpyAsync(box, box0, sizeof(box0), cudaMemcpyHostToDevice, st), "box init");
    if (n) k_bbox<<<std::min(grid_of(n, 256), 1024u), 256, 0, st>>>(cloud, un, box);
    uint32_t hbox[8];
    DB_CUDA(cudaMemcpyAsync(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost, st), "box read");
    DB_CUDA(cudaStreamSynchronize(st), "bounding box");
    if (hbox[6]) { err = "non-finite coordinate in points"; return CAPT_E_NONFINITE; }
    for (int d = 0; d < 3; d++) {
        out.box_lo[d] = n ? key_float(hbox[d]) : INFINITY;
        out.box_hi[d] = n ? key_float(hbox[3 + d]) : -INFINITY;
    }

    // --- the three sorted orders ---
    const uint32_t nsb = grid_of(N, kSortThreads);
    DB_ALLOC(hist, uint32_t, 256 * (size_t)nsb);
    DB_ALLOC(kt, uint32_t, N);
    DB_ALLOC(vt, uint32_t, N);
    uint32_t* ord[3];
    for (int d = 0; d < 3; d++) {
        DB_ALLOC(o, uint32_t, N);
        DB_ALLOC(keys, uint32_t, N);
        ord[d] = o;
        k_init_keys<<<grid_of(N, 256), 256, 0, st>>>(cloud, un, N, d, keys, o);
        uint32_t *ka = keys, *va = o, *kb = kt, *vb = vt;
        for (int pass = 0; pass < 4; pass++) {   // an even count: the result ends in keys / o
            k_radix_hist<<<nsb, kSortThreads, 0, st>>>(ka, N, 8 * pass, hist, nsb);
            k_scan_exclusive<<<1, 1024, 0, st>>>(hist, 256 * nsb);
            k_radix_scatter<<<nsb, kSortThreads, 0, st>>>(ka, va, N, 8 * pass, hist, nsb, kb, vb);
            std::swap(ka, kb);
            std::swap(va, vb);
        }
    }

    // --- medians, level by level ---
    DB_ALLOC(Tplain, float, std::max<uint32_t>(N - 1, 1));
    DB_ALLOC(left, uint8_t, N);
    DB_ALLOC(rank, uint32_t, N);
    DB_ALLOC(tile_left, uint32_t, grid_of(N, kTile));
    DB_ALLOC(ord_tmp, uint32_t, N);
    for (int l = 0; l < L; l++) {
        const int d = l % 3, lg_m = L - l;
        k_level_split<<<grid_of(N, 256), 256, 0, st>>>(cloud, un, N, lg_m, d, ord[d], (1u << l) - 1u, Tplain, left);
        for (int e = 0; e < 3; e++) {
            if (e == d) continue;
            k_part_tiles<<<grid_of(N, kTile), kTile, 0, st>>>(ord[e], N, lg_m, left, rank, tile_left);
            if ((1u << lg_m) > kTile) {
                const uint32_t per_seg = (1u << lg_m) / kTile, nseg = N >> lg_m;
                k_part_segments<<<grid_of(nseg, 128), 128, 0, st>>>(tile_left, nseg, per_seg);
            }
            k_part_scatter<<<grid_of(N, 256), 256, 0, st>>>(ord[e], N, lg_m, left, rank, tile_left, ord_tmp);
            std::swap(ord[e], ord_tmp);
        }
    }
    const uint32_t* rep = ord[0];   // every order now lists the leaves' representatives

    // --- uniform grid over the cloud, cells of edge >= the reach ---
    SetArgs a;
    a.pts = cloud;
    a.n = un;
    a.N = N;
    a.L = L;
    a.T = Tplain;
    a.rep = rep;
    const double ra = (double)r_max * (1.0 + 1e-5), rp = (double)r_min * (1.0 - 1e-5);
    a.thr_afford = ra * ra;
    a.thr_prune = rp * rp;
    a.reach = ra * (1.0 + 1e-6);
    if (a.thr_afford >= 1e-30 && a.thr_afford <= 1e30) {
        a.f32_in = (float)(a.thr_afford * (1.0 - 1e-5));
        a.f32_out = (float)(a.thr_afford * (1.0 + 1e-5));
    } else {   // outside the range where the FP32 error bound holds
        a.f32_in = -1.f;
        a.f32_out = INFINITY;
    }
    GridDesc gd;
    for (int d = 0; d < 3; d++) gd.origin[d] = n ? (double)out.box_lo[d] - a.reach : 0.0;
    gd.g = std::max(a.reach, 1e-30);
    for (;;) {
        uint64_t cells = 1;
        for (int d = 0; d < 3; d++) {
            const double ext = n ? (double)out.box_hi[d] - (double)out.box_lo[d] + 2 * a.reach : 0.0;
            gd.dims[d] = (int)std::min(1.0e6, std::floor(ext / gd.g) + 1.0);
            cells *= (uint64_t)gd.dims[d];
        }
        if (cells <= (uint64_t(1) << 22)) break;
        gd.g *= 2.0;
    }
    a.gd = gd;
    const uint32_t ncell = (uint32_t)gd.dims[0] * gd.dims[1] * gd.dims[2];
    DB_ALLOC(cell_of, uint32_t, n);
    DB_ALLOC(cell_start, uint32_t, (size_t)ncell + 1);
    DB_ALLOC(cursor, uint32_t, (size_t)ncell + 1);
    DB_ALLOC(items, uint32_t, n);
    DB_CUDA(cudaMemsetAsync(cell_start, 0, ((size_t)ncell + 1) * sizeof(uint32_t), st), "grid clear");
    if (n) k_grid_count<<<grid_of(n, 256), 256, 0, st>>>(cloud, un, gd, cell_of, cell_start);
    k_scan_exclusive<<<1, 1024, 0, st>>>(cell_start, ncell + 1);
    DB_CUDA(cudaMemcpyAsync(cursor, cell_start, ((size_t)ncell + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
            "grid cursor");
    if (n) k_grid_fill<<<grid_of(n, 256), 256, 0, st>>>(un, cell_of, cursor, items);
    a.cell_start = cell_start;
    a.items = items;

    // --- set sizes and offsets ---
    DB_ALLOC(sizes, uint32_t, N);
    DB_ALLOC(pruned, uint8_t, N);
    DB_ALLOC(set_begin, unsigned long long, (size_t)N + 1);
    DB_ALLOC(nblocks, uint32_t, N);
    DB_ALLOC(blk_begin, unsigned long long, (size_t)N + 1);
    const unsigned set_grid = std::min<unsigned>(grid_of((uint64_t)N * 32, 256), (unsigned)sm_count() * 8);
    k_leaf_sets<false><<<set_grid, 256, 0, st>>>(a, sizes, pruned, nullptr, nullptr, nullptr);
    k_scan64<<<1, 1024, 0, st>>>(sizes, N, set_begin);
    k_blocks_of<<<grid_of(N, 256), 256, 0, st>>>(sizes, N, nblocks);
    k_scan64<<<1, 1024, 0, st>>>(nblocks, N, blk_begin);
    unsigned long long tot[2];
    DB_CUDA(cudaMemcpyAsync(&tot[0], set_begin + N, 8, cudaMemcpyDeviceToHost, st), "set total");
    DB_CUDA(cudaMemcpyAsync(&tot[1], blk_begin + N, 8, cudaMemcpyDeviceToHost, st), "block total");
    DB_CUDA(cudaStreamSynchronize(st), "set sizes");
    if (tot[1] >= (1ull << 32)) { err = "affordance sets too large for 32-bit block offsets"; return CAPT_E_RANGE; }
    out.total = tot[0];
    out.total_blocks = tot[1];

    // --- sets, sorted and laid out ---
    DB_ALLOC(set_idx, uint32_t, out.total);
    DB_ALLOC(set_tmp, uint32_t, out.total);
    k_leaf_sets<true><<<set_grid, 256, 0, st>>>(a, sizes, nullptr, set_begin, set_idx, box + 7);
    const uint64_t plane = std::max<uint64_t>(out.total_blocks, 1);
    DB_ALLOC(blocks, float, 12 * plane);
    DB_ALLOC(ids, uint32_t, 4 * plane);
    DB_ALLOC(leaves, LeafRec, N);
    if (out.total_blocks == 0) {   // the one unused block of an empty layout
        k_fill_f32<<<1, 32, 0, st>>>(blocks, 12, INFINITY);
        DB_CUDA(cudaMemsetAsync(ids, 0xff, 4 * sizeof(uint32_t), st), "ids");
    }
    int passes = 0;
    for (uint64_t v = n; v > 0; v >>= 8) passes++;
    passes += passes & 1;
    k_leaf_layout<<<set_grid, 256, 0, st>>>(N, cloud, sizes, set_begin, blk_begin, set_idx, set_tmp, passes, plane,
                                            blocks, ids, leaves);

    // --- blocked split array ---
    blocked_shape(L, out.bs);
    DB_ALLOC(Tb, float, out.bs.total_floats);
    k_fill_f32<<<std::min(grid_of(out.bs.total_floats, 256), 4096u), 256, 0, st>>>(Tb, out.bs.total_floats, INFINITY);
    {
        const uint64_t nb = out.bs.tail_off / 8 + (out.bs.R ? (1ull << (3 * out.bs.K)) : 0ull);
        if (nb) k_blocked_splits<<<grid_of(nb, 256), 256, 0, st>>>(Tplain, out.bs.K, out.bs.R, out.bs.tail_off, Tb);
    }
    DB_CUDA(cudaMemcpyAsync(&hbox[7], box + 7, 4, cudaMemcpyDeviceToHost, st), "check word");
    DB_CUDA(cudaGetLastError(), "build kernels");
    DB_CUDA(cudaStreamSynchronize(st), "build");
    if (hbox[7]) { err = "device build: the two passes over the sets disagree"; return CAPT_E_BOUNDS; }

    out.Tb = Tb;
    out.Tplain = Tplain;
    out.leaves = leaves;
    out.blocks = blocks;
    out.ids = ids;
    out.cloud = cloud;
    out.set_idx = set_idx;
    out.set_begin = set_begin;
    out.pruned = pruned;
    out.bytes = out.bs.total_floats * 4 + (size_t)N * sizeof(LeafRec) + 48 * plane + 16 * plane +
                12 * std::max<size_t>(n, 1);
    for (void* p : {(void*)Tb, (void*)Tplain, (void*)leaves, (void*)blocks, (void*)ids, (void*)cloud, (void*)set_idx,
                    (void*)set_begin, (void*)pruned})
        scratch.keep(p);
    return CAPT_OK;
}

}  // namespace capt
