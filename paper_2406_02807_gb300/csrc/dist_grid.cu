// Distance-bound grid: an exact classifier in front of the descent (this build's
// addition; the paper's query starts with the descent of Alg. 3).
//
// A uniform grid of cubic cells of side h covers the cloud's bounding box grown by
// r_max.  Each cell (grown by delta = h / 100 on every side) stores two bytes, in units
// of unit = r_max / 128:
//   lb: a lower bound of the distance from any point of the cell to the cloud, rounded
//       down (saturating at 255);
//   ub: an upper bound of the same distance, rounded up (255: none known).
// A query sphere (x, r) is then
//   rejected  when fl(lb * unit) > r: it misses every point under the FP32 test;
//   accepted  when x lies inside the grid box and fl(ub * unit) < r: it hits the
//             nearest point under the FP32 test;
//   undecided otherwise (it descends as usual).
//
// Why both decisions are exact:
//  1. The cell the kernel computes holds x.  The kernel takes u = fl(fl(x - org) *
//     fl(1 / h)) and i = floor(u) clamped to [0, n - 1].  With three roundings
//     |u - (x - org) / h| <= 3 * 2^-24 * n < 0.003 cells for n <= 16384 cells per axis,
//     so an x inside the grid box lies in cell i grown by delta.  An x outside it is
//     clamped to the border cell that holds its projection P(x) onto the grid box; the
//     grid box is convex and holds every cloud point p, so |P(x) - p| <= |x - p| and the
//     lower bound still holds (the upper bound is not used outside the box).
//  2. The bounds.  Let m be a point of the grown cell and rho >= max |x - m| over it
//     (rounded up).  The distance D(x) to the cloud is 1-Lipschitz, so D(m) - rho <=
//     D(x) <= D(m) + rho.  D(m) comes from the tree: m descends to its leaf by the
//     exact comparisons of Alg. 3, and an unpruned leaf's set holds every point within
//     r_max of the leaf's closed cell (Alg. 1, affordance with the margin of the
//     builder), hence every point within r_max of m.  So with s the exact minimum over
//     the set, min(s, r_max) <= D(m) <= s.  A leaf holding one point may be a pruned one
//     (Alg. 1 keeps {t} only): there D(m) <= |m - t| still holds, and the lower bound is
//     taken as 0.  Every operation is rounded toward the safe side (gaps, squares, sums
//     and square roots down for the lower bound, up for the upper bound).
//  3. Quantisation: lb_q = floor(lb * 0.99999 / unit) and ub_q = ceil(ub * 1.00001 /
//     unit), rounded the safe way, so fl(lb_q * unit) < lb (1 - 9.8e-6) and
//     fl(ub_q * unit) > ub (1 + 9.8e-6).
//  4. The FP32 test ((x0-p0)^2 + (x1-p1)^2) + (x2-p2)^2 <= fl(r * r) can only pass when
//     the true distance is at most r (1 + 1.8e-7), and passes whenever it is at most
//     r (1 - 1.8e-7) (five rounded operations on the left, one on the right).
//     fl(lb_q * unit) > r gives D(x) > r (1 + 9.8e-6): no point hits.  fl(ub_q * unit)
//     < r gives D(x) < r (1 - 9.8e-6): the nearest point hits.
// Lemma 1 makes the CAPT's answer the FP32 brute force's, so deciding a sphere either
// way by the grid gives the same flag.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "kernels.h"

namespace capt {

GridShape grid_shape(const float lo[3], const float hi[3], float r_max, uint64_t n_points, uint64_t max_cells) {
    GridShape g;
    if (n_points == 0 || !(r_max > 0.f) || !std::isfinite(r_max) || max_cells < 1) return g;
    double blo[3], bhi[3], ext[3];
    for (int d = 0; d < 3; d++) {
        if (!(lo[d] <= hi[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d])) return g;
        blo[d] = (double)lo[d] - (double)r_max;
        bhi[d] = (double)hi[d] + (double)r_max;
        ext[d] = bhi[d] - blo[d];
    }
    double h = std::cbrt(ext[0] * ext[1] * ext[2] / (double)max_cells);
    for (int it = 0; it < 4096; it++, h *= 1.02) {
        const float hf = (float)h;
        if (!(hf > 0.f)) continue;
        uint64_t cells = 1;
        int n[3];
        float org[3];
        bool ok = true;
        for (int d = 0; d < 3; d++) {
            float o = (float)blo[d];
            if ((double)o > blo[d]) o = std::nextafter(o, -INFINITY);
            org[d] = o;
            const double nd = std::ceil((bhi[d] - (double)o) / (double)hf);
            if (nd > (double)kGridMaxAxis) ok = false;
            n[d] = (int)std::max(1.0, std::min(nd, (double)kGridMaxAxis));
            cells *= (uint64_t)n[d];
        }
        if (!ok || cells > max_cells) continue;
        for (int d = 0; d < 3; d++) {
            g.org[d] = org[d];
            g.n[d] = n[d];
        }
        g.h = hf;
        g.inv_h = (float)(1.0 / (double)hf);
        g.unit = (float)((double)r_max / 128.0);
        g.cells = (uint32_t)cells;
        return g;
    }
    return g;
}

namespace {

constexpr int kGridThreads = 128;

// Bounds of |a - b| for FP32 a, b: lo <= |a - b| <= hi.
__device__ __forceinline__ void abs_diff_bounds(float a, float b, float& lo, float& hi) {
    const float dn = __fsub_rd(a, b), up = __fsub_ru(a, b);
    lo = dn > 0.f ? dn : (up < 0.f ? -up : 0.f);
    hi = fmaxf(fabsf(dn), fabsf(up));
}

// Cell c grown by h / 100 on every side: the box [L, U] (rounded outward), its
// representative point m and rho >= max |x - m| over the box (rounded up).
__device__ __forceinline__ void cell_box(const GridShape& g, uint32_t c, float L[3], float U[3], float m[3],
                                         float& rho) {
    const uint32_t nx = (uint32_t)g.n[0], ny = (uint32_t)g.n[1];
    const uint32_t idx[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
    const float dl = __fmul_ru(g.h, 0.01f);
    float rho2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        L[d] = __fsub_rd(__fadd_rd(g.org[d], __fmul_rd((float)idx[d], g.h)), dl);
        U[d] = __fadd_ru(__fadd_ru(g.org[d], __fmul_ru((float)(idx[d] + 1u), g.h)), dl);
        m[d] = __fmul_rn(__fadd_rn(L[d], U[d]), 0.5f);
        const float e = fmaxf(__fsub_ru(m[d], L[d]), __fsub_ru(U[d], m[d]));
        rho2 = __fadd_ru(rho2, __fmul_ru(e, e));
    }
    rho = __fsqrt_ru(rho2);
}

// One thread per cell: the bounds of the distance from the grown cell to the cloud,
// through the cell's representative point m and its leaf's set.
__global__ void __launch_bounds__(kGridThreads) k_dist_grid(DevArgs t, GridShape g, uchar2* __restrict__ out) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.cells) return;
    float L[3], U[3], m[3], rho;
    cell_box(g, c, L, U, m, rho);
    const uint32_t leaf = descend(m[0], m[1], m[2], t, nullptr);
    float4 a, b;
    load_leaf(t.leaves, leaf, a, b);
    const uint32_t cnt = __float_as_uint(b.w);
    const uint32_t b0 = __float_as_uint(a.w);
    float lo2 = INFINITY, hi2 = INFINITY;   // smallest lower / upper bound of the squared distance
    const uint64_t pl = 4ull * t.plane;
    for (uint32_t j = 0; j < cnt; j++) {
        const float* s = t.blocks + 4ull * (b0 + j / 4u) + (j & 3u);
        float l0, h0, l1, h1, l2, h2;
        abs_diff_bounds(m[0], s[0], l0, h0);
        abs_diff_bounds(m[1], s[pl], l1, h1);
        abs_diff_bounds(m[2], s[2 * pl], l2, h2);
        lo2 = fminf(lo2, __fadd_rd(__fadd_rd(__fmul_rd(l0, l0), __fmul_rd(l1, l1)), __fmul_rd(l2, l2)));
        hi2 = fminf(hi2, __fadd_ru(__fadd_ru(__fmul_ru(h0, h0), __fmul_ru(h1, h1)), __fmul_ru(h2, h2)));
    }
    // D(m) >= min(s, r_max) (an unpruned leaf), >= 0 (a leaf of one point may be pruned);
    // D(m) <= s whenever the set is not empty
    const float lbm = cnt == 1u ? 0.f : fminf(__fsqrt_rd(lo2), t.r_max);
    const float ubm = cnt == 0u ? INFINITY : __fsqrt_ru(hi2);
    const float lb = fmaxf(__fsub_rd(lbm, rho), 0.f);
    const float ub = __fadd_ru(ubm, rho);
    const float ql = floorf(__fdiv_rd(__fmul_rd(lb, 0.99999f), g.unit));
    const float qu = ceilf(__fdiv_ru(__fmul_ru(ub, 1.00001f), g.unit));
    uchar2 q;
    q.x = (unsigned char)(ql >= 255.f ? 255.f : ql);
    q.y = (unsigned char)(qu >= 255.f ? 255.f : qu);   // 255 also when ub is infinite
    out[c] = q;
}

}  // namespace

int launch_dist_grid(const DevArgs& t, const GridShape& g, uint8_t* out, cudaStream_t st, std::string& err) {
    if (g.cells == 0) return CAPT_OK;
    const unsigned blocks = (g.cells + kGridThreads - 1) / kGridThreads;
    k_dist_grid<<<blocks, kGridThreads, 0, st>>>(t, g, reinterpret_cast<uchar2*>(out));
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { err = std::string("distance grid launch: ") + cudaGetErrorString(ce); return CAPT_E_CUDA; }
    return CAPT_OK;
}

// ------------------------------------------------------------------------------------
// Nearest-candidate lists of the clearance (this build's addition; the paper's
// clearance scans the whole set of the centre's leaf, Lemma 1 case 1).
//
// For each cell C of the grid (grown by h / 100, centre m, rho as above) the list holds
// the cloud points of the sets of every leaf whose closed cell meets C that lie within
//   R_C = min(ub_C, r_max) (1 + 2^-20) + rho          (rounded up)
// of m, each point once; ub_C is the grid's rounded-up upper bound of the distance
// from C to the cloud.  Why a centre x of C gets the paper's answer from its cell's
// list (the FP32 argmin over the list, ties to the lowest point index):
//  a. The paper's answer is p*, the lowest-index point of minimal FP32 squared
//     distance in S_x, the set of x's leaf, reported when its distance is below r_max.
//     x lies in C (argument 1 above) and in the closed cell of its leaf, so that leaf
//     meets C and S_x is among the sets the list is cut from.
//  b. A reported p* has |x - p*| < r_max (1 + 2.5e-7) (five rounded operations and a
//     rounded square root).  Then D(x) < r_max (1 + 1e-5), so the nearest cloud point
//     is in S_x (the builder's affordance radius) and |x - p*| <= D(x) (1 + 3e-7) <=
//     ub_C (1 + 3e-7).  So |m - p*| <= |x - p*| + rho <= R_C: p* is in the list.
//  c. Any point p that beats p* in FP32, or is reportable at all, lies within
//     r_max (1 + 2.5e-7) of x and therefore in S_x, where p* already beats it.  So the
//     argmin over the list is p*, and when the paper reports nothing no list point is
//     reportable either: the distance and index are the paper's, bit for bit (the same
//     FP32 expression).
//  d. A centre outside the grid box is farther than r_max + h / 300 from every point:
//     both paths answer r_max, -1 whatever they scan.
// Cells that the grid proves farther than r_max from the cloud (the reject rule at
// r = r_max) get an empty list.  A cell whose leaves or points overflow the builder's
// per-warp buffers is marked kNearFallback and its centres take the paper's path.
// The membership test is conservative (the FP32 distance from m rounded down against
// R_C^2 rounded up), so extra points may enter a list; by c they change nothing.
// ------------------------------------------------------------------------------------

namespace {

constexpr int kNearThreads = 128;              // four warps, one cell each at a time
constexpr uint32_t kNearMaxLeaves = 32;        // leaves meeting one cell
constexpr uint32_t kNearMaxCand = 1024;        // points collected for one cell
constexpr int kNearScanThreads = 1024;         // cells per block of the offset scan

struct NearScratch {
    uint32_t leaf[kNearMaxLeaves];
    uint32_t seg[kNearMaxLeaves + 1];   // first entry of each leaf's points in cand
    uint32_t cand[kNearMaxCand];
};

// Split value of the node at depth lev reached by `path` (lev decisions, the first one
// most significant, 1 = right) in the blocked split array of the descent.
__device__ __forceinline__ float split_at(const DevArgs& t, int lev, uint32_t path) {
    const int k = lev / 3, j = lev - 3 * k;
    if (k < t.K) {
        uint32_t u = 0;
        for (int i = 0; i < k; i++) u = 8u * u + 1u + ((path >> (lev - 3 * (i + 1))) & 7u);
        const float* b = t.T + 8ull * u;
        if (j == 0) return __ldg(b);
        if (j == 1) return __ldg(b + ((path & 1u) ? 2 : 1));
        return __ldg(b + 3 + 2 * ((path >> 1) & 1u) + (path & 1u));
    }
    const uint32_t bits = path >> (lev - 3 * t.K);   // the decisions of the full super-levels
    const float* q = t.T + (size_t)t.tail_off + 4ull * bits;
    return j == 0 ? __ldg(q) : __ldg(q + ((path & 1u) ? 2 : 1));
}

// Warp per cell.  COUNT: cell[2c + 1] = the cell's entries (its points rounded up to a
// multiple of 4; 0: empty; kNearFallback).  FILL: the entries at cand[cell[2c] ...]
// (padded with `pad`, the index of the point at +inf); the same deterministic walk
// finds the same points, and a count that differs is flagged in *bad with no write
// past the counted entries.
template <bool FILL>
__global__ void __launch_bounds__(kNearThreads) k_near_lists(DevArgs t, GridShape g, const uchar2* __restrict__ grid,
                                                             uint32_t* __restrict__ cell, uint32_t* __restrict__ cand,
                                                             uint32_t pad, unsigned long long* __restrict__ n_fallback,
                                                             uint32_t* __restrict__ bad) {
    __shared__ NearScratch sh[kNearThreads / 32];
    NearScratch& s = sh[threadIdx.x >> 5];
    const uint32_t lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t pl = 4ull * t.plane;
    for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < g.cells; c += warps) {
        const uchar2 q = grid[c];
        uint32_t result = 0;
        const uint32_t limit = FILL ? cell[2 * (size_t)c + 1] : 0u;
        const uint32_t cap = limit == kNearFallback ? 0u : limit;   // entries reserved for the cell
        const uint32_t base = FILL ? cell[2 * (size_t)c] : 0u;
        if (!(__fmul_rn((float)q.x, g.unit) > t.r_max)) {
            float L[3], U[3], m[3], rho;
            cell_box(g, c, L, U, m, rho);
            const float R = __fadd_ru(__fmul_ru(fminf(__fmul_ru((float)q.y, g.unit), t.r_max), 1.00000095367431640625f),
                                      rho);
            const float R2 = __fmul_ru(R, R);
            // leaves whose closed cell meets [L, U]: depth-first over the splits, every
            // lane walking the same nodes (left child: x_d <= T, right child: x_d >= T)
            uint32_t nl = 0;
            bool over = false;
            uint64_t stk[34];
            int sp = 0;
            stk[sp++] = 0;
            while (sp > 0) {
                const uint64_t e = stk[--sp];
                const int lev = (int)(e >> 32);
                const uint32_t path = (uint32_t)e;
                if (lev == t.L) {
                    if (nl == kNearMaxLeaves) {
                        over = true;
                        break;
                    }
                    if (lane == 0) s.leaf[nl] = path;
                    nl++;
                    continue;
                }
                const float T = split_at(t, lev, path);
                const int ax = lev % 3;
                const uint64_t child = (uint64_t)(lev + 1) << 32;
                if (U[ax] >= T) stk[sp++] = child | ((path << 1) | 1u);
                if (L[ax] <= T) stk[sp++] = child | (path << 1);
            }
            __syncwarp();
            uint32_t n = 0;
            if (!over) {
                // their points within R_C of m, leaf by leaf: the set's 32-slot chunks
                // are tested by their boxes first (one chunk per lane; a box holds its
                // points, so a chunk whose box is farther than R_C has none), then the
                // slots of the chunks that pass, in slot order
                for (uint32_t k = 0; k < nl; k++) {
                    if (lane == 0) s.seg[k] = n;
                    float4 a, b;
                    load_leaf(t.leaves, s.leaf[k], a, b);
                    const uint32_t b0 = __float_as_uint(a.w), cnt = __float_as_uint(b.w);
                    if (cnt == 0) continue;
                    const uint64_t s_lo = 4ull * b0, s_hi = s_lo + cnt;   // the set's slots
                    const uint64_t c_lo = b0 / kChunkBlocks, c_hi = (b0 + (cnt + 3u) / 4u - 1u) / kChunkBlocks;
                    for (uint64_t c0 = c_lo; c0 <= c_hi; c0 += 32) {
                        bool reach = false;
                        if (c0 + lane <= c_hi) {
                            const float4* cb = reinterpret_cast<const float4*>(t.cbox) + 2 * (c0 + lane);
                            const float4 lo = __ldg(cb), hi = __ldg(cb + 1);
                            float g2 = 0.f;
                            const float lv[3] = {lo.x, lo.y, lo.z}, hv[3] = {hi.x, hi.y, hi.z};
#pragma unroll
                            for (int d = 0; d < 3; d++) {
                                const float gd = fmaxf(fmaxf(__fsub_rd(lv[d], m[d]), __fsub_rd(m[d], hv[d])), 0.f);
                                g2 = __fadd_rd(g2, __fmul_rd(gd, gd));
                            }
                            reach = g2 <= R2;
                        }
                        uint32_t pm = __ballot_sync(0xffffffffu, reach);
                        while (pm) {
                            const uint64_t slot = 32ull * (c0 + (uint32_t)(__ffs(pm) - 1)) + lane;
                            pm &= pm - 1u;
                            bool in = false;
                            uint32_t id = 0;
                            if (slot >= s_lo && slot < s_hi) {
                                const float* p = t.blocks + slot;
                                float l0, h0, l1, h1, l2, h2;
                                abs_diff_bounds(m[0], __ldg(p), l0, h0);
                                abs_diff_bounds(m[1], __ldg(p + pl), l1, h1);
                                abs_diff_bounds(m[2], __ldg(p + 2 * pl), l2, h2);
                                const float lo2 =
                                    __fadd_rd(__fadd_rd(__fmul_rd(l0, l0), __fmul_rd(l1, l1)), __fmul_rd(l2, l2));
                                in = lo2 <= R2;
                                id = __ldg(t.ids + slot);
                            }
                            const uint32_t mask = __ballot_sync(0xffffffffu, in);
                            const uint32_t pos = n + __popc(mask & lt);
                            if (in && pos < kNearMaxCand) s.cand[pos] = id;
                            n += __popc(mask);
                        }
                    }
                }
                if (lane == 0) s.seg[nl] = n;
                over = n > kNearMaxCand;
            }
            __syncwarp();
            if (over) {
                result = kNearFallback;
            } else {
                // each point once: an entry is dropped when an earlier leaf's points hold it
                uint32_t u = 0;
                for (uint32_t i0 = 0; i0 < n; i0 += 32) {
                    const uint32_t i = i0 + lane;
                    bool keep = false;
                    uint32_t id = 0;
                    if (i < n) {
                        id = s.cand[i];
                        uint32_t first = 0;   // start of i's leaf segment
                        for (uint32_t k = 1; k < nl; k++)
                            if (s.seg[k] <= i) first = s.seg[k];
                        keep = true;
                        for (uint32_t j = 0; j < first; j++)
                            if (s.cand[j] == id) {
                                keep = false;
                                break;
                            }
                    }
                    const uint32_t mask = __ballot_sync(0xffffffffu, keep);
                    const uint32_t pos = u + __popc(mask & lt);
                    if constexpr (FILL) {
                        if (keep && pos < cap) cand[(size_t)base + pos] = id;
                    }
                    u += __popc(mask);
                }
                result = (u + 3u) & ~3u;
                if constexpr (FILL) {
                    for (uint32_t i = u + lane; i < result && i < cap; i += 32) cand[(size_t)base + i] = pad;
                }
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (!FILL) {
                cell[2 * (size_t)c + 1] = result;
                if (result == kNearFallback) atomicAdd(n_fallback, 1ull);
            } else if (result != limit) {
                atomicOr(bad, 1u);
            }
        }
    }
}

__device__ __forceinline__ uint32_t near_entries(uint32_t v) { return v == kNearFallback ? 0u : v; }

// Entries of each block of kNearScanThreads cells.
__global__ void __launch_bounds__(kNearScanThreads) k_near_block_sums(const uint32_t* __restrict__ cell, uint32_t cells,
                                                                       uint32_t* __restrict__ bsum) {
    __shared__ uint32_t ws[32];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = i < cells ? near_entries(cell[2 * (size_t)i + 1]) : 0u;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31u) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0u;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = w;
    }
}

// First entry of each cell: the block's exclusive prefix plus the prefix of the blocks
// before it (boff, 64-bit; the host refuses totals of 2^32 entries or more).
__global__ void __launch_bounds__(kNearScanThreads) k_near_offsets(uint32_t* __restrict__ cell, uint32_t cells,
                                                                    const unsigned long long* __restrict__ boff) {
    __shared__ uint32_t ws[32];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t v = i < cells ? near_entries(cell[2 * (size_t)i + 1]) : 0u;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (blockDim.x >> 5) ? ws[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const uint32_t before = (warp ? ws[warp - 1] : 0u) + incl - v;
    if (i < cells) cell[2 * (size_t)i] = (uint32_t)(boff[blockIdx.x] + before);
}

// The cloud as 4 floats per point, then one point at +inf (the padding entry).
__global__ void k_near_cloud(const float* __restrict__ cloud, uint32_t n, float4* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4(cloud[3 * (size_t)i], cloud[3 * (size_t)i + 1], cloud[3 * (size_t)i + 2], 0.f);
    else if (i == n) out[i] = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
}

}  // namespace

void NearLists::release() {
    for (void* p : {cell, cand, cloud})
        if (p) cudaFree(p);
    cell = cand = cloud = nullptr;
    entries = fallback_cells = 0;
    bytes = 0;
}

#define NL_CUDA(call, what)                                              \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) {                                         \
            err = std::string(what) + ": " + cudaGetErrorString(_e);     \
            rc = _e == cudaErrorMemoryAllocation ? CAPT_E_NOMEM : CAPT_E_CUDA; \
            goto done;                                                   \
        }                                                                \
    } while (0)

int device_near_lists(const DevArgs& t, size_t n, cudaStream_t st, NearLists& out, std::string& err) {
    out = NearLists();
    const GridShape& g = t.g;
    if (!t.grid || g.cells == 0) {
        err = "the nearest-candidate lists need the distance-bound grid";
        return CAPT_E_STATE;
    }
    int rc = CAPT_OK;
    const uint32_t nb = (g.cells + kNearScanThreads - 1) / kNearScanThreads;
    uint32_t* bsum = nullptr;
    unsigned long long* boff = nullptr;   // nb + 1 offsets, then the fallback count and the bad flag
    unsigned long long h_tail[3] = {0, 0, 0};
    unsigned walk_blocks = 0;
    {
        int sms = sm_count();
        walk_blocks = (unsigned)std::min<uint64_t>(((uint64_t)g.cells + 3) / 4, (uint64_t)sms * 16);
    }
    NL_CUDA(cudaMalloc(&out.cell, 8 * (size_t)g.cells), "near lists: cell table");
    NL_CUDA(cudaMalloc((void**)&bsum, 4 * (size_t)nb), "near lists: scratch");
    NL_CUDA(cudaMalloc((void**)&boff, 8 * ((size_t)nb + 3)), "near lists: scratch");
    NL_CUDA(cudaMalloc(&out.cloud, 16 * (n + 1)), "near lists: cloud");
    NL_CUDA(cudaMemsetAsync(boff + nb + 1, 0, 16, st), "near lists: memset");
    k_near_cloud<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(t.cloud, (uint32_t)n,
                                                                  static_cast<float4*>(out.cloud));
    k_near_lists<false><<<walk_blocks, kNearThreads, 0, st>>>(t, g, reinterpret_cast<const uchar2*>(t.grid),
                                                               static_cast<uint32_t*>(out.cell), nullptr, 0u,
                                                               boff + nb + 1, nullptr);
    k_near_block_sums<<<nb, kNearScanThreads, 0, st>>>(static_cast<const uint32_t*>(out.cell), g.cells, bsum);
    NL_CUDA(cudaGetLastError(), "near lists: launch");
    rc = launch_scan64(bsum, nb, boff, st, err);
    if (rc) goto done;
    k_near_offsets<<<nb, kNearScanThreads, 0, st>>>(static_cast<uint32_t*>(out.cell), g.cells, boff);
    NL_CUDA(cudaGetLastError(), "near lists: launch");
    NL_CUDA(cudaMemcpyAsync(h_tail, boff + nb, 16, cudaMemcpyDeviceToHost, st), "near lists: D2H");
    NL_CUDA(cudaStreamSynchronize(st), "near lists: count");
    if (h_tail[0] >= (1ull << 32)) {
        err = "the nearest-candidate lists would hold 2^32 entries or more (use a coarser grid)";
        rc = CAPT_E_RANGE;
        goto done;
    }
    out.entries = h_tail[0];
    out.fallback_cells = h_tail[1];
    NL_CUDA(cudaMalloc(&out.cand, 4 * std::max<size_t>((size_t)out.entries, 4)), "near lists: entries");
    k_near_lists<true><<<walk_blocks, kNearThreads, 0, st>>>(
        t, g, reinterpret_cast<const uchar2*>(t.grid), static_cast<uint32_t*>(out.cell),
        static_cast<uint32_t*>(out.cand), (uint32_t)n, nullptr, reinterpret_cast<uint32_t*>(boff + nb + 2));
    NL_CUDA(cudaGetLastError(), "near lists: launch");
    NL_CUDA(cudaMemcpyAsync(h_tail + 2, boff + nb + 2, 8, cudaMemcpyDeviceToHost, st), "near lists: D2H");
    NL_CUDA(cudaStreamSynchronize(st), "near lists: fill");
    if (h_tail[2] != 0) {
        err = "nearest-candidate lists: the fill walk disagreed with the count walk";
        rc = CAPT_E_BOUNDS;
        goto done;
    }
    out.bytes = 8 * (size_t)g.cells + 4 * std::max<size_t>((size_t)out.entries, 4) + 16 * (n + 1);
done:
    if (bsum) cudaFree(bsum);
    if (boff) cudaFree(boff);
    if (rc) out.release();
    return rc;
}

}  // namespace capt
