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

// One thread per cell: the bounds of the distance from the grown cell to the cloud,
// through the cell's representative point m and its leaf's set.
__global__ void __launch_bounds__(kGridThreads) k_dist_grid(DevArgs t, GridShape g, uchar2* __restrict__ out) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.cells) return;
    const uint32_t nx = (uint32_t)g.n[0], ny = (uint32_t)g.n[1];
    const uint32_t idx[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
    const float dl = __fmul_ru(g.h, 0.01f);
    float m[3];
    float rho2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float L = __fsub_rd(__fadd_rd(g.org[d], __fmul_rd((float)idx[d], g.h)), dl);
        const float U = __fadd_ru(__fadd_ru(g.org[d], __fmul_ru((float)(idx[d] + 1u), g.h)), dl);
        m[d] = __fmul_rn(__fadd_rn(L, U), 0.5f);
        const float e = fmaxf(__fsub_ru(m[d], L), __fsub_ru(U, m[d]));
        rho2 = __fadd_ru(rho2, __fmul_ru(e, e));
    }
    const float rho = __fsqrt_ru(rho2);
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

}  // namespace capt
