// Host CAPT construction (Alg. 1, Sec. IV-A/B) and the flattening into the device
// layout.  Compiled with -ffp-contract=off: the affordance and prune predicates are
// FP64 expressions evaluated one rounded operation at a time.
//
// Construction is the paper's recursive median partition with the afforded set z
// carried down the recursion.  Differences from a literal reading, none of which
// changes the result:
//  - the median is found with std::nth_element on (coordinate, index) instead of a
//    full sort (the first half is the same set either way);
//  - for points of the node's own halves, the distance to the sibling cell is the
//    distance along the split axis only (those points already lie inside the parent's
//    closed cell, so the other two clamped differences are exactly zero);
//  - the top levels of the recursion run on separate threads.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <system_error>
#include <thread>

#include "capt_internal.h"
#include "host_internal.h"

namespace capt {
namespace {

struct Cell {
    double lo[3], hi[3];
};

struct Builder {
    const float* pts;
    size_t n, N;
    double thr_afford, thr_prune;
    std::vector<uint32_t> perm;                  // N entries; index >= n is a pad at +inf
    std::vector<float>* T;
    std::vector<std::vector<uint32_t>> sets;     // per leaf
    std::vector<uint8_t> pruned;

    float key(uint32_t i, int d) const { return i < n ? pts[3 * (size_t)i + d] : INFINITY; }

    // FP64 squared distance from point i to the closed cell c (clamped per axis).
    bool affords(const Cell& c, uint32_t i) const {
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
            double v = pts[3 * (size_t)i + d], q = v;
            if (q < c.lo[d]) q = c.lo[d];
            if (q > c.hi[d]) q = c.hi[d];
            double e = v - q;
            s = s + e * e;
        }
        return s <= thr_afford;
    }

    // Same predicate for a point known to lie inside the parent's closed cell, tested
    // against the child that excludes it along axis d (only that axis differs).
    bool affords_axis(double plane, uint32_t i, int d) const {
        double e = (double)pts[3 * (size_t)i + d] - plane;
        double s = 0.0;
        s = s + e * e;
        return s <= thr_afford;
    }

    bool within_rmin(const Cell& c, uint32_t i) const {
        double s = 0.0;
        for (int d = 0; d < 3; d++) {
            if (!std::isfinite(c.lo[d]) || !std::isfinite(c.hi[d])) return false;
            double v = pts[3 * (size_t)i + d];
            double a = std::fabs(v - c.lo[d]), b = std::fabs(c.hi[d] - v);
            double e = a > b ? a : b;
            s = s + e * e;
        }
        return s <= thr_prune;
    }

    void node(size_t lo, size_t hi, const Cell& c, std::vector<uint32_t> z, size_t i, int d, int spawn_depth) {
        size_t m = hi - lo;
        if (m == 1) {
            size_t leaf = i - (N - 1);
            uint32_t rep = perm[lo];
            std::vector<uint32_t>& P = sets[leaf];
            bool pr = false;
            if (rep < n) pr = within_rmin(c, rep);
            if (pr) {
                P.assign(1, rep);
            } else {
                P = std::move(z);
                if (rep < n) P.push_back(rep);
                std::sort(P.begin(), P.end());
            }
            pruned[leaf] = pr ? 1 : 0;
            return;
        }
        size_t h = m / 2;
        auto first = perm.begin() + (ptrdiff_t)lo, last = perm.begin() + (ptrdiff_t)hi;
        auto cmp = [this, d](uint32_t a, uint32_t b) {
            float ka = key(a, d), kb = key(b, d);
            return ka < kb || (ka == kb && a < b);
        };
        std::nth_element(first, first + (ptrdiff_t)(h - 1), last, cmp);
        float Ti = key(perm[lo + h - 1], d);
        (*T)[i] = Ti;
        Cell c1 = c, c2 = c;
        c1.hi[d] = Ti;
        c2.lo[d] = Ti;
        std::vector<uint32_t> z1, z2;
        z1.reserve(z.size() + 16);
        z2.reserve(z.size() + 16);
        for (uint32_t p : z) {
            if (affords(c1, p)) z1.push_back(p);
            if (affords(c2, p)) z2.push_back(p);
        }
        z.clear();
        z.shrink_to_fit();
        for (size_t j = lo + h; j < hi; j++) {           // B2 against c1
            uint32_t p = perm[j];
            if (p < n && affords_axis(Ti, p, d)) z1.push_back(p);
        }
        for (size_t j = lo; j < lo + h; j++) {           // B1 against c2
            uint32_t p = perm[j];
            if (p < n && affords_axis(Ti, p, d)) z2.push_back(p);
        }
        int nd = (d + 1) % 3;
        if (spawn_depth > 0) {
            std::thread left([&, c1]() mutable { node(lo, lo + h, c1, std::move(z1), 2 * i + 1, nd, spawn_depth - 1); });
            node(lo + h, hi, c2, std::move(z2), 2 * i + 2, nd, spawn_depth - 1);
            left.join();
        } else {
            node(lo, lo + h, c1, std::move(z1), 2 * i + 1, nd, 0);
            node(lo + h, hi, c2, std::move(z2), 2 * i + 2, nd, 0);
        }
    }
};

}  // namespace

int build_host_tree(const float* points, size_t n, float r_min, float r_max, int threads, HostTree& out,
                    std::string& err) {
    auto t0 = std::chrono::steady_clock::now();
    if (n && !points) { err = "points is NULL"; return CAPT_E_ARG; }
    if (n >= (size_t(1) << 31)) { err = "n must be below 2^31"; return CAPT_E_ARG; }
    if (!(r_min >= 0.f) || !(r_max >= r_min) || !std::isfinite(r_max)) {
        err = "need 0 <= r_min <= r_max < inf";
        return CAPT_E_RANGE;
    }
    for (size_t j = 0; j < 3 * n; j++)
        if (!std::isfinite(points[j])) { err = "non-finite coordinate in points"; return CAPT_E_NONFINITE; }
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    try {
        out = HostTree();
        size_t N = 1;
        int L = 0;
        while (N < n) { N *= 2; L++; }
        out.n = n; out.N = N; out.L = L; out.r_min = r_min; out.r_max = r_max;
        out.build_threads = threads;
        out.pts.assign(points, points + 3 * n);
        out.T.assign(N > 1 ? N - 1 : 0, 0.f);
        Builder b;
        b.pts = out.pts.data();
        b.n = n; b.N = N;
        double ra = (double)r_max * (1.0 + 1e-5), rp = (double)r_min * (1.0 - 1e-5);
        b.thr_afford = ra * ra;
        b.thr_prune = rp * rp;
        b.perm.resize(N);
        for (size_t j = 0; j < N; j++) b.perm[j] = (uint32_t)j;
        b.T = &out.T;
        b.sets.resize(N);
        b.pruned.assign(N, 0);
        int spawn = 0;
        while ((1 << spawn) < threads && spawn < L && spawn < 6) spawn++;
        Cell root;
        for (int d = 0; d < 3; d++) { root.lo[d] = -INFINITY; root.hi[d] = INFINITY; }
        b.node(0, N, root, {}, 0, 0, spawn);
        // flatten the ragged sets
        out.set_begin.resize(N + 1);
        uint64_t tot = 0;
        for (size_t l = 0; l < N; l++) { out.set_begin[l] = tot; tot += b.sets[l].size(); }
        out.set_begin[N] = tot;
        out.set_idx.resize(tot);
        out.aabb.resize(6 * N);
        for (size_t l = 0; l < N; l++) {
            const auto& P = b.sets[l];
            std::copy(P.begin(), P.end(), out.set_idx.begin() + (ptrdiff_t)out.set_begin[l]);
            float* a = &out.aabb[6 * l];
            for (int e = 0; e < 3; e++) { a[e] = INFINITY; a[3 + e] = -INFINITY; }
            for (uint32_t p : P)
                for (int e = 0; e < 3; e++) {
                    float v = out.pts[3 * (size_t)p + e];
                    a[e] = std::min(a[e], v);
                    a[3 + e] = std::max(a[3 + e], v);
                }
        }
        out.pruned = std::move(b.pruned);
    } catch (const std::bad_alloc&) {
        err = "host allocation failed while building";
        return CAPT_E_NOMEM;
    } catch (const std::system_error& e) {
        err = std::string("thread creation failed: ") + e.what();
        return CAPT_E_NOMEM;
    }
    out.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return CAPT_OK;
}

// The descent reads T three levels at a time: the subtree of the level-3k node with
// Eytzinger index i is stored as 8 floats {T_i, T_2i+1, T_2i+2, T_4i+3, T_4i+4,
// T_4i+5, T_4i+6, +inf}, the subtrees in 8-ary heap order (children of block u are
// 8u+1 .. 8u+8), so one step is two 16-byte loads and three compares on x, y, z.
// The last L mod 3 levels follow as one 4-float block per level-3K node
// {T_i, T_2i+1, T_2i+2, +inf} (only T_i used when one level remains).
void blocked_shape(int L, BlockedSplits& out) {
    out.K = L / 3;
    out.R = L % 3;
    uint64_t nblk = 0, p8 = 1;
    for (int k = 0; k < out.K; k++) { nblk += p8; p8 *= 8; }
    const uint64_t ntail = out.R ? (uint64_t(1) << (3 * out.K)) : 0;
    out.tail_off = (uint32_t)(8 * nblk);
    out.total_floats = 8 * nblk + 4 * ntail + 4;
    // shared-memory prefix: at most 4 super-levels (585 blocks, 18.7 KB), plus the tail
    // when every super-level fits and the tail is at most 16 KB
    out.Ks = out.K < 4 ? out.K : 4;
    uint64_t sblk = 0;
    p8 = 1;
    for (int k = 0; k < out.Ks; k++) { sblk += p8; p8 *= 8; }
    out.stage_floats = (uint32_t)(8 * sblk);
    out.tail_staged = 0;
    if (out.Ks == out.K && ntail && 4 * ntail <= 4096) {
        out.stage_floats += (uint32_t)(4 * ntail);
        out.tail_staged = 1;
    }
}

void blocked_splits(const HostTree& t, BlockedSplits& out) {
    blocked_shape(t.L, out);
    out.data.assign(out.total_floats, INFINITY);
    const auto& T = t.T;
    const uint64_t ntail = out.R ? (uint64_t(1) << (3 * out.K)) : 0;
    uint64_t base_u = 0;
    for (int k = 0; k < out.K; k++) {
        const uint64_t width = uint64_t(1) << (3 * k);
        for (uint64_t s = 0; s < width; s++) {
            const uint64_t i = width - 1 + s, u = base_u + s;
            float* b = &out.data[8 * u];
            b[0] = T[i];
            b[1] = T[2 * i + 1];
            b[2] = T[2 * i + 2];
            b[3] = T[4 * i + 3];
            b[4] = T[4 * i + 4];
            b[5] = T[4 * i + 5];
            b[6] = T[4 * i + 6];
        }
        base_u += width;
    }
    for (uint64_t s = 0; s < ntail; s++) {
        const uint64_t i = ntail - 1 + s;
        float* b = &out.data[out.tail_off + 4 * s];
        b[0] = T[i];
        if (out.R == 2) {
            b[1] = T[2 * i + 1];
            b[2] = T[2 * i + 2];
        }
    }
}

void flatten(const HostTree& t, Layout& out) {
    out.leaves.resize(t.N);
    uint64_t blocks = 0;
    for (size_t l = 0; l < t.N; l++) {
        uint64_t cnt = t.set_begin[l + 1] - t.set_begin[l];
        LeafRec& r = out.leaves[l];
        for (int e = 0; e < 3; e++) { r.lo[e] = t.aabb[6 * l + e]; r.hi[e] = t.aabb[6 * l + 3 + e]; }
        r.block = (uint32_t)blocks;
        r.count = (uint32_t)cnt;
        blocks += (cnt + 3) / 4;
    }
    out.total_blocks = blocks;
    // three planes of 4-point quads: all x quads, then all y quads, then all z quads, so
    // that consecutive blocks read by consecutive lanes are contiguous in each plane
    const uint64_t plane = std::max<uint64_t>(blocks, 1);
    out.blocks.assign(12 * plane, INFINITY);
    out.ids.assign(4 * plane, 0xffffffffu);
    for (size_t l = 0; l < t.N; l++) {
        uint64_t b0 = out.leaves[l].block;
        uint64_t beg = t.set_begin[l], cnt = t.set_begin[l + 1] - beg;
        for (uint64_t j = 0; j < cnt; j++) {
            uint32_t p = t.set_idx[beg + j];
            uint64_t blk = b0 + j / 4, lane = j % 4;
            for (int e = 0; e < 3; e++) out.blocks[4 * (e * plane + blk) + lane] = t.pts[3 * (size_t)p + e];
            out.ids[4 * blk + lane] = p;
        }
    }
}

}  // namespace capt
