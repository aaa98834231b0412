// Host space-filling-curve filter (Alg. 2, Sec. IV-C).  Compiled with -ffp-contract=off.
//
// Per pass: the surviving points, taken in ascending index order, are sorted by their
// 63-bit Morton key with a stable LSD radix sort (so equal keys stay in index order),
// then one linear sweep keeps a point iff its FP32 squared distance to the last kept
// point exceeds fl(r^2).
#include <cmath>
#include <cstring>
#include <vector>

#include "capt_internal.h"
#include "host_internal.h"

namespace capt {
namespace {

// Spread the low 21 bits of v so that bit b moves to bit 3b.
inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

const int kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

inline float d2f(const float* a, const float* b) {
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    float s = dx * dx + dy * dy;
    s = s + dz * dz;
    return s;
}

}  // namespace

int host_sfc_filter(const float* pts, size_t n, float r, uint32_t* kept, size_t* n_out, std::string& err) {
    if (!n_out || (n && (!pts || !kept))) { err = "NULL argument"; return CAPT_E_ARG; }
    if (!(r >= 0.f)) { err = "min_spacing must be >= 0"; return CAPT_E_RANGE; }
    if (n >= (size_t(1) << 32)) { err = "n must be below 2^32"; return CAPT_E_ARG; }
    *n_out = 0;
    if (n == 0) return CAPT_OK;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) lo[a] = hi[a] = pts[a];
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            float v = pts[3 * j + a];
            if (!std::isfinite(v)) { err = "non-finite coordinate in points"; return CAPT_E_NONFINITE; }
            lo[a] = v < lo[a] ? v : lo[a];
            hi[a] = v > hi[a] ? v : hi[a];
        }
    try {
        std::vector<uint64_t> sp(3 * n);              // spread quantised coordinates
        for (size_t j = 0; j < n; j++)
            for (int a = 0; a < 3; a++) {
                double ext = (double)hi[a] - (double)lo[a];
                uint32_t v = 0;
                if (ext > 0.0) {
                    double f = std::floor(((double)pts[3 * j + a] - (double)lo[a]) / ext * 2097152.0);
                    v = f >= 2097151.0 ? 2097151u : (uint32_t)f;
                }
                sp[3 * j + a] = spread3(v);
            }
        std::vector<uint32_t> cur(n), asc(n), tmp(n);
        std::vector<uint64_t> key(n), ktmp(n);
        std::vector<uint8_t> alive(n, 1);
        std::vector<uint32_t> hist(1 << 11);
        for (size_t j = 0; j < n; j++) cur[j] = (uint32_t)j;
        size_t m = n;
        float r2 = r * r;
        for (int p = 0; p < 6; p++) {
            // survivors in ascending index order
            size_t k = 0;
            for (size_t j = 0; j < n; j++) if (alive[j]) asc[k++] = (uint32_t)j;
            const int* X = kPerms[p];
            for (size_t j = 0; j < m; j++) {
                const uint64_t* s = &sp[3 * (size_t)asc[j]];
                key[j] = (s[X[0]] << 2) | (s[X[1]] << 1) | s[X[2]];
            }
            // stable LSD radix sort by key: 6 digits of 11 bits cover 63 bits
            for (int shift = 0; shift < 63; shift += 11) {
                std::fill(hist.begin(), hist.end(), 0u);
                for (size_t j = 0; j < m; j++) hist[(key[j] >> shift) & 2047u]++;
                if (hist[(key[0] >> shift) & 2047u] == m) continue;     // constant digit
                uint32_t run = 0;
                for (auto& h : hist) { uint32_t c = h; h = run; run += c; }
                for (size_t j = 0; j < m; j++) {
                    uint32_t dst = hist[(key[j] >> shift) & 2047u]++;
                    tmp[dst] = asc[j];
                    ktmp[dst] = key[j];
                }
                asc.swap(tmp);
                key.swap(ktmp);
            }
            // greedy sweep against the last kept point
            size_t i = 0;
            cur[0] = asc[0];
            for (size_t j = 1; j < m; j++) {
                uint32_t pj = asc[j];
                if (d2f(pts + 3 * (size_t)cur[i], pts + 3 * (size_t)pj) > r2) {
                    cur[++i] = pj;
                } else {
                    alive[pj] = 0;
                }
            }
            m = i + 1;
        }
        std::memcpy(kept, cur.data(), m * sizeof(uint32_t));
        *n_out = m;
    } catch (const std::bad_alloc&) {
        err = "host allocation failed in sfc_filter";
        return CAPT_E_NOMEM;
    }
    return CAPT_OK;
}

int host_morton_order(const float* pts, size_t n, uint32_t* order, std::string& err) {
    if (n && (!pts || !order)) { err = "NULL argument"; return CAPT_E_ARG; }
    if (n >= (size_t(1) << 32)) { err = "n must be below 2^32"; return CAPT_E_ARG; }
    if (n == 0) return CAPT_OK;
    float lo[3], hi[3];
    for (int a = 0; a < 3; a++) lo[a] = hi[a] = pts[a];
    for (size_t j = 0; j < n; j++)
        for (int a = 0; a < 3; a++) {
            float v = pts[3 * j + a];
            if (!std::isfinite(v)) { err = "non-finite coordinate in points"; return CAPT_E_NONFINITE; }
            lo[a] = v < lo[a] ? v : lo[a];
            hi[a] = v > hi[a] ? v : hi[a];
        }
    try {
        std::vector<uint64_t> key(n), ktmp(n);
        std::vector<uint32_t> idx(n), tmp(n);
        for (size_t j = 0; j < n; j++) {
            uint64_t k = 0;
            for (int a = 0; a < 3; a++) {
                double ext = (double)hi[a] - (double)lo[a];
                uint32_t v = 0;
                if (ext > 0.0) {
                    double f = std::floor(((double)pts[3 * j + a] - (double)lo[a]) / ext * 2097152.0);
                    v = f >= 2097151.0 ? 2097151u : (uint32_t)f;
                }
                k |= spread3(v) << (2 - a);   // x most significant in every bit triple
            }
            key[j] = k;
            idx[j] = (uint32_t)j;
        }
        std::vector<uint32_t> hist(1 << 11);
        for (int shift = 0; shift < 63; shift += 11) {   // stable LSD radix sort by key
            std::fill(hist.begin(), hist.end(), 0u);
            for (size_t j = 0; j < n; j++) hist[(key[j] >> shift) & 2047u]++;
            uint32_t run = 0;
            for (auto& h : hist) { uint32_t c = h; h = run; run += c; }
            for (size_t j = 0; j < n; j++) {
                uint32_t dst = hist[(key[j] >> shift) & 2047u]++;
                tmp[dst] = idx[j];
                ktmp[dst] = key[j];
            }
            idx.swap(tmp);
            key.swap(ktmp);
        }
        std::memcpy(order, idx.data(), n * sizeof(uint32_t));
    } catch (const std::bad_alloc&) {
        err = "host allocation failed in capt_morton_order";
        return CAPT_E_NOMEM;
    }
    return CAPT_OK;
}

}  // namespace capt
