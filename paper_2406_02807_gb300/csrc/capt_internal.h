// Internal structures of the CAPT library (host side).  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/capt.h"

namespace capt {

// Host form of a built tree: T in Eytzinger order, ragged sets, per-leaf boxes.
struct HostTree {
    size_t n = 0, N = 1;
    int L = 0;
    float r_min = 0.f, r_max = 0.f;
    std::vector<float> pts;            // [n][3]
    std::vector<float> T;              // N-1
    std::vector<uint64_t> set_begin;   // N+1
    std::vector<uint32_t> set_idx;     // sum |P_i|, ascending within a set
    std::vector<float> aabb;           // [N][6] lo xyz, hi xyz (+inf/-inf when empty)
    std::vector<uint8_t> pruned;       // [N]
    double build_ms = 0.0;
    int build_threads = 1;
};

// 32-byte leaf record of the device layout.
struct LeafRec {
    float lo[3];
    uint32_t block;   // first 4-point block of the set
    float hi[3];
    uint32_t count;   // |P_i|
};
static_assert(sizeof(LeafRec) == 32, "leaf record is one 32-byte sector");

// Flattened device layout, built on the host then copied.
struct Layout {
    std::vector<LeafRec> leaves;      // N
    std::vector<float> blocks;        // three planes (x, y, z) of 4 floats per block
    std::vector<uint32_t> ids;        // 4 per block
    uint64_t total_blocks = 0;
};

// Blocked copy of T used by the descent (see blocked_splits).
struct BlockedSplits {
    std::vector<float> data;
    uint32_t tail_off = 0;      // float offset of the tail blocks
    int K = 0, R = 0;           // full 3-level super-levels, remaining levels (L = 3K + R)
    uint32_t stage_floats = 0;  // prefix copied to shared memory by the staged kernels
    int Ks = 0;                 // super-levels inside that prefix
    int tail_staged = 0;        // 1 if the tail is inside it too
    uint64_t total_floats = 0;  // size of data
};
void blocked_shape(int L, BlockedSplits& out);   // every field but data
void blocked_splits(const HostTree& t, BlockedSplits& out);

// Blocks per chunk of the point buffer: chunk k holds blocks [8k, 8k + 8) (a chunk may
// straddle two sets); its box is the FP32 min / max of the finite coordinates in it.
constexpr uint32_t kChunkBlocks = 8;
inline uint64_t chunk_count(uint64_t total_blocks) {
    return ((total_blocks > 0 ? total_blocks : 1) + kChunkBlocks - 1) / kChunkBlocks;
}

// Distance-bound grid (dist_grid.cu): a uniform grid of cubic cells over the cloud's
// bounding box grown by r_max, two bytes per cell (a lower and an upper bound of the
// distance from the cell to the cloud, in units of `unit`).  Cell (i, j, k) is the box
// [org + (i, j, k) h, org + (i + 1, j + 1, k + 1) h], computed exactly from the FP32
// org and h, stored at (k n[1] + j) n[0] + i.
constexpr uint64_t kGridDefaultCells = 1ull << 22;
constexpr int kGridMaxAxis = 16384;
struct GridShape {
    float org[3] = {0.f, 0.f, 0.f};
    float h = 0.f, inv_h = 0.f, unit = 0.f, pad = 0.f;
    int n[3] = {0, 0, 0};
    uint32_t cells = 0;   // 0: no grid
};
GridShape grid_shape(const float lo[3], const float hi[3], float r_max, uint64_t n_points, uint64_t max_cells);

// Entry count of a grid cell whose centres take the paper's path (descent and full set
// scan) instead of a nearest-candidate list.
constexpr uint32_t kNearFallback = 0xffffffffu;

// Kernel view of an uploaded tree (raw device pointers, passed by value).
struct DevArgs {
    const float* T = nullptr;        // blocked split array (BlockedSplits::data)
    uint32_t tail_off = 0;
    int K = 0, R = 0, Ks = 0, tail_staged = 0;
    uint32_t stage_floats = 0;
    const LeafRec* leaves = nullptr; // N records
    const float* blocks = nullptr;   // 4-point blocks in three planes of float4 (x, y, z quads)
    uint64_t plane = 1;              // blocks per plane (float4 stride between the planes)
    const uint32_t* ids = nullptr;   // 4 per block
    const float* cbox = nullptr;     // chunk boxes: 8 floats each {lo.xyz, 0, hi.xyz, 0}
    const float* cloud = nullptr;    // [n][3]
    // compact (de-duplicated) sets: null until capt_compact
    const LeafRec* cleaves = nullptr;  // N records: {lo, first list entry, hi, chunks}
    const uint32_t* clist = nullptr;   // chunk ids of each leaf, ascending
    const float* cblocks = nullptr;    // the cloud in Z-order, 4-point blocks in three planes
    uint64_t cplane = 1;               // blocks per plane of cblocks
    const float* ccbox = nullptr;      // boxes of the cloud's 32-point chunks
    int* status = nullptr;           // latched device status bits
    uint32_t N = 1;
    int L = 0;
    float r_min = 0.f, r_max = 0.f;
    float lo[3] = {0.f, 0.f, 0.f};   // bounding box of the cloud (empty cloud: lo > hi)
    float hi[3] = {-1.f, -1.f, -1.f};
    const uint8_t* grid = nullptr;   // distance-bound grid, 2 g.cells bytes (null: none)
    GridShape g;
    // nearest-candidate lists of the clearance (null: none): per grid cell two words
    // {first entry, entries (a multiple of 4), or kNearFallback}, the entries (point
    // indices, padded with n), and the cloud as 4 floats per point plus a point at
    // +inf (index n)
    const uint32_t* nl_cell = nullptr;
    const uint32_t* nl_cand = nullptr;
    const float* nl_cloud = nullptr;
    // always -0: the zero addend of the packed exact products (f2_mulz), passed as an
    // argument so that the code generator cannot see its value
    float nzero = -0.f;
};

}  // namespace capt
