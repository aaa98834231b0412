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
    std::vector<float> blocks;        // 12 floats per block
    std::vector<uint32_t> ids;        // 4 per block
    uint64_t total_blocks = 0;
};

// Kernel view of an uploaded tree (raw device pointers, passed by value).
struct DevArgs {
    const float* T = nullptr;        // N-1 split values, padded to a multiple of 4 floats
    const LeafRec* leaves = nullptr; // N records
    const float* blocks = nullptr;   // 12 floats per 4-point block (float4 x 3)
    const uint32_t* ids = nullptr;   // 4 per block
    const float* cloud = nullptr;    // [n][3]
    int* status = nullptr;           // latched device status bits
    uint32_t N = 1;
    int L = 0;
    float r_min = 0.f, r_max = 0.f;
};

int build_host_tree(const float* points, size_t n, float r_min, float r_max, int threads, HostTree& out,
                    std::string& err);
void flatten(const HostTree& t, Layout& out);
int host_sfc_filter(const float* points, size_t n, float r, uint32_t* kept, size_t* n_out, std::string& err);

}  // namespace capt
