// GPU construction of a CAPT (internal; see device_build.cu).
#pragma once

#include <cuda_runtime_api.h>

#include <cstdint>
#include <string>

#include "capt_internal.h"

namespace capt {

// Device arrays of a tree built on the GPU.  Tb .. cloud are the query layout (the
// same arrays capt_upload makes from a host tree); Tplain, set_idx, set_begin and
// pruned are the plain arrays the host form holds, kept for export.
struct DeviceTree {
    float* Tb = nullptr;                   // blocked split array, bs.total_floats floats
    float* Tplain = nullptr;               // N - 1 split values in Eytzinger order
    LeafRec* leaves = nullptr;             // N records
    float* blocks = nullptr;               // 3 planes of 4 * max(total_blocks, 1) floats
    uint32_t* ids = nullptr;               // 4 * max(total_blocks, 1)
    float* cloud = nullptr;                // [n][3]
    uint32_t* set_idx = nullptr;           // total, ascending within each set
    unsigned long long* set_begin = nullptr;   // N + 1
    uint8_t* pruned = nullptr;             // N
    size_t n = 0;
    uint32_t N = 1;
    int L = 0;
    uint64_t total = 0, total_blocks = 0;
    BlockedSplits bs;                      // shape only (data stays empty)
    float box_lo[3] = {0.f, 0.f, 0.f}, box_hi[3] = {0.f, 0.f, 0.f};
    size_t bytes = 0;                      // bytes of the query layout

    void release();   // cudaFree every array (the device must be current)
};

// Build on the current device from d_points (device float[n][3]); every stage runs on
// st and the call returns after the stream has finished it.  Temporary buffers are
// allocated and freed inside.  Returns a capt_status; on failure `out` owns nothing.
int device_build(const float* d_points, size_t n, float r_min, float r_max, cudaStream_t st, DeviceTree& out,
                 std::string& err);

}  // namespace capt
