// Host-side launchers of the CAPT kernels (internal; each returns a capt_status).
#pragma once

#include <cuda_runtime_api.h>

#include <string>

#include "capt_internal.h"

namespace capt {

enum QueryMode { kModeSpheres = 0, kModeConfigs = 1 };

// Persistent query kernel: flags per sphere (mode 0) or per configuration (mode 1).
// ctr: a work counter zeroed on st before the launch (the warps take tiles from it), or
// nullptr for the static schedule (warp w takes tiles w, w + warps, ...).
int launch_query(const DevArgs& t, int mode, const float* centers, const float* radii, uint64_t n_items, int S,
                 uint8_t* out, const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st,
                 std::string& err);

// Sequential Alg. 3 work counters for configuration queries.
int launch_count_configs(const DevArgs& t, const float* centers, const float* radii, uint64_t C, int S, bool per_sphere,
                         bool use_grid, uint64_t* counts, cudaStream_t st, std::string& err);

// Boxes of the chunks of kChunkBlocks blocks (cbox: 8 floats per chunk, chunk_count).
int launch_chunk_boxes(const float* blocks, uint64_t total_blocks, float* cbox, cudaStream_t st, std::string& err);

int launch_leaves(const DevArgs& t, const float* centers, uint64_t m, uint32_t* leaves, cudaStream_t st,
                  std::string& err);

// Distance-bound grid: 2 bytes per cell of g (dist_grid.cu).
int launch_dist_grid(const DevArgs& t, const GridShape& g, uint8_t* out, cudaStream_t st, std::string& err);

// Nearest-candidate lists of the clearance over the tree's grid (dist_grid.cu): device
// buffers owned by the tree once built (release() frees them).
struct NearLists {
    void* cell = nullptr;    // 2 uint32 per grid cell: {first entry, entries or kNearFallback}
    void* cand = nullptr;    // uint32 point indices, each list padded to a multiple of 4 with n
    void* cloud = nullptr;   // float4 per point, then one at +inf
    uint64_t entries = 0, fallback_cells = 0;
    size_t bytes = 0;
    void release();
};
// Builds them from the tree's grid, sets and cloud (n points).  Synchronises st.
int device_near_lists(const DevArgs& t, size_t n, cudaStream_t st, NearLists& out, std::string& err);

// Clearance forward / backward.
int launch_count_clearance(const DevArgs& t, const float* centers, uint64_t m, bool lists, uint64_t* counts,
                           cudaStream_t st, std::string& err);
int launch_clearance_fwd(const DevArgs& t, const float* centers, const float* radii, uint64_t T, int W, int S,
                         float margin, float* cost, float* dist, int32_t* argmin, const capt_launch_cfg& cfg,
                         cudaStream_t st, std::string& err);
int launch_clearance_bwd(const DevArgs& t, const float* centers, const float* radii, const float* dist,
                         const int32_t* argmin, const float* grad_cost, uint64_t T, int W, int S, float margin,
                         float* grad, cudaStream_t st, std::string& err);

// Edge validation: scratch holds (E + 1) uint32 work-item offsets plus one counter.
size_t edge_scratch_words(size_t E);
// Word of the edge scratch that holds the 64-bit count of configurations evaluated.
__host__ __device__ __forceinline__ uint32_t edge_eval_word(uint32_t E) { return (E + 3u) & ~1u; }
int launch_edges_persistent(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                            const int32_t* ns, uint64_t E, uint8_t* valid, uint32_t* scratch,
                            const capt_launch_cfg& cfg, cudaStream_t st, std::string& err);
int launch_edges_per_edge(const DevArgs& t, const capt_arm& arm, const float* qa, const float* qb,
                          const int32_t* h_ns, uint64_t E, uint8_t* valid, const capt_launch_cfg& cfg,
                          cudaStream_t st, std::string& err);

// Configurations given by joint angles q [C][J]: kinematics in-kernel, one flag each.
int launch_joint_configs(const DevArgs& t, const capt_arm& arm, const float* q, uint64_t C, uint8_t* out,
                         const capt_launch_cfg& cfg, unsigned long long* ctr, cudaStream_t st, std::string& err);

// Alg. 2 on the device: d_points [n][3] -> kept indices (d_kept, caller-owned, n
// entries) in the last pass's curve order, *n_out = their count.  Synchronises st.
int device_sfc_filter(const float* d_points, size_t n, float r, uint32_t* d_kept, size_t* n_out, cudaStream_t st,
                      std::string& err);

// out[i] = pts[idx[i]] for i < m (points [.][3]).
int launch_gather_points(const float* pts, const uint32_t* idx, size_t m, float* out, cudaStream_t st,
                         std::string& err);

// Stable LSD radix sort of n (key, value) pairs by the `passes` lowest 8-bit digits of
// the 32-bit keys, through kb / vb; an even number of passes leaves the result in ka /
// va.  hist: 256 * ceil(n / 256) words of scratch.
int launch_sort_pairs(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t n, int passes, uint32_t* hist,
                      cudaStream_t st, std::string& err);

// Exclusive scan of v[0..len) into 64-bit offsets out[0..len], out[len] = total (one block).
int launch_scan64(const uint32_t* v, uint32_t len, unsigned long long* out, cudaStream_t st, std::string& err);

// Compact (de-duplicated) affordance sets of an uploaded tree: device buffers owned by
// the tree once built (release() frees them).
struct CompactSets {
    void* cleaves = nullptr;   // N leaf records {lo, first list entry, hi, number of chunks}
    void* clist = nullptr;     // uint32 chunk ids, ascending per leaf
    void* cblocks = nullptr;   // the Z-ordered cloud: n_chunks x 8 blocks in three planes
    void* ccbox = nullptr;     // n_chunks boxes of 8 floats
    uint64_t n_chunks = 0, list_len = 0;
    size_t bytes = 0;
    void release();
};

// Builds the compact sets from the tree's device sets (t.leaves, t.ids, t.cloud), with
// the cloud ordered along its Z-order curve on the device.  Synchronises st.
int device_compact(const DevArgs& t, size_t n, cudaStream_t st, CompactSets& out, std::string& err);

// Number of SMs of the current device (cached per device).
int sm_count();

}  // namespace capt
