// C ABI of the CAPT library: argument checking, tree lifecycle, upload, dispatch to
// the kernels, the host-buffer pipeline, the autotuner and CUDA-graph edge plans.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/capt.h"
#include "capt_internal.h"
#include "host_internal.h"
#include "device_build.h"
#include "kernels.h"

using capt::DevArgs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(CAPT_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(call, what)                        \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// Restores the caller's current device when it goes out of scope.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool valid_cfg(int kernel, const capt_launch_cfg& c) {
    if (c.warps_per_block < 1 || c.warps_per_block > 16) return false;
    if (c.staging != CAPT_STAGE_GLOBAL && c.staging != CAPT_STAGE_SMEM) return false;
    if (c.prefetch < 0 || c.prefetch > CAPT_MAX_PREFETCH) return false;
    if (c.prefetch != 0 && kernel != CAPT_KERNEL_CONFIGS && kernel != CAPT_KERNEL_CLEARANCE) return false;
    if (c.grid != 0 && c.grid != 1) return false;
    const int spl = c.spheres_per_lane;
    const bool scan_mode = c.chunk >= CAPT_SCAN_SETS && c.chunk <= CAPT_SCAN_COMPACT;
    if (kernel == CAPT_KERNEL_SPHERES) return (spl == 1 || spl == 2 || spl == 4 || spl == 8) && scan_mode;
    if (kernel == CAPT_KERNEL_CONFIGS) return (spl == 2 || spl == 4 || spl == 8 || spl == 16) && scan_mode;
    if (kernel == CAPT_KERNEL_EDGES) return c.chunk >= 1 && c.chunk <= 1024;   // one configuration per lane
    if (kernel == CAPT_KERNEL_CLEARANCE) return true;
    if (kernel == CAPT_KERNEL_JOINTS) return true;   // one configuration per lane
    return false;
}

}  // namespace

// Device status allocation: the latched status word (first 256 bytes), then the work
// counters of the query kernels.
constexpr size_t kStatusBytes = 256 + 64 * sizeof(unsigned long long);

struct capt_tree {
    capt::HostTree h;
    int device = -1;
    void* d_T = nullptr;
    void* d_leaves = nullptr;
    void* d_blocks = nullptr;
    void* d_ids = nullptr;
    void* d_cloud = nullptr;
    void* d_cbox = nullptr;      // chunk boxes (chunk_count(total_blocks) x 8 floats)
    uint8_t* d_grid = nullptr;   // distance-bound grid of capt_build_grid (2 bytes per cell)
    capt::GridShape gshape;
    capt::NearLists nl;          // nearest-candidate lists of capt_build_near_lists (over the grid)
    int* d_status = nullptr;
    uint64_t total_blocks = 0;
    size_t dev_bytes = 0;
    uint32_t tail_off = 0, stage_floats = 0;
    float box_lo[3] = {INFINITY, INFINITY, INFINITY};     // bounding box of every point
    float box_hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int K = 0, R = 0, Ks = 0, tail_staged = 0;
    capt_launch_cfg cfg[CAPT_N_KERNELS];
    // host-buffer pipeline
    float* d_pipe_c[2] = {nullptr, nullptr};
    uint8_t* d_pipe_f[2] = {nullptr, nullptr};
    size_t pipe_cap = 0;   // floats per centre buffer
    size_t pipe_fbytes = 0;   // bytes per flag buffer
    cudaStream_t pipe_stream = nullptr;
    cudaEvent_t pipe_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    uint8_t* d_zc_flags = nullptr;  // flags of the zero-copy path when h_flags is pageable
    size_t zc_cap = 0;
    // edge validation scratch (persistent mode without a plan)
    uint32_t* d_edge_scratch = nullptr;
    size_t edge_scratch_cap = 0;
    // tree built on the device: its plain arrays stay there until the host form is
    // first needed (host_pending)
    bool host_pending = false;
    void* d_Tplain = nullptr;
    void* d_set_idx = nullptr;
    void* d_set_begin = nullptr;
    void* d_pruned = nullptr;
    // compact (de-duplicated) sets, built by capt_compact; full_dropped: the replicated
    // device sets (blocks, ids, chunk boxes) were freed after it
    capt::CompactSets cs;
    bool full_dropped = false;
    // live edge plans (their graphs hold the device pointers); shared so that a plan
    // freed after its tree does not touch the tree
    std::shared_ptr<std::atomic<int>> n_plans = std::make_shared<std::atomic<int>>(0);
    // work counters of the persistent query kernels (dynamic tile scheduling), in the
    // status allocation after its first 256 bytes; a slot is zeroed for a launch only
    // after the launch that last used it has finished (its event)
    static constexpr int kCtrSlots = 64;
    unsigned long long* d_ctr = nullptr;
    mutable cudaEvent_t ctr_ev[kCtrSlots] = {};
    mutable bool ctr_pending[kCtrSlots] = {};
    mutable uint32_t ctr_next = 0;
    mutable std::mutex ctr_mu;
    std::mutex mu;

    capt_tree() {
        cfg[CAPT_KERNEL_SPHERES] = {8, 2, CAPT_STAGE_SMEM, 0};
        cfg[CAPT_KERNEL_CONFIGS] = {4, 8, CAPT_STAGE_GLOBAL, 1};
        cfg[CAPT_KERNEL_EDGES] = {8, 2, CAPT_STAGE_SMEM, 32};
        cfg[CAPT_KERNEL_CLEARANCE] = {16, 2, CAPT_STAGE_GLOBAL, 0, 0, 1};   // lists once built
        cfg[CAPT_KERNEL_JOINTS] = {4, 1, CAPT_STAGE_GLOBAL, 0};
    }

    DevArgs args() const {
        DevArgs a;
        a.T = static_cast<const float*>(d_T);
        a.tail_off = tail_off;
        a.K = K;
        a.R = R;
        a.Ks = Ks;
        a.tail_staged = tail_staged;
        a.stage_floats = stage_floats;
        a.leaves = static_cast<const capt::LeafRec*>(d_leaves);
        a.blocks = static_cast<const float*>(d_blocks);
        a.plane = total_blocks > 0 ? total_blocks : 1;
        a.ids = static_cast<const uint32_t*>(d_ids);
        a.cbox = static_cast<const float*>(d_cbox);
        a.cloud = static_cast<const float*>(d_cloud);
        a.cleaves = static_cast<const capt::LeafRec*>(cs.cleaves);
        a.clist = static_cast<const uint32_t*>(cs.clist);
        a.cblocks = static_cast<const float*>(cs.cblocks);
        a.cplane = cs.n_chunks > 0 ? cs.n_chunks * capt::kChunkBlocks : 1;
        a.ccbox = static_cast<const float*>(cs.ccbox);
        a.status = d_status;
        a.grid = gshape.cells ? d_grid : nullptr;
        a.g = gshape;
        a.nl_cell = static_cast<const uint32_t*>(nl.cell);
        a.nl_cand = static_cast<const uint32_t*>(nl.cand);
        a.nl_cloud = static_cast<const float*>(nl.cloud);
        a.N = (uint32_t)h.N;
        a.L = h.L;
        a.r_min = h.r_min;
        a.r_max = h.r_max;
        for (int d = 0; d < 3; d++) {
            a.lo[d] = box_lo[d];
            a.hi[d] = box_hi[d];
        }
        return a;
    }

    void free_device() {
        if (device < 0) return;
        DeviceGuard g(device);
        for (void* p : {d_T, d_leaves, d_blocks, d_ids, d_cloud, d_cbox, (void*)d_status, (void*)d_pipe_c[0], (void*)d_pipe_c[1],
                        (void*)d_pipe_f[0], (void*)d_pipe_f[1], (void*)d_edge_scratch, (void*)d_zc_flags, (void*)d_grid,
                        d_Tplain,
                        d_set_idx, d_set_begin, d_pruned})
            if (p) cudaFree(p);
        cs.release();
        nl.release();
        full_dropped = false;
        for (int i = 0; i < kCtrSlots; i++) {
            if (ctr_ev[i]) cudaEventDestroy(ctr_ev[i]);
            ctr_ev[i] = nullptr;
            ctr_pending[i] = false;
        }
        d_ctr = nullptr;   // part of the status allocation
        for (auto& e : pipe_ev)
            if (e) cudaEventDestroy(e);
        if (pipe_stream) cudaStreamDestroy(pipe_stream);
        d_T = d_leaves = d_blocks = d_ids = d_cloud = d_cbox = nullptr;
        d_grid = nullptr;
        gshape = capt::GridShape();
        d_Tplain = d_set_idx = d_set_begin = d_pruned = nullptr;
        d_status = nullptr;
        d_pipe_c[0] = d_pipe_c[1] = nullptr;
        d_pipe_f[0] = d_pipe_f[1] = nullptr;
        d_edge_scratch = nullptr;
        d_zc_flags = nullptr;
        zc_cap = 0;
        for (auto& e : pipe_ev) e = nullptr;
        pipe_stream = nullptr;
        pipe_cap = 0;
        pipe_fbytes = 0;
        edge_scratch_cap = 0;
        dev_bytes = 0;
        device = -1;
    }
};

namespace {

// Device address of a page-locked host allocation that the current device can reach,
// or nullptr for pageable (or device) memory.
const void* mapped_device_pointer(const void* h) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// The tree must be uploaded and the caller's current device must be the tree's.
int check_ready(const capt_tree* t) {
    if (!t) return fail(CAPT_E_ARG, "tree is NULL");
    if (t->device < 0) return fail(CAPT_E_STATE, "tree is not uploaded (call capt_upload)");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != t->device)
        return fail(CAPT_E_STATE, "current CUDA device differs from the tree's device");
    return CAPT_OK;
}

// check_ready, and the replicated device sets are still there (not dropped by capt_compact).
int check_full(const capt_tree* t) {
    const int rc = check_ready(t);
    if (rc) return rc;
    if (t->full_dropped)
        return fail(CAPT_E_STATE, "the replicated sets were dropped by capt_compact (only the compact scan remains)");
    return CAPT_OK;
}

// Launch a persistent query kernel with dynamic tile scheduling: it gets a counter slot
// of the tree's pool, zeroed on `st` after the launch that last used the slot has
// finished.  Inside a stream capture the launch keeps the static schedule (no counter,
// no events), so a captured graph has no hidden state.
template <class F>
int with_counter(const capt_tree* t, cudaStream_t st, F&& launch) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!t->d_ctr || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return launch(nullptr);
    }
    std::lock_guard<std::mutex> lk(t->ctr_mu);
    const int slot = (int)(t->ctr_next++ % capt_tree::kCtrSlots);
    if (!t->ctr_ev[slot] && cudaEventCreateWithFlags(&t->ctr_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        t->ctr_ev[slot] = nullptr;
        return launch(nullptr);
    }
    cudaError_t e = cudaSuccess;
    if (t->ctr_pending[slot]) e = cudaStreamWaitEvent(st, t->ctr_ev[slot], 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_ctr + slot, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "work counter");
    const int rc = launch(t->d_ctr + slot);
    e = cudaEventRecord(t->ctr_ev[slot], st);
    if (e != cudaSuccess) {
        t->ctr_pending[slot] = false;
        return rc ? rc : cuda_fail(e, "work counter event");
    }
    t->ctr_pending[slot] = true;
    return rc;
}

// The scan mode of a sphere / configuration launch has its data on the device.
int check_scan(const capt_tree* t, const capt_launch_cfg& c) {
    if (c.chunk == CAPT_SCAN_COMPACT && !t->cs.clist)
        return fail(CAPT_E_STATE, "scan mode CAPT_SCAN_COMPACT needs capt_compact first");
    if (c.chunk != CAPT_SCAN_COMPACT && t->full_dropped)
        return fail(CAPT_E_STATE, "the replicated sets were dropped by capt_compact: use CAPT_SCAN_COMPACT");
    return CAPT_OK;
}

// Candidate scan modes for the autotuners: those whose data is on the device.
std::vector<int> scan_modes(const capt_tree* t) {
    std::vector<int> m;
    if (!t->full_dropped) {
        m.push_back(CAPT_SCAN_SETS);
        m.push_back(CAPT_SCAN_CHUNKED);
    }
    if (t->cs.clist) m.push_back(CAPT_SCAN_COMPACT);
    return m;
}

// Two chunk buffers of `chunk` configurations of S spheres (+ slack for the radii),
// their flag buffers, a copy stream and events, kept by the tree.
bool ensure_pipe(capt_tree* t, size_t chunk, int S) {
    const size_t cfloats = chunk * (size_t)S * 3;
    if (t->pipe_cap >= cfloats + 64) return true;
    for (int i = 0; i < 2; i++) {
        if (t->d_pipe_c[i]) cudaFree(t->d_pipe_c[i]);
        if (t->d_pipe_f[i]) cudaFree(t->d_pipe_f[i]);
        t->d_pipe_c[i] = nullptr;
        t->d_pipe_f[i] = nullptr;
    }
    t->pipe_cap = 0;
    t->pipe_fbytes = 0;
    for (int i = 0; i < 2; i++) {
        if (cudaMalloc((void**)&t->d_pipe_c[i], (cfloats + 64) * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&t->d_pipe_f[i], chunk + 256) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    t->pipe_cap = cfloats + 64;
    t->pipe_fbytes = chunk + 256;
    if (!t->pipe_stream && cudaStreamCreateWithFlags(&t->pipe_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (auto& e : t->pipe_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}

// A device flag buffer of at least C bytes (zero-copy path with pageable flags).
bool ensure_flags(capt_tree* t, size_t C) {
    if (t->zc_cap >= C) return true;
    if (t->d_zc_flags) cudaFree(t->d_zc_flags);
    t->d_zc_flags = nullptr;
    t->zc_cap = 0;
    if (cudaMalloc((void**)&t->d_zc_flags, C) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    t->zc_cap = C;
    return true;
}

}  // namespace

extern "C" {

const char* capt_last_error(void) { return g_err.c_str(); }

int capt_build_threads(const float* points, size_t n, float r_min, float r_max, int n_threads, capt_tree** out) {
    if (!out) return fail(CAPT_E_ARG, "out is NULL");
    *out = nullptr;
    capt_tree* t = nullptr;
    try {
        t = new capt_tree();
    } catch (...) {
        return fail(CAPT_E_NOMEM, "host allocation failed");
    }
    std::string err;
    int rc = capt::build_host_tree(points, n, r_min, r_max, n_threads, t->h, err);
    if (rc != CAPT_OK) {
        delete t;
        return fail(rc, err);
    }
    *out = t;
    return CAPT_OK;
}

int capt_build(const float* points, size_t n, float r_min, float r_max, capt_tree** out) {
    return capt_build_threads(points, n, r_min, r_max, 0, out);
}

namespace {

// Fill the host form of a tree built on the device from its device arrays.
int materialize_host(capt_tree* t) {
    if (!t->host_pending) return CAPT_OK;
    DeviceGuard g(t->device);
    auto& h = t->h;
    try {
        h.pts.resize(3 * h.n);
        h.T.resize(h.N > 1 ? h.N - 1 : 0);
        h.set_begin.resize(h.N + 1);
        h.pruned.resize(h.N);
        h.aabb.resize(6 * h.N);
        std::vector<capt::LeafRec> rec(h.N);
        CUDA_TRY(cudaMemcpy(h.set_begin.data(), t->d_set_begin, (h.N + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost),
                 "set offsets to host");
        h.set_idx.resize(h.set_begin[h.N]);
        if (!h.pts.empty())
            CUDA_TRY(cudaMemcpy(h.pts.data(), t->d_cloud, h.pts.size() * sizeof(float), cudaMemcpyDeviceToHost),
                     "points to host");
        if (!h.T.empty())
            CUDA_TRY(cudaMemcpy(h.T.data(), t->d_Tplain, h.T.size() * sizeof(float), cudaMemcpyDeviceToHost),
                     "splits to host");
        if (!h.set_idx.empty())
            CUDA_TRY(cudaMemcpy(h.set_idx.data(), t->d_set_idx, h.set_idx.size() * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost),
                     "sets to host");
        CUDA_TRY(cudaMemcpy(h.pruned.data(), t->d_pruned, h.N, cudaMemcpyDeviceToHost), "prune flags to host");
        CUDA_TRY(cudaMemcpy(rec.data(), t->d_leaves, h.N * sizeof(capt::LeafRec), cudaMemcpyDeviceToHost),
                 "leaf records to host");
        for (size_t l = 0; l < h.N; l++)
            for (int d = 0; d < 3; d++) {
                h.aabb[6 * l + d] = rec[l].lo[d];
                h.aabb[6 * l + 3 + d] = rec[l].hi[d];
            }
    } catch (const std::bad_alloc&) {
        return fail(CAPT_E_NOMEM, "host allocation failed while copying the tree to the host");
    }
    t->host_pending = false;
    return CAPT_OK;
}

}  // namespace

int capt_build_device(const float* d_points, size_t n, float r_min, float r_max, void* stream, capt_tree** out) {
    if (!out) return fail(CAPT_E_ARG, "out is NULL");
    *out = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    capt_tree* t = nullptr;
    try {
        t = new capt_tree();
    } catch (...) {
        return fail(CAPT_E_NOMEM, "host allocation failed");
    }
    capt::DeviceTree d;
    std::string err;
    int rc = capt::device_build(d_points, n, r_min, r_max, static_cast<cudaStream_t>(stream), d, err);
    if (rc != CAPT_OK) {
        delete t;
        return fail(rc, err);
    }
    int* status = nullptr;
    void* cbox = nullptr;
    const size_t sz_cbox = capt::chunk_count(d.total_blocks) * 8 * sizeof(float);
    cudaError_t e = cudaMalloc((void**)&status, kStatusBytes);
    if (e == cudaSuccess) e = cudaMemset(status, 0, kStatusBytes);
    if (e == cudaSuccess) e = cudaMalloc(&cbox, sz_cbox);
    if (e == cudaSuccess) {
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (capt::launch_chunk_boxes(d.blocks, d.total_blocks, static_cast<float*>(cbox), st, err) != CAPT_OK)
            e = cudaErrorLaunchFailure;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (status) cudaFree(status);
        if (cbox) cudaFree(cbox);
        d.release();
        delete t;
        return cuda_fail(e, "status word and chunk boxes");
    }
    auto& h = t->h;
    h.n = n;
    h.N = d.N;
    h.L = d.L;
    h.r_min = r_min;
    h.r_max = r_max;
    h.build_threads = 0;
    t->device = dev;
    t->d_T = d.Tb;
    t->d_leaves = d.leaves;
    t->d_blocks = d.blocks;
    t->d_ids = d.ids;
    t->d_cloud = d.cloud;
    t->d_cbox = cbox;
    t->d_status = status;
    t->d_ctr = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(status) + 256);
    t->d_Tplain = d.Tplain;
    t->d_set_idx = d.set_idx;
    t->d_set_begin = d.set_begin;
    t->d_pruned = d.pruned;
    t->total_blocks = d.total_blocks;
    t->tail_off = d.bs.tail_off;
    t->K = d.bs.K;
    t->R = d.bs.R;
    t->Ks = d.bs.Ks;
    t->tail_staged = d.bs.tail_staged;
    t->stage_floats = d.bs.stage_floats;
    for (int k = 0; k < 3; k++) {
        t->box_lo[k] = d.box_lo[k];
        t->box_hi[k] = d.box_hi[k];
    }
    t->dev_bytes = d.bytes + sz_cbox + kStatusBytes;
    t->host_pending = true;

    h.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = t;
    return CAPT_OK;
}

int capt_build_frame_device(const float* d_points, size_t n, float r_filter, float r_min, float r_max,
                            uint32_t* d_kept, size_t* n_kept, void* stream, capt_tree** out) {
    if (!out || !n_kept) return fail(CAPT_E_ARG, "NULL argument");
    *out = nullptr;
    *n_kept = 0;
    if (n && !d_points) return fail(CAPT_E_ARG, "points is NULL");
    if (!(r_min >= 0.f) || !(r_max >= r_min) || !std::isfinite(r_max)) return fail(CAPT_E_RANGE, "need 0 <= r_min <= r_max < inf");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::string err;
    uint32_t* kept = d_kept;
    float* pts = nullptr;
    int rc = CAPT_OK;
    if (n && !kept && cudaMalloc((void**)&kept, n * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(CAPT_E_NOMEM, "cudaMalloc of the kept indices failed");
    }
    size_t m = 0;
    rc = capt::device_sfc_filter(d_points, n, r_filter, kept, &m, st, err);
    if (!rc && m && cudaMalloc((void**)&pts, m * 3 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        rc = CAPT_E_NOMEM;
        err = "cudaMalloc of the filtered points failed";
    }
    if (!rc) rc = capt::launch_gather_points(d_points, kept, m, pts, st, err);
    if (!rc) {
        rc = capt_build_device(pts, m, r_min, r_max, stream, out);   // synchronises the stream
        if (rc) err = g_err;
    }
    if (pts) cudaFree(pts);
    if (kept != d_kept && kept) cudaFree(kept);
    if (rc) return fail(rc, err);
    *n_kept = m;
    return CAPT_OK;
}

int sfc_filter(const float* points, size_t n, float min_spacing, uint32_t* kept_idx, size_t* n_out) {
    std::string err;
    int rc = capt::host_sfc_filter(points, n, min_spacing, kept_idx, n_out, err);
    return rc == CAPT_OK ? rc : fail(rc, err);
}

int capt_morton_order(const float* points, size_t n, uint32_t* order) {
    std::string err;
    int rc = capt::host_morton_order(points, n, order, err);
    return rc == CAPT_OK ? rc : fail(rc, err);
}

int sfc_filter_device(const float* d_points, size_t n, float min_spacing, uint32_t* d_kept, size_t* n_out,
                      void* stream) {
    std::string err;
    int rc = capt::device_sfc_filter(d_points, n, min_spacing, d_kept, n_out, static_cast<cudaStream_t>(stream), err);
    return rc == CAPT_OK ? rc : fail(rc, err);
}

int capt_stats(const capt_tree* t, capt_tree_stats* s) {
    if (!t || !s) return fail(CAPT_E_ARG, "NULL argument");
    {
        capt_tree* m = const_cast<capt_tree*>(t);
        std::lock_guard<std::mutex> lk(m->mu);
        const int rc = materialize_host(m);
        if (rc) return rc;
    }
    std::memset(s, 0, sizeof(*s));
    const auto& h = t->h;
    s->n_points = h.n;
    s->n_leaves = h.N;
    s->depth = (uint32_t)h.L;
    s->total_afforded = h.set_idx.size();
    uint64_t blocks = 0, mx = 0, pr = 0, em = 0;
    for (size_t l = 0; l < h.N; l++) {
        uint64_t c = h.set_begin[l + 1] - h.set_begin[l];
        blocks += (c + 3) / 4;
        mx = std::max(mx, c);
        pr += h.pruned[l];
        em += c == 0;
    }
    s->total_blocks = blocks;
    s->max_set = (uint32_t)mx;
    s->pruned_leaves = pr;
    s->empty_leaves = em;
    s->device_bytes = t->dev_bytes;
    s->build_ms = h.build_ms;
    s->r_min = h.r_min;
    s->r_max = h.r_max;
    s->device = t->device;
    s->build_threads = h.build_threads;
    s->compact_chunks = t->cs.n_chunks;
    s->compact_entries = t->cs.list_len;
    s->compact_bytes = t->cs.bytes;
    s->scratch_bytes = (uint64_t)t->edge_scratch_cap * sizeof(uint32_t) +
                       2 * ((uint64_t)t->pipe_cap * sizeof(float) + t->pipe_fbytes) + (uint64_t)t->zc_cap;
    for (int d = 0; d < 3; d++) s->grid_dims[d] = t->gshape.cells ? (uint32_t)t->gshape.n[d] : 0u;
    s->grid_cell = t->gshape.cells ? t->gshape.h : 0.f;
    s->near_entries = t->nl.entries;
    s->near_bytes = t->nl.bytes;
    s->near_fallback_cells = t->nl.fallback_cells;
    s->full_dropped = t->full_dropped ? 1 : 0;
    return CAPT_OK;
}

int capt_export(const capt_tree* t, float* T, uint64_t* set_begin, uint32_t* set_idx, float* aabb) {
    if (!t) return fail(CAPT_E_ARG, "tree is NULL");
    {
        capt_tree* m = const_cast<capt_tree*>(t);
        std::lock_guard<std::mutex> lk(m->mu);
        const int rc = materialize_host(m);
        if (rc) return rc;
    }
    const auto& h = t->h;
    if (T && !h.T.empty()) std::memcpy(T, h.T.data(), h.T.size() * sizeof(float));
    if (set_begin) std::memcpy(set_begin, h.set_begin.data(), h.set_begin.size() * sizeof(uint64_t));
    if (set_idx && !h.set_idx.empty()) std::memcpy(set_idx, h.set_idx.data(), h.set_idx.size() * sizeof(uint32_t));
    if (aabb) std::memcpy(aabb, h.aabb.data(), h.aabb.size() * sizeof(float));
    return CAPT_OK;
}

void capt_free(capt_tree* t) {
    if (!t) return;
    t->free_device();
    delete t;
}

int capt_upload(capt_tree* t, int device, void* stream) {
    if (!t) return fail(CAPT_E_ARG, "tree is NULL");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(CAPT_E_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(t->mu);
    int mrc = materialize_host(t);
    if (mrc) return mrc;
    t->free_device();
    DeviceGuard g(device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    capt::Layout lay;
    try {
        capt::flatten(t->h, lay);
    } catch (const std::bad_alloc&) {
        return fail(CAPT_E_NOMEM, "host allocation failed while flattening");
    }
    const auto& h = t->h;
    capt::BlockedSplits bs;
    try {
        capt::blocked_splits(h, bs);
    } catch (const std::bad_alloc&) {
        return fail(CAPT_E_NOMEM, "host allocation failed while blocking T");
    }
    const size_t sz_T = bs.data.size() * sizeof(float);
    const size_t sz_leaves = lay.leaves.size() * sizeof(capt::LeafRec);
    const size_t sz_blocks = lay.blocks.size() * sizeof(float);
    const size_t sz_ids = lay.ids.size() * sizeof(uint32_t);
    const size_t sz_cloud = std::max<size_t>(1, h.pts.size()) * sizeof(float);
    t->device = device;   // from here on free_device() releases what was allocated
    auto alloc = [&](void** p, size_t bytes, const char* what) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            t->free_device();
            return fail(e == cudaErrorMemoryAllocation ? CAPT_E_NOMEM : CAPT_E_CUDA,
                        std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
        }
        return CAPT_OK;
    };
    int rc;
    const size_t sz_cbox = capt::chunk_count(lay.total_blocks) * 8 * sizeof(float);
    if ((rc = alloc(&t->d_T, sz_T, "T")) || (rc = alloc(&t->d_leaves, sz_leaves, "leaves")) ||
        (rc = alloc(&t->d_blocks, sz_blocks, "blocks")) || (rc = alloc(&t->d_ids, sz_ids, "ids")) ||
        (rc = alloc(&t->d_cloud, sz_cloud, "cloud")) || (rc = alloc(&t->d_cbox, sz_cbox, "chunk boxes")) ||
        (rc = alloc((void**)&t->d_status, kStatusBytes, "status")))
        return rc;
    t->d_ctr = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(t->d_status) + 256);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_T, bs.data.data(), sz_T, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_leaves, lay.leaves.data(), sz_leaves, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_blocks, lay.blocks.data(), sz_blocks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_ids, lay.ids.data(), sz_ids, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !h.pts.empty())
        e = cudaMemcpyAsync(t->d_cloud, h.pts.data(), h.pts.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_status, 0, kStatusBytes, st);
    if (e == cudaSuccess) {
        std::string cerr;
        if (capt::launch_chunk_boxes(static_cast<const float*>(t->d_blocks), lay.total_blocks,
                                     static_cast<float*>(t->d_cbox), st, cerr) != CAPT_OK)
            e = cudaErrorLaunchFailure;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the staging vectors die here
    if (e != cudaSuccess) {
        t->free_device();
        return cuda_fail(e, "upload");
    }
    t->total_blocks = lay.total_blocks;
    for (int d = 0; d < 3; d++) {
        t->box_lo[d] = INFINITY;
        t->box_hi[d] = -INFINITY;
    }
    for (size_t j = 0; j < h.n; j++)
        for (int d = 0; d < 3; d++) {
            t->box_lo[d] = std::min(t->box_lo[d], h.pts[3 * j + d]);
            t->box_hi[d] = std::max(t->box_hi[d], h.pts[3 * j + d]);
        }
    t->tail_off = bs.tail_off;
    t->K = bs.K;
    t->R = bs.R;
    t->Ks = bs.Ks;
    t->tail_staged = bs.tail_staged;
    t->stage_floats = bs.stage_floats;
    t->dev_bytes = sz_T + sz_leaves + sz_blocks + sz_ids + sz_cloud + sz_cbox + kStatusBytes;
    return CAPT_OK;
}

int capt_build_grid(capt_tree* t, uint64_t max_cells, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (max_cells == 0) max_cells = capt::kGridDefaultCells;
    if (max_cells > (1ull << 28)) return fail(CAPT_E_ARG, "max_cells must be at most 2^28");
    std::lock_guard<std::mutex> lk(t->mu);
    DeviceGuard g(t->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const capt::GridShape gs = capt::grid_shape(t->box_lo, t->box_hi, t->h.r_max, t->h.n, max_cells);
    if (t->nl.cell) {   // the lists belong to the old grid
        CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
        t->dev_bytes -= std::min<size_t>(t->dev_bytes, t->nl.bytes);
        t->nl.release();
    }
    if (t->d_grid) {
        CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
        cudaFree(t->d_grid);
        t->dev_bytes -= std::min<size_t>(t->dev_bytes, 2 * (size_t)t->gshape.cells);
        t->d_grid = nullptr;
        t->gshape = capt::GridShape();
    }
    if (gs.cells == 0) return CAPT_OK;   // no points or r_max = 0: nothing to bound
    const size_t bytes = 2 * (size_t)gs.cells;
    cudaError_t e = cudaMalloc((void**)&t->d_grid, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        t->d_grid = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? CAPT_E_NOMEM : CAPT_E_CUDA, "cudaMalloc of the grid failed");
    }
    std::string err;
    rc = capt::launch_dist_grid(t->args(), gs, t->d_grid, st, err);
    if (rc == CAPT_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { rc = CAPT_E_CUDA; err = std::string("grid: ") + cudaGetErrorString(e); }
    }
    if (rc) {
        cudaFree(t->d_grid);
        t->d_grid = nullptr;
        return fail(rc, err);
    }
    t->gshape = gs;
    t->dev_bytes += bytes;
    return CAPT_OK;
}

int capt_grid_export(const capt_tree* t, capt_grid_info* info, uint8_t* h_cells) {
    if (!t || !info) return fail(CAPT_E_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    const capt::GridShape& g = t->gshape;
    if (!t->d_grid || g.cells == 0) return CAPT_OK;
    for (int d = 0; d < 3; d++) {
        info->origin[d] = g.org[d];
        info->dims[d] = g.n[d];
    }
    info->cell = g.h;
    info->inv_cell = g.inv_h;
    info->unit = g.unit;
    info->cells = g.cells;
    if (h_cells) {
        DeviceGuard dg(t->device);
        CUDA_TRY(cudaMemcpy(h_cells, t->d_grid, 2 * (size_t)g.cells, cudaMemcpyDeviceToHost), "grid D2H");
    }
    return CAPT_OK;
}

int capt_build_near_lists(capt_tree* t, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (t->h.r_min != 0.f) return fail(CAPT_E_STATE, "the nearest-candidate lists need a tree built with r_min = 0");
    if (t->h.n == 0 || !(t->h.r_max > 0.f)) return CAPT_OK;   // no cloud to be near: nothing to list
    if (!t->d_grid || t->gshape.cells == 0)
        return fail(CAPT_E_STATE, "the nearest-candidate lists need the distance-bound grid (capt_build_grid)");
    std::lock_guard<std::mutex> lk(t->mu);
    DeviceGuard g(t->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t->nl.cell) {
        CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
        t->dev_bytes -= std::min<size_t>(t->dev_bytes, t->nl.bytes);
        t->nl.release();
    }
    std::string err;
    capt::DevArgs a = t->args();
    rc = capt::device_near_lists(a, t->h.n, st, t->nl, err);
    if (rc) return fail(rc, err);
    t->dev_bytes += t->nl.bytes;
    return CAPT_OK;
}

int capt_compact(capt_tree* t, int drop_full, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (drop_full != 0 && drop_full != 1) return fail(CAPT_E_ARG, "drop_full must be 0 or 1");
    std::lock_guard<std::mutex> lk(t->mu);
    if (drop_full && *t->n_plans > 0) return fail(CAPT_E_STATE, "edge plans of this tree still use its replicated sets");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::string err;
    t->dev_bytes -= std::min(t->dev_bytes, t->cs.bytes);
    t->cs.release();
    rc = capt::device_compact(t->args(), t->h.n, st, t->cs, err);
    if (rc) return fail(rc, err);
    t->dev_bytes += t->cs.bytes;
    if (drop_full) {
        CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
        for (void* p : {t->d_blocks, t->d_ids, t->d_cbox})
            if (p) cudaFree(p);
        t->d_blocks = t->d_ids = t->d_cbox = nullptr;
        const size_t full = t->total_blocks * 16 * sizeof(float) + capt::chunk_count(t->total_blocks) * 8 * sizeof(float);
        t->dev_bytes = t->dev_bytes > full ? t->dev_bytes - full : 0;
        t->full_dropped = true;
    }
    return CAPT_OK;
}

int capt_query_spheres(const capt_tree* t, const float* d_centers, const float* d_radii, size_t m, uint8_t* d_flags,
                       void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (m == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    if ((rc = check_scan(t, t->cfg[CAPT_KERNEL_SPHERES]))) return rc;
    std::string err;
    rc = with_counter(t, static_cast<cudaStream_t>(stream), [&](unsigned long long* ctr) {
        return capt::launch_query(t->args(), capt::kModeSpheres, d_centers, d_radii, m, 1, d_flags,
                                  t->cfg[CAPT_KERNEL_SPHERES], ctr, static_cast<cudaStream_t>(stream), err);
    });
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_query_configs(const capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                       uint8_t* d_flags, void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (S < 1 || S > CAPT_MAX_SPHERES) return fail(CAPT_E_ARG, "S must be in [1, 64]");
    if (C == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    if ((rc = check_scan(t, t->cfg[CAPT_KERNEL_CONFIGS]))) return rc;
    std::string err;
    rc = with_counter(t, static_cast<cudaStream_t>(stream), [&](unsigned long long* ctr) {
        return capt::launch_query(t->args(), capt::kModeConfigs, d_centers, d_radii, C, S, d_flags,
                                  t->cfg[CAPT_KERNEL_CONFIGS], ctr, static_cast<cudaStream_t>(stream), err);
    });
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_query_configs_host(capt_tree* t, const float* h_centers, const float* h_radii, size_t C, int S,
                            uint8_t* h_flags, void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (S < 1 || S > CAPT_MAX_SPHERES) return fail(CAPT_E_ARG, "S must be in [1, 64]");
    if (C == 0) return CAPT_OK;
    if (!h_centers || !h_radii || !h_flags) return fail(CAPT_E_ARG, "NULL host pointer");
    if ((rc = check_scan(t, t->cfg[CAPT_KERNEL_CONFIGS]))) return rc;
    std::lock_guard<std::mutex> lk(t->mu);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    std::string err;
    // Page-locked host memory is mapped into the device's address space: the kernel then
    // reads every centre once, straight from host memory (over NVLink-C2C on Grace
    // systems), with no staging copy.  Flags go to page-locked host memory the same way,
    // else through a small device buffer.
    const void* dc = mapped_device_pointer(h_centers);
    if (dc) {
        if (!ensure_pipe(t, 1, S)) return fail(CAPT_E_NOMEM, "cudaMalloc of the host-pipeline buffers failed");
        float* d_r = t->d_pipe_c[0];
        CUDA_TRY(cudaMemcpyAsync(d_r, h_radii, (size_t)S * sizeof(float), cudaMemcpyHostToDevice, user), "radii H2D");
        void* df = const_cast<void*>(mapped_device_pointer(h_flags));
        if (df) {
            rc = with_counter(t, user, [&](unsigned long long* ctr) {
                return capt::launch_query(t->args(), capt::kModeConfigs, static_cast<const float*>(dc), d_r, C, S,
                                          static_cast<uint8_t*>(df), t->cfg[CAPT_KERNEL_CONFIGS], ctr, user, err);
            });
            if (rc) return fail(rc, err);
        } else {
            if (!ensure_flags(t, C)) return fail(CAPT_E_NOMEM, "cudaMalloc of the flag buffer failed");
            rc = with_counter(t, user, [&](unsigned long long* ctr) {
                return capt::launch_query(t->args(), capt::kModeConfigs, static_cast<const float*>(dc), d_r, C, S,
                                          t->d_zc_flags, t->cfg[CAPT_KERNEL_CONFIGS], ctr, user, err);
            });
            if (rc) return fail(rc, err);
            CUDA_TRY(cudaMemcpyAsync(h_flags, t->d_zc_flags, C, cudaMemcpyDeviceToHost, user), "flags D2H");
        }
        CUDA_TRY(cudaStreamSynchronize(user), "synchronize");
        return CAPT_OK;
    }
    // chunk: 64 Ki configurations (about 47 MB of centres for S = 60)
    const size_t chunk = std::min<size_t>(C, 65536);
    const size_t cfloats = chunk * (size_t)S * 3;
    if (!ensure_pipe(t, chunk, S)) return fail(CAPT_E_NOMEM, "cudaMalloc of the host-pipeline buffers failed");
    // radii live in the tail of buffer 0's slack (S <= 64 floats)
    float* d_r = t->d_pipe_c[0] + cfloats;
    cudaStream_t cp = t->pipe_stream;
    (void)err;
    // the copies start after the caller's queued work
    CUDA_TRY(cudaEventRecord(t->pipe_ev[2], user), "event record");
    CUDA_TRY(cudaStreamWaitEvent(cp, t->pipe_ev[2], 0), "wait");
    CUDA_TRY(cudaMemcpyAsync(d_r, h_radii, (size_t)S * sizeof(float), cudaMemcpyHostToDevice, cp), "radii H2D");
    const size_t nchunks = (C + chunk - 1) / chunk;
    for (size_t k = 0; k < nchunks; k++) {
        const int b = (int)(k & 1);
        const size_t c0 = k * chunk, cn = std::min(chunk, C - c0);
        if (k >= 2) CUDA_TRY(cudaStreamWaitEvent(cp, t->pipe_ev[b], 0), "wait compute");   // buffer b free again
        CUDA_TRY(cudaMemcpyAsync(t->d_pipe_c[b], h_centers + c0 * (size_t)S * 3, cn * (size_t)S * 3 * sizeof(float),
                                 cudaMemcpyHostToDevice, cp),
                 "centres H2D");
        CUDA_TRY(cudaEventRecord(t->pipe_ev[3], cp), "event record");
        CUDA_TRY(cudaStreamWaitEvent(user, t->pipe_ev[3], 0), "wait copy");
        rc = with_counter(t, user, [&](unsigned long long* ctr) {
            return capt::launch_query(t->args(), capt::kModeConfigs, t->d_pipe_c[b], d_r, cn, S, t->d_pipe_f[b],
                                      t->cfg[CAPT_KERNEL_CONFIGS], ctr, user, err);
        });
        if (rc) return fail(rc, err);
        CUDA_TRY(cudaMemcpyAsync(h_flags + c0, t->d_pipe_f[b], cn, cudaMemcpyDeviceToHost, user), "flags D2H");
        CUDA_TRY(cudaEventRecord(t->pipe_ev[b], user), "event record");
    }
    CUDA_TRY(cudaStreamSynchronize(user), "synchronize");
    return CAPT_OK;
}

int capt_count_config_work(const capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                           uint64_t* d_counts, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (S < 1 || S > CAPT_MAX_SPHERES) return fail(CAPT_E_ARG, "S must be in [1, 64]");
    if (C == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_counts) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_count_configs(t->args(), d_centers, d_radii, C, S, false, t->cfg[CAPT_KERNEL_CONFIGS].grid != 0,
                                    d_counts, static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_count_sphere_work(const capt_tree* t, const float* d_centers, const float* d_radii, size_t m,
                           uint64_t* d_counts, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (m == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_counts) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_count_configs(t->args(), d_centers, d_radii, m, 1, true, t->cfg[CAPT_KERNEL_SPHERES].grid != 0,
                                    d_counts, static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_query_leaves(const capt_tree* t, const float* d_centers, size_t m, uint32_t* d_leaves, void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (m == 0) return CAPT_OK;
    if (!d_centers || !d_leaves) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_leaves(t->args(), d_centers, m, d_leaves, static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_device_status(const capt_tree* t, void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int word = 0;
    CUDA_TRY(cudaMemcpyAsync(&word, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "status D2H");
    CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), st), "status clear");
    CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
    if (word & 1) return fail(CAPT_E_TIMEOUT, "a bounded device wait gave up");
    if (word & 2) return fail(CAPT_E_BOUNDS, "a device-side index or size check failed (e.g. an edge batch over 2^31 work items)");
    return CAPT_OK;
}

int capt_set_launch_cfg(capt_tree* t, int kernel, const capt_launch_cfg* cfg) {
    if (!t || !cfg || kernel < 0 || kernel >= CAPT_N_KERNELS) return fail(CAPT_E_ARG, "bad argument");
    if (!valid_cfg(kernel, *cfg)) return fail(CAPT_E_ARG, "unsupported launch configuration");
    t->cfg[kernel] = *cfg;
    return CAPT_OK;
}

int capt_get_launch_cfg(const capt_tree* t, int kernel, capt_launch_cfg* cfg) {
    if (!t || !cfg || kernel < 0 || kernel >= CAPT_N_KERNELS) return fail(CAPT_E_ARG, "bad argument");
    *cfg = t->cfg[kernel];
    return CAPT_OK;
}

namespace {

// Time each candidate launch configuration of the sphere or configuration kernel on
// these inputs (CUDA events, best of two after one untimed run) and keep the fastest.
int autotune_query(capt_tree* t, int kernel, const std::vector<capt_launch_cfg>& cands, const float* d_centers,
                   const float* d_radii, size_t n, int S, uint8_t* d_flags, cudaStream_t st, capt_launch_cfg* best,
                   float* best_ms) {
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "event");
    CUDA_TRY(cudaEventCreate(&e1), "event");
    float best_t = INFINITY;
    capt_launch_cfg best_c = t->cfg[kernel];
    std::string err;
    const int mode = kernel == CAPT_KERNEL_CONFIGS ? capt::kModeConfigs : capt::kModeSpheres;
    int rc = CAPT_OK;
    for (const capt_launch_cfg& c : cands) {
        float tt = INFINITY;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, st);
            rc = with_counter(t, st, [&](unsigned long long* ctr) {
                return capt::launch_query(t->args(), mode, d_centers, d_radii, n, S, d_flags, c, ctr, st, err);
            });
            cudaEventRecord(e1, st);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = CAPT_E_CUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tt = std::min(tt, ms);
        }
        if (rc) break;
        if (tt < best_t) { best_t = tt; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return fail(rc, err.empty() ? "autotune failed" : err);
    t->cfg[kernel] = best_c;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return CAPT_OK;
}

}  // namespace

int capt_autotune_configs(capt_tree* t, const float* d_centers, const float* d_radii, size_t C, int S,
                          uint8_t* d_flags, void* stream, capt_launch_cfg* best, float* best_ms) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (S < 1 || S > CAPT_MAX_SPHERES || C == 0) return fail(CAPT_E_ARG, "need C > 0 and S in [1, 64]");
    if (!d_centers || !d_radii || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    std::vector<capt_launch_cfg> cands;
    for (int warps : {4, 8, 16})
        for (int spl : {2, 4, 8, 16})
            for (int stage : {CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM})
                for (int mode : scan_modes(t))
                    for (int pf : {0, 1})
                        for (int grid : {0, 1})
                            // the grid path has no staged variant
                            if (!grid || (t->d_grid && stage == CAPT_STAGE_GLOBAL))
                                cands.push_back({warps, spl, stage, mode, pf, grid});
    return autotune_query(t, CAPT_KERNEL_CONFIGS, cands, d_centers, d_radii, C, S, d_flags,
                          static_cast<cudaStream_t>(stream), best, best_ms);
}

int capt_autotune_spheres(capt_tree* t, const float* d_centers, const float* d_radii, size_t m, uint8_t* d_flags,
                          void* stream, capt_launch_cfg* best, float* best_ms) {
    int rc = check_ready(t);
    if (rc) return rc;
    if (m == 0) return fail(CAPT_E_ARG, "need m > 0");
    if (!d_centers || !d_radii || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    std::vector<capt_launch_cfg> cands;
    for (int warps : {4, 8, 16})
        for (int spl : {1, 2, 4, 8})
            for (int stage : {CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM})
                for (int mode : scan_modes(t))
                    for (int grid : {0, 1})
                        if (!grid || t->d_grid) cands.push_back({warps, spl, stage, mode, 0, grid});
    return autotune_query(t, CAPT_KERNEL_SPHERES, cands, d_centers, d_radii, m, 1, d_flags,
                          static_cast<cudaStream_t>(stream), best, best_ms);
}

}  // extern "C"

// Internal accessors for entry points defined in other translation units.
int capt_internal_tree_args(const capt_tree* t, capt::DevArgs* out, int* device) {
    int rc = check_ready(t);
    if (rc) return rc;
    *out = t->args();
    *device = t->device;
    return CAPT_OK;
}

const char* capt_internal_set_error(int code, const char* msg) {
    fail(code, msg ? msg : "");
    return g_err.c_str();
}

// ------------------------------------------------------------------------------------
// Edges and clearance entry points
// ------------------------------------------------------------------------------------
namespace {

int check_arm(const capt_arm* arm) {
    if (!arm) return fail(CAPT_E_ARG, "arm is NULL");
    if (arm->n_joints < 1 || arm->n_joints > CAPT_MAX_JOINTS) return fail(CAPT_E_ARG, "n_joints must be in [1, 16]");
    if (arm->n_spheres < 1 || arm->n_spheres > CAPT_MAX_SPHERES) return fail(CAPT_E_ARG, "n_spheres must be in [1, 64]");
    for (int j = 0; j < arm->n_joints; j++)
        if (arm->axis[j] < 0 || arm->axis[j] > 2) return fail(CAPT_E_ARG, "joint axis must be 0, 1 or 2");
    for (int s = 0; s < arm->n_spheres; s++)
        if (arm->sphere_link[s] < 0 || arm->sphere_link[s] >= arm->n_joints)
            return fail(CAPT_E_ARG, "sphere_link out of range");
    return CAPT_OK;
}

}  // namespace

struct capt_edge_plan {
    capt_tree* tree = nullptr;
    std::shared_ptr<std::atomic<int>> tree_plans;
    int device = -1;
    uint32_t* d_scratch = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    capt_launch_cfg cfg{};
    float tuned_ms = 0.f;
    size_t E = 0;
};

extern "C" {

int capt_validate_edges(capt_tree* t, const capt_arm* arm, const float* d_qa, const float* d_qb,
                        const int32_t* d_nsteps, size_t E, uint8_t* d_valid, int mode, void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if ((rc = check_arm(arm))) return rc;
    if (mode != CAPT_EDGES_PERSISTENT && mode != CAPT_EDGES_PER_EDGE) return fail(CAPT_E_ARG, "unknown mode");
    if (E == 0) return CAPT_OK;
    if (!d_qa || !d_qb || !d_nsteps || !d_valid) return fail(CAPT_E_ARG, "NULL device pointer");
    if (E >= (size_t(1) << 31)) return fail(CAPT_E_ARG, "too many edges");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::string err;
    if (mode == CAPT_EDGES_PER_EDGE) {
        std::vector<int32_t> ns(E);
        CUDA_TRY(cudaMemcpyAsync(ns.data(), d_nsteps, E * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "nsteps D2H");
        CUDA_TRY(cudaStreamSynchronize(st), "synchronize");
        rc = capt::launch_edges_per_edge(t->args(), *arm, d_qa, d_qb, ns.data(), E, d_valid, t->cfg[CAPT_KERNEL_EDGES],
                                         st, err);
        return rc ? fail(rc, err) : CAPT_OK;
    }
    std::lock_guard<std::mutex> lk(t->mu);
    const size_t words = capt::edge_scratch_words(E);
    if (t->edge_scratch_cap < words) {
        if (t->d_edge_scratch) cudaFree(t->d_edge_scratch);
        t->d_edge_scratch = nullptr;
        t->edge_scratch_cap = 0;
        if (cudaMalloc((void**)&t->d_edge_scratch, words * sizeof(uint32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(CAPT_E_NOMEM, "cudaMalloc of the edge scratch failed");
        }
        t->edge_scratch_cap = words;
    }
    rc = capt::launch_edges_persistent(t->args(), *arm, d_qa, d_qb, d_nsteps, E, d_valid, t->d_edge_scratch,
                                       t->cfg[CAPT_KERNEL_EDGES], st, err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_query_joint_configs(const capt_tree* t, const capt_arm* arm, const float* d_q, size_t C, uint8_t* d_flags,
                             void* stream) {
    int rc = check_ready(t);
    if (rc) return rc;
    if ((rc = check_arm(arm))) return rc;
    if (C == 0) return CAPT_OK;
    if (!d_q || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = with_counter(t, static_cast<cudaStream_t>(stream), [&](unsigned long long* ctr) {
        return capt::launch_joint_configs(t->args(), *arm, d_q, C, d_flags, t->cfg[CAPT_KERNEL_JOINTS], ctr,
                                          static_cast<cudaStream_t>(stream), err);
    });
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_autotune_joint_configs(capt_tree* t, const capt_arm* arm, const float* d_q, size_t C, uint8_t* d_flags,
                                void* stream, capt_launch_cfg* best, float* best_ms) {
    int rc = check_ready(t);
    if (rc) return rc;
    if ((rc = check_arm(arm))) return rc;
    if (C == 0) return fail(CAPT_E_ARG, "need C > 0");
    if (!d_q || !d_flags) return fail(CAPT_E_ARG, "NULL device pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "event");
    CUDA_TRY(cudaEventCreate(&e1), "event");
    float best_t = INFINITY;
    capt_launch_cfg best_c = t->cfg[CAPT_KERNEL_JOINTS];
    std::string err;
    for (int warps : {2, 4, 8, 16})
        for (int stage : {CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM})
            for (int grid : {0, 1}) {
            if (grid && !t->d_grid) continue;
            capt_launch_cfg c = {warps, 1, stage, 0, 0, grid};
            float tt = INFINITY;
            for (int rep = 0; rep < 3; rep++) {
                cudaEventRecord(e0, st);
                rc = with_counter(t, st, [&](unsigned long long* ctr) {
                    return capt::launch_joint_configs(t->args(), *arm, d_q, C, d_flags, c, ctr, st, err);
                });
                cudaEventRecord(e1, st);
                if (rc) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { rc = CAPT_E_CUDA; break; }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tt = std::min(tt, ms);
            }
            if (rc) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(rc, err.empty() ? "autotune failed" : err);
            }
            if (tt < best_t) { best_t = tt; best_c = c; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->cfg[CAPT_KERNEL_JOINTS] = best_c;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return CAPT_OK;
}

void capt_edge_plan_free(capt_edge_plan* p) {
    if (!p) return;
    if (p->tree_plans) --*p->tree_plans;
    DeviceGuard g(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_scratch) cudaFree(p->d_scratch);
    delete p;
}

int capt_edge_plan_create(capt_tree* t, const capt_arm* arm, const float* d_qa, const float* d_qb,
                          const int32_t* d_nsteps, size_t E, uint8_t* d_valid, const capt_launch_cfg* cfg,
                          void* stream, capt_edge_plan** out) {
    if (!out) return fail(CAPT_E_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_ready(t);
    if (rc) return rc;
    if ((rc = check_arm(arm))) return rc;
    if (E == 0 || !d_qa || !d_qb || !d_nsteps || !d_valid) return fail(CAPT_E_ARG, "need E > 0 and device buffers");
    if (E >= (size_t(1) << 31)) return fail(CAPT_E_ARG, "too many edges");
    if (cfg && !valid_cfg(CAPT_KERNEL_EDGES, *cfg)) return fail(CAPT_E_ARG, "unsupported launch configuration");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    capt_edge_plan* p = new (std::nothrow) capt_edge_plan();
    if (!p) return fail(CAPT_E_NOMEM, "host allocation failed");
    p->tree = t;
    p->E = E;
    p->device = t->device;
    p->tree_plans = t->n_plans;
    ++*p->tree_plans;
    const size_t words = capt::edge_scratch_words(E);
    if (cudaMalloc((void**)&p->d_scratch, words * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(CAPT_E_NOMEM, "cudaMalloc of the plan scratch failed");
    }
    std::string err;
    const DevArgs a = t->args();
    if (cfg) {
        p->cfg = *cfg;
    } else {
        // autotune: warps per block x spheres per lane x staging x chunk
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = INFINITY;
        capt_launch_cfg bc = t->cfg[CAPT_KERNEL_EDGES];
        for (int warps : {4, 8, 16})
            for (int stage : {CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM})
                for (int chunk : {32, 64, 128})
                    for (int grid : {0, 1}) {
                        if (grid && !t->d_grid) continue;
                        capt_launch_cfg c = {warps, 1, stage, chunk, 0, grid};
                        float tt = INFINITY;
                        for (int rep = 0; rep < 3 && !rc; rep++) {
                            cudaEventRecord(e0, st);
                            rc = capt::launch_edges_persistent(a, *arm, d_qa, d_qb, d_nsteps, E, d_valid, p->d_scratch,
                                                               c, st, err);
                            cudaEventRecord(e1, st);
                            if (!rc && cudaEventSynchronize(e1) != cudaSuccess) { rc = CAPT_E_CUDA; err = "autotune sync"; }
                            float ms = 0;
                            cudaEventElapsedTime(&ms, e0, e1);
                            if (rep > 0) tt = std::min(tt, ms);
                        }
                        if (rc) break;
                        if (tt < best) { best = tt; bc = c; }
                    }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) {
            capt_edge_plan_free(p);
            return fail(rc, err);
        }
        p->cfg = bc;
        p->tuned_ms = best;
    }
    // capture {reset, prefix, persistent kernel} into a graph on a private stream
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = capt::launch_edges_persistent(a, *arm, d_qa, d_qb, d_nsteps, E, d_valid, p->d_scratch, p->cfg, cap, err);
        cudaError_t e2 = cudaStreamEndCapture(cap, &p->graph);
        if (!rc && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && !rc) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess || rc) {
        capt_edge_plan_free(p);
        return rc ? fail(rc, err) : cuda_fail(e, "edge plan capture");
    }
    *out = p;
    return CAPT_OK;
}

int capt_edge_plan_launch(capt_edge_plan* p, void* stream) {
    if (!p || !p->exec) return fail(CAPT_E_ARG, "plan is NULL");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device)
        return fail(CAPT_E_STATE, "current CUDA device differs from the plan's device");
    CUDA_TRY(cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)), "cudaGraphLaunch");
    return CAPT_OK;
}

int capt_edge_plan_work(const capt_edge_plan* p, uint64_t* configs_evaluated) {
    if (!p || !configs_evaluated) return fail(CAPT_E_ARG, "NULL argument");
    DeviceGuard g(p->device);
    unsigned long long v = 0;
    CUDA_TRY(cudaMemcpy(&v, p->d_scratch + capt::edge_eval_word((uint32_t)p->E), sizeof(v), cudaMemcpyDeviceToHost),
             "edge work D2H");
    *configs_evaluated = v;
    return CAPT_OK;
}

int capt_edge_plan_info(const capt_edge_plan* p, capt_launch_cfg* cfg, float* tuned_ms) {
    if (!p) return fail(CAPT_E_ARG, "plan is NULL");
    if (cfg) *cfg = p->cfg;
    if (tuned_ms) *tuned_ms = p->tuned_ms;
    return CAPT_OK;
}

int capt_clearance_fwd(const capt_tree* t, const float* d_centers, const float* d_radii, size_t T, int W, int S,
                       float margin, float* d_cost, float* d_dist, int32_t* d_argmin, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (t->h.r_min != 0.f) return fail(CAPT_E_STATE, "clearance needs a tree built with r_min = 0 (no prune)");
    if (S < 1 || S > CAPT_MAX_SPHERES || W < 1) return fail(CAPT_E_ARG, "need 1 <= S <= 64 and W >= 1");
    if (!std::isfinite(margin)) return fail(CAPT_E_ARG, "margin must be finite");
    if (T == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_cost || !d_dist || !d_argmin) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_clearance_fwd(t->args(), d_centers, d_radii, T, W, S, margin, d_cost, d_dist, d_argmin,
                                    t->cfg[CAPT_KERNEL_CLEARANCE], static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_autotune_clearance(capt_tree* t, const float* d_centers, const float* d_radii, size_t T, int W, int S,
                            float margin, float* d_cost, float* d_dist, int32_t* d_argmin, void* stream,
                            capt_launch_cfg* best, float* best_ms) {
    int rc = check_full(t);
    if (rc) return rc;
    if (t->h.r_min != 0.f) return fail(CAPT_E_STATE, "clearance needs a tree built with r_min = 0 (no prune)");
    if (S < 1 || S > CAPT_MAX_SPHERES || W < 1) return fail(CAPT_E_ARG, "need 1 <= S <= 64 and W >= 1");
    if (!std::isfinite(margin)) return fail(CAPT_E_ARG, "margin must be finite");
    if (T == 0) return fail(CAPT_E_ARG, "need T > 0");
    if (!d_centers || !d_radii || !d_cost || !d_dist || !d_argmin) return fail(CAPT_E_ARG, "NULL device pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "event");
    CUDA_TRY(cudaEventCreate(&e1), "event");
    float best_t = INFINITY;
    capt_launch_cfg best_c = t->cfg[CAPT_KERNEL_CLEARANCE];
    std::string err;
    for (int warps : {4, 8, 16})
        for (int stage : {CAPT_STAGE_GLOBAL, CAPT_STAGE_SMEM})
            for (int pf : {0, 1})
                for (int grid : {0, 1}) {
                    if (grid && !t->nl.cell) continue;
                    const capt_launch_cfg c = {warps, 2, stage, 0, pf, grid};
                    float tt = INFINITY;
                    for (int rep = 0; rep < 3; rep++) {
                        cudaEventRecord(e0, st);
                        rc = capt::launch_clearance_fwd(t->args(), d_centers, d_radii, T, W, S, margin, d_cost, d_dist,
                                                        d_argmin, c, st, err);
                        cudaEventRecord(e1, st);
                        if (rc) break;
                        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = CAPT_E_CUDA; break; }
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (rep > 0) tt = std::min(tt, ms);
                    }
                    if (rc) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return fail(rc, err.empty() ? "autotune failed" : err);
                    }
                    if (tt < best_t) { best_t = tt; best_c = c; }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t->cfg[CAPT_KERNEL_CLEARANCE] = best_c;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return CAPT_OK;
}

int capt_count_clearance_work(const capt_tree* t, const float* d_centers, size_t m, uint64_t* d_counts,
                              void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (t->h.r_min != 0.f) return fail(CAPT_E_STATE, "clearance needs a tree built with r_min = 0 (no prune)");
    if (m == 0) return CAPT_OK;
    if (!d_centers || !d_counts) return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_count_clearance(t->args(), d_centers, m, t->cfg[CAPT_KERNEL_CLEARANCE].grid != 0, d_counts,
                                      static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

int capt_clearance_bwd(const capt_tree* t, const float* d_centers, const float* d_radii, const float* d_dist,
                       const int32_t* d_argmin, const float* d_grad_cost, size_t T, int W, int S, float margin,
                       float* d_grad_centers, void* stream) {
    int rc = check_full(t);
    if (rc) return rc;
    if (t->h.r_min != 0.f) return fail(CAPT_E_STATE, "clearance needs a tree built with r_min = 0 (no prune)");
    if (S < 1 || S > CAPT_MAX_SPHERES || W < 1) return fail(CAPT_E_ARG, "need 1 <= S <= 64 and W >= 1");
    if (T == 0) return CAPT_OK;
    if (!d_centers || !d_radii || !d_dist || !d_argmin || !d_grad_cost || !d_grad_centers)
        return fail(CAPT_E_ARG, "NULL device pointer");
    std::string err;
    rc = capt::launch_clearance_bwd(t->args(), d_centers, d_radii, d_dist, d_argmin, d_grad_cost, T, W, S, margin,
                                    d_grad_centers, static_cast<cudaStream_t>(stream), err);
    return rc ? fail(rc, err) : CAPT_OK;
}

}  // extern "C"
