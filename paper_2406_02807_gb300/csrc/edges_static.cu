// Edge validation without any device allocation.
//
// capt_validate_edges (persistent mode) keeps its work-item scratch in a buffer the
// tree allocates on first use; capt_edge_plan_create allocates one per plan.  Some
// callers cannot let the library allocate: a planner inside a real-time control loop
// must not enter the CUDA allocator (cudaMalloc and cudaFree can synchronise the device
// and take unbounded time), and a host application whose device memory is owned by
// another allocator (a caching allocator, a fixed arena) cannot have raw allocations
// appear behind its back.  capt_validate_edges_static serves them: its scratch is a
// fixed array in the library's own device memory, reserved when the library's device
// code is loaded into a device's context (with CUDA's lazy module loading, at the first
// call that needs it, at the latest this entry point's first call on that device) and
// held until the context ends.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/capt.h"
#include "capt_internal.h"
#include "kernels.h"

namespace {

constexpr int kMaxDevices = 64;

// The shared scratch: (E + 1) work-item offsets, the work counter and slack, for at most
// CAPT_STATIC_MAX_EDGES edges (about 256 KB on every device that loads the library).
static __device__ __align__(256) uint32_t g_edge_scratch[CAPT_STATIC_MAX_EDGES + 64];

std::mutex g_mu;
// Per device: the array's device address and the unique ID of the context it belongs
// to.  A reset of the device (cudaDeviceReset) ends that context and the next runtime
// call creates a new one with a new ID, in which the array has a new address; the ID
// tells the two apart, so a stale address is never used.
uint32_t* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

thread_local std::string g_static_err;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The two driver calls that identify the current context, found through the runtime
// (no link-time dependency on the driver library).
bool ctx_fns(CtxGetCurrentFn* cur, CtxGetIdFn* id) {
    static CtxGetCurrentFn s_cur = nullptr;
    static CtxGetIdFn s_id = nullptr;
    static bool s_done = false;
    if (!s_done) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            s_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            s_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
        s_done = true;
    }
    *cur = s_cur;
    *id = s_id;
    return s_cur && s_id;
}

// ID of the context current on this thread, or 0 when none is bound yet.
unsigned long long current_ctx_id(CtxGetCurrentFn cur, CtxGetIdFn id) {
    CUcontext c = nullptr;
    unsigned long long v = 0;
    if (cur(&c) != CUDA_SUCCESS || !c) return 0;
    if (id(c, &v) != CUDA_SUCCESS) return 0;
    return v;
}

// Device address of g_edge_scratch on the current device.  In host code the name of a
// __device__ array is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with that device current, once per device and context (the
// set-up), and cached.
int scratch_for_current_device(uint32_t** out, int* dev_out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_static_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return CAPT_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_static_err = "device ordinal beyond the library's static table";
        return CAPT_E_STATE;
    }
    std::lock_guard<std::mutex> g(g_mu);
    CtxGetCurrentFn cur;
    CtxGetIdFn idf;
    if (!ctx_fns(&cur, &idf)) {
        g_static_err = "the driver does not provide cuCtxGetCurrent / cuCtxGetId";
        return CAPT_E_CUDA;
    }
    const unsigned long long ctx = current_ctx_id(cur, idf);
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_edge_scratch);   // binds the device's context if needed
        if (e != cudaSuccess || !p) {
            g_static_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return CAPT_E_CUDA;
        }
        const unsigned long long now = current_ctx_id(cur, idf);
        if (now == 0) {
            g_static_err = "no CUDA context is current after cudaGetSymbolAddress";
            return CAPT_E_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
        g_scratch_ctx[dev] = now;
    }
    *out = g_scratch_addr[dev];
    *dev_out = dev;
    return CAPT_OK;
}

}  // namespace

// Reaches the tree's device view through the same accessor the other entry points use.
int capt_internal_tree_args(const capt_tree* t, capt::DevArgs* out, int* device);
const char* capt_internal_set_error(int code, const char* msg);

extern "C" int capt_validate_edges_static(const capt_tree* t, const capt_arm* arm, const float* d_qa,
                                          const float* d_qb, const int32_t* d_nsteps, size_t E, uint8_t* d_valid,
                                          void* stream) {
    capt::DevArgs a;
    int tree_dev = -1;
    int rc = capt_internal_tree_args(t, &a, &tree_dev);
    if (rc) return rc;
    if (!arm || arm->n_joints < 1 || arm->n_joints > CAPT_MAX_JOINTS || arm->n_spheres < 1 ||
        arm->n_spheres > CAPT_MAX_SPHERES) {
        capt_internal_set_error(CAPT_E_ARG, "arm is NULL or has an unsupported joint or sphere count");
        return CAPT_E_ARG;
    }
    for (int j = 0; j < arm->n_joints; j++)
        if (arm->axis[j] < 0 || arm->axis[j] > 2) {
            capt_internal_set_error(CAPT_E_ARG, "joint axis must be 0, 1 or 2");
            return CAPT_E_ARG;
        }
    for (int s = 0; s < arm->n_spheres; s++)
        if (arm->sphere_link[s] < 0 || arm->sphere_link[s] >= arm->n_joints) {
            capt_internal_set_error(CAPT_E_ARG, "sphere_link out of range");
            return CAPT_E_ARG;
        }
    if (E > (size_t)CAPT_STATIC_MAX_EDGES) {
        capt_internal_set_error(CAPT_E_ARG, "capt_validate_edges_static takes at most CAPT_STATIC_MAX_EDGES "
                                            "(65536) edges per call");
        return CAPT_E_ARG;
    }
    if (E == 0) return CAPT_OK;
    if (!d_qa || !d_qb || !d_nsteps || !d_valid) {
        capt_internal_set_error(CAPT_E_ARG, "NULL device pointer");
        return CAPT_E_ARG;
    }
    uint32_t* scratch = nullptr;
    int dev = -1;
    rc = scratch_for_current_device(&scratch, &dev);
    if (rc) {
        capt_internal_set_error(rc, g_static_err.c_str());
        return rc;
    }
    if (dev != tree_dev) {
        capt_internal_set_error(CAPT_E_STATE, "current CUDA device differs from the tree's device");
        return CAPT_E_STATE;
    }
    capt_launch_cfg cfg;
    capt_get_launch_cfg(t, CAPT_KERNEL_EDGES, &cfg);
    std::string err;
    rc = capt::launch_edges_persistent(a, *arm, d_qa, d_qb, d_nsteps, E, d_valid, scratch, cfg,
                                       static_cast<cudaStream_t>(stream), err);
    if (rc) capt_internal_set_error(rc, err.c_str());
    return rc;
}
