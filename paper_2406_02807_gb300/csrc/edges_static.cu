// Edge validation without any device allocation.
//
// capt_validate_edges (persistent mode) keeps its work-item scratch in a buffer the
// tree allocates on first use; capt_edge_plan_create allocates one per plan.  Some
// callers cannot let the library allocate: a planner inside a real-time control loop
// must not enter the CUDA allocator (cudaMalloc and cudaFree can synchronise the device
// and take unbounded time), and a host application whose device memory is owned by
// another allocator (a caching allocator, a fixed arena) cannot have raw allocations
// appear behind its back.  capt_validate_edges_static serves them: its scratch is a
// fixed array in the library's own device memory, reserved when the library is loaded
// on a device and held until the process exits.
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
uint32_t* g_scratch_addr[kMaxDevices] = {};

thread_local std::string g_static_err;

// Device address of g_edge_scratch on the current device.  In host code the name of a
// __device__ array is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
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
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_edge_scratch);
        if (e != cudaSuccess || !p) {
            g_static_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return CAPT_E_CUDA;
        }
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
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
