// heff_apply_noalloc: heff_apply for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under another framework's memory
// manager which has already reserved the device memory it may use, or code on a
// latency-critical path where cudaMalloc's implicit device synchronisation is not
// acceptable.  This entry point takes the plan's workspace from a fixed array compiled
// into the library instead of from the caller.  The paper has no counterpart of it.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

using heff::fail;

namespace {

// One copy per GPU that loads the library, held until the process exits.  Every call
// shares it and it keeps the last call's contents; two calls that overlap on the GPU
// (different streams, or different threads on one device) race on it.
static __device__ __align__(256) unsigned char g_noalloc_ws[HEFF_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_ws[kMaxDevices] = {};   // device address of g_noalloc_ws, per device ordinal

// Resolve the array's device address on the current device (once per device).  The host
// symbol g_noalloc_ws is only a stand-in; kernels must be given this address.
int static_workspace(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ws[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
        if (e != cudaSuccess)
            return fail(HEFF_ERR_CUDA, "cudaGetSymbolAddress(static workspace): %s", cudaGetErrorString(e));
        g_ws[dev] = p;
    }
    *out = g_ws[dev];
    return HEFF_OK;
}

}  // namespace

extern "C" int heff_apply_noalloc(heff_plan* plan, const void* L, const void* W1, const void* W2,
                                  const void* R, const void* x, void* y, void* stream) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_apply_noalloc: null plan");
    size_t need = 0;
    heff_plan_workspace_size(plan, &need);
    if (need > (size_t)HEFF_NOALLOC_WORKSPACE_BYTES)
        return fail(HEFF_ERR_WORKSPACE,
                    "heff_apply_noalloc: the plan needs %zu bytes of workspace, the built-in array holds %zu "
                    "(HEFF_NOALLOC_WORKSPACE_BYTES); use heff_apply with a caller-owned workspace",
                    need, (size_t)HEFF_NOALLOC_WORKSPACE_BYTES);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(HEFF_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    if (plan->uploaded && dev != plan->device)
        return fail(HEFF_ERR_INVALID_ARG, "heff_apply_noalloc: plan lives on device %d, current device is %d",
                    plan->device, dev);
    void* ws = nullptr;
    int rc = static_workspace(dev, &ws);
    if (rc) return rc;
    // the device error flag must start at zero; everything else is written before it is read
    e = cudaMemsetAsync(static_cast<char*>(ws) + plan->off_flags, 0, 256,
                        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return heff_apply(plan, L, W1, W2, R, x, y, ws, (size_t)HEFF_NOALLOC_WORKSPACE_BYTES, stream);
}

// Read and clear the error flag of the built-in workspace: an expired bounded wait inside a
// heff_apply_noalloc call leaves it set (heff_apply_noalloc clears it when it starts, so read
// it after each call whose result matters).  No allocation either.
extern "C" int heff_apply_noalloc_status(const heff_plan* plan, void* stream) {
    heff::clear_error();
    if (!plan) return fail(HEFF_ERR_INVALID_ARG, "heff_apply_noalloc_status: null plan");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HEFF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(HEFF_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    void* ws = nullptr;
    int rc = static_workspace(dev, &ws);
    if (rc) return rc;
    return heff_workspace_status(plan, ws, (size_t)HEFF_NOALLOC_WORKSPACE_BYTES, stream);
}
