// fmx_step_static: the staged step for callers that cannot allocate device
// memory.  Its workspace is a file-scope device array of fixed size that
// every GPU loading the library holds until the process exits.  The paper
// has no counterpart; see include/fmx.h for the contract.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "fmx.h"
#include "fmx_internal.h"

namespace fmx {
size_t staged_workspace_bytes(const fmx_params *p);
fmx_status staged_steps_on(const fmx_params *p, void *const E[3], void *const B[3], const void *const J[3],
                           void *work, size_t work_bytes, int nsteps);
void set_last_error(const char *msg);
}  // namespace fmx

namespace {

// The shared scratch.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[FMX_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, resolved once per
// device (with that device current) and cached.
fmx_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        fmx::set_last_error("fmx_step_static: cudaGetDevice failed");
        return FMX_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        fmx::set_last_error("fmx_step_static: device ordinal out of range");
        return FMX_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            char msg[200];
            snprintf(msg, sizeof(msg), "fmx_step_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            fmx::set_last_error(msg);
            return FMX_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FMX_OK;
}

}  // namespace

extern "C" fmx_status fmx_step_static(const fmx_params *p, void *const *E, void *const *B, const void *const *J,
                                      int nsteps) {
    if (!p || !E || !B) {
        fmx::set_last_error("fmx_step_static: NULL argument");
        return FMX_EINVAL;
    }
    const size_t need = fmx::staged_workspace_bytes(p);
    if (need == 0) return fmx::staged_steps_on(p, E, B, J, nullptr, 0, nsteps);  // reports the invalid parameter
    if (need > (size_t)FMX_STATIC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "fmx_step_static: this grid needs %zu bytes of scratch, the static scratch holds %zu; "
                 "use fmx_create/fmx_bind with a caller-allocated workspace instead",
                 need, (size_t)FMX_STATIC_SCRATCH_BYTES);
        fmx::set_last_error(msg);
        return FMX_EINVAL;
    }
    void *scratch = nullptr;
    fmx_status s = scratch_address(&scratch);
    if (s != FMX_OK) return s;
    // The scratch belongs to the current device: the fields must live there too.
    int dev = -1;
    cudaPointerAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, E[0]) != cudaSuccess) {
        cudaGetLastError();
        fmx::set_last_error("fmx_step_static: E[0] is not a pointer the CUDA runtime knows");
        return FMX_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        fmx::set_last_error("fmx_step_static: E[0] is not device memory");
        return FMX_EINVAL;
    }
    if (a.device != dev) {
        char msg[160];
        snprintf(msg, sizeof(msg), "fmx_step_static: the fields are on device %d but device %d is current", a.device,
                 dev);
        fmx::set_last_error(msg);
        return FMX_EINVAL;
    }
    return fmx::staged_steps_on(p, E, B, J, scratch, FMX_STATIC_SCRATCH_BYTES, nsteps);
}
