// trsyl_lu_noalloc: the FP64 triangular Sylvester solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA
// graph that is being captured, where an allocation would break the capture;
// plugins and real-time loops that must not allocate after start-up; and
// hosts whose allocator is owned by another framework.  They can still pass
// their own input and output buffers, so this entry point takes everything
// trsyl_lu takes except the workspace, and uses a fixed scratch area in the
// library's own device memory instead.
//
// The scratch is a file-scope device array of kScratchBytes (1 MiB).  Every
// GPU that loads this library holds it until the process exits.  In host code
// the array's name is only a host-side stand-in, not a device address, so the
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device; because of that set-up
// the first call on each device should come before any stream capture.  All
// calls share the one array: calls that overlap on the GPU race on it, so
// they must be ordered (one stream, or events).  The array keeps the last
// call's contents; the solve's pre-pass rewrites every part it reads (queue
// heads, size bins, the sorted order) at the start of each call.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/smallsolve.h"

namespace {

constexpr size_t kScratchBytes = 1u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per
// device), or nullptr if the lookup failed.
void *scratch_address()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return nullptr;
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

}  // namespace

extern "C" int trsyl_lu_noalloc(int batch, int max_n, const int *d_n,
                                const double *const *d_L, const int *d_ldl,
                                const double *const *d_U, const int *d_ldu,
                                const double *const *d_C, const int *d_ldc,
                                double *const *d_X, const int *d_ldx, int *d_info, void *stream)
{
    if (batch < 0) return -1;
    if (max_n < 0 || max_n > SS_MAX_N) return -2;
    size_t need = 0;
    if (ss_workspace_size(SS_OP_TRSYL, batch, max_n, SS_MODE_FP64, &need) != 0) return -1;
    if (need > kScratchBytes) return SS_ERR_SCRATCH_LIMIT;
    if (batch == 0) return 0;
    void *scratch = scratch_address();
    if (scratch == nullptr) return SS_ERR_CUDA;
    return trsyl_lu(batch, max_n, d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info,
                    SS_MODE_FP64, SS_CFG_DEFAULT, scratch, kScratchBytes, stream);
}
