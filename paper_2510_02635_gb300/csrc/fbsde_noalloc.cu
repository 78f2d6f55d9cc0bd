// fbsde_noalloc.cu -- fbsde_solve_noalloc(): the solve for callers that cannot allocate
// device memory.  Its workspace is a file-scope device array of fixed size that lives
// in the library's own module, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fbsde.h"
#include "fbsde_internal.cuh"

namespace {

// The scratch workspace.  Every GPU that loads this library reserves these bytes for
// the lifetime of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FBSDE_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.  The cache is not refreshed: after a
// cudaDeviceReset the module is loaded again and the array may move, so this entry point
// is not supported on a device after it has been reset.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FBSDE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FBSDE_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return FBSDE_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FBSDE_OK;
}

}  // namespace

extern "C" int fbsde_solve_noalloc(const fbsde_problem *P, int32_t Q, const double *x0,
                                   uint64_t seed, uint32_t solve_index0, double *u0,
                                   double *grad_u0, fbsde_stream_t stream)
{
    const size_t need = fbsde_workspace_bytes(P, Q);
    if (need == 0) return FBSDE_ERR_ARG;
    if (need > (size_t)FBSDE_NOALLOC_MAX_BYTES) return FBSDE_ERR_WORKSPACE;
    void *scratch = nullptr;
    const int st = scratch_address(&scratch);
    if (st != FBSDE_OK) return st;
    // every CG pass is launched on the stream: the cached CUDA graphs of fbsde_solve would
    // create streams and instantiate graphs, which may allocate
    return fbsde::solve_launches_only(P, Q, x0, seed, solve_index0, u0, grad_u0, scratch,
                                      (size_t)FBSDE_NOALLOC_MAX_BYTES,
                                      reinterpret_cast<cudaStream_t>(stream));
}
