// vp_noalloc.cu -- vp_apply_noalloc: the potential apply for callers that may
// not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they apply the
// operator: code that runs inside another framework whose allocator owns the
// device memory and forbids raw allocations, real-time or latency-bound loops
// where an allocation's implicit synchronisation is not acceptable, or
// plug-ins that may only allocate during their initialisation.  They create
// the plan at set-up (that allocates the precomputed multiplier) and then call
// this entry point, which takes its scratch from a fixed array compiled into
// the library instead of the plan's lazily allocated workspace.
//
// The scratch is a file-scope __device__ array of VP_NOALLOC_SCRATCH_BYTES.
// In host code the array's name is only a host-side stand-in for the symbol;
// the device address is looked up with cudaGetSymbolAddress once per device,
// the first time this entry point runs on that device, with the plan's device
// current.  That first call should therefore come before any stream capture.
// Under lazy module loading (CUDA's default) the lookup also loads this
// file's module, i.e. allocates the array on that device; it then stays until
// the process exits.  The cached address is per process and per device: a
// cudaDeviceReset between calls would leave it stale.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/vp.h"
#include "vp_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)VP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" vp_status vp_apply_noalloc(vp_plan plan, const void* f, void* phi, vp_dtype dtype) {
  if (!plan) return VP_ERR_INVALID_ARG;
  const int dev = vp::plan_device(plan);
  if (dev < 0 || dev >= kMaxDevices) return VP_ERR_UNSUPPORTED;
  vp::DeviceGuard dg_(dev);
  if (dg_.error() != cudaSuccess) return VP_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return VP_ERR_CUDA;
      g_scratch_addr[dev] = ptr;
    }
    scratch = g_scratch_addr[dev];
  }
  return vp::apply_with_workspace(plan, f, phi, dtype, scratch, kScratchBytes);
}
