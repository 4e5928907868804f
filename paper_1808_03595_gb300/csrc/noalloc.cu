// semmg_smooth_noalloc: star smoothing whose scratch is a fixed array compiled
// into the library, for callers that must not allocate device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds its SEMMG_NOALLOC_SCRATCH_BYTES until the process exits.  In
// host code the name g_smooth_scratch is only a host-side stand-in for that
// variable, never a device address: the device address is looked up with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// with that device current, and cached.
#include <mutex>

#include "semmg_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_smooth_scratch[SEMMG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int semmg_smooth_noalloc(semmg_ctx* ctx, int level, int dtype, const void* r_hat, void* du_hat,
                                    void* stream) {
  if (!ctx) return SEMMG_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_smooth_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return SEMMG_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return semmg::smooth_with_scratch(ctx, level, dtype, r_hat, du_hat, scratch, SEMMG_NOALLOC_SCRATCH_BYTES,
                                    (cudaStream_t)stream);
}
