// semmg_smooth_noalloc: star smoothing whose scratch is a fixed array compiled
// into the library, for callers that must not allocate device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds its SEMMG_NOALLOC_SCRATCH_BYTES until the process exits.  In
// host code the name g_smooth_scratch is only a host-side stand-in for that
// variable, never a device address: every call looks the device address up
// with cudaGetSymbolAddress (which allocates nothing) for the device current
// at the call, so no address outlives a reset of the device or of its primary
// context.  The first lookup on a device may load the library's device code
// there, which is why the first call on a device should come before any
// stream capture.
#include "semmg_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_smooth_scratch[SEMMG_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int semmg_smooth_noalloc(semmg_ctx* ctx, int level, int dtype, const void* r_hat, void* du_hat,
                                    void* stream) {
  if (!ctx) return SEMMG_ERR_INVALID_ARG;
  void* scratch = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&scratch, g_smooth_scratch);
  if (e != cudaSuccess || !scratch) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  return semmg::smooth_with_scratch(ctx, level, dtype, r_hat, du_hat, scratch, SEMMG_NOALLOC_SCRATCH_BYTES,
                                    (cudaStream_t)stream);
}
