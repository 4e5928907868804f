// Arithmetic peak of the current GPU, measured: independent fused multiply-add
// chains (eight per thread, four blocks of 256 threads per SM), timed with CUDA
// events.  The FP64 rate is the denominator of the FP64 kernels' roofline
// fraction (the chip's FP64 pipe is far narrower than its FP32 one).
#include "semmg_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.2345e30) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

}  // namespace

extern "C" int semmg_peak_tflops(int dtype, double* tflops, void* stream) {
  if (!tflops || (dtype != SEMMG_F64 && dtype != SEMMG_F32)) return SEMMG_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  const int grid = 4 * nsm, block = 256;
  // about 10 ms at the expected rates (FP64 ~1.2, FP32 ~70 TFLOP/s)
  const int iters = dtype == SEMMG_F64 ? 4096 : 262144;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up; the second is timed
    cudaEventRecord(e0, st);
    if (dtype == SEMMG_F64)
      k_fma_chains<double><<<grid, block, 0, st>>>(nullptr, iters, 0.999999, 1e-7);
    else
      k_fma_chains<float><<<grid, block, 0, st>>>(nullptr, iters, 0.9999f, 1e-7f);
    cudaEventRecord(e1, st);
  }
  const cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || !(ms > 0.f)) return SEMMG_ERR_CUDA;
  const double flops = 2.0 * 8.0 * iters * (double)grid * block;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SEMMG_OK;
}
