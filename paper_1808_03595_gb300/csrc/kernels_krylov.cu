// Algorithm 5 (Krylov-accelerated multigrid, Sec. 4.1): the vector steps of
// the inexact preconditioned CG iteration with the V-cycle as preconditioner.
// The scalars gamma, gamma0, delta, beta, alpha live in device memory and
// are updated by one-block kernels, so an iteration needs no host round trip
// and can be captured in a graph.  Every reduction has a fixed partition
// (npart blocks, fixed block size, fixed tree), so results are reproducible
// run to run.
#include "semmg_internal.h"

namespace semmg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double s = red[0];
  __syncthreads();
  return s;
}

// part[b] = sum z.r, part[npart + b] = sum z.s over block b's grid-strided range
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot2_partial(const T* __restrict__ z, const double* __restrict__ r,
                                                            const double* __restrict__ s, int64_t n,
                                                            double* __restrict__ part) {
  __shared__ double red[kThreads];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)z[i];
    a += zi * r[i];
    b += zi * s[i];
  }
  const double sa = block_sum(a, red);
  const double sb = block_sum(b, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sa;
    part[gridDim.x + blockIdx.x] = sb;
  }
}

// gamma = z.r, gamma0 = z.s, beta = (gamma - gamma0) / delta, delta = gamma
__global__ void __launch_bounds__(kThreads) k_krylov_beta(const double* __restrict__ part, int npart,
                                                           KrylovScal* k) {
  __shared__ double red[kThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) {
    a += part[i];
    b += part[npart + i];
  }
  const double g = block_sum(a, red);
  const double g0 = block_sum(b, red);
  if (threadIdx.x == 0) {
    k->gamma = g;
    k->gamma0 = g0;
    k->beta = (g - g0) / k->delta;
    k->delta = g;
  }
}

// p = beta p + z
template <typename T>
__global__ void __launch_bounds__(kThreads) k_krylov_dir(double* __restrict__ p, const T* __restrict__ z,
                                                          const KrylovScal* __restrict__ k, int64_t n) {
  const double beta = k->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = beta * p[i] + (double)z[i];
}

__global__ void __launch_bounds__(kThreads) k_dot_partial(const double* __restrict__ x, const double* __restrict__ y,
                                                           int64_t n, double* __restrict__ part) {
  __shared__ double red[kThreads];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  const double s = block_sum(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = gamma / (q.p)
__global__ void __launch_bounds__(kThreads) k_krylov_alpha(const double* __restrict__ part, int npart,
                                                            KrylovScal* k) {
  __shared__ double red[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) a += part[i];
  const double qp = block_sum(a, red);
  if (threadIdx.x == 0) {
    k->qp = qp;
    k->alpha = k->gamma / qp;
  }
}

// s = r; u += alpha p; r -= alpha q; part[b] = block sum of r_new^2
__global__ void __launch_bounds__(kThreads) k_krylov_update(double* __restrict__ u, double* __restrict__ r,
                                                             double* __restrict__ s, const double* __restrict__ p,
                                                             const double* __restrict__ q,
                                                             const KrylovScal* __restrict__ k, int64_t n,
                                                             double* __restrict__ part) {
  __shared__ double red[kThreads];
  const double alpha = k->alpha;
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    s[i] = ri;
    u[i] += alpha * p[i];
    const double rn = ri - alpha * q[i];
    r[i] = rn;
    a += rn * rn;
  }
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_krylov_sum(const double* __restrict__ part, int npart, double* __restrict__ out) {
  __shared__ double red[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) a += part[i];
  const double s = block_sum(a, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_krylov_init(KrylovScal* k) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *k = KrylovScal{0.0, 0.0, 1.0, 0.0, 0.0, 0.0};
}

}  // namespace

void launch_krylov_init(KrylovScal* k, cudaStream_t st) { k_krylov_init<<<1, 32, 0, st>>>(k); }

template <typename T>
void launch_krylov_beta_dir(const T* z, const double* r, const double* s, double* p, int64_t n, double* part,
                            int npart, KrylovScal* k, cudaStream_t st) {
  k_dot2_partial<T><<<npart, kThreads, 0, st>>>(z, r, s, n, part);
  k_krylov_beta<<<1, kThreads, 0, st>>>(part, npart, k);
  k_krylov_dir<T><<<npart, kThreads, 0, st>>>(p, z, k, n);
}

void launch_krylov_alpha(const double* q, const double* p, int64_t n, double* part, int npart, KrylovScal* k,
                         cudaStream_t st) {
  k_dot_partial<<<npart, kThreads, 0, st>>>(q, p, n, part);
  k_krylov_alpha<<<1, kThreads, 0, st>>>(part, npart, k);
}

void launch_krylov_update(double* u, double* r, double* s, const double* p, const double* q, int64_t n,
                          double* part, int npart, const KrylovScal* k, double* rnorm2, cudaStream_t st) {
  k_krylov_update<<<npart, kThreads, 0, st>>>(u, r, s, p, q, k, n, part);
  k_krylov_sum<<<1, kThreads, 0, st>>>(part, npart, rnorm2);
}

template void launch_krylov_beta_dir<double>(const double*, const double*, const double*, double*, int64_t, double*,
                                             int, KrylovScal*, cudaStream_t);
template void launch_krylov_beta_dir<float>(const float*, const double*, const double*, double*, int64_t, double*,
                                            int, KrylovScal*, cudaStream_t);

}  // namespace semmg
