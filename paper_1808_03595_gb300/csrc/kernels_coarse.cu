// Exact coarse solve at degree p0 (Sec. 4.1 coarse-grid solver), FP64.
//
// The full degree-p0 system on the tensor-product mesh is a Kronecker sum of
// assembled 1D matrices, so it is inverted by global fast diagonalisation
// (eq. fast_diagonalization on the whole domain):
//   H^{-1} = (S3(x)S2(x)S1) (lam + Lam1 + Lam2 + Lam3)^{-1} (S3(x)S2(x)S1)^T
// with S_d^T Mg_d S_d = I, S_d^T Lg_d S_d = Lam_d on the K_d grid points of
// axis d that are unknowns (all but the points on a Dirichlet face).  The condensed right-hand side is embedded
// with zeros at the element-interior nodes; by the embedding argument of
// Sec. 3.1 the skeleton part of the full solution is the condensed solution.
// At p0 = 1 there are no interior nodes and this is the condensed system itself.
#include "semmg_internal.h"

namespace semmg {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

__global__ void k_coarse_embed(Geo G, CoarseTabs ct, const double* __restrict__ F0, double* __restrict__ X) {
  const int K1 = ct.K[0], K2 = ct.K[1], K3 = ct.K[2];
  const int64_t n = (int64_t)K1 * K2 * K3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % K1), k2 = (int)((i / K1) % K2), k3 = (int)(i / ((int64_t)K1 * K2));
    const int64_t s = skel_index(G, k1 + ct.g0[0], k2 + ct.g0[1], k3 + ct.g0[2]);
    X[i] = s >= 0 ? F0[s] : 0.0;
  }
}

// One 1D transform along `axis` of the K1 x K2 x K3 array; forward: out[k] =
// sum_j S[j][k] in[j]; backward: out[j] = sum_k S[j][k] in[k].  With `divide`
// the result is divided by lam + Lam1 + Lam2 + Lam3.
__global__ void k_coarse_tx(CoarseTabs ct, double lam, int axis, int backward, int divide,
                            const double* __restrict__ X, double* __restrict__ Y) {
  const int K1 = ct.K[0], K2 = ct.K[1], K3 = ct.K[2];
  const int64_t n = (int64_t)K1 * K2 * K3;
  const int Ka = ct.K[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? K1 : (int64_t)K1 * K2);
  const double* S = ct.S[axis];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % K1), k2 = (int)((i / K1) % K2), k3 = (int)(i / ((int64_t)K1 * K2));
    const int ko = axis == 0 ? k1 : (axis == 1 ? k2 : k3);
    const double* x = X + (i - ko * stride);
    double s = 0;
    if (!backward)
      for (int j = 0; j < Ka; ++j) s += S[j * Ka + ko] * x[j * stride];
    else
      for (int k = 0; k < Ka; ++k) s += S[ko * Ka + k] * x[k * stride];
    if (divide) s /= lam + ct.lam[0][k1] + ct.lam[1][k2] + ct.lam[2][k3];
    Y[i] = s;
  }
}

__global__ void k_coarse_extract(Geo G, CoarseTabs ct, const double* __restrict__ X, double* __restrict__ U0) {
  const int K1 = ct.K[0], K2 = ct.K[1], K3 = ct.K[2];
  const int64_t n = (int64_t)K1 * K2 * K3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k1 = (int)(i % K1), k2 = (int)((i / K1) % K2), k3 = (int)(i / ((int64_t)K1 * K2));
    const int64_t s = skel_index(G, k1 + ct.g0[0], k2 + ct.g0[1], k3 + ct.g0[2]);
    if (s >= 0) U0[s] = X[i];
  }
}

}  // namespace

void launch_coarse_solve(const Geo& G0, const CoarseTabs& ct, const double* F0, double* U0, double* X, double* Y,
                         cudaStream_t st) {
  cudaMemsetAsync(U0, 0, sizeof(double) * G0.size, st);
  const int64_t n = (int64_t)ct.K[0] * ct.K[1] * ct.K[2];
  if (n == 0) return;
  const int gr = grid_for(n);
  k_coarse_embed<<<gr, kThreads, 0, st>>>(G0, ct, F0, X);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 0, 0, 0, X, Y);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 1, 0, 0, Y, X);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 2, 0, 1, X, Y);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 2, 1, 0, Y, X);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 1, 1, 0, X, Y);
  k_coarse_tx<<<gr, kThreads, 0, st>>>(ct, G0.lam, 0, 1, 0, Y, X);
  k_coarse_extract<<<gr, kThreads, 0, st>>>(G0, ct, X, U0);
}

}  // namespace semmg
