// Skeleton-parallel kernels: one thread per condensed slot.
//
// On the tensor-product mesh the assembled operator is the Kronecker sum of
// the assembled 1D matrices (Sec. 2.1 and 3.2: "one-dimensional matrices
// assembled from the elements"):
//   H = lam Mg3(x)Mg2(x)Mg1 + Mg3(x)Mg2(x)Lg1 + Mg3(x)Lg2(x)Mg1 + Lg3(x)Mg2(x)Mg1,
// so the skeleton block H_BB of a node is a sum of three 1D line sums over the
// skeleton nodes of the lines through it.  The Schur complement term
// -H_BI H_II^{-1} H_IB arrives per element and face from the element kernel
// (buffer Z[e][f][m^2]) and is added here, two elements per face node.
#include "semmg_internal.h"
#include "skel_ops.cuh"

namespace semmg {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

// Schur-complement contributions of the two elements sharing a face node.
template <typename T>
__device__ __forceinline__ T face_z(const Geo& G, const T* __restrict__ Z, int type, const int* g) {
  const int p = G.p, m = G.m;
  const int64_t mm = (int64_t)m * m;
  int a[3], q[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = divp(G, g[d]);
    q[d] = g[d] - a[d] * p;
  }
  const int d = type;  // face normal axis (ENT_F1..F3 == 0..2)
  const int ia = (d == 0) ? 1 : 0, ib = (d == 2) ? 1 : 2;
  const int64_t loc = (int64_t)(q[ib] - 1) * m + (q[ia] - 1);
  int e[3] = {a[0], a[1], a[2]};
  T z = 0;
  if (a[d] > 0 || G.per[d]) {  // element on the minus side (absent at a low non-periodic face): this face is its side p
    e[d] = wrape(G, d, a[d] - 1);
    const int64_t em = ((int64_t)e[2] * G.n2 + e[1]) * G.n1 + e[0];
    z += Z[(em * 6 + 2 * d + 1) * mm + loc];
  }
  if (a[d] < ncount(G, d)) {  // element on the plus side (absent at the high face): side 0
    e[d] = a[d];
    const int64_t ep = ((int64_t)e[2] * G.n2 + e[1]) * G.n1 + e[0];
    z += Z[(ep * 6 + 2 * d) * mm + loc];
  }
  return z;
}

// mode 0: out = F - Hhat u;  mode 1: out = Hhat u.  Arithmetic in T, F and out
// of type TF (float TF with double T: the mixed form's level residuals).
template <typename T, typename TF = T>
__global__ void __launch_bounds__(kThreads) k_assemble(Geo G, Tabs<T> t, const TF* __restrict__ F,
                                                        const T* __restrict__ u, const T* __restrict__ Z,
                                                        TF* __restrict__ out, int mode) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    const int type = skel_decode(G, s, g, &bd);
    if (bd) {
      out[s] = 0;
      continue;
    }
    T Hu = node_hbb(G, t, u, s, type, g);
    if (type <= ENT_F3 && Z) Hu -= face_z(G, Z, type, g);
    out[s] = (TF)(mode == 0 ? (T)F[s] - Hu : Hu);
  }
}

// Fhat = (M f)_B - H_BI H_II^{-1} F_I
__global__ void __launch_bounds__(kThreads) k_assemble_rhs(Geo G, Tabs<double> t, const double* __restrict__ f,
                                                            const double* __restrict__ Z, double* __restrict__ Fh) {
  const int nd[3] = {G.n1, G.n2, G.n3};
  const int64_t N1 = (int64_t)G.n1 * G.p + 1, N2 = (int64_t)G.n2 * G.p + 1;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    const int type = skel_decode(G, s, g, &bd);
    if (bd) {
      Fh[s] = 0;
      continue;
    }
    double v = mass1d(G, t, 0, g[0], nd[0]) * mass1d(G, t, 1, g[1], nd[1]) * mass1d(G, t, 2, g[2], nd[2]) *
               f[((int64_t)g[2] * N2 + g[1]) * N1 + g[0]];
    if (type <= ENT_F3 && G.m > 0) v -= face_z(G, Z, type, g);
    Fh[s] = v;
  }
}

__global__ void k_pack(Geo G, const double* __restrict__ nodal, double* __restrict__ hat) {
  const int64_t N1 = (int64_t)G.n1 * G.p + 1, N2 = (int64_t)G.n2 * G.p + 1;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    skel_decode(G, s, g, &bd);
    hat[s] = bd ? 0.0 : nodal[((int64_t)g[2] * N2 + g[1]) * N1 + g[0]];
  }
}

// E g: the nodal values on Dirichlet faces in their skeleton slots, 0 elsewhere.
__global__ void k_pack_dirichlet(Geo G, const double* __restrict__ nodal, double* __restrict__ hat) {
  const int64_t N1 = (int64_t)G.n1 * G.p + 1, N2 = (int64_t)G.n2 * G.p + 1;
  const int top[3] = {G.n1 * G.p, G.n2 * G.p, G.n3 * G.p};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    skel_decode(G, s, g, &bd);
    bool on = false;
    for (int d = 0; d < 3; ++d) on |= (g[d] == 0 && G.dir[2 * d]) || (g[d] == top[d] && G.dir[2 * d + 1]);
    hat[s] = on ? nodal[((int64_t)g[2] * N2 + g[1]) * N1 + g[0]] : 0.0;
  }
}

// Every skeleton node of the nodal array; a periodic image takes the value of
// the unknown it repeats (the slot skel_index maps it to).
__global__ void k_unpack(Geo G, const double* __restrict__ hat, double* __restrict__ nodal) {
  const int64_t N1 = (int64_t)G.n1 * G.p + 1, N2 = (int64_t)G.n2 * G.p + 1;
  const bool anyper = G.per[0] || G.per[1] || G.per[2];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    skel_decode(G, s, g, &bd);
    nodal[((int64_t)g[2] * N2 + g[1]) * N1 + g[0]] = anyper ? hat[skel_index(G, g[0], g[1], g[2])] : hat[s];
  }
}

// Delta u at a skeleton node: sum of the weighted star outputs of every star
// (and every plane of that star) the node lies on (Algorithm 2, last line).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_star_gather(Geo G, const T* __restrict__ Ob, T* __restrict__ du,
                                                           int accumulate) {
  const int p = G.p, m = G.m, nS = G.nS;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    skel_decode(G, s, g, &bd);
    if (bd) {
      if (!accumulate) du[s] = 0;
      continue;
    }
    int c[3][2], j[3][2], no[3];
    for (int d = 0; d < 3; ++d) {
      const int a = divp(G, g[d]), q = g[d] - a * p;
      if (q == 0) {
        no[d] = 1;
        c[d][0] = a;
        j[d][0] = 0;
      } else {
        no[d] = 2;
        c[d][0] = a;
        j[d][0] = q;
        c[d][1] = (G.per[d] && a + 1 == ncount(G, d)) ? 0 : a + 1;  // periodic: the star at plane 0
        j[d][1] = q - p;
      }
    }
    T acc = 0;
    for (int o3 = 0; o3 < no[2]; ++o3)
      for (int o2 = 0; o2 < no[1]; ++o2)
        for (int o1 = 0; o1 < no[0]; ++o1) {
          const int64_t st = ((int64_t)c[2][o3] * G.nv2 + c[1][o2]) * G.nv1 + c[0][o1];
          const int jj[3] = {j[0][o1], j[1][o2], j[2][o3]};
          const T* ob = Ob + st * 3 * (int64_t)nS * nS;
          if (jj[0] == 0) acc += ob[(0 * nS + jj[2] + m) * nS + jj[1] + m];
          if (jj[1] == 0) acc += ob[(1 * nS + jj[2] + m) * nS + jj[0] + m];
          if (jj[2] == 0) acc += ob[(2 * nS + jj[1] + m) * nS + jj[0] + m];
        }
    du[s] = accumulate ? du[s] + acc : acc;
  }
}

template <typename T>
__global__ void k_norm2_partial(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[kThreads];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double red[kThreads];
  double s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <typename TY, typename TX>
__global__ void k_axpy(TY* __restrict__ y, const TX* __restrict__ x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (TY)((double)y[i] + a * (double)x[i]);
}

template <typename TO, typename TI>
__global__ void k_copy(TO* __restrict__ y, const TI* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

}  // namespace

template <typename T>
void launch_assemble(const Geo& G, const Tabs<T>& t, const T* F, const T* u, const T* Z, T* out, int mode,
                     cudaStream_t st) {
  k_assemble<T><<<grid_for(G.size), kThreads, 0, st>>>(G, t, F, u, G.m > 0 ? Z : nullptr, out, mode);
}

void launch_assemble_mixed(const Geo& G, const Tabs<double>& t, const float* F, const double* u, const double* Z,
                           float* out, int mode, cudaStream_t st) {
  k_assemble<double, float><<<grid_for(G.size), kThreads, 0, st>>>(G, t, F, u, G.m > 0 ? Z : nullptr, out, mode);
}

void launch_assemble_rhs(const Geo& G, const Tabs<double>& t, const double* f, const double* Z, double* Fh,
                         cudaStream_t st) {
  k_assemble_rhs<<<grid_for(G.size), kThreads, 0, st>>>(G, t, f, Z, Fh);
}

void launch_pack(const Geo& G, const double* nodal, double* hat, cudaStream_t st) {
  k_pack<<<grid_for(G.size), kThreads, 0, st>>>(G, nodal, hat);
}

void launch_pack_dirichlet(const Geo& G, const double* nodal, double* hat, cudaStream_t st) {
  k_pack_dirichlet<<<grid_for(G.size), kThreads, 0, st>>>(G, nodal, hat);
}

void launch_unpack(const Geo& G, const double* hat, double* nodal, cudaStream_t st) {
  k_unpack<<<grid_for(G.size), kThreads, 0, st>>>(G, hat, nodal);
}

template <typename T>
void launch_star_gather(const Geo& G, const T* Ob, T* du, int accumulate, cudaStream_t st) {
  k_star_gather<T><<<grid_for(G.size), kThreads, 0, st>>>(G, Ob, du, accumulate);
}

template <typename T>
void launch_norm2(const T* x, int64_t n, double* partial, int npart, double* out, cudaStream_t st) {
  k_norm2_partial<T><<<npart, kThreads, 0, st>>>(x, n, partial);
  k_sum_final<<<1, kThreads, 0, st>>>(partial, npart, out);
}

template <typename TY, typename TX>
void launch_axpy(TY* y, const TX* x, double a, int64_t n, cudaStream_t st) {
  k_axpy<TY, TX><<<grid_for(n), kThreads, 0, st>>>(y, x, a, n);
}

template <typename TO, typename TI>
void launch_copy(TO* y, const TI* x, int64_t n, cudaStream_t st) {
  k_copy<TO, TI><<<grid_for(n), kThreads, 0, st>>>(y, x, n);
}

template void launch_assemble<double>(const Geo&, const Tabs<double>&, const double*, const double*, const double*,
                                      double*, int, cudaStream_t);
template void launch_assemble<float>(const Geo&, const Tabs<float>&, const float*, const float*, const float*,
                                     float*, int, cudaStream_t);
template void launch_star_gather<double>(const Geo&, const double*, double*, int, cudaStream_t);
template void launch_star_gather<float>(const Geo&, const float*, float*, int, cudaStream_t);
template void launch_norm2<double>(const double*, int64_t, double*, int, double*, cudaStream_t);
template void launch_norm2<float>(const float*, int64_t, double*, int, double*, cudaStream_t);
template void launch_axpy<double, double>(double*, const double*, double, int64_t, cudaStream_t);
template void launch_axpy<double, float>(double*, const float*, double, int64_t, cudaStream_t);
template void launch_axpy<float, float>(float*, const float*, double, int64_t, cudaStream_t);
template void launch_copy<double, double>(double*, const double*, int64_t, cudaStream_t);
template void launch_copy<float, double>(float*, const double*, int64_t, cudaStream_t);
template void launch_copy<double, float>(double*, const float*, int64_t, cudaStream_t);
template void launch_copy<float, float>(float*, const float*, int64_t, cudaStream_t);
template void launch_copy<ff, float>(ff*, const float*, int64_t, cudaStream_t);

}  // namespace semmg
