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

namespace semmg {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

// Assembled 1D mass at global index g along axis d.
template <typename T>
__device__ __forceinline__ T mass1d(const Geo& G, const Tabs<T>& t, int d, int g, int nd) {
  const int a = divp(G, g), q = g - a * G.p;
  if (q) return (T)0.5 * t.h[d][a] * t.w[q];
  T s = 0;
  if (a > 0 || G.per[d]) s += (T)0.5 * t.h[d][wrape(G, d, a - 1)] * t.w[G.p];  // periodic: the last element
  if (a < nd) s += (T)0.5 * t.h[d][a] * t.w[0];
  return s;
}

// Line sum (Lg_d u)(g) over the skeleton nodes of the line through node s
// along axis d.  `other` tells whether the node has a vertex-plane coordinate
// on another axis, in which case every node of the line is a skeleton node.
template <typename T>
__device__ T line_sum(const Geo& G, const Tabs<T>& t, const T* __restrict__ u, int64_t s, int type, const int* g,
                      int d, bool other) {
  const int nd = ncount(G, d);
  const int p = G.p;
  const int a = divp(G, g[d]), q = g[d] - a * p;
  int gg[3] = {g[0], g[1], g[2]};
  const T* Ls = t.Ls;
  const int P1 = p + 1;
  if (q) {
    // inside element a along d: endpoints are skeleton, the run is this entity
    const T k = t.hx[d][6 * a + 1];  // 2 / h
    const T* row = Ls + q * P1;
    T acc = 0;
    gg[d] = a * p;
    acc += row[0] * u[skel_index(G, gg[0], gg[1], gg[2])];
    gg[d] = a * p + p;
    acc += row[p] * u[skel_index(G, gg[0], gg[1], gg[2])];
    const int st = run_stride(G, type, d);
    const T* ur = u + s - (int64_t)(q - 1) * st;  // slot of local index 1
    for (int j = 1; j < p; ++j) acc += row[j] * ur[(int64_t)(j - 1) * st];
    return k * acc;
  }
  // on vertex plane c = a; the element on either side may be missing at a
  // (Neumann) face of the domain: 0 <= c <= n_d; neighbour nodes past a
  // periodic end wrap in skel_index
  // (on a periodic axis the element left of plane 0 is the last one)
  const bool hasL = a > 0 || G.per[d], hasR = a < nd;
  const T kL = hasL ? t.hx[d][6 * wrape(G, d, a - 1) + 1] : (T)0, kR = hasR ? t.hx[d][6 * a + 1] : (T)0;  // 2 / h
  T acc = (kL * Ls[p * P1 + p] + kR * Ls[0]) * u[s];
  if (hasL) {
    gg[d] = (a - 1) * p;
    acc += kL * Ls[p * P1 + 0] * u[skel_index(G, gg[0], gg[1], gg[2])];
  }
  if (hasR) {
    gg[d] = (a + 1) * p;
    acc += kR * Ls[0 * P1 + p] * u[skel_index(G, gg[0], gg[1], gg[2])];
  }
  if (other && p > 1) {
    T sL = 0, sR = 0;
    if (hasL) {
      int rt;
      gg[d] = (a - 1) * p + 1;
      const int64_t bL = skel_index(G, gg[0], gg[1], gg[2], &rt);
      const int st = run_stride(G, rt, d);
      for (int j = 1; j < p; ++j) sL += Ls[p * P1 + j] * u[bL + (int64_t)(j - 1) * st];
    }
    if (hasR) {
      int rt;
      gg[d] = a * p + 1;
      const int64_t bR = skel_index(G, gg[0], gg[1], gg[2], &rt);
      const int st = run_stride(G, rt, d);
      for (int j = 1; j < p; ++j) sR += Ls[0 * P1 + j] * u[bR + (int64_t)(j - 1) * st];
    }
    acc += kL * sL + kR * sR;
  }
  return acc;
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
  const int nd[3] = {G.n1, G.n2, G.n3};
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    const int type = skel_decode(G, s, g, &bd);
    if (bd) {
      out[s] = 0;
      continue;
    }
    bool on[3];
    for (int d = 0; d < 3; ++d) on[d] = (g[d] - divp(G, g[d]) * G.p) == 0;
    T M[3], L[3];
    for (int d = 0; d < 3; ++d) {
      M[d] = mass1d(G, t, d, g[d], nd[d]);
      const bool other = on[(d + 1) % 3] || on[(d + 2) % 3];
      L[d] = line_sum(G, t, u, s, type, g, d, other);
    }
    T Hu = (T)G.lam * M[0] * M[1] * M[2] * u[s] + M[1] * M[2] * L[0] + M[0] * M[2] * L[1] + M[0] * M[1] * L[2];
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

}  // namespace semmg
