// Element kernels of the statically condensed operator (Sec. 2.2).
//
// For a cuboidal element with widths (h1, h2, h3) the interior block is
//   H_II = lam M3(x)M2(x)M1 + M3(x)M2(x)L1 + M3(x)L2(x)M1 + L3(x)M2(x)M1
// restricted to the interior nodes, M_d = (h_d/2) M_S, L_d = (2/h_d) L_S.
// With the reference interior eigenpairs Sref^T L_II Sref = Lam,
// Sref^T M_II Sref = I, the scaled S_d = sqrt(2/h_d) Sref diagonalise it:
//   H_II^{-1} = (S3(x)S2(x)S1) D^{-1} (S3(x)S2(x)S1)^T,
//   D(k) = lam + (4/h1^2) Lam[k1] + (4/h2^2) Lam[k2] + (4/h3^2) Lam[k3]
// (eq. fast_diagonalization for one element).  H_IB touches the interiors of
// the six faces only: the face at side s of axis d couples through the
// single column L_d[.][s], so in the eigenbasis a face contributes
//   alpha_d a_s[k_d] * c_f (Sh^T U_f Sh)(k_a, k_b),
// alpha_d = (2/h_d)^{3/2}, c_f = sqrt(h_a h_b)/2, Sh = diag(w_I) Sref,
// a_s[k] = sum_i Sref[i][k] L_S[i][s].  H_BI is the transpose.  This gives the
// O(p^3) Schur complement term H_BI H_II^{-1} H_IB on the six faces.
#include "semmg_internal.h"

namespace semmg {

namespace {

template <typename T>
struct ElemScal {
  T sf[6];      // c_f alpha_d for the six faces
  T e[3];       // 4 / h_d^2
};

template <typename T>
__device__ __forceinline__ ElemScal<T> elem_scalars(const Tabs<T>& t, int a1, int a2, int a3) {
  ElemScal<T> s;
  const double h1 = (double)t.h[0][a1], h2 = (double)t.h[1][a2], h3 = (double)t.h[2][a3];
  const double c1 = 0.5 * sqrt(h2 * h3), c2 = 0.5 * sqrt(h1 * h3), c3 = 0.5 * sqrt(h1 * h2);
  const double al1 = pow(2.0 / h1, 1.5), al2 = pow(2.0 / h2, 1.5), al3 = pow(2.0 / h3, 1.5);
  s.sf[0] = s.sf[1] = (T)(c1 * al1);
  s.sf[2] = s.sf[3] = (T)(c2 * al2);
  s.sf[4] = s.sf[5] = (T)(c3 * al3);
  s.e[0] = (T)(4.0 / (h1 * h1));
  s.e[1] = (T)(4.0 / (h2 * h2));
  s.e[2] = (T)(4.0 / (h3 * h3));
  return s;
}

// Forward 2D transform of the six face interiors held in X[f][ib][ia]:
// X[f][kb][ka] <- sf[f] * sum Sh[ib][kb] Sh[ia][ka] X[f][ib][ia].
template <typename T>
__device__ void faces_forward(int m, const T* __restrict__ Sh, T* X, T* Tt, const ElemScal<T>& sc) {
  const int mm = m * m;
  for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm, ib = r / m, ka = r - ib * m;
    const T* x = X + f * mm + ib * m;
    T s = 0;
    for (int ia = 0; ia < m; ++ia) s += x[ia] * Sh[ia * m + ka];
    Tt[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm, kb = r / m, ka = r - kb * m;
    const T* tt = Tt + f * mm + ka;
    T s = 0;
    for (int ib = 0; ib < m; ++ib) s += Sh[ib * m + kb] * tt[ib * m];
    X[idx] = sc.sf[f] * s;
  }
  __syncthreads();
}

// Backward 2D transform: out[f][ib][ia] = sf[f] * sum Sh[ib][kb] Sh[ia][ka] X[f][kb][ka].
template <typename T, typename Store>
__device__ void faces_backward(int m, const T* __restrict__ Sh, const T* X, T* Tt, const ElemScal<T>& sc,
                               Store store) {
  const int mm = m * m;
  for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm, kb = r / m, ia = r - kb * m;
    const T* x = X + f * mm + kb * m;
    T s = 0;
    for (int ka = 0; ka < m; ++ka) s += x[ka] * Sh[ia * m + ka];
    Tt[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm, ib = r / m, ia = r - ib * m;
    const T* tt = Tt + f * mm + ia;
    T s = 0;
    for (int kb = 0; kb < m; ++kb) s += Sh[ib * m + kb] * tt[kb * m];
    store(idx, sc.sf[f] * s);
  }
}

// Sum of the six face contributions at eigen-point k (face data in X).
template <typename T>
__device__ __forceinline__ T face_expand(int m, const T* a0, const T* ap, const T* X, int k1, int k2, int k3) {
  const int mm = m * m;
  return a0[k1] * X[0 * mm + k3 * m + k2] + ap[k1] * X[1 * mm + k3 * m + k2]
       + a0[k2] * X[2 * mm + k3 * m + k1] + ap[k2] * X[3 * mm + k3 * m + k1]
       + a0[k3] * X[4 * mm + k2 * m + k1] + ap[k3] * X[5 * mm + k2 * m + k1];
}

// X[f][kb][ka] <- sum_{k_d} a_side[k_d] W(k) for the six faces.
template <typename T>
__device__ void faces_reduce(int m, const T* a0, const T* ap, const T* W, T* X) {
  const int mm = m * m;
  for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm, kb = r / m, ka = r - kb * m;
    const T* a = (f & 1) ? ap : a0;
    T s = 0;
    switch (f >> 1) {
      case 0: { const T* w = W + (kb * m + ka) * m; for (int k = 0; k < m; ++k) s += a[k] * w[k]; } break;
      case 1: { const T* w = W + kb * mm + ka; for (int k = 0; k < m; ++k) s += a[k] * w[k * m]; } break;
      default: { const T* w = W + kb * m + ka; for (int k = 0; k < m; ++k) s += a[k] * w[k * mm]; } break;
    }
    X[idx] = s;
  }
}

template <typename T>
__device__ void load_tables(int m, const Tabs<T>& t, T* Sh, T* a0, T* ap, T* lI) {
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Sh[i] = t.Sh[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    a0[i] = t.a0[i];
    ap[i] = t.ap[i];
    lI[i] = t.lamI[i];
  }
}

// y_e = H_BI H_II^{-1} H_IB u on the six faces of every element -> Z[e][f][.]
// Work regions: 0 tables (Sh, a0, ap, Lam), 1 X (6 m^2), 2 Tt (6 m^2), 3 W (m^3).
template <typename T>
__global__ void __launch_bounds__(256) k_elem_schur(Geo G, Tabs<T> t, const T* __restrict__ u, T* __restrict__ Z,
                                                     T* ws, WsPlan wp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = G.m, mm = m * m;
  T* Sh = ws_ptr<T>(wp, 0, smem_raw, ws);
  T* a0 = Sh + mm;
  T* ap = a0 + m;
  T* lI = ap + m;
  T* X = ws_ptr<T>(wp, 1, smem_raw, ws);
  T* Tt = ws_ptr<T>(wp, 2, smem_raw, ws);
  T* W = ws_ptr<T>(wp, 3, smem_raw, ws);
  load_tables(m, t, Sh, a0, ap, lI);
  const T lam = (T)G.lam;
  for (int64_t e = blockIdx.x; e < G.nelem; e += gridDim.x) {
    const int a1 = (int)(e % G.n1), a2 = (int)((e / G.n1) % G.n2), a3 = (int)(e / ((int64_t)G.n1 * G.n2));
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
      const int f = idx / mm;
      X[idx] = u[elem_face_base(G, a1, a2, a3, f) + (idx - f * mm)];
    }
    __syncthreads();
    faces_forward(m, Sh, X, Tt, sc);
    for (int idx = threadIdx.x; idx < m * mm; idx += blockDim.x) {
      const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
      const T D = lam + sc.e[0] * lI[k1] + sc.e[1] * lI[k2] + sc.e[2] * lI[k3];
      W[idx] = face_expand(m, a0, ap, X, k1, k2, k3) / D;
    }
    __syncthreads();
    faces_reduce(m, a0, ap, W, X);
    __syncthreads();
    T* Ze = Z + e * 6 * mm;
    faces_backward(m, Sh, X, Tt, sc, [&](int idx, T v) { Ze[idx] = v; });
  }
}

// Interior 3D transforms with the reference eigenvectors (scale applied by the caller).
// forward: B[k3][k2][k1] = sum Sref[i1][k1] Sref[i2][k2] Sref[i3][k3] A[i3][i2][i1]; A is clobbered.
__device__ void interior_forward(int m, const double* Sr, double* A, double* B) {
  const int mm = m * m, mmm = mm * m;
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x1
    const int k1 = idx % m, r = idx - k1;
    double s = 0;
    for (int i = 0; i < m; ++i) s += A[r + i] * Sr[i * m + k1];
    B[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x2
    const int k1 = idx % m, k2 = (idx / m) % m, i3 = idx / mm;
    const double* b = B + i3 * mm + k1;
    double s = 0;
    for (int i = 0; i < m; ++i) s += Sr[i * m + k2] * b[i * m];
    A[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x3
    const int r = idx % mm, k3 = idx / mm;
    const double* a = A + r;
    double s = 0;
    for (int i = 0; i < m; ++i) s += Sr[i * m + k3] * a[i * mm];
    B[idx] = s;
  }
  __syncthreads();
}

// backward: A[i3][i2][i1] = sum Sref[i1][k1] Sref[i2][k2] Sref[i3][k3] B[k3][k2][k1]; B is clobbered.
__device__ void interior_backward(int m, const double* Sr, double* B, double* A) {
  const int mm = m * m, mmm = mm * m;
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x3
    const int r = idx % mm, i3 = idx / mm;
    const double* b = B + r;
    double s = 0;
    for (int k = 0; k < m; ++k) s += Sr[i3 * m + k] * b[k * mm];
    A[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x2
    const int k1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
    const double* a = A + i3 * mm + k1;
    double s = 0;
    for (int k = 0; k < m; ++k) s += Sr[i2 * m + k] * a[k * m];
    B[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {  // along x1
    const int i1 = idx % m, r = idx - i1;
    double s = 0;
    for (int k = 0; k < m; ++k) s += B[r + k] * Sr[i1 * m + k];
    A[idx] = s;
  }
  __syncthreads();
}

struct FdmSmem {
  double *Sh, *Sr, *a0, *ap, *lI, *X, *Tt, *A, *B;
};

// Work regions: 0 tables (Sh, Sref, a0, ap, Lam), 1 X (6 m^2), 2 Tt (6 m^2), 3 A+B (2 m^3).
__device__ FdmSmem fdm_layout(int m, unsigned char* smem, double* ws, const WsPlan& wp) {
  const int mm = m * m;
  FdmSmem s;
  s.Sh = ws_ptr<double>(wp, 0, smem, ws);
  s.Sr = s.Sh + mm;
  s.a0 = s.Sr + mm;
  s.ap = s.a0 + m;
  s.lI = s.ap + m;
  s.X = ws_ptr<double>(wp, 1, smem, ws);
  s.Tt = ws_ptr<double>(wp, 2, smem, ws);
  s.A = ws_ptr<double>(wp, 3, smem, ws);
  s.B = s.A + (int64_t)mm * m;
  return s;
}

// Z[e][f] = (H_BI H_II^{-1} F_I) on the faces, F_I = (M f)_I element-local.
__global__ void __launch_bounds__(256) k_elem_condense(Geo G, Tabs<double> t, const double* __restrict__ f,
                                                        double* __restrict__ Z, double* ws, WsPlan wp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = G.m, mm = m * m, mmm = mm * m, p = G.p;
  FdmSmem s = fdm_layout(m, smem_raw, ws, wp);
  load_tables(m, t, s.Sh, s.a0, s.ap, s.lI);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) s.Sr[i] = t.Sref[i];
  const int N1 = G.n1 * p + 1, N2 = G.n2 * p + 1;
  for (int64_t e = blockIdx.x; e < G.nelem; e += gridDim.x) {
    const int a1 = (int)(e % G.n1), a2 = (int)((e / G.n1) % G.n2), a3 = (int)(e / ((int64_t)G.n1 * G.n2));
    const ElemScal<double> sc = elem_scalars(t, a1, a2, a3);
    const double h1 = t.h[0][a1], h2 = t.h[1][a2], h3 = t.h[2][a3];
    const double vol = h1 * h2 * h3 / 8.0;
    const double sig = sqrt(8.0 / (h1 * h2 * h3));
    __syncthreads();
    for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
      const int i1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
      const int64_t g = ((int64_t)(a3 * p + i3 + 1) * N2 + (a2 * p + i2 + 1)) * N1 + (a1 * p + i1 + 1);
      s.A[idx] = vol * t.w[i1 + 1] * t.w[i2 + 1] * t.w[i3 + 1] * f[g];
    }
    __syncthreads();
    interior_forward(m, s.Sr, s.A, s.B);
    for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
      const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
      const double D = G.lam + sc.e[0] * s.lI[k1] + sc.e[1] * s.lI[k2] + sc.e[2] * s.lI[k3];
      s.B[idx] = sig * s.B[idx] / D;
    }
    __syncthreads();
    faces_reduce(m, s.a0, s.ap, s.B, s.X);
    __syncthreads();
    double* Ze = Z + e * 6 * mm;
    faces_backward(m, s.Sh, s.X, s.Tt, sc, [&](int idx, double v) { Ze[idx] = v; });
  }
}

// u_I = H_II^{-1} (F_I - H_IB uhat) written into the nodal array.
__global__ void __launch_bounds__(256) k_elem_recover(Geo G, Tabs<double> t, const double* __restrict__ f,
                                                       const double* __restrict__ uh, double* __restrict__ un,
                                                       double* ws, WsPlan wp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = G.m, mm = m * m, mmm = mm * m, p = G.p;
  FdmSmem s = fdm_layout(m, smem_raw, ws, wp);
  load_tables(m, t, s.Sh, s.a0, s.ap, s.lI);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) s.Sr[i] = t.Sref[i];
  const int N1 = G.n1 * p + 1, N2 = G.n2 * p + 1;
  for (int64_t e = blockIdx.x; e < G.nelem; e += gridDim.x) {
    const int a1 = (int)(e % G.n1), a2 = (int)((e / G.n1) % G.n2), a3 = (int)(e / ((int64_t)G.n1 * G.n2));
    const ElemScal<double> sc = elem_scalars(t, a1, a2, a3);
    const double h1 = t.h[0][a1], h2 = t.h[1][a2], h3 = t.h[2][a3];
    const double vol = h1 * h2 * h3 / 8.0;
    const double sig = sqrt(8.0 / (h1 * h2 * h3));
    __syncthreads();
    for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
      const int i1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
      const int64_t g = ((int64_t)(a3 * p + i3 + 1) * N2 + (a2 * p + i2 + 1)) * N1 + (a1 * p + i1 + 1);
      s.A[idx] = vol * t.w[i1 + 1] * t.w[i2 + 1] * t.w[i3 + 1] * f[g];
    }
    for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
      const int fc = idx / mm;
      s.X[idx] = uh[elem_face_base(G, a1, a2, a3, fc) + (idx - fc * mm)];
    }
    __syncthreads();
    interior_forward(m, s.Sr, s.A, s.B);
    faces_forward(m, s.Sh, s.X, s.Tt, sc);
    for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
      const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
      const double D = G.lam + sc.e[0] * s.lI[k1] + sc.e[1] * s.lI[k2] + sc.e[2] * s.lI[k3];
      s.B[idx] = (sig * s.B[idx] - face_expand(m, s.a0, s.ap, s.X, k1, k2, k3)) / D;
    }
    __syncthreads();
    interior_backward(m, s.Sr, s.B, s.A);
    for (int idx = threadIdx.x; idx < mmm; idx += blockDim.x) {
      const int i1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
      const int64_t g = ((int64_t)(a3 * p + i3 + 1) * N2 + (a2 * p + i2 + 1)) * N1 + (a1 * p + i1 + 1);
      un[g] = sig * s.A[idx];
    }
  }
}

constexpr size_t kSmemCap = 112 * 1024;

}  // namespace

template <typename T>
LaunchCfg plan_elem_schur(const Geo& G, int nsm) {
  LaunchCfg c;
  const size_t m = G.m, mm = m * m;
  const size_t sizes[4] = {mm + 3 * m, 6 * mm, 6 * mm, mm * m};
  c.ws = plan_regions(sizes, 4, sizeof(T), kSmemCap, &c.smem);
  c.ok = plan_ok(c.ws, sizes, 4, sizeof(T), c.smem);
  const int64_t grid = (int64_t)nsm * blocks_per_sm(c.smem);
  c.grid = (int)(G.nelem < grid ? G.nelem : grid);
  if (c.grid < 1) c.grid = 1;
  return c;
}

template <typename T>
void launch_elem_schur(const Geo& G, const Tabs<T>& t, const T* u, T* Z, T* ws, const LaunchCfg& c,
                       cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  k_elem_schur<T><<<c.grid, c.block, c.smem, st>>>(G, t, u, Z, ws, c.ws);
}

LaunchCfg plan_elem_fdm(const Geo& G, int nsm) {
  LaunchCfg c;
  const size_t m = G.m, mm = m * m;
  const size_t sizes[4] = {2 * mm + 3 * m, 6 * mm, 6 * mm, 2 * mm * m};
  c.ws = plan_regions(sizes, 4, sizeof(double), kSmemCap, &c.smem);
  c.ok = plan_ok(c.ws, sizes, 4, sizeof(double), c.smem);
  const int64_t grid = (int64_t)nsm * blocks_per_sm(c.smem);
  c.grid = (int)(G.nelem < grid ? G.nelem : grid);
  if (c.grid < 1) c.grid = 1;
  return c;
}

void launch_elem_condense(const Geo& G, const Tabs<double>& t, const double* f, double* Z, double* ws,
                          const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  k_elem_condense<<<c.grid, c.block, c.smem, st>>>(G, t, f, Z, ws, c.ws);
}

void launch_elem_recover(const Geo& G, const Tabs<double>& t, const double* f, const double* uh, double* un,
                         double* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  k_elem_recover<<<c.grid, c.block, c.smem, st>>>(G, t, f, uh, un, ws, c.ws);
}

template LaunchCfg plan_elem_schur<double>(const Geo&, int);
template LaunchCfg plan_elem_schur<float>(const Geo&, int);
template void launch_elem_schur<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                        const LaunchCfg&, cudaStream_t);
template void launch_elem_schur<float>(const Geo&, const Tabs<float>&, const float*, float*, float*,
                                       const LaunchCfg&, cudaStream_t);

int set_elem_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_elem_schur<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_condense, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_recover, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

}  // namespace semmg
