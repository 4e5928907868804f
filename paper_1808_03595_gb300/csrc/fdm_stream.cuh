// Condensation and recovery (Sec. 2.2, Algorithm 4) with the interior
// transforms staged through shared memory.
//
// The element's interior fast diagonalisation applies Sref^T along x1, x2 and
// x3 (condensation) or Sref along x3, x2, x1 (recovery) to an m^3 array, which
// at high p does not fit in shared memory.  Instead of streaming the whole
// array through global memory for each of the six fold / transform passes
// (elem_kernel.cuh), the work is split into two shared-memory passes:
//   pass A: x3-planes, NP at a time: the x1 and x2 transforms of a plane need
//           only that plane;
//   pass B: k2-tiles (all k1 and k3 for TK values of k2): the x3 transform of a
//           column needs only that column, and the face contractions of
//           condensation come out of the tile directly: the sums over k1
//           (faces 0, 1) and over k3 (faces 4, 5) are complete in a tile, the
//           sums over k2 (faces 2, 3) are added tile by tile, in order.
// The m^3 array crosses global memory once between the passes.  Elements are
// handed to teams of one CTA or a cluster of two (Team, elem_kernel.cuh); the
// CTAs of a team take alternate planes and tiles, and the partial face-2/3 sums
// of the second CTA are added to the first's after the first's, so every output
// has a fixed summation order.  The face transforms (faces_forward /
// faces_backward) run over the team on face arrays in global memory.
#pragma once
#include "elem_kernel.cuh"

namespace semmg {

namespace {

constexpr size_t kFsSmemMax = 224 * 1024;  // one CTA per SM: the planes and tiles take what is left

// Shared memory: Sh (m^2), Sr (m^2), a0 (m), lI (m), then the pass buffers:
// pass A two plane buffers of NP m^2, pass B two tile buffers of TK m^2 and the
// face-2/3 accumulators (2 m^2).
struct FsShape {
  int np, tk;
  size_t smem_elems;
};

__host__ __device__ inline FsShape fs_shape(int m, size_t esize) {
  const size_t mm = (size_t)m * m, tables = 2 * mm + 2 * (size_t)m;
  const size_t budget = kFsSmemMax / esize > tables ? kFsSmemMax / esize - tables : 0;
  FsShape s;
  s.np = (int)(budget / (2 * mm));
  s.tk = budget > 2 * mm ? (int)((budget - 2 * mm) / (2 * mm)) : 0;
  if (s.np > m) s.np = m;
  if (s.tk > m) s.tk = m;
  const size_t a = 2 * (size_t)s.np * mm, b = 2 * (size_t)s.tk * mm + 2 * mm;
  s.smem_elems = tables + (a > b ? a : b);
  return s;
}

// Global elements of one team: the m^3 array between the passes, the face arrays
// X and their transform scratch Tt (6 m^2 each), the second CTA's face-2/3 sums.
__host__ __device__ inline int64_t fs_team_elems(int m) {
  const int64_t mm = (int64_t)m * m;
  return mm * m + 14 * mm;
}

template <typename T>
struct FsPtrs {
  T *Sh, *Sr, *a0, *lI, *W;      // shared
  T *gA, *gX, *gT, *gP;          // the team's global slice
};

template <typename T>
__device__ __forceinline__ FsPtrs<T> fs_ptrs(int m, unsigned char* smem, T* ws, int64_t team) {
  const int mm = m * m;
  FsPtrs<T> p;
  p.Sh = reinterpret_cast<T*>(smem);
  p.Sr = p.Sh + mm;
  p.a0 = p.Sr + mm;
  p.lI = p.a0 + m;
  p.W = p.lI + m;
  p.gA = ws + team * fs_team_elems(m);
  p.gX = p.gA + (int64_t)mm * m;
  p.gT = p.gX + 6 * mm;
  p.gP = p.gT + 6 * mm;
  return p;
}

template <typename T>
__device__ __forceinline__ void fs_load_tables(int m, const Tabs<T>& t, const FsPtrs<T>& s) {
  load_tables(m, t, s.Sh, s.a0, s.lI);
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) s.Sr[i] = t.Sref[i];
}

// Z[e][f] = (H_BI H_II^{-1} F_I) on the faces, F_I = (M f)_I, with the scaled
// interior eigen-coefficients of every element saved in Gsave when given (as
// k_elem_condense).  PC > 0 compiles the kernel for degree PC (constant
// extents, the same arithmetic in the same order); PC = 0 reads it from G.
template <typename T, int PC>
__global__ void __launch_bounds__(512, 1) k_fs_condense(Geo G, Tabs<T> t, const double* __restrict__ f,
                                                      double* __restrict__ Z, T* __restrict__ Gsave, T* ws, int cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m, ne = (m + 1) / 2;
  const int64_t mmm = (int64_t)mm * m;
  const FsShape sh = fs_shape(m, sizeof(T));
  const Team tm = team_of(cs);
  const int rank = tm.id / (int)blockDim.x;
  const FsPtrs<T> s = fs_ptrs(m, smem_raw, ws, blockIdx.x / cs);
  fs_load_tables(m, t, s);
  const Lines F{m, m / 2, ne, m, m, 6 * mm};
  const T lam = (T)G.lam;
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    const T* x1 = t.hx[0] + 6 * a1;
    const T* x2 = t.hx[1] + 6 * a2;
    const T* x3 = t.hx[2] + 6 * a3;
    const T vol = (T)0.125 * x1[0] * x2[0] * x3[0];  // h1 h2 h3 / 8
    const T sig = x1[5] * x2[5] * x3[5];             // sqrt(8 / (h1 h2 h3))
    tm.sync();  // the team's global arrays of the previous element are consumed
    // pass A: x1 and x2 transforms, NP planes at a time
    for (int p0 = rank * sh.np; p0 < m; p0 += cs * sh.np) {
      const int np = m - p0 < sh.np ? m - p0 : sh.np;
      const Lines P{m, m / 2, ne, m, m, np * mm};
      T* Pb = s.W;
      T* Qb = s.W + sh.np * mm;
      __syncthreads();  // the previous round's planes are stored
      // (the staging loops are unrolled so that several global loads are in flight per thread)
#pragma unroll 4
      for (int idx = threadIdx.x; idx < np * mm; idx += blockDim.x) {
        const int i1 = idx % m, i2 = (idx / m) % m, i3 = p0 + idx / mm;
        Pb[idx] = vol * t.w[i1 + 1] * t.w[i2 + 1] * t.w[i3 + 1] *
                  (T)f[interior_node3(G, a1, a2, a3, i1, i2, i3)];
      }
      __syncthreads();
      fold_lines(P, 0, Pb, Qb);
      __syncthreads();
      tx_lines_g(P, 0, s.Sr, Qb, Pb, (T)1, (const T*)nullptr);
      __syncthreads();
      fold_lines(P, 1, Pb, Qb);
      __syncthreads();
      tx_lines_g(P, 1, s.Sr, Qb, Pb, (T)1, (const T*)nullptr);
      __syncthreads();
      for (int idx = threadIdx.x; idx < np * mm; idx += blockDim.x) s.gA[(int64_t)p0 * mm + idx] = Pb[idx];
    }
    tm.sync();  // every plane of the element is in gA
    // pass B: x3 transform, 1/D and the face contractions, TK values of k2 at a time
    T* C = s.W;
    T* D = s.W + sh.tk * mm;
    T* acc = s.W + 2 * sh.tk * mm;  // faces 2 / 3: [class][k3][k1]
    T* Ge = Gsave ? Gsave + e * mmm : nullptr;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * mm; idx += blockDim.x) acc[idx] = (T)0;
    for (int b0 = rank * sh.tk; b0 < m; b0 += cs * sh.tk) {
      const int tk = m - b0 < sh.tk ? m - b0 : sh.tk;
      const Lines Cl{m, m / 2, ne, m, tk, tk * mm};  // C[i3][t][k1], lines along i3
      __syncthreads();  // the previous tile is consumed
#pragma unroll 4
      for (int idx = threadIdx.x; idx < tk * mm; idx += blockDim.x) {
        const int k1 = idx % m, tt = (idx / m) % tk, i3 = idx / (m * tk);
        C[idx] = s.gA[((int64_t)i3 * m + b0 + tt) * m + k1];
      }
      __syncthreads();
      fold_lines(Cl, 2, C, D);
      __syncthreads();
      tx_lines_g(Cl, 2, s.Sr, D, C, sig, (const T*)nullptr);
      __syncthreads();
#pragma unroll 4
      for (int idx = threadIdx.x; idx < tk * mm; idx += blockDim.x) {
        const int k1 = idx % m, tt = (idx / m) % tk, k3 = idx / (m * tk), k2 = b0 + tt;
        const int64_t gi = ((int64_t)k3 * m + k2) * m + k1;
        const T v = C[idx] * inv_d(t, sc, s.lI, lam, gi, k1, k2, k3, mmm);
        C[idx] = v;
        if (Ge) Ge[gi] = v;
      }
      __syncthreads();
      // faces 0 / 1 at (k3, k2): sums over k1 of each class; faces 4 / 5 at (k2, k1): over k3
      for (int o = threadIdx.x; o < 4 * m * tk; o += blockDim.x) {
        const int grp = o / (m * tk), r = o - grp * (m * tk), par = grp & 1;
        const int lo = par ? ne : 0, hi = par ? m : ne;
        T s0 = (T)0, s1 = (T)0;
        if (grp < 2) {  // r = k3 tk + tt
          const int k3 = r / tk, tt = r - (r / tk) * tk;
          const T* c = C + ((int64_t)k3 * tk + tt) * m;
          int k = lo;
          for (; k + 1 < hi; k += 2) {
            s0 = madd(s.a0[k], c[k], s0);
            s1 = madd(s.a0[k + 1], c[k + 1], s1);
          }
          if (k < hi) s0 = madd(s.a0[k], c[k], s0);
          s.gX[(int64_t)(0 + par) * mm + k3 * m + b0 + tt] = s0 + s1;
        } else {  // r = tt m + k1
          const int tt = r / m, k1 = r - tt * m;
          const T* c = C + tt * m + k1;
          const int st = tk * m;
          int k = lo;
          for (; k + 1 < hi; k += 2) {
            s0 = madd(s.a0[k], c[(int64_t)k * st], s0);
            s1 = madd(s.a0[k + 1], c[(int64_t)(k + 1) * st], s1);
          }
          if (k < hi) s0 = madd(s.a0[k], c[(int64_t)k * st], s0);
          s.gX[(int64_t)(4 + par) * mm + (b0 + tt) * m + k1] = s0 + s1;
        }
      }
      // faces 2 / 3 at (k3, k1): this tile's k2 added to the class's running sum, in order
      for (int o = threadIdx.x; o < mm; o += blockDim.x) {
        const int k3 = o / m, k1 = o - k3 * m;
        T ev = acc[o], od = acc[mm + o];
        for (int tt = 0; tt < tk; ++tt) {
          const int k2 = b0 + tt;
          const T v = C[((int64_t)k3 * tk + tt) * m + k1];
          if (k2 < ne)
            ev = madd(s.a0[k2], v, ev);
          else
            od = madd(s.a0[k2], v, od);
        }
        acc[o] = ev;
        acc[mm + o] = od;
      }
    }
    __syncthreads();
    // the team's face-2/3 sums: the first CTA's, then the second's added
    if (cs > 1 && rank == 1)
      for (int idx = threadIdx.x; idx < 2 * mm; idx += blockDim.x) s.gP[idx] = acc[idx];
    tm.sync();
    if (rank == 0)
      for (int idx = threadIdx.x; idx < 2 * mm; idx += blockDim.x)
        s.gX[2 * mm + idx] = cs > 1 ? acc[idx] + s.gP[idx] : acc[idx];
    tm.sync();
    double* Ze = Z + e * 6 * mm;
    faces_backward(F, s.Sh, s.gX, s.gT, sc, [&](int idx, T v) { Ze[idx] = (double)v; }, tm);
  }
}

// u_I = H_II^{-1} (F_I - H_IB uhat) into the nodal array, from the coefficients
// Gin that k_fs_condense saved for the same f (as k_elem_recover with Gin).
// PC as for k_fs_condense.
template <typename T, int PC>
__global__ void __launch_bounds__(512, 1) k_fs_recover(Geo G, Tabs<T> t, const T* __restrict__ Gin,
                                                     const double* __restrict__ uh, double* __restrict__ un, T* ws,
                                                     int cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m, ne = (m + 1) / 2;
  const int64_t mmm = (int64_t)mm * m;
  const FsShape sh = fs_shape(m, sizeof(T));
  const Team tm = team_of(cs);
  const int rank = tm.id / (int)blockDim.x;
  const FsPtrs<T> s = fs_ptrs(m, smem_raw, ws, blockIdx.x / cs);
  fs_load_tables(m, t, s);
  const Lines F{m, m / 2, ne, m, m, 6 * mm};
  const T lam = (T)G.lam;
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    const T sig = t.hx[0][6 * a1 + 5] * t.hx[1][6 * a2 + 5] * t.hx[2][6 * a3 + 5];  // sqrt(8 / (h1 h2 h3))
    tm.sync();
    // the six faces of u_hat in the face eigenbasis, pair sums / differences
    for (int idx = tm.id; idx < 6 * mm; idx += tm.n) {
      const int fc = idx / mm;
      s.gX[idx] = (T)uh[elem_face_base(G, a1, a2, a3, fc) + (idx - fc * mm)];
    }
    tm.sync();
    face_pairs(mm, s.gX, tm);
    tm.sync();
    faces_forward(F, s.Sh, s.gX, s.gT, sc, tm);
    // pass B: the eigenspace values and the x3 back transform, TK values of k2 at a time
    const T* Ge = Gin + e * mmm;
    T* C = s.W;
    T* D = s.W + sh.tk * mm;
    for (int b0 = rank * sh.tk; b0 < m; b0 += cs * sh.tk) {
      const int tk = m - b0 < sh.tk ? m - b0 : sh.tk;
      const Lines Cl{m, m / 2, ne, m, tk, tk * mm};
      __syncthreads();
#pragma unroll 4
      for (int idx = threadIdx.x; idx < tk * mm; idx += blockDim.x) {
        const int k1 = idx % m, tt = (idx / m) % tk, k3 = idx / (m * tk), k2 = b0 + tt;
        const int64_t gi = ((int64_t)k3 * m + k2) * m + k1;
        C[idx] = Ge[gi] - face_expand(m, ne, s.a0, s.gX, k1, k2, k3) * inv_d(t, sc, s.lI, lam, gi, k1, k2, k3, mmm);
      }
      __syncthreads();
      txT_lines_g(Cl, 2, s.Sr, C, D);
      __syncthreads();
      unfold_lines(Cl, 2, D, C);
      __syncthreads();
      for (int idx = threadIdx.x; idx < tk * mm; idx += blockDim.x) {
        const int k1 = idx % m, tt = (idx / m) % tk, i3 = idx / (m * tk);
        s.gA[((int64_t)i3 * m + b0 + tt) * m + k1] = C[idx];
      }
    }
    tm.sync();  // the x3 back transform of every column is in gA
    // pass A: x2 and x1 back transforms, NP planes at a time, and the store
    for (int p0 = rank * sh.np; p0 < m; p0 += cs * sh.np) {
      const int np = m - p0 < sh.np ? m - p0 : sh.np;
      const Lines P{m, m / 2, ne, m, m, np * mm};
      T* Pb = s.W;
      T* Qb = s.W + sh.np * mm;
      __syncthreads();
#pragma unroll 4
      for (int idx = threadIdx.x; idx < np * mm; idx += blockDim.x) Pb[idx] = s.gA[(int64_t)p0 * mm + idx];
      __syncthreads();
      txT_lines_g(P, 1, s.Sr, Pb, Qb);
      __syncthreads();
      unfold_lines(P, 1, Qb, Pb);
      __syncthreads();
      txT_lines_g(P, 0, s.Sr, Pb, Qb);
      __syncthreads();
      for (int idx = threadIdx.x; idx < np * mm; idx += blockDim.x) {
        const int i1 = idx % m, i2 = (idx / m) % m, i3 = p0 + idx / mm;
        un[interior_node3(G, a1, a2, a3, i1, i2, i3)] = (double)(sig * unfold_at(P, 0, Qb, idx));
      }
    }
  }
}

}  // namespace

// Launch shape: one 512-thread CTA per SM, two CTAs per element (a cluster) when
// that shortens the rounds per SM; the work arrays' global slices per team.
template <typename T>
LaunchCfg plan_fs(const Geo& G, int nsm) {
  LaunchCfg c;
  const FsShape sh = fs_shape(G.m, sizeof(T));
  c.block = 512;
  c.smem = sh.smem_elems * sizeof(T);
  c.ok = G.m >= 1 && sh.np >= 1 && sh.tk >= 1 && c.smem <= kFsSmemMax;
  const int64_t r1 = (G.nelem + nsm - 1) / nsm, r2 = (2 * G.nelem + nsm - 1) / nsm;
  c.cluster = (nsm >= 2 && r2 < 2 * r1) ? 2 : 1;
  const int64_t teams = nsm / c.cluster;
  const int64_t nt = G.nelem < teams ? G.nelem : teams;
  c.grid = (int)((nt < 1 ? 1 : nt) * c.cluster);
  // per-CTA stride of the workspace such that grid x stride covers every team's slice
  c.ws.gstride = (fs_team_elems(G.m) + c.cluster - 1) / c.cluster;
  return c;
}

template <typename T>
void launch_fs_condense(const Geo& G, const Tabs<T>& t, const double* f, double* Z, T* Gsave, T* ws,
                        const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 32: launch_clustered(k_fs_condense<T, 32>, c, st, G, t, f, Z, Gsave, ws, c.cluster); break;
    case 48: launch_clustered(k_fs_condense<T, 48>, c, st, G, t, f, Z, Gsave, ws, c.cluster); break;
    default: launch_clustered(k_fs_condense<T, 0>, c, st, G, t, f, Z, Gsave, ws, c.cluster); break;
  }
}

template <typename T>
void launch_fs_recover(const Geo& G, const Tabs<T>& t, const T* Gin, const double* uh, double* un, T* ws,
                       const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  switch (G.p) {
    case 32: launch_clustered(k_fs_recover<T, 32>, c, st, G, t, Gin, uh, un, ws, c.cluster); break;
    case 48: launch_clustered(k_fs_recover<T, 48>, c, st, G, t, Gin, uh, un, ws, c.cluster); break;
    default: launch_clustered(k_fs_recover<T, 0>, c, st, G, t, Gin, uh, un, ws, c.cluster); break;
  }
}

template <typename T, int PC>
int fs_attrs_pc() {
  int bad = cudaFuncSetAttribute(k_fs_condense<T, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFsSmemMax);
  bad |= cudaFuncSetAttribute(k_fs_recover<T, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFsSmemMax);
  return bad;
}

template <typename T>
int fs_attrs() {
  return fs_attrs_pc<T, 0>() | fs_attrs_pc<T, 32>() | fs_attrs_pc<T, 48>();
}

}  // namespace semmg
