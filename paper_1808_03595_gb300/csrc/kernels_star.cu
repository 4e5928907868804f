// Star smoother: Algorithm 2 around Algorithm 1 (Sec. 3.2), one CTA per star.
//
// The star of vertex c is every skeleton node strictly inside its 2x2x2
// element block; after condensation it is three planes of n_S x n_S points
// (n_S = 2p-1) through the vertex, perpendicular to x1, x2, x3 (Sec. 2.3).
// Embedding the condensed star system in the full block system (Sec. 3.1)
// lets the block's fast diagonalisation act on the plane data only:
//   1. divide the residual on each plane by the number of planes the node
//      lies on (1, 2 or 3);
//   2. transform each plane with the two in-plane eigenvector matrices and
//      expand it along its normal with the vertex row s_d = S_d[vertex, :];
//   3. divide by D(k) = lam + Lam_1[k1] + Lam_2[k2] + Lam_3[k3];
//   4. contract back onto each plane with s_d and the in-plane matrices.
// The 1D tables S_d, Lam_d of a vertex line come from the assembled block
// matrices of the two elements beside it, with identity / 1 padding at the
// Dirichlet boundary (Sec. 3.3).  The plane outputs are weighted with the
// degree-7 weights W_i (Sec. 3.2) and the multiplicity, and written to a
// per-star buffer; k_star_gather sums them per skeleton node.
#include "semmg_internal.h"

namespace semmg {

namespace {

// Work regions: 0 S tables (3 nS^2; optional), 1 P (3 nS^2), 2 Tt (3 nS^2),
// 3 V (nS^3), 4 Lam + act (3 nS each, as T).
//
// Plane dd (normal to axis dd) is stored [jb][ja] with a = the lower and b
// the higher of the two in-plane axes.  Centrosymmetric lines (every interior
// vertex line of a uniform mesh) have even eigenvectors in columns 0..m and
// odd ones in m+1..2m, so a 1D transform folds the data about the vertex
// (x[m+j] +- x[m-j]) and multiplies with the half-size blocks: half the
// multiply-adds.  Odd eigenvectors vanish at the vertex (s_d[k] = 0 for
// k > m), so the contractions along the normals run over the even half only.

// Plane pass helpers: axis index of the fast (a) and slow (b) in-plane axes.
__device__ __forceinline__ int ax_fast(int dd) { return dd == 0 ? 1 : 0; }
__device__ __forceinline__ int ax_slow(int dd) { return dd == 2 ? 1 : 2; }

// Fold (sym) or copy a 3-plane array along the fast (along=0) or slow (along=1) index.
template <typename T>
__device__ void fold_pass(int nS, int m, const int* sym, int along, const T* X, T* Y) {
  const int n2 = nS * nS;
  for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
    const int dd = idx / n2, rr = idx - dd * n2, row = rr / nS, col = rr - row * nS;
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const T* x = X + dd * n2;
    T v;
    if (!sym[ax]) {
      v = x[rr];
    } else {
      const int j = along == 0 ? col : row;  // folded index
      const int jj = j <= m ? j : j - m;     // distance from the vertex
      const int ip = along == 0 ? row * nS + (m + jj) : (m + jj) * nS + col;
      const int im = along == 0 ? row * nS + (m - jj) : (m - jj) * nS + col;
      if (j == 0) v = x[ip];
      else if (j <= m) v = x[ip] + x[im];
      else v = x[ip] - x[im];
    }
    Y[idx] = v;
  }
}

// Forward 1D transform of folded data along the fast (along=0) / slow (along=1)
// index: out[k] = sum_j S[j][k] x[j] (folded sums on symmetric lines).
template <typename T>
__device__ void tx_pass(int nS, int m, const int* sym, const T* const* S, int along, const T* Y, T* Z) {
  const int n2 = nS * nS;
  for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
    const int dd = idx / n2, rr = idx - dd * n2, row = rr / nS, col = rr - row * nS;
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const T* Sa = S[ax];
    const T* y = Y + dd * n2;
    const int k = along == 0 ? col : row;
    const int str = along == 0 ? 1 : nS;
    const T* yy = along == 0 ? y + row * nS : y + col;
    T s = 0;
    if (!sym[ax]) {
      for (int j = 0; j < nS; ++j) s += Sa[j * nS + k] * yy[j * str];
    } else if (k <= m) {
      for (int j = 0; j <= m; ++j) s += Sa[(m + j) * nS + k] * yy[j * str];
    } else {
      for (int j = 1; j <= m; ++j) s += Sa[(m + j) * nS + k] * yy[(m + j) * str];
    }
    Z[idx] = s;
  }
}

// Transposed 1D transform into folded form: symmetric lines give E_j (j <= m)
// and O_j (stored at m+j); others give x[j] = sum_k S[j][k] b[k].
template <typename T>
__device__ void txT_pass(int nS, int m, const int* sym, const T* const* S, int along, const T* B, T* Y) {
  const int n2 = nS * nS;
  for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
    const int dd = idx / n2, rr = idx - dd * n2, row = rr / nS, col = rr - row * nS;
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const T* Sa = S[ax];
    const T* b = B + dd * n2;
    const int j = along == 0 ? col : row;
    const int str = along == 0 ? 1 : nS;
    const T* bb = along == 0 ? b + row * nS : b + col;
    T s = 0;
    if (!sym[ax]) {
      const T* sr = Sa + j * nS;
      for (int k = 0; k < nS; ++k) s += sr[k] * bb[k * str];
    } else if (j <= m) {
      const T* sr = Sa + (m + j) * nS;
      for (int k = 0; k <= m; ++k) s += sr[k] * bb[k * str];
    } else {
      const T* sr = Sa + j * nS;  // row m + (j - m)
      for (int k = m + 1; k < nS; ++k) s += sr[k] * bb[k * str];
    }
    Y[idx] = s;
  }
}

// Unfold E/O pairs (or copy) back to natural order along the fast / slow index.
template <typename T>
__device__ __forceinline__ T unfold_value(int nS, int m, const int* sym, int along, const T* Y, int dd, int row,
                                          int col) {
  const int n2 = nS * nS;
  const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
  const T* y = Y + dd * n2;
  if (!sym[ax]) return y[row * nS + col];
  const int j = along == 0 ? col : row;  // natural index
  const int dist = j >= m ? j - m : m - j;
  const int ie = along == 0 ? row * nS + dist : dist * nS + col;
  if (dist == 0) return y[ie];
  const int io = along == 0 ? row * nS + m + dist : (m + dist) * nS + col;
  return j > m ? y[ie] + y[io] : y[ie] - y[io];
}

template <typename T>
__global__ void __launch_bounds__(256) k_star(Geo G, Tabs<T> t, const T* __restrict__ r, T* __restrict__ Ob,
                                               T* ws, WsPlan wp, int S_copy, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  __shared__ int s_sym[3];
  const int p = G.p, m = G.m, nS = G.nS, n2 = nS * nS;
  T* Sbuf = ws_ptr<T>(wp, 0, smem_raw, ws);
  T* P = ws_ptr<T>(wp, 1, smem_raw, ws);
  T* Tt = ws_ptr<T>(wp, 2, smem_raw, ws);
  T* V = ws_ptr<T>(wp, 3, smem_raw, ws);
  T* Lm = ws_ptr<T>(wp, 4, smem_raw, ws);
  T* Ac = Lm + 3 * nS;
  const T lam = (T)G.lam;
  int64_t st = blockIdx.x;
  while (st < G.nstar) {
    const int c[3] = {(int)(st % G.nv1), (int)((st / G.nv1) % G.nv2), (int)(st / ((int64_t)G.nv1 * G.nv2))};
    const T* S[3];
    __syncthreads();
    if (threadIdx.x < 3) s_sym[threadIdx.x] = t.starSym[threadIdx.x][c[threadIdx.x]];
    for (int d = 0; d < 3; ++d) {
      const T* src = t.starS[d] + (int64_t)c[d] * n2;
      if (S_copy) {
        for (int i = threadIdx.x; i < n2; i += blockDim.x) Sbuf[d * n2 + i] = src[i];
        S[d] = Sbuf + d * n2;
      } else {
        S[d] = src;
      }
      for (int i = threadIdx.x; i < nS; i += blockDim.x) {
        Lm[d * nS + i] = t.starLam[d][(int64_t)c[d] * nS + i];
        Ac[d * nS + i] = (T)t.act[d][(int64_t)c[d] * nS + i];
      }
    }
    __syncthreads();
    const int* sym = s_sym;
    // 1. gather the three planes, divided by the multiplicity, zero where not a star node
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS - m, ja = rr % nS - m;
      const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
      T v = 0;
      if (Ac[dd * nS + m] != (T)0 && Ac[ax_a * nS + ja + m] != (T)0 && Ac[ax_b * nS + jb + m] != (T)0) {
        int g[3];
        g[dd] = c[dd] * p;
        g[ax_a] = c[ax_a] * p + ja;
        g[ax_b] = c[ax_b] * p + jb;
        const T mult = (T)(1 + (ja == 0) + (jb == 0));
        v = r[skel_index(G, g[0], g[1], g[2])] / mult;
      }
      P[idx] = v;
    }
    __syncthreads();
    // 2a. in-plane transforms A = S_b^T P S_a (fold, transform; fast then slow index)
    fold_pass(nS, m, sym, 0, P, Tt);
    __syncthreads();
    tx_pass(nS, m, sym, S, 0, Tt, P);
    __syncthreads();
    fold_pass(nS, m, sym, 1, P, Tt);
    __syncthreads();
    tx_pass(nS, m, sym, S, 1, Tt, P);
    __syncthreads();
    // 2b + 3. expansion along the normals with the vertex rows, times 1/D
    const T* s1 = S[0] + m * nS;
    const T* s2 = S[1] + m * nS;
    const T* s3 = S[2] + m * nS;
    const int64_t n3 = (int64_t)n2 * nS;
    const T* R = nullptr;
    if (t.Rtab) {
      const int64_t cls = ((int64_t)t.starCls[0][c[0]] * t.ncls[1] + t.starCls[1][c[1]]) * t.ncls[2] + t.starCls[2][c[2]];
      R = t.Rtab + cls * n3;
    }
    for (int64_t idx = threadIdx.x; idx < n3; idx += blockDim.x) {
      const int k1 = (int)(idx % nS), k2 = (int)((idx / nS) % nS), k3 = (int)(idx / n2);
      const T E = s1[k1] * P[k3 * nS + k2] + s2[k2] * P[n2 + k3 * nS + k1] + s3[k3] * P[2 * n2 + k2 * nS + k1];
      V[idx] = R ? E * R[idx] : E / (lam + Lm[k1] + Lm[nS + k2] + Lm[2 * nS + k3]);
    }
    __syncthreads();
    // 4a. contraction along the normals: B1[k3][k2], B2[k3][k1], B3[k2][k1]
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, kb = rr / nS, ka = rr % nS;
      const int nz = sym[dd] ? m + 1 : nS;  // odd eigenvectors vanish at the vertex
      T s = 0;
      if (dd == 0) {
        const T* v = V + (int64_t)(kb * nS + ka) * nS;
        for (int k = 0; k < nz; ++k) s += s1[k] * v[k];
      } else if (dd == 1) {
        const T* v = V + (int64_t)kb * n2 + ka;
        for (int k = 0; k < nz; ++k) s += s2[k] * v[k * nS];
      } else {
        const T* v = V + (int64_t)kb * nS + ka;
        for (int k = 0; k < nz; ++k) s += s3[k] * v[(int64_t)k * n2];
      }
      P[idx] = s;
    }
    __syncthreads();
    // 4b. back to the planes: O = S_b B S_a^T (slow index first, then fast)
    txT_pass(nS, m, sym, S, 1, P, Tt);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, row = rr / nS, col = rr - row * nS;
      P[idx] = unfold_value(nS, m, sym, 1, Tt, dd, row, col);
    }
    __syncthreads();
    txT_pass(nS, m, sym, S, 0, P, Tt);
    __syncthreads();
    T* ob = Ob + st * 3 * (int64_t)n2;
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS, ja = rr % nS;
      const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
      const T s = unfold_value(nS, m, sym, 0, Tt, dd, jb, ja);
      const bool active = Ac[dd * nS + m] != (T)0 && Ac[ax_a * nS + ja] != (T)0 && Ac[ax_b * nS + jb] != (T)0;
      const int oa = ja - m, obb = jb - m;
      const T wgt = t.w1d[oa < 0 ? -oa : oa] * t.w1d[obb < 0 ? -obb : obb];
      const T mult = (T)(1 + (oa == 0) + (obb == 0));
      ob[idx] = active ? wgt * s / mult : (T)0;
    }
    // next star: from the shared counter when given (dynamic balance), else grid-strided
    if (counter) {
      __syncthreads();
      if (threadIdx.x == 0) s_next = atomicAdd(&counter[0], 1) + (int)gridDim.x;
      __syncthreads();
      st = s_next;
    } else {
      st += gridDim.x;
    }
  }
  if (counter) {
    // the last block to finish resets the counter for the next launch on the stream
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const int done = atomicAdd(&counter[1], 1);
      if (done == (int)gridDim.x - 1) {
        counter[0] = 0;
        counter[1] = 0;
        __threadfence();
      }
    }
  }
}

constexpr size_t kStarSmemCap = 112 * 1024;

}  // namespace

template <typename T>
LaunchCfg plan_star(const Geo& G, int nsm) {
  LaunchCfg c;
  const size_t nS = G.nS, n2 = nS * nS;
  const size_t sizes[5] = {3 * n2, 3 * n2, 3 * n2, n2 * nS, 6 * nS};
  // priority: small tables, planes, transform temp, S tables, eigenspace
  const int order[5] = {4, 1, 2, 0, 3};
  c.ws = plan_regions(sizes, 5, sizeof(T), kStarSmemCap, &c.smem, order);
  c.ok = plan_ok(c.ws, sizes, 5, sizeof(T), c.smem);
  const int64_t grid = (int64_t)nsm * blocks_per_sm(c.smem);
  c.grid = (int)(G.nstar < grid ? G.nstar : grid);
  if (c.grid < 1) c.grid = 1;
  return c;
}

template <typename T>
void launch_star(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, int* counter,
                 cudaStream_t st) {
  if (G.nstar == 0 || !c.ok) return;
  // copy the S tables into the CTA's work memory only when that is shared memory
  const int S_copy = c.ws.in_smem[0];
  k_star<T><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter);
}

template LaunchCfg plan_star<double>(const Geo&, int);
template LaunchCfg plan_star<float>(const Geo&, int);
template void launch_star<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                  const LaunchCfg&, int*, cudaStream_t);
template void launch_star<float>(const Geo&, const Tabs<float>&, const float*, float*, float*, const LaunchCfg&, int*,
                                 cudaStream_t);

int set_star_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_star<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

}  // namespace semmg
