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
template <typename T>
__global__ void __launch_bounds__(256) k_star(Geo G, Tabs<T> t, const T* __restrict__ r, T* __restrict__ Ob,
                                               T* ws, WsPlan wp, int S_copy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = G.p, m = G.m, nS = G.nS, n2 = nS * nS;
  T* Sbuf = ws_ptr<T>(wp, 0, smem_raw, ws);
  T* P = ws_ptr<T>(wp, 1, smem_raw, ws);
  T* Tt = ws_ptr<T>(wp, 2, smem_raw, ws);
  T* V = ws_ptr<T>(wp, 3, smem_raw, ws);
  T* Lm = ws_ptr<T>(wp, 4, smem_raw, ws);
  T* Ac = Lm + 3 * nS;
  const T lam = (T)G.lam;
  for (int64_t st = blockIdx.x; st < G.nstar; st += gridDim.x) {
    const int c[3] = {(int)(st % G.nv1), (int)((st / G.nv1) % G.nv2), (int)(st / ((int64_t)G.nv1 * G.nv2))};
    const T* S[3];
    __syncthreads();
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
    // 1. gather the three planes, divided by the multiplicity, zero where not a star node
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS - m, ja = rr % nS - m;
      const int ax_a = dd == 0 ? 1 : 0, ax_b = dd == 2 ? 1 : 2;
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
    // 2a. in-plane transforms: A_dd[kb][ka] = sum S_b[jb][kb] S_a[ja][ka] P[jb][ja]
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS, ka = rr % nS;
      const T* Sa = S[dd == 0 ? 1 : 0];
      const T* pr = P + dd * n2 + jb * nS;
      T s = 0;
      for (int ja = 0; ja < nS; ++ja) s += pr[ja] * Sa[ja * nS + ka];
      Tt[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, kb = rr / nS, ka = rr % nS;
      const T* Sb = S[dd == 2 ? 1 : 2];
      const T* tc = Tt + dd * n2 + ka;
      T s = 0;
      for (int jb = 0; jb < nS; ++jb) s += Sb[jb * nS + kb] * tc[jb * nS];
      P[idx] = s;
    }
    __syncthreads();
    // 2b + 3. expansion along the normals and the inverse eigenvalues
    const T* s1 = S[0] + m * nS;
    const T* s2 = S[1] + m * nS;
    const T* s3 = S[2] + m * nS;
    const int64_t n3 = (int64_t)n2 * nS;
    for (int64_t idx = threadIdx.x; idx < n3; idx += blockDim.x) {
      const int k1 = (int)(idx % nS), k2 = (int)((idx / nS) % nS), k3 = (int)(idx / n2);
      const T E = s1[k1] * P[k3 * nS + k2] + s2[k2] * P[n2 + k3 * nS + k1] + s3[k3] * P[2 * n2 + k2 * nS + k1];
      V[idx] = E / (lam + Lm[k1] + Lm[nS + k2] + Lm[2 * nS + k3]);
    }
    __syncthreads();
    // 4a. contraction along the normals: B1[k3][k2], B2[k3][k1], B3[k2][k1]
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, kb = rr / nS, ka = rr % nS;
      T s = 0;
      if (dd == 0) {
        const T* v = V + (int64_t)(kb * nS + ka) * nS;
        for (int k = 0; k < nS; ++k) s += s1[k] * v[k];
      } else if (dd == 1) {
        const T* v = V + (int64_t)kb * n2 + ka;
        for (int k = 0; k < nS; ++k) s += s2[k] * v[k * nS];
      } else {
        const T* v = V + (int64_t)kb * nS + ka;
        for (int k = 0; k < nS; ++k) s += s3[k] * v[(int64_t)k * n2];
      }
      P[idx] = s;
    }
    __syncthreads();
    // 4b. back to the planes: O[jb][ja] = sum S_b[jb][kb] S_a[ja][ka] B[kb][ka]
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, kb = rr / nS, ja = rr % nS;
      const T* Sa = S[dd == 0 ? 1 : 0];
      const T* pr = P + dd * n2 + kb * nS;
      const T* sa = Sa + ja * nS;
      T s = 0;
      for (int ka = 0; ka < nS; ++ka) s += pr[ka] * sa[ka];
      Tt[idx] = s;
    }
    __syncthreads();
    T* ob = Ob + st * 3 * (int64_t)n2;
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS, ja = rr % nS;
      const int ax_a = dd == 0 ? 1 : 0, ax_b = dd == 2 ? 1 : 2;
      const T* Sb = S[ax_b] + jb * nS;
      const T* tc = Tt + dd * n2 + ja;
      T s = 0;
      for (int kb = 0; kb < nS; ++kb) s += Sb[kb] * tc[kb * nS];
      const bool active = Ac[dd * nS + m] != (T)0 && Ac[ax_a * nS + ja] != (T)0 && Ac[ax_b * nS + jb] != (T)0;
      const int oa = ja - m, obb = jb - m;
      const T wgt = t.w1d[oa < 0 ? -oa : oa] * t.w1d[obb < 0 ? -obb : obb];
      const T mult = (T)(1 + (oa == 0) + (obb == 0));
      ob[idx] = active ? wgt * s / mult : (T)0;
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
void launch_star(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.nstar == 0 || !c.ok) return;
  // copy the S tables into the CTA's work memory only when that is shared memory
  const int S_copy = c.ws.in_smem[0];
  k_star<T><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy);
}

template LaunchCfg plan_star<double>(const Geo&, int);
template LaunchCfg plan_star<float>(const Geo&, int);
template void launch_star<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                  const LaunchCfg&, cudaStream_t);
template void launch_star<float>(const Geo&, const Tabs<float>&, const float*, float*, float*, const LaunchCfg&,
                                 cudaStream_t);

int set_star_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_star<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  bad |= cudaFuncSetAttribute(k_star<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  return bad;
}

}  // namespace semmg
