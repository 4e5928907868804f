// Element-centred block smoother (Sec. 3.4): one CTA per element block.
//
// The block of element c is the 3x3x3 element block around it (full overlap).
// Along each axis it holds n_E = 3p - 1 nodes strictly inside (line index j at
// global index (c_d - 1) p + 1 + j); after condensation only the six planes
// through the faces of element c remain, two per axis, at j = p - 1 and
// j = 2p - 1 (q_0, q_1), each n_E x n_E.  As for the star (Sec. 3.1), the
// condensed block system embeds in the full block system, so the block's fast
// diagonalisation acts on the plane data only:
//   1. divide the residual on each plane by the number of the six planes the
//      node lies on (1, 2 or 3);
//   2. transform each plane with its two in-plane eigenvector matrices,
//      A = S_b^T P S_a (4 n_E^3 operations per plane);
//   3. expand along the normals with the plane rows s_{d,s} = S_d[q_s, :],
//      divide by D(k) = lam + Lam_1[k1] + Lam_2[k2] + Lam_3[k3] and contract
//      back onto each plane with the same rows (25 n_E^3 for the six planes);
//   4. transform back, O = S_b B S_a^T.
// In total 73 n_E^3 operations per block, the count the paper gives.  Each
// plane output is weighted with the block's weight at its node (a product of
// per-axis factors from the host) and divided by the node's plane count, and
// stored per block; k_eblock_gather sums the outputs of every block and plane
// a skeleton node lies on.
//
// Plane pl = 2 d + s (normal d, position q_s) is stored [jb][ja], a the lower
// and b the higher in-plane axis.  The 1D tables S_d (n_E x n_E, S[j][k]) and
// Lam_d of a block line come per axis and element from the host (assembled
// matrices of the three elements, identity padding where a node is not an
// unknown).  Work regions: 0 P (6 n_E^2), 1 X (6 n_E^2), 2 V slab (ts n_E^2),
// 3 plane rows and eigenvalues (9 n_E); each in shared memory or in the
// CTA's slice of the global workspace (plan_eblock).
#include "semmg_internal.h"

namespace semmg {

namespace {

constexpr int kEbThreads = 512;
constexpr int kEbRegions = 4;

__device__ __forceinline__ int eb_axis_a(int d) { return d == 0 ? 1 : 0; }
__device__ __forceinline__ int eb_axis_b(int d) { return d == 2 ? 1 : 2; }

// Global node index along axis d of line index j of the block of element c,
// wrapped on a periodic axis; -1 outside the domain.
__device__ __forceinline__ int eb_global(const Geo& G, int d, int c, int j) {
  const int nd = ncount(G, d);
  int g = (c - 1) * G.p + 1 + j;
  if (G.per[d]) {
    const int L = nd * G.p;
    g = g < 0 ? g + L : (g >= L ? g - L : g);
    return g;
  }
  return (g < 0 || g > nd * G.p) ? -1 : g;
}

// Whether a node (global indices, each >= 0) is an unknown: no coordinate on a
// Dirichlet vertex plane.
__device__ __forceinline__ bool eb_unknown(const Geo& G, const int* g) {
  for (int d = 0; d < 3; ++d) {
    const int a = divp(G, g[d]);
    if (g[d] == a * G.p && dir_plane(G, d, a)) return false;
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kEbThreads, 1)
    k_eblock(Geo G, Tabs<T> t, const T* __restrict__ r, T* __restrict__ Ob, T* ws, WsPlan wp, int ts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = G.p, nE = 3 * p - 1, nn = nE * nE;
  const int q0 = p - 1, q1 = 2 * p - 1;
  T* P = ws_ptr<T>(wp, 0, smem_raw, ws);
  T* X = ws_ptr<T>(wp, 1, smem_raw, ws);
  T* V = ws_ptr<T>(wp, 2, smem_raw, ws);
  T* sq = ws_ptr<T>(wp, 3, smem_raw, ws);  // sq[(2 d + s) nE + k] = S_d[q_s][k]
  T* Lm = sq + 6 * nE;                     // Lm[d nE + k]
  const int nT = blockDim.x;
  for (int64_t blk = blockIdx.x; blk < G.nelem; blk += gridDim.x) {
    const int c1 = (int)(blk % G.n1), c2 = (int)((blk / G.n1) % G.n2), c3 = (int)(blk / ((int64_t)G.n1 * G.n2));
    const int cc[3] = {c1, c2, c3};
    const T* S[3];
    const T* ST[3];
    for (int d = 0; d < 3; ++d) {
      S[d] = t.ebS[d] + (int64_t)cc[d] * nn;
      ST[d] = t.ebST[d] + (int64_t)cc[d] * nn;
    }
    // 1/D of the block's line-class triple, when tabulated
    const T* Rd = nullptr;
    if (t.ebR) {
      const int64_t cls = ((int64_t)t.ebCls[2][c3] * t.ebNcls[1] + t.ebCls[1][c2]) * t.ebNcls[0] + t.ebCls[0][c1];
      Rd = t.ebR + cls * nn * nE;
    }
    __syncthreads();  // previous block done with every region
    for (int i = threadIdx.x; i < 9 * nE; i += nT) {
      if (i < 6 * nE) {
        const int pl = i / nE, k = i - pl * nE;
        sq[i] = S[pl >> 1][(int64_t)((pl & 1) ? q1 : q0) * nE + k];
      } else {
        const int d = (i - 6 * nE) / nE, k = i - 6 * nE - d * nE;
        Lm[i - 6 * nE] = t.ebLam[d][(int64_t)cc[d] * nE + k];
      }
    }
    // 1. gather the six planes divided by the plane count; zero where not an unknown
    for (int i = threadIdx.x; i < 6 * nn; i += nT) {
      const int pl = i / nn, rem = i - pl * nn, jb = rem / nE, ja = rem - jb * nE;
      const int d = pl >> 1, a = eb_axis_a(d), b = eb_axis_b(d);
      int g[3];
      g[d] = eb_global(G, d, cc[d], (pl & 1) ? q1 : q0);
      g[a] = eb_global(G, a, cc[a], ja);
      g[b] = eb_global(G, b, cc[b], jb);
      T v = 0;
      if (g[0] >= 0 && g[1] >= 0 && g[2] >= 0 && eb_unknown(G, g)) {
        const int mult = 1 + (ja == q0 || ja == q1) + (jb == q0 || jb == q1);
        v = r[skel_index(G, g[0], g[1], g[2])] / (T)mult;
      }
      P[i] = v;
    }
    __syncthreads();
    // 2. forward: X[pl][jb][ka] = sum_ja P[pl][jb][ja] S_a[ja][ka]; four rows jb per thread
    const int nq = (nE + 3) / 4;  // row groups of four
    for (int i = threadIdx.x; i < 6 * nq * nE; i += nT) {
      const int pl = i / (nq * nE), rem = i - pl * nq * nE, jb0 = 4 * (rem / nE), ka = rem % nE;
      const T* Sa = S[eb_axis_a(pl >> 1)] + ka;
      const T* Pr = P + (int64_t)pl * nn + (int64_t)jb0 * nE;
      const int nr = min(4, nE - jb0);
      T acc[4] = {0, 0, 0, 0};
      for (int ja = 0; ja < nE; ++ja) {
        const T sv = Sa[(int64_t)ja * nE];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < nr) acc[r] += Pr[r * nE + ja] * sv;
      }
      for (int r = 0; r < nr; ++r) X[(int64_t)pl * nn + (int64_t)(jb0 + r) * nE + ka] = acc[r];
    }
    __syncthreads();
    //    P[pl][kb][ka] = sum_jb S_b[jb][kb] X[pl][jb][ka] (A of the plane); four kb per thread
    for (int i = threadIdx.x; i < 6 * nq * nE; i += nT) {
      const int pl = i / (nq * nE), rem = i - pl * nq * nE, kb0 = 4 * (rem / nE), ka = rem % nE;
      const T* Sb = S[eb_axis_b(pl >> 1)] + kb0;
      const T* Xc = X + (int64_t)pl * nn + ka;
      const int nr = min(4, nE - kb0);
      T acc[4] = {0, 0, 0, 0};
      for (int jb = 0; jb < nE; ++jb) {
        const T xv = Xc[(int64_t)jb * nE];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < nr) acc[r] += Sb[(int64_t)jb * nE + r] * xv;
      }
      for (int r = 0; r < nr; ++r) P[(int64_t)pl * nn + (int64_t)(kb0 + r) * nE + ka] = acc[r];
    }
    __syncthreads();
    // 3. eigenspace in slabs of ts k3-planes.  B accumulators in X:
    //    B[0 + s][k3][k2], B[2 + s][k3][k1] per slab; B[4 + s][k2][k1] summed over the slabs
    for (int i = threadIdx.x; i < 2 * nn; i += nT) X[4 * nn + i] = 0;
    for (int k30 = 0; k30 < nE; k30 += ts) {
      const int tc = min(ts, nE - k30);
      __syncthreads();
      for (int i = threadIdx.x; i < tc * nn; i += nT) {
        const int tt = i / nn, rem = i - tt * nn, k2 = rem / nE, k1 = rem - k2 * nE;
        const int k3 = k30 + tt;
        T e = 0;
        for (int s = 0; s < 2; ++s) {
          e += sq[(0 + s) * nE + k1] * P[(int64_t)(0 + s) * nn + k3 * nE + k2];
          e += sq[(2 + s) * nE + k2] * P[(int64_t)(2 + s) * nn + k3 * nE + k1];
          e += sq[(4 + s) * nE + k3] * P[(int64_t)(4 + s) * nn + k2 * nE + k1];
        }
        V[i] = Rd ? e * Rd[(int64_t)k3 * nn + rem] : e / ((T)G.lam + Lm[k1] + Lm[nE + k2] + Lm[2 * nE + k3]);
      }
      __syncthreads();
      const int n0 = tc * nE;
      for (int i = threadIdx.x; i < 2 * n0 + nn; i += nT) {
        if (i < n0) {  // B[s][k3][k2] = sum_k1 s1 V
          const int tt = i / nE, k2 = i - tt * nE;
          const T* Vr = V + (int64_t)tt * nn + (int64_t)k2 * nE;
          T a0 = 0, a1 = 0;
          for (int k1 = 0; k1 < nE; ++k1) {
            a0 += sq[0 * nE + k1] * Vr[k1];
            a1 += sq[1 * nE + k1] * Vr[k1];
          }
          X[(int64_t)0 * nn + (k30 + tt) * nE + k2] = a0;
          X[(int64_t)1 * nn + (k30 + tt) * nE + k2] = a1;
        } else if (i < 2 * n0) {  // B[2 + s][k3][k1] = sum_k2 s2 V
          const int j = i - n0, tt = j / nE, k1 = j - tt * nE;
          const T* Vc = V + (int64_t)tt * nn + k1;
          T a0 = 0, a1 = 0;
          for (int k2 = 0; k2 < nE; ++k2) {
            a0 += sq[2 * nE + k2] * Vc[(int64_t)k2 * nE];
            a1 += sq[3 * nE + k2] * Vc[(int64_t)k2 * nE];
          }
          X[(int64_t)2 * nn + (k30 + tt) * nE + k1] = a0;
          X[(int64_t)3 * nn + (k30 + tt) * nE + k1] = a1;
        } else {  // B[4 + s][k2][k1] += sum_k3 s3 V over the slab
          const int j = i - 2 * n0;
          T a0 = X[(int64_t)4 * nn + j], a1 = X[(int64_t)5 * nn + j];
          for (int tt = 0; tt < tc; ++tt) {
            const T v = V[(int64_t)tt * nn + j];
            a0 += sq[4 * nE + k30 + tt] * v;
            a1 += sq[5 * nE + k30 + tt] * v;
          }
          X[(int64_t)4 * nn + j] = a0;
          X[(int64_t)5 * nn + j] = a1;
        }
      }
    }
    __syncthreads();
    // 4. backward: P[pl][jb][ka] = sum_kb S_b[jb][kb] B[pl][kb][ka]; four jb per thread
    for (int i = threadIdx.x; i < 6 * nq * nE; i += nT) {
      const int pl = i / (nq * nE), rem = i - pl * nq * nE, jb0 = 4 * (rem / nE), ka = rem % nE;
      const T* Sb = S[eb_axis_b(pl >> 1)] + (int64_t)jb0 * nE;
      const T* Bc = X + (int64_t)pl * nn + ka;
      const int nr = min(4, nE - jb0);
      T acc[4] = {0, 0, 0, 0};
      for (int kb = 0; kb < nE; ++kb) {
        const T bv = Bc[(int64_t)kb * nE];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < nr) acc[r] += Sb[(int64_t)r * nE + kb] * bv;
      }
      for (int r = 0; r < nr; ++r) P[(int64_t)pl * nn + (int64_t)(jb0 + r) * nE + ka] = acc[r];
    }
    __syncthreads();
    //    O[pl][jb][ja] = sum_ka P[pl][jb][ka] S_a[ja][ka] (S_a^T[ka][ja] from the transposed
    //    table), four jb per thread, weighted, into the block's output
    T* Oblk = Ob + blk * 6 * (int64_t)nn;
    for (int i = threadIdx.x; i < 6 * nq * nE; i += nT) {
      const int pl = i / (nq * nE), rem = i - pl * nq * nE, jb0 = 4 * (rem / nE), ja = rem % nE;
      const int d = pl >> 1, a = eb_axis_a(d), b = eb_axis_b(d);
      const T* SaT = ST[a] + ja;
      const T* Pr = P + (int64_t)pl * nn + (int64_t)jb0 * nE;
      const int nr = min(4, nE - jb0);
      T acc[4] = {0, 0, 0, 0};
      for (int ka = 0; ka < nE; ++ka) {
        const T sv = SaT[(int64_t)ka * nE];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < nr) acc[r] += Pr[r * nE + ka] * sv;
      }
      for (int r = 0; r < nr; ++r) {
        const int jb = jb0 + r;
        int g[3];
        g[d] = eb_global(G, d, cc[d], (pl & 1) ? q1 : q0);
        g[a] = eb_global(G, a, cc[a], ja);
        g[b] = eb_global(G, b, cc[b], jb);
        T v = 0;
        if (g[0] >= 0 && g[1] >= 0 && g[2] >= 0 && eb_unknown(G, g)) {
          const int mult = 1 + (ja == q0 || ja == q1) + (jb == q0 || jb == q1);
          int j[3];
          j[d] = (pl & 1) ? q1 : q0;
          j[a] = ja;
          j[b] = jb;
          v = acc[r] * t.ebW[0][(int64_t)cc[0] * nE + j[0]] * t.ebW[1][(int64_t)cc[1] * nE + j[1]] *
              t.ebW[2][(int64_t)cc[2] * nE + j[2]] / (T)mult;
        }
        Oblk[(int64_t)pl * nn + (int64_t)jb * nE + ja] = v;
      }
    }
  }
}

// du at a skeleton node: the weighted outputs of every block and plane it lies on.
template <typename T>
__global__ void k_eblock_gather(Geo G, const T* __restrict__ Ob, T* __restrict__ du, int accumulate) {
  const int p = G.p, nE = 3 * p - 1, q0 = p - 1, q1 = 2 * p - 1;
  const int64_t nn = (int64_t)nE * nE;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < G.size; s += (int64_t)gridDim.x * blockDim.x) {
    int g[3];
    bool bd;
    skel_decode(G, s, g, &bd);
    if (bd) {
      if (!accumulate) du[s] = 0;
      continue;
    }
    // per axis: the blocks holding the node and its line index in each
    int cs[3][3], js[3][3], nc[3];
    for (int d = 0; d < 3; ++d) {
      const int nd = ncount(G, d);
      const int a = divp(G, g[d]), q = g[d] - a * p;
      nc[d] = 0;
      const int chi = q == 0 ? a : a + 1;  // a vertex plane lies in blocks a-1, a; other nodes in a-1..a+1
      for (int c = a - 1; c <= chi; ++c) {
        int cw = c;
        if (G.per[d]) cw = c < 0 ? c + nd : (c >= nd ? c - nd : c);
        if (cw < 0 || cw >= nd) continue;
        cs[d][nc[d]] = cw;
        js[d][nc[d]] = g[d] - (c - 1) * p - 1;  // offset from the unwrapped centre
        ++nc[d];
      }
    }
    T acc = 0;
    for (int i3 = 0; i3 < nc[2]; ++i3)
      for (int i2 = 0; i2 < nc[1]; ++i2)
        for (int i1 = 0; i1 < nc[0]; ++i1) {
          const int64_t blk = ((int64_t)cs[2][i3] * G.n2 + cs[1][i2]) * G.n1 + cs[0][i1];
          const int j[3] = {js[0][i1], js[1][i2], js[2][i3]};
          const T* ob = Ob + blk * 6 * nn;
          for (int d = 0; d < 3; ++d) {
            if (j[d] != q0 && j[d] != q1) continue;
            const int pl = 2 * d + (j[d] == q1);
            acc += ob[pl * nn + (int64_t)j[eb_axis_b(d)] * nE + j[eb_axis_a(d)]];
          }
        }
    du[s] = accumulate ? du[s] + acc : acc;
  }
}

}  // namespace

template <typename T>
LaunchCfg plan_eblock(const Geo& G, int nsm) {
  LaunchCfg c{};
  const int nE = 3 * G.p - 1;
  const size_t nn = (size_t)nE * nE, es = sizeof(T);
  int ts = (int)((96 * 1024) / (nn * es));
  ts = ts < 1 ? 1 : (ts > nE ? nE : ts);
  const size_t sizes[kEbRegions] = {6 * nn, 6 * nn, (size_t)ts * nn, 9 * (size_t)nE};
  const int order[kEbRegions] = {3, 0, 2, 1};
  size_t smem = 0;
  c.ws = plan_regions(sizes, kEbRegions, es, 200 * 1024, &smem, order);
  c.smem = smem;
  c.block = kEbThreads;
  c.depth = ts;
  int64_t grid = G.nelem < nsm ? G.nelem : nsm;
  c.grid = (int)(grid < 1 ? 1 : grid);
  c.ok = plan_ok(c.ws, sizes, kEbRegions, es, smem);
  return c;
}

template <typename T>
void launch_eblock(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, cudaStream_t st) {
  k_eblock<T><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, c.depth);
}

template <typename T>
void launch_eblock_gather(const Geo& G, const T* Ob, T* du, int accumulate, cudaStream_t st) {
  int64_t g = (G.size + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_eblock_gather<T><<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(G, Ob, du, accumulate);
}

int set_eblock_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_eblock<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_eblock<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

template LaunchCfg plan_eblock<double>(const Geo&, int);
template LaunchCfg plan_eblock<float>(const Geo&, int);
template void launch_eblock<double>(const Geo&, const Tabs<double>&, const double*, double*, double*,
                                    const LaunchCfg&, cudaStream_t);
template void launch_eblock<float>(const Geo&, const Tabs<float>&, const float*, float*, float*, const LaunchCfg&,
                                   cudaStream_t);
template void launch_eblock_gather<double>(const Geo&, const double*, double*, int, cudaStream_t);
template void launch_eblock_gather<float>(const Geo&, const float*, float*, int, cudaStream_t);

}  // namespace semmg
