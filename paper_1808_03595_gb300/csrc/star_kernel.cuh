// Star smoother: Algorithm 2 around Algorithm 1 (Sec. 3.2), one CTA per star.
// Kernel templates; kernels_star_f64.cu and kernels_star_f32.cu instantiate
// them for one element type each (two translation units compile in parallel).
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
#pragma once
#include "semmg_internal.h"

#include <type_traits>

namespace semmg {

namespace {

// Work regions: 0 S tables (3 nS^2; optional), 1 P (3 nS^2), 2 Tt (3 nS^2),
// 3 V slab (ts nS^2), 4 Lam (3 nS) and s3^2 (nS, in a 3 nS slot).
//
// Plane dd (normal to axis dd) is stored [jb][ja] with a = the lower and b
// the higher of the two in-plane axes.  Centrosymmetric lines (every interior
// vertex line of a uniform mesh) have even eigenvectors in columns 0..m and
// odd ones in m+1..2m, so a 1D transform folds the data about the vertex
// (x[m+j] +- x[m-j]) and multiplies with the half-size blocks: half the
// multiply-adds.  Odd eigenvectors vanish at the vertex (s_d[k] = 0 for
// k > m), so the contractions along the normals run over the even half only.

// a / b: IEEE division in FP64, the hardware approximate quotient (about 2 ulp)
// in FP32, where the smoother sits inside FP64 iterative refinement.
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
__device__ __forceinline__ float fast_div(float a, float b) { return a * rcp_approx(b); }

// k3-planes of the eigenspace held at once.
__host__ __device__ __forceinline__ int slab_thickness(int nS) { return star_slab_thickness(nS); }

// The n pairs j = o2 w + o1 of a segment, j strided by the block: the thread's
// first pair and the block-size step, decoded once per star (integer division
// goes through the FP64 pipe, which the FP64 kernel needs for its arithmetic).
struct PairSeg {
  int n, w, b1, b2, q, r, o1, o2;
};

__device__ __forceinline__ PairSeg pair_seg(int n, int w, int b1, int b2) {
  PairSeg s{n, w, b1, b2, 0, 0, 0, 0};
  if (n <= 0 || w <= 0) {
    s.n = 0;
    return s;
  }
  const int nT = blockDim.x;
  s.q = nT / w;
  s.r = nT - s.q * w;
  s.o2 = threadIdx.x / w;
  s.o1 = threadIdx.x - s.o2 * w;
  return s;
}

// f(b1 + o1, b2 + o2) for this thread's pairs of the segment
template <typename F>
__device__ __forceinline__ void for_pairs(const PairSeg& s, F f) {
  int o1 = s.o1, o2 = s.o2;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    f(s.b1 + o1, s.b2 + o2);
    o1 += s.r;
    o2 += s.q;
    if (o1 >= s.w) {
      o1 -= s.w;
      ++o2;
    }
  }
}

// Plane pass helpers: axis index of the fast (a) and slow (b) in-plane axes.
__device__ __forceinline__ int ax_fast(int dd) { return dd == 0 ? 1 : 0; }
__device__ __forceinline__ int ax_slow(int dd) { return dd == 2 ? 1 : 2; }

// Fold (sym) or copy a 3-plane array along the fast (along=0) or slow (along=1) index.
template <typename T>
__device__ __forceinline__ void fold_pass(int nS, int m, const int* sym, int along, const T* X, T* Y) {
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

// ---- grouped passes: each thread computes kG outputs of one line that share
// the input loads (kG independent multiply-add chains per thread).
constexpr int kG = kStarGroup;

// Output block of group g on a line: [k0, k1) and the input range of that block.
struct Block {
  int k0, k1;   // outputs
  int j0, j1;   // folded inputs
  int even;     // 1: even block (inputs j use row m + j), 0: odd block or unfolded (row j)
};

// Index ranges of a star, per axis d: the active range [lo[d], hi[d]) of the
// vertex line (all nS points inside the domain; for a line whose vertex lies
// on a face of the domain, the points on the inner side: m of them beside a
// Dirichlet vertex, m + 1 including a Neumann vertex), and pa[d]: whether the
// plane through the vertex normal to d holds active points (the vertex itself
// is active along d).  Points outside the active ranges are
// identity-padded with zero data, so every sum and every eigen index outside
// them contributes exactly zero and is skipped.
struct Ranges {
  int lo[3], hi[3], pa[3];
};

__device__ __forceinline__ int groups_per_line(int m, int symax, int lo, int hi) {
  return symax ? (m + 1 + kG - 1) / kG + (m + kG - 1) / kG : (hi - lo + kG - 1) / kG;
}

__device__ __forceinline__ Block block_of(int m, int symax, int lo, int hi, int g) {
  Block b;
  if (!symax) {
    b.k0 = lo + g * kG; b.k1 = min(b.k0 + kG, hi); b.j0 = lo; b.j1 = hi; b.even = 0;
  } else {
    const int ge = (m + 1 + kG - 1) / kG;
    if (g < ge) {
      b.k0 = g * kG; b.k1 = min(b.k0 + kG, m + 1); b.j0 = 0; b.j1 = m + 1; b.even = 1;
    } else {
      b.k0 = m + 1 + (g - ge) * kG; b.k1 = min(b.k0 + kG, 2 * m + 1); b.j0 = m + 1; b.j1 = 2 * m + 1; b.even = 0;
    }
  }
  return b;
}

// Work items of a grouped pass: per active plane, the active lines (indexed
// along the other in-plane axis) times the output groups of a line.
struct PassItems {
  int gpl[3], acc[4];
};

__device__ __forceinline__ PassItems pass_items(int m, const int* sym, const Ranges& R, int along) {
  PassItems it;
  it.acc[0] = 0;
  for (int dd = 0; dd < 3; ++dd) {
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const int ox = along == 0 ? ax_slow(dd) : ax_fast(dd);
    it.gpl[dd] = R.pa[dd] ? groups_per_line(m, sym[ax], R.lo[ax], R.hi[ax]) : 0;
    it.acc[dd + 1] = it.acc[dd] + (R.hi[ox] - R.lo[ox]) * it.gpl[dd];
  }
  return it;
}

// Z = forward transform of folded Y along `along` (0: fast index, 1: slow index), grouped.
template <typename T>
__device__ __forceinline__ void tx_pass_g(int nS, int m, const int* sym, const Ranges& R, const T* const* S,
                                          int along, const T* Y, T* Z) {
  const int n2 = nS * nS;
  const PassItems pi = pass_items(m, sym, R, along);
  for (int it = threadIdx.x; it < pi.acc[3]; it += blockDim.x) {
    const int dd = it < pi.acc[1] ? 0 : (it < pi.acc[2] ? 1 : 2);
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const int ox = along == 0 ? ax_slow(dd) : ax_fast(dd);
    const int r = it - pi.acc[dd], line = R.lo[ox] + r / pi.gpl[dd], g = r % pi.gpl[dd];
    const Block b = block_of(m, sym[ax], R.lo[ax], R.hi[ax], g);
    const T* Sa = S[ax];
    const T* y = Y + dd * n2 + (along == 0 ? line * nS : line);
    const int ys = along == 0 ? 1 : nS;
    T a[kG];
#pragma unroll
    for (int q = 0; q < kG; ++q) a[q] = 0;
    for (int j = b.j0; j < b.j1; ++j) {
      const T yv = y[j * ys];
      const T* sr = Sa + (b.even ? m + j : j) * nS + b.k0;
#pragma unroll
      for (int q = 0; q < kG; ++q)
        if (b.k0 + q < b.k1) a[q] += sr[q] * yv;
    }
    T* z = Z + dd * n2;
#pragma unroll
    for (int q = 0; q < kG; ++q)
      if (b.k0 + q < b.k1) z[along == 0 ? line * nS + b.k0 + q : (b.k0 + q) * nS + line] = a[q];
  }
}

// Y = transposed transform into folded form (E_j / O_j), grouped over outputs j.
template <typename T>
__device__ __forceinline__ void txT_pass_g(int nS, int m, const int* sym, const Ranges& R, const T* const* S,
                                           int along, const T* B, T* Y) {
  const int n2 = nS * nS;
  const PassItems pi = pass_items(m, sym, R, along);
  for (int it = threadIdx.x; it < pi.acc[3]; it += blockDim.x) {
    const int dd = it < pi.acc[1] ? 0 : (it < pi.acc[2] ? 1 : 2);
    const int ax = along == 0 ? ax_fast(dd) : ax_slow(dd);
    const int ox = along == 0 ? ax_slow(dd) : ax_fast(dd);
    const int r = it - pi.acc[dd], line = R.lo[ox] + r / pi.gpl[dd], g = r % pi.gpl[dd];
    // the group's outputs are folded positions [k0, k1); their sums run over the
    // eigen-index block of the same parity, [j0, j1) (same ranges as the forward pass)
    const Block blk = block_of(m, sym[ax], R.lo[ax], R.hi[ax], g);
    const T* Sa = S[ax];
    const T* bb = B + dd * n2 + (along == 0 ? line * nS : line);
    const int bs = along == 0 ? 1 : nS;
    T a[kG];
    const T* sr[kG];
#pragma unroll
    for (int q = 0; q < kG; ++q) {
      a[q] = 0;
      const int jo = min(blk.k0 + q, blk.k1 - 1);
      sr[q] = Sa + (blk.even ? m + jo : jo) * nS;
    }
    for (int k = blk.j0; k < blk.j1; ++k) {
      const T bv = bb[k * bs];
#pragma unroll
      for (int q = 0; q < kG; ++q) a[q] += sr[q][k] * bv;
    }
    T* yv = Y + dd * n2;
#pragma unroll
    for (int q = 0; q < kG; ++q)
      if (blk.k0 + q < blk.k1) yv[along == 0 ? line * nS + blk.k0 + q : (blk.k0 + q) * nS + line] = a[q];
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

// PC > 0 compiles the kernel for degree PC (constant extents, unrolled loops);
// PC = 0 takes the degree from G.
template <typename T, int PC, int NB>
__global__ void __launch_bounds__(512, NB) k_star(Geo G, Tabs<T> t, const T* __restrict__ r, T* __restrict__ Ob,
                                               T* ws, WsPlan wp, int S_copy, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  __shared__ int s_sym[3];
  __shared__ Ranges s_rg;
  __shared__ int Ac[3 * (2 * SEMMG_MAX_DEGREE - 1)];  // active flags of the three vertex lines
  const int p = PC ? PC : G.p, m = p - 1, nS = 2 * p - 1, n2 = nS * nS;
  T* Sbuf = ws_ptr<T>(wp, 0, smem_raw, ws);
  T* P = ws_ptr<T>(wp, 1, smem_raw, ws);
  T* Tt = ws_ptr<T>(wp, 2, smem_raw, ws);
  T* V = ws_ptr<T>(wp, 3, smem_raw, ws);
  T* Lm = ws_ptr<T>(wp, 4, smem_raw, ws);
  T* s3sq = Lm + 3 * nS;  // s3[k]^2
  const T lam = (T)G.lam;
  // 1 / (number of planes a node lies on): 1, 2 or 3 planes
  const T rcp_mult[3] = {(T)1, (T)0.5, (T)1 / (T)3};
  // position in the star order (most work first when the level has an order table)
  int64_t it = blockIdx.x;
  while (it < G.nstar) {
    const int64_t st = t.order ? (int64_t)t.order[it] : it;
    const int c[3] = {(int)(st % G.nv1), (int)((st / G.nv1) % G.nv2), (int)(st / ((int64_t)G.nv1 * G.nv2))};
    // the last vertex plane of a periodic axis repeats plane 0: its stars are never read
    const bool alias = (G.per[0] && c[0] == G.n1) || (G.per[1] && c[1] == G.n2) || (G.per[2] && c[2] == G.n3);
    if (!alias) {
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
        Ac[d * nS + i] = t.act[d][(int64_t)c[d] * nS + i];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nS; i += blockDim.x) {
      const T v = S[2][m * nS + i];
      s3sq[i] = v * v;
    }
    if (threadIdx.x < 3) {
      const int d = threadIdx.x;
      int lo = 0, hi = nS;
      while (lo < nS && !Ac[d * nS + lo]) ++lo;
      while (hi > lo && !Ac[d * nS + hi - 1]) --hi;
      s_rg.lo[d] = lo;
      s_rg.hi[d] = hi;
      s_rg.pa[d] = Ac[d * nS + m];
    }
    __syncthreads();
    const int* sym = s_sym;
    const Ranges rg = s_rg;
    // 1. gather the three planes, divided by the multiplicity, zero where not a star node
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS - m, ja = rr % nS - m;
      const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
      T v = 0;
      if (Ac[dd * nS + m] && Ac[ax_a * nS + ja + m] && Ac[ax_b * nS + jb + m])
        v = r[star_plane_slot(G, dd, c[0], c[1], c[2], ja, jb)] * rcp_mult[(ja == 0) + (jb == 0)];
      P[idx] = v;
    }
    __syncthreads();
    // 2a. in-plane transforms A = S_b^T P S_a (fold, transform; fast then slow index)
    fold_pass(nS, m, sym, 0, P, Tt);
    __syncthreads();
    tx_pass_g(nS, m, sym, rg, S, 0, Tt, P);
    __syncthreads();
    fold_pass(nS, m, sym, 1, P, Tt);
    __syncthreads();
    tx_pass_g(nS, m, sym, rg, S, 1, Tt, P);
    __syncthreads();
    // 2b + 3 + 4a. expansion along the normals with the vertex rows, times 1/D,
    // and the contractions back along the normals, in slabs of `ts` k3-planes
    // held in shared memory: B1[k3][k2] = sum_k1 s1 V and B2[k3][k1] = sum_k2 s2 V
    // per slab, B3[k2][k1] = sum_k3 s3 V accumulated over the slabs.
    // Odd eigenvectors vanish at the vertex, so on symmetric axes the sums run
    // over the even half only.  Results land in Tt (B1, B2, B3).
    const T* s1 = S[0] + m * nS;
    const T* s2 = S[1] + m * nS;
    const T* s3 = S[2] + m * nS;
    const int64_t n3 = (int64_t)n2 * nS;
    const T* R = nullptr;
    if (t.Rtab && sizeof(T) == sizeof(double)) {
      const int64_t cls = ((int64_t)t.starCls[0][c[0]] * t.ncls[1] + t.starCls[1][c[1]]) * t.ncls[2] + t.starCls[2][c[2]];
      R = t.Rtab + cls * n3;
    }
    // live ranges [lo_d, lo_d + nz_d) of the vertex rows: s_d[k] may be non-zero
    // only there (odd eigenvectors vanish at the vertex; a vertex on a Dirichlet
    // face makes the whole row zero on the active range)
    const int lo1 = rg.lo[0], w1 = rg.hi[0] - rg.lo[0], lo2 = rg.lo[1], w2 = rg.hi[1] - rg.lo[1];
    const int lo3 = rg.lo[2], w3 = rg.hi[2] - rg.lo[2];
    const int nz1 = rg.pa[0] ? (sym[0] ? m + 1 : w1) : 0;
    const int nz2 = rg.pa[1] ? (sym[1] ? m + 1 : w2) : 0;
    const int nz3 = rg.pa[2] ? (sym[2] ? m + 1 : w3) : 0;
    // (k1, k2) pairs in three segments, each its own loop so that warps stay on
    // one branch: k2 live (any k1), then k2 dead with k1 live, then both dead (only
    // the x3-plane term, so only when that plane is active); the live k_d are the
    // first nz_d indices of the active range
    const int seg1 = nz2 * w1, seg2 = (w2 - nz2) * nz1, nlive = seg1 + seg2;
    const int npair = nlive + (rg.pa[2] ? (w2 - nz2) * (w1 - nz1) : 0);
    const int ts = slab_thickness(nS);
    // the four pair segments (the same for every slab of the star)
    const PairSeg sg_both = pair_seg(nz2 * nz1, nz1, lo1, lo2);                  // k1, k2 live
    const PairSeg sg_k2 = pair_seg(nz2 * (w1 - nz1), w1 - nz1, lo1 + nz1, lo2);  // k2 live, k1 dead
    const PairSeg sg_k1 = pair_seg(seg2, nz1, lo1, lo2 + nz2);                    // k1 live, k2 dead
    const PairSeg sg_dead = pair_seg(rg.pa[2] ? npair - nlive : 0, w1 - nz1, lo1 + nz1, lo2 + nz2);
    T* B1 = Tt;
    T* B2 = Tt + n2;
    T* B3 = Tt + 2 * n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) B3[i] = 0;
    for (int k3s = rg.lo[2]; k3s < rg.hi[2]; k3s += ts) {
      const int tn = rg.hi[2] - k3s < ts ? rg.hi[2] - k3s : ts;
      __syncthreads();
      // which = 0: s1[k1] and s2[k2] may both be non-zero; 1: only s1[k1] (k2 dead);
      // 2: only s2[k2] (k1 dead) -- the zero term is left out
      auto live = [&](auto which, int k1, int k2) {
        constexpr int W = decltype(which)::value;
        const int pr = k2 * nS + k1;
        const T a3 = rg.pa[2] ? P[2 * n2 + pr] : (T)0;
        {
          const T c1 = k1 - lo1 < nz1 ? s1[k1] : (T)0, c2 = k2 - lo2 < nz2 ? s2[k2] : (T)0;
          T b3 = 0;
          // bounded by the slab thickness, a constant in the degree-specialised builds
#pragma unroll
          for (int kk = 0; kk < ts; ++kk) {
            if (kk >= tn) break;
            const int k3 = k3s + kk;
            T E;
            if constexpr (W == 0) E = c1 * P[k3 * nS + k2] + c2 * P[n2 + k3 * nS + k1];
            if constexpr (W == 1) E = c1 * P[k3 * nS + k2];
            if constexpr (W == 2) E = c2 * P[n2 + k3 * nS + k1];
            if (k3 - lo3 < nz3) E += s3[k3] * a3;
            const int64_t pt = (int64_t)k3 * n2 + pr;
            const T v = R ? E * R[pt] : fast_div(E, lam + Lm[k1] + Lm[nS + k2] + Lm[2 * nS + k3]);
            V[kk * n2 + pr] = v;
            if (k3 - lo3 < nz3) b3 += s3[k3] * v;
          }
          if (nz3) B3[pr] += b3;
        }
      };
      auto live_both = [&](int k1, int k2) { live(std::integral_constant<int, 0>{}, k1, k2); };
      auto live_1 = [&](int k1, int k2) { live(std::integral_constant<int, 1>{}, k1, k2); };
      auto live_2 = [&](int k1, int k2) { live(std::integral_constant<int, 2>{}, k1, k2); };
      auto dead = [&](int k1, int k2) {
        const int pr = k2 * nS + k1;
        const T a3 = rg.pa[2] ? P[2 * n2 + pr] : (T)0;
        {
          // s1[k1] = s2[k2] = 0: V = s3 a3 / D is read only by B3, which gets
          // a3 sum_k3 s3^2 / D
          T b3 = 0;
          for (int kk = 0; kk < tn; ++kk) {
            const int k3 = k3s + kk;
            if (k3 - lo3 >= nz3) break;
            const int64_t pt = (int64_t)k3 * n2 + pr;
            b3 += R ? s3sq[k3] * R[pt] : fast_div(s3sq[k3], lam + Lm[k1] + Lm[nS + k2] + Lm[2 * nS + k3]);
          }
          B3[pr] += a3 * b3;
        }
      };
      for_pairs(sg_both, live_both);
      for_pairs(sg_k2, live_2);
      for_pairs(sg_k1, live_1);
      for_pairs(sg_dead, dead);
      __syncthreads();
      // B1[k3][k2] = sum_k1 s1 V (plane 0 active), B2[k3][k1] = sum_k2 s2 V (plane 1 active)
      const int nb1 = rg.pa[0] ? tn * w2 : 0, nb2 = rg.pa[1] ? tn * w1 : 0;
      if constexpr (sizeof(T) == sizeof(double)) {
        // four consecutive lanes per output, lane q summing the terms k = q (mod 4) of the
        // full groups of four and lane 0 also the leftover ones -- the four partial sums and
        // their combination (s0 + s1) + (s2 + s3) of a one-thread four-chain loop
        const int nq = 4 * (nb1 + nb2);
        for (int base = 0; base < nq; base += blockDim.x) {  // same trip count for every thread
          const int o4 = base + (int)threadIdx.x, q = o4 & 3, o = o4 >> 2;
          T sq = 0;
          bool first = false;
          int kk = 0, kx = 0;
          if (o4 < nq) {
            first = o < nb1;
            const int wx = first ? w2 : w1;
            int rr = first ? o : o - nb1;
            while (rr >= wx) {  // rr / wx < tn <= slab depth: subtract instead of dividing
              rr -= wx;
              ++kk;
            }
            kx = (first ? lo2 : lo1) + rr;
            const T* vs = V + kk * n2;
            const int nz = first ? nz1 : nz2, full = nz & ~3;
            const T* sv = first ? s1 + lo1 : s2 + lo2;
            const T* v = first ? vs + kx * nS + lo1 : vs + kx + lo2 * nS;
            const int vst = first ? 1 : nS;
            for (int k = q; k < full; k += 4) sq += sv[k] * v[k * vst];
            if (q == 0)
              for (int k = full; k < nz; ++k) sq += sv[k] * v[k * vst];
          }
          const T t1 = sq + __shfl_down_sync(0xffffffffu, sq, 1, 4);  // lanes 0, 2: s0 + s1, s2 + s3
          const T t2 = t1 + __shfl_down_sync(0xffffffffu, t1, 2, 4);  // lane 0: (s0 + s1) + (s2 + s3)
          if (o4 < nq && q == 0) {
            if (first)
              B1[(k3s + kk) * nS + kx] = t2;
            else
              B2[(k3s + kk) * nS + kx] = t2;
          }
        }
      } else {
        // one thread per output, four independent partial sums
        for (int o = threadIdx.x; o < nb1 + nb2; o += blockDim.x) {
          const bool first = o < nb1;
          const int wx = first ? w2 : w1;
          int rr = first ? o : o - nb1, kk = 0;
          while (rr >= wx) {  // rr / wx < tn <= slab depth: subtract instead of dividing
            rr -= wx;
            ++kk;
          }
          const int kx = (first ? lo2 : lo1) + rr;
          const T* vs = V + kk * n2;
          T s = 0;
          T s_1 = 0, s_2 = 0, s_3 = 0;  // four independent partial sums
          if (first) {  // sum over k1
            const T* v = vs + kx * nS + lo1;
            const T* sv = s1 + lo1;
            int k = 0;
            for (; k + 3 < nz1; k += 4) {
              s += sv[k] * v[k];
              s_1 += sv[k + 1] * v[k + 1];
              s_2 += sv[k + 2] * v[k + 2];
              s_3 += sv[k + 3] * v[k + 3];
            }
            for (; k < nz1; ++k) s += sv[k] * v[k];
            B1[(k3s + kk) * nS + kx] = (s + s_1) + (s_2 + s_3);
          } else {      // sum over k2
            const T* v = vs + kx + lo2 * nS;
            const T* sv = s2 + lo2;
            int k = 0;
            for (; k + 3 < nz2; k += 4) {
              s += sv[k] * v[k * nS];
              s_1 += sv[k + 1] * v[(k + 1) * nS];
              s_2 += sv[k + 2] * v[(k + 2) * nS];
              s_3 += sv[k + 3] * v[(k + 3) * nS];
            }
            for (; k < nz2; ++k) s += sv[k] * v[k * nS];
            B2[(k3s + kk) * nS + kx] = (s + s_1) + (s_2 + s_3);
          }
        }
      }
    }
    __syncthreads();
    // 4b. back to the planes: O = S_b B S_a^T (slow index first, then fast)
    txT_pass_g(nS, m, sym, rg, S, 1, Tt, P);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, row = rr / nS, col = rr - row * nS;
      Tt[idx] = unfold_value(nS, m, sym, 1, P, dd, row, col);
    }
    __syncthreads();
    txT_pass_g(nS, m, sym, rg, S, 0, Tt, P);
    __syncthreads();
    T* ob = Ob + st * 3 * (int64_t)n2;
    for (int idx = threadIdx.x; idx < 3 * n2; idx += blockDim.x) {
      const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS, ja = rr % nS;
      const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
      const T s = unfold_value(nS, m, sym, 0, P, dd, jb, ja);
      const bool active = Ac[dd * nS + m] && Ac[ax_a * nS + ja] && Ac[ax_b * nS + jb];
      const int oa = ja - m, obb = jb - m;
      const T wgt = t.w1d[oa < 0 ? -oa : oa] * t.w1d[obb < 0 ? -obb : obb] * rcp_mult[(oa == 0) + (obb == 0)];
      ob[idx] = active ? wgt * s : (T)0;
    }
    }  // !alias
    // next star: from the shared counter when given (dynamic balance), else grid-strided
    if (counter) {
      __syncthreads();
      if (threadIdx.x == 0) s_next = atomicAdd(&counter[0], 1) + (int)gridDim.x;
      __syncthreads();
      it = s_next;
    } else {
      it += gridDim.x;
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

constexpr size_t kStarSmemCap = 200 * 1024;

}  // namespace

template <typename T>
LaunchCfg plan_star(const Geo& G, int nsm, size_t cap, int block, int wide) {
  LaunchCfg c;
  if (cap == 0) cap = kStarSmemCap;
  const size_t nS = G.nS, n2 = nS * nS;
  const size_t sizes[5] = {3 * n2, 3 * n2, 3 * n2, (size_t)slab_thickness((int)nS) * n2, 6 * nS};
  // priority: small tables, planes, transform temp, eigenspace slab, S tables
  const int order[5] = {4, 1, 2, 3, 0};
  c.ws = plan_regions(sizes, 5, sizeof(T), cap, &c.smem, order);
  c.ok = plan_ok(c.ws, sizes, 5, sizeof(T), c.smem);
  c.block = block ? block : (c.smem > 100 * 1024 ? 512 : 256);  // a block that owns the SM brings more warps
  const int bps = resident_blocks(c, wide);
  const int64_t grid = (int64_t)nsm * bps;
  c.grid = (int)(G.nstar < grid ? G.nstar : grid);
  if (c.grid < 1) c.grid = 1;
  return c;
}

template <typename T, int NB>
void launch_star_nb(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, int* counter,
                    cudaStream_t st) {
  // copy the S tables into the CTA's work memory only when that is shared memory
  const int S_copy = c.ws.in_smem[0];
  switch (G.p) {
    case 2: k_star<T, 2, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
    case 4: k_star<T, 4, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
    case 8: k_star<T, 8, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
    case 16: k_star<T, 16, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
    case 32: k_star<T, 32, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
    default: k_star<T, 0, NB><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, ws, c.ws, S_copy, counter); break;
  }
}

template <typename T>
void launch_star(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, int* counter,
                 cudaStream_t st) {
  if (G.nstar == 0 || !c.ok) return;
  if (c.wide)
    launch_star_nb<T, 1>(G, t, r, Ob, ws, c, counter, st);
  else
    launch_star_nb<T, 2>(G, t, r, Ob, ws, c, counter, st);
}

template <typename T, int NB>
static int star_attrs_nb() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_star<T, 0, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<T, 2, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<T, 4, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<T, 8, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<T, 16, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star<T, 32, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

template <typename T>
static int star_attrs() {
  return star_attrs_nb<T, 1>() | star_attrs_nb<T, 2>();
}

}  // namespace semmg
