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
//
// The interior block is centrosymmetric, so Sref splits into even and odd
// eigenvectors (columns 0..ne-1 even, ne..m-1 odd, ne = (m+1)/2): every 1D
// transform folds a line about its middle and multiplies half-size blocks,
// and a_p[k] = +a_0[k] (even k) / -a_0[k] (odd k), so the two faces of one
// axis enter as their sum (even k_d) and difference (odd k_d).  1/D comes from
// a table per distinct width triple when one was built.
#pragma once
#include "semmg_internal.h"

namespace semmg {

namespace {

// The threads working on one element: the CTA, or the two CTAs of a cluster.
// Work items are spread over all of them (id, n) and phases are separated by
// sync(): a CTA barrier, or a cluster barrier with release / acquire
// semantics, which orders the global-memory work arrays the two CTAs share.
struct Team {
  int id, n, cs;
  __device__ __forceinline__ static Team block() { return Team{(int)threadIdx.x, (int)blockDim.x, 1}; }
  __device__ __forceinline__ void sync() const {
    if (cs == 1)
      __syncthreads();
    else
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  }
};

// The team of a kernel launched with clusters of cs CTAs (cs = 1: no clusters).
__device__ __forceinline__ Team team_of(int cs) {
  unsigned rank = 0;
  if (cs > 1) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  return Team{(int)(rank * blockDim.x + threadIdx.x), (int)(cs * blockDim.x), cs};
}

template <typename T>
struct ElemScal {
  T sf[3];      // c_f alpha_d for the two faces of axis d
  T al[3];      // alpha_d alone (faces transformed beforehand, scaled by c_f there)
  T e[3];       // 4 / h_d^2
  int64_t cls;  // width-class triple of the element (for the 1/D table)
  // sf[d] and al[d] for a run-time axis d, by selection: an indexed read would
  // place the whole struct in local memory
  __device__ __forceinline__ T sfd(int d) const { return d == 0 ? sf[0] : (d == 1 ? sf[1] : sf[2]); }
  __device__ __forceinline__ T ald(int d) const { return d == 0 ? al[0] : (d == 1 ? al[1] : al[2]); }
};

template <typename T>
__device__ __forceinline__ ElemScal<T> elem_scalars(const Tabs<T>& t, int a1, int a2, int a3) {
  ElemScal<T> s;
  // c_f = sqrt(h_a h_b) / 2 and alpha_d = (2/h_d)^(3/2) from the per-width tables
  const T* x1 = t.hx[0] + 6 * a1;
  const T* x2 = t.hx[1] + 6 * a2;
  const T* x3 = t.hx[2] + 6 * a3;
  s.sf[0] = (T)0.5 * x2[3] * x3[3] * x1[4];
  s.sf[1] = (T)0.5 * x1[3] * x3[3] * x2[4];
  s.sf[2] = (T)0.5 * x1[3] * x2[3] * x3[4];
  s.al[0] = x1[4];
  s.al[1] = x2[4];
  s.al[2] = x3[4];
  s.e[0] = x1[2];
  s.e[1] = x2[2];
  s.e[2] = x3[2];
  s.cls = ((int64_t)t.hcls[0][a1] * t.nhcls[1] + t.hcls[1][a2]) * t.nhcls[2] + t.hcls[2][a3];
  return s;
}

// ---------------------------------------------------------------- folded line transforms
// Arrays are [D2][D1][D0] (D0 fastest); a line runs along axis ax (0: D0, 1:
// D1, 2: D2) and has n = m points.  Folded coordinates of a line: even
// position j < ne pairs points h+j and n-1-(h+j) (h = n/2), odd position
// q >= ne pairs points q and n-1-q.

struct Lines {
  int n, h, ne, D0, D1, total;
  __device__ __forceinline__ int stride(int ax) const { return ax == 0 ? 1 : (ax == 1 ? D0 : D0 * D1); }
  __device__ __forceinline__ int pos(int idx, int ax) const {
    return ax == 0 ? idx % D0 : (ax == 1 ? (idx / D0) % D1 : idx / (D0 * D1));
  }
};

// The float-float builds of the line operations run as straight-line code: a float-float
// step is long (about twelve FP32 operations), so unrolling costs little code and removes the
// loop's own instructions, and selects in place of branches keep a warp's lanes together.
// FP64 and FP32 builds keep the compiler's choices (their 64-register builds would spill).
template <typename T>
constexpr bool kStraight = std::is_same<T, ff>::value;

template <typename T>
__device__ __forceinline__ void fold_lines(const Lines& L, int ax, const T* X, T* Y, const Team& tm = Team::block()) {
  const int str = L.stride(ax);
  for (int idx = tm.id; idx < L.total; idx += tm.n) {
    const int j = L.pos(idx, ax);
    const int base = idx - j * str;
    T v;
    if constexpr (kStraight<T>) {
      // E_j = x[h + j] + x[n-1-h-j] (the middle point alone), O_j = x[j] - x[n-1-j]
      const bool ev = j < L.ne;
      const int i = ev ? L.h + j : j, mi = L.n - 1 - i;
      const T xb = X[base + mi * str];
      v = X[base + i * str] + (ev ? (i == mi ? T(0) : xb) : -xb);
    } else if (j < L.ne) {
      const int i = L.h + j, mi = L.n - 1 - i;
      v = (i == mi) ? X[base + i * str] : X[base + i * str] + X[base + mi * str];
    } else {
      v = X[base + j * str] - X[base + (L.n - 1 - j) * str];
    }
    Y[idx] = v;
  }
}

// ---- grouped line transforms: each thread computes kG outputs of one line
// that share the input loads (independent multiply-add chains).
constexpr int kG = 4;

__device__ __forceinline__ int nlines(const Lines& L) { return L.total / L.n; }

// First element and stride of line l along axis ax.
__device__ __forceinline__ void line_of(const Lines& L, int ax, int l, int* base, int* str, int* i2) {
  if (ax == 0) {
    *base = l * L.D0;
    *str = 1;
    *i2 = l / L.D1;
  } else if (ax == 1) {
    const int a2 = l / L.D0, a0 = l - a2 * L.D0;
    *base = a2 * L.D1 * L.D0 + a0;
    *str = L.D0;
    *i2 = a2;
  } else {
    *base = l;
    *str = L.D0 * L.D1;
    *i2 = 0;
  }
}

__device__ __forceinline__ int line_groups(const Lines& L) {
  return (L.ne + kG - 1) / kG + (L.n - L.ne + kG - 1) / kG;
}

// Outputs k0, k0 + ks, k0 + 2 ks, ... below k1 of group g, and the folded input range
// [j0, j1); even: inputs use row h + j.  The groups of a half interleave (stride ks = the
// half's number of groups), so the neighbouring groups of a warp read neighbouring entries
// of S at each step: no shared-memory bank conflicts between them.
__device__ __forceinline__ void line_block(const Lines& L, int g, int* k0, int* ks, int* k1, int* j0, int* j1,
                                           int* even) {
  const int ge = (L.ne + kG - 1) / kG, go = (L.n - L.ne + kG - 1) / kG;
  if (g < ge) {
    *k0 = g;
    *ks = ge;
    *k1 = L.ne;
    *j0 = 0;
    *j1 = L.ne;
    *even = 1;
  } else {
    *k0 = L.ne + (g - ge);
    *ks = go;
    *k1 = L.n;
    *j0 = L.ne;
    *j1 = L.n;
    *even = 0;
  }
}

// The input loops below run over the odd half's length tc = n - ne for every group, so that
// all lanes of a warp take the same trip count (known at compile time where n is); the even
// half's one extra input (n odd) is added after them.  Each output's terms are summed in
// input order.

// Z = (scale or sc2[i2]) * forward transform of folded Y along ax.
template <typename T>
__device__ __forceinline__ void tx_lines_g(const Lines& L, int ax, const T* __restrict__ S, const T* Y, T* Z,
                                           T scale, const T* sc2, const Team& tm = Team::block()) {
  const int G = line_groups(L), n = L.n, tc = L.n - L.ne;
  const int items = nlines(L) * G;
  for (int it = tm.id; it < items; it += tm.n) {
    const int l = it / G, g = it - l * G;
    int base, str, i2, k0, ks, k1, j0, j1, even;
    line_of(L, ax, l, &base, &str, &i2);
    line_block(L, g, &k0, &ks, &k1, &j0, &j1, &even);
    const T* yp = Y + base + j0 * str;
    const T* sp = S + (even ? L.h : L.ne) * n + k0;  // row of input j0, first output column
    // column offsets of the outputs; in the float-float build a slot past the group's end
    // repeats its last column (summed, not stored), so that every step is the same
    // straight-line code; the other builds skip that slot
    int kq[kG];
    Acc<T> a[kG];
#pragma unroll
    for (int q = 0; q < kG; ++q) {
      a[q] = Acc<T>::zero();
      kq[q] = kStraight<T> ? min(q * ks, k1 - 1 - k0) : q * ks;
    }
    auto step = [&](int t) {
      const T yv = yp[t * str];
      const T* sr = sp + t * n;
#pragma unroll
      for (int q = 0; q < kG; ++q) {
        if constexpr (kStraight<T>)
          a[q].add(sr[kq[q]], yv);
        else if (k0 + q * ks < k1)
          a[q].add(sr[q * ks], yv);
      }
    };
    if constexpr (kStraight<T>) {
#pragma unroll 4
      for (int t = 0; t < tc; ++t) step(t);
    } else {
      for (int t = 0; t < tc; ++t) step(t);
    }
    if (j1 - j0 > tc) step(tc);
    const T s = sc2 ? sc2[i2] : scale;
#pragma unroll
    for (int q = 0; q < kG; ++q)
      if (k0 + q * ks < k1) Z[base + (k0 + q * ks) * str] = s * a[q].value();
  }
}

// Y = transposed transform of B along ax into folded form (E_j, O_q).
template <typename T>
__device__ __forceinline__ void txT_lines_g(const Lines& L, int ax, const T* __restrict__ S, const T* B, T* Y,
                                            const Team& tm = Team::block()) {
  const int G = line_groups(L), n = L.n, tc = L.n - L.ne;
  const int items = nlines(L) * G;
  for (int it = tm.id; it < items; it += tm.n) {
    const int l = it / G, g = it - l * G;
    int base, str, i2, k0, ks, k1, j0, j1, even;
    line_of(L, ax, l, &base, &str, &i2);
    line_block(L, g, &k0, &ks, &k1, &j0, &j1, &even);
    const T* bp = B + base + j0 * str;
    Acc<T> a[kG];
    const T* sr[kG];
#pragma unroll
    for (int q = 0; q < kG; ++q) {
      a[q] = Acc<T>::zero();
      const int jo = min(k0 + q * ks, k1 - 1);
      sr[q] = S + (even ? L.h + jo : jo) * n + j0;
    }
    auto step = [&](int t) {
      const T bv = bp[t * str];
#pragma unroll
      for (int q = 0; q < kG; ++q) a[q].add(sr[q][t], bv);
    };
    if constexpr (kStraight<T>) {
#pragma unroll 4
      for (int t = 0; t < tc; ++t) step(t);
    } else {
      for (int t = 0; t < tc; ++t) step(t);
    }
    if (j1 - j0 > tc) step(tc);
#pragma unroll
    for (int q = 0; q < kG; ++q)
      if (k0 + q * ks < k1) Y[base + (k0 + q * ks) * str] = a[q].value();
  }
}

// Natural-order value at element idx from folded E/O data.
template <typename T>
__device__ __forceinline__ T unfold_at(const Lines& L, int ax, const T* Y, int idx) {
  const int str = L.stride(ax);
  const int i = L.pos(idx, ax);
  const int base = idx - i * str;
  const int mi = L.n - 1 - i;
  if constexpr (kStraight<T>) {
    // u = max(i, mi): E at u - h plus (i > mi) or minus (i < mi) O at u; the middle point E alone
    const int u = i > mi ? i : mi;
    const T ob = Y[base + u * str];
    return Y[base + (u - L.h) * str] + (i == mi ? T(0) : (i > mi ? ob : -ob));
  }
  if (i == mi) return Y[base + (i - L.h) * str];
  if (i > mi) return Y[base + (i - L.h) * str] + Y[base + i * str];
  return Y[base + (mi - L.h) * str] - Y[base + mi * str];
}

template <typename T>
__device__ __forceinline__ void unfold_lines(const Lines& L, int ax, const T* Y, T* X, const Team& tm = Team::block()) {
  for (int idx = tm.id; idx < L.total; idx += tm.n) X[idx] = unfold_at(L, ax, Y, idx);
}

// ---------------------------------------------------------------- face helpers
// Six faces X[f][ib][ia] (f = 2d + side) -> pair sums and differences
// X[2d] = X[2d] + X[2d+1], X[2d+1] = X[2d] - X[2d+1].
template <typename T>
__device__ __forceinline__ void face_pairs(int mm, T* X, const Team& tm = Team::block()) {
  for (int idx = tm.id; idx < 3 * mm; idx += tm.n) {
    const int d = idx / mm, r = idx - d * mm;
    const T a = X[(2 * d) * mm + r], b = X[(2 * d + 1) * mm + r];
    X[(2 * d) * mm + r] = a + b;
    X[(2 * d + 1) * mm + r] = a - b;
  }
}

// forward 2D transform of the six face arrays, scaled by c_f alpha_d
template <typename T>
__device__ __forceinline__ void faces_forward(const Lines& F, const T* Sh, T* X, T* Tt, const ElemScal<T>& sc,
                                              const Team& tm = Team::block()) {
  __shared__ T sc6[6];
  if (threadIdx.x < 6) sc6[threadIdx.x] = sc.sfd(threadIdx.x >> 1);
  fold_lines(F, 0, X, Tt, tm);
  tm.sync();
  tx_lines_g(F, 0, Sh, Tt, X, (T)1, (const T*)nullptr, tm);
  tm.sync();
  fold_lines(F, 1, X, Tt, tm);
  tm.sync();
  tx_lines_g(F, 1, Sh, Tt, X, (T)1, (const T*)sc6, tm);
  tm.sync();
}

// Back transform of the six reduced arrays (pairs: even / odd parts of axis d)
// and store of both faces: Z[2d] = sf (Ye + Yo), Z[2d+1] = sf (Ye - Yo).
template <typename T, typename Store>
__device__ __forceinline__ void faces_backward(const Lines& F, const T* Sh, T* X, T* Tt, const ElemScal<T>& sc, Store store,
                                               const Team& tm = Team::block()) {
  txT_lines_g(F, 0, Sh, X, Tt, tm);
  tm.sync();
  unfold_lines(F, 0, Tt, X, tm);
  tm.sync();
  txT_lines_g(F, 1, Sh, X, Tt, tm);
  tm.sync();
  const int mm = F.D0 * F.D1;
  for (int idx = tm.id; idx < 3 * mm; idx += tm.n) {
    const int d = idx / mm, r = idx - d * mm;
    const T ye = unfold_at(F, 1, Tt, (2 * d) * mm + r);
    const T yo = unfold_at(F, 1, Tt, (2 * d + 1) * mm + r);
    store((2 * d) * mm + r, sc.sfd(d) * (ye + yo));
    store((2 * d + 1) * mm + r, sc.sfd(d) * (ye - yo));
  }
}

// Face contribution at eigen-point k from the pair sums (even k_d) / differences (odd k_d).
template <typename T>
__device__ __forceinline__ T face_expand(int m, int ne, const T* a0, const T* X, int k1, int k2, int k3) {
  const int mm = m * m;
  return a0[k1] * X[(k1 < ne ? 0 : 1) * mm + k3 * m + k2] + a0[k2] * X[(k2 < ne ? 2 : 3) * mm + k3 * m + k1] +
         a0[k3] * X[(k3 < ne ? 4 : 5) * mm + k2 * m + k1];
}

// X[2d + parity][kb][ka] <- sum over k_d of that parity of a0[k_d] W(k)
template <typename T>
__device__ __forceinline__ void faces_reduce(int m, int ne, const T* a0, const T* W, T* X, const Team& tm = Team::block()) {
  const int mm = m * m;
  for (int idx = tm.id; idx < 6 * mm; idx += tm.n) {
    const int f = idx / mm, r = idx - f * mm, kb = r / m, ka = r - kb * m;
    const int k0 = (f & 1) ? ne : 0, k1 = (f & 1) ? m : ne;
    const T* w;
    int ws;
    switch (f >> 1) {
      case 0: w = W + (kb * m + ka) * m; ws = 1; break;
      case 1: w = W + kb * mm + ka; ws = m; break;
      default: w = W + kb * m + ka; ws = mm; break;
    }
    T s0 = 0, s1 = 0;  // two independent partial sums
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      s0 = madd(a0[k], w[k * ws], s0);
      s1 = madd(a0[k + 1], w[(k + 1) * ws], s1);
    }
    if (k < k1) s0 = madd(a0[k], w[k * ws], s0);
    X[idx] = s0 + s1;
  }
}

// The Schur kernel's reduction order: faces 0..3 (sums over k1 or k2 at fixed
// k3) as in faces_reduce; faces 4, 5 (sums over k3) in slabs of schur_slab(m)
// k3-values, one chain per slab, slabs added in order (shorter dependent chains).
__host__ __device__ __forceinline__ int schur_slab(int m) { return m > 31 ? 4 : 8; }

// Faces 0..3 at the k3 rows [r0, r1) of the eigenspace slab W (rows r0..r1-1
// stored from W[0]): X[f][k3][.] for f < 4.
template <typename T>
__device__ __forceinline__ void faces_reduce_rows(int m, int ne, const T* a0, const T* W, int r0, int r1, T* X) {
  const int mm = m * m, nr = r1 - r0;
  for (int idx = threadIdx.x; idx < 4 * nr * m; idx += blockDim.x) {
    const int f = idx / (nr * m), r = idx - f * nr * m, k3 = r0 + r / m, kx = r - (r / m) * m;
    const int k0 = (f & 1) ? ne : 0, k1 = (f & 1) ? m : ne;
    const T* w;
    int ws;
    if (f < 2) {
      w = W + ((k3 - r0) * m + kx) * m;  // along k1 at (k3, k2 = kx)
      ws = 1;
    } else {
      w = W + (k3 - r0) * mm + kx;       // along k2 at (k3, k1 = kx)
      ws = m;
    }
    T s0 = 0, s1 = 0;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      s0 = madd(a0[k], w[k * ws], s0);
      s1 = madd(a0[k + 1], w[(k + 1) * ws], s1);
    }
    if (k < k1) s0 = madd(a0[k], w[k * ws], s0);
    X[f * mm + k3 * m + kx] = s0 + s1;
  }
}

// Partial sums of faces 4, 5 over the k3 rows [r0, r1) of one slab (W as above):
// P[f - 4][k2][k1], one chain over k3 within the parity range of the face.
template <typename T>
__device__ __forceinline__ void faces_reduce_slab45(int m, int ne, const T* a0, const T* W, int r0, int r1, T* P) {
  const int mm = m * m;
  for (int idx = threadIdx.x; idx < 2 * mm; idx += blockDim.x) {
    const int f = idx / mm, r = idx - f * mm;
    const int lo = max(r0, f ? ne : 0), hi = min(r1, f ? m : ne);
    T acc = 0;
    for (int k3 = lo; k3 < hi; ++k3) acc = madd(a0[k3], W[(k3 - r0) * mm + r], acc);
    P[idx] = acc;
  }
}

__device__ __forceinline__ double inv_d(const Tabs<double>& t, const ElemScal<double>& sc, const double* lI,
                                        double lam, int64_t idx, int k1, int k2, int k3, int64_t n3) {
  if (t.Relem) return t.Relem[sc.cls * n3 + idx];
  return 1.0 / (lam + sc.e[0] * lI[k1] + sc.e[1] * lI[k2] + sc.e[2] * lI[k3]);
}

// float-float: the table's value, or the refined reciprocal of the sum
__device__ __forceinline__ ff inv_d(const Tabs<ff>& t, const ElemScal<ff>& sc, const ff* lI, ff lam, int64_t idx,
                                    int k1, int k2, int k3, int64_t n3) {
  if (t.Relem) return t.Relem[sc.cls * n3 + idx];
  return ff_recip(lam + sc.e[0] * lI[k1] + sc.e[1] * lI[k2] + sc.e[2] * lI[k3]);
}

// FP32 (inside FP64 iterative refinement): approximate reciprocal, no table read
__device__ __forceinline__ float inv_d(const Tabs<float>&, const ElemScal<float>& sc, const float* lI, float lam,
                                       int64_t, int k1, int k2, int k3, int64_t) {
  return rcp_approx(lam + sc.e[0] * lI[k1] + sc.e[1] * lI[k2] + sc.e[2] * lI[k3]);
}

template <typename T>
__device__ __forceinline__ void load_tables(int m, const Tabs<T>& t, T* Sh, T* a0, T* lI) {
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) Sh[i] = t.Sh[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    a0[i] = t.a0[i];
    lI[i] = t.lamI[i];
  }
}

__device__ __forceinline__ void elem_coords(const Geo& G, int64_t e, int* a1, int* a2, int* a3) {
  *a1 = (int)(e % G.n1);
  *a2 = (int)((e / G.n1) % G.n2);
  *a3 = (int)(e / ((int64_t)G.n1 * G.n2));
}

// y_e = H_BI H_II^{-1} H_IB u on the six faces of every element -> Z[e][f][.]
// Work regions: 0 tables (Sh, a0, Lam), 1 X (6 m^2), 2 Tt (6 m^2; empty in eigenbasis mode), 3 W (m^3).
// PC > 0 compiles the kernel for degree PC (constant extents); PC = 0 reads it from G.
// pre = 1: u holds every face already in the eigenbasis, c_f Sh^T U_f Sh (the
// transform is the same for the two elements sharing the face, so it is done
// once per face), and Z receives the element's face terms in that basis,
// alpha_d (X_even +- X_odd), for one back transform per face after the two
// elements' terms are summed.
template <typename T, int PC, int NB>
__global__ void __launch_bounds__(512, NB) k_elem_schur(Geo G, Tabs<T> t, const T* __restrict__ u,
                                                         T* __restrict__ Z, T* ws, WsPlan wp, int pre, int cs) {
  // cs = 2 (eigenbasis mode, W in global memory): the two CTAs of a cluster share an
  // element: each keeps its own copy of the face data X, the expansion into W is split
  // over both (one cluster barrier), and each reduces and stores its own half of the
  // in-face index r, so nothing else crosses CTAs; every output has the summation order
  // of cs = 1
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m;
  const int64_t n3 = (int64_t)mm * m;
  const Team tm = team_of(cs);
  const int crank = tm.id / (int)blockDim.x;
  auto at = [&](int i) {
    return wp.in_smem[i] ? reinterpret_cast<T*>(smem_raw) + wp.off[i] : ws + (blockIdx.x / cs) * wp.gstride + wp.off[i];
  };
  T* Sh = at(0);
  T* a0 = Sh + mm;
  T* lI = a0 + m;
  T* X = at(1);
  T* Tt = at(2);
  T* W = at(3);
  load_tables(m, t, Sh, a0, lI);
  const Lines F{m, m / 2, (m + 1) / 2, m, m, 6 * mm};
  const int ne = F.ne;
  const T lam = (T)G.lam;
  const int rlo = crank * mm / cs, rhi = (crank + 1) * mm / cs, nr = rhi - rlo;  // this CTA's r range
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    tm.sync();  // W (shared by the cluster) is free again
    for (int idx = threadIdx.x; idx < 6 * mm; idx += blockDim.x) {
      const int f = idx / mm;
      X[idx] = u[elem_face_base(G, a1, a2, a3, f) + (idx - f * mm)];
    }
    __syncthreads();
    if (pre) {
      // pair sums / differences of the transformed faces, scaled by alpha_d
      for (int idx = threadIdx.x; idx < 3 * mm; idx += blockDim.x) {
        const int d = idx / mm, r = idx - d * mm;
        const T a = X[(2 * d) * mm + r], b = X[(2 * d + 1) * mm + r];
        X[(2 * d) * mm + r] = sc.ald(d) * (a + b);
        X[(2 * d + 1) * mm + r] = sc.ald(d) * (a - b);
      }
      __syncthreads();
    } else {
      face_pairs(mm, X);
      __syncthreads();
      faces_forward(F, Sh, X, Tt, sc);
    }
    for (int64_t idx = tm.id; idx < n3; idx += tm.n) {
      const int k1 = (int)(idx % m), k2 = (int)((idx / m) % m), k3 = (int)(idx / mm);
      W[idx] = face_expand(m, ne, a0, X, k1, k2, k3) * inv_d(t, sc, lI, lam, idx, k1, k2, k3, n3);
    }
    tm.sync();
    if (cs == 1) {
      faces_reduce_rows(m, ne, a0, W, 0, m, X);
    } else {
      // faces 0..3 on this CTA's r range, each output as faces_reduce_rows sums it
      for (int idx = threadIdx.x; idx < 4 * nr; idx += blockDim.x) {
        const int f = idx / nr, r = rlo + (idx - f * nr), k3 = r / m, kx = r - k3 * m;
        const int k0 = (f & 1) ? ne : 0, k1 = (f & 1) ? m : ne;
        const T* w = f < 2 ? W + (k3 * m + kx) * m : W + k3 * mm + kx;
        const int wst = f < 2 ? 1 : m;
        T s0 = 0, s1 = 0;
        int k = k0;
        for (; k + 1 < k1; k += 2) {
          s0 = madd(a0[k], w[k * wst], s0);
          s1 = madd(a0[k + 1], w[(k + 1) * wst], s1);
        }
        if (k < k1) s0 = madd(a0[k], w[k * wst], s0);
        X[f * mm + r] = s0 + s1;
      }
    }
    // faces 4, 5: slab partials in order (schur_slab(m) k3-rows each)
    const int slab = schur_slab(m);
    for (int idx = threadIdx.x; idx < 2 * nr; idx += blockDim.x) {
      const int f = idx / nr, r = rlo + (idx - f * nr);
      const int flo = f ? ne : 0, fhi = f ? m : ne;
      T tot = 0;
      for (int r0 = 0; r0 < m; r0 += slab) {
        const int lo = max(r0, flo), hi = min(r0 + slab, fhi);
        T acc = 0;
        for (int k3 = lo; k3 < hi; ++k3) acc = madd(a0[k3], W[k3 * mm + r], acc);
        tot = r0 == 0 ? acc : tot + acc;
      }
      X[(4 + f) * mm + r] = tot;
    }
    __syncthreads();
    T* Ze = Z + e * 6 * mm;
    if (pre) {
      for (int idx = threadIdx.x; idx < 3 * nr; idx += blockDim.x) {
        const int d = idx / nr, r = rlo + (idx - d * nr);
        const T xe = X[(2 * d) * mm + r], xo = X[(2 * d + 1) * mm + r];
        Ze[(2 * d) * mm + r] = sc.ald(d) * (xe + xo);
        Ze[(2 * d + 1) * mm + r] = sc.ald(d) * (xe - xo);
      }
    } else {
      faces_backward(F, Sh, X, Tt, sc, [&](int idx, T v) { Ze[idx] = v; });
    }
  }
}

// Interior 3D transforms with the folded reference eigenvectors.
// forward: A <- scale * (Sref^T (x) Sref^T (x) Sref^T) A, B is scratch.
template <typename T>
__device__ __forceinline__ void interior_forward(const Lines& I, const T* Sr, T* A, T* B, T scale, const Team& tm) {
  fold_lines(I, 0, A, B, tm);
  tm.sync();
  tx_lines_g(I, 0, Sr, B, A, (T)1, (const T*)nullptr, tm);
  tm.sync();
  fold_lines(I, 1, A, B, tm);
  tm.sync();
  tx_lines_g(I, 1, Sr, B, A, (T)1, (const T*)nullptr, tm);
  tm.sync();
  fold_lines(I, 2, A, B, tm);
  tm.sync();
  tx_lines_g(I, 2, Sr, B, A, scale, (const T*)nullptr, tm);
  tm.sync();
}

// backward along x3 and x2 (natural order in A afterwards), then the x1
// transposed transform into B; the caller unfolds B along x1.
template <typename T>
__device__ __forceinline__ void interior_backward(const Lines& I, const T* Sr, T* A, T* B, const Team& tm) {
  txT_lines_g(I, 2, Sr, A, B, tm);
  tm.sync();
  unfold_lines(I, 2, B, A, tm);
  tm.sync();
  txT_lines_g(I, 1, Sr, A, B, tm);
  tm.sync();
  unfold_lines(I, 1, B, A, tm);
  tm.sync();
  txT_lines_g(I, 0, Sr, A, B, tm);
  tm.sync();
}

template <typename T>
struct FdmSmem {
  T *Sh, *Sr, *a0, *lI, *X, *Tt, *A, *B;
};

// Work regions: 0 tables (Sh, Sref, a0, Lam), 1 X (6 m^2), 2 Tt (6 m^2), 3 A+B (2 m^3).
// Work arrays of the team: shared memory of this CTA, or the team's slice of the global
// workspace (slice = the team's index: the CTA, or the cluster, in the grid).
template <typename T>
__device__ FdmSmem<T> fdm_layout(int m, unsigned char* smem, T* ws, const WsPlan& wp, int64_t slice) {
  const int mm = m * m;
  auto at = [&](int i) {
    return wp.in_smem[i] ? reinterpret_cast<T*>(smem) + wp.off[i] : ws + slice * wp.gstride + wp.off[i];
  };
  FdmSmem<T> s;
  s.Sh = at(0);
  s.Sr = s.Sh + mm;
  s.a0 = s.Sr + mm;
  s.lI = s.a0 + m;
  s.X = at(1);
  s.Tt = at(2);
  s.A = at(3);
  s.B = s.A + (int64_t)mm * m;
  return s;
}

// nodal index of interior point (i1, i2, i3) of element (a1, a2, a3)
__device__ __forceinline__ int64_t interior_node3(const Geo& G, int a1, int a2, int a3, int i1, int i2, int i3) {
  const int p = G.p;
  const int64_t N1 = (int64_t)G.n1 * p + 1, N2 = (int64_t)G.n2 * p + 1;
  return ((int64_t)(a3 * p + i3 + 1) * N2 + (a2 * p + i2 + 1)) * N1 + (a1 * p + i1 + 1);
}

__device__ __forceinline__ int64_t interior_node(const Geo& G, int a1, int a2, int a3, int idx) {
  const int m = G.m;
  return interior_node3(G, a1, a2, a3, idx % m, (idx / m) % m, idx / (m * m));
}

// Z[e][f] = (H_BI H_II^{-1} F_I) on the faces, F_I = (M f)_I element-local.
// When Gsave is given, the scaled interior eigen-coefficients
// D^{-1} (S^T x S^T x S^T) F_I of every element are also stored there
// (m^3 per element), for the recovery of the same solve.  cs = 2: launched in
// clusters of two CTAs that share each element's work (global work arrays).
// T: the arithmetic (FP64, or float-float); f and Z are FP64, Gsave of type T.
template <typename T, int PC>
__global__ void __launch_bounds__(512, 1) k_elem_condense(Geo G, Tabs<T> t, const double* __restrict__ f,
                                                        double* __restrict__ Z, T* __restrict__ Gsave, T* ws,
                                                        WsPlan wp, int cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m, mmm = mm * m;
  const Team tm = team_of(cs);
  FdmSmem<T> s = fdm_layout(m, smem_raw, ws, wp, blockIdx.x / cs);
  load_tables(m, t, s.Sh, s.a0, s.lI);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) s.Sr[i] = t.Sref[i];
  const Lines F{m, m / 2, (m + 1) / 2, m, m, 6 * mm};
  const Lines I{m, m / 2, (m + 1) / 2, m, m, mmm};
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    const T* x1 = t.hx[0] + 6 * a1;
    const T* x2 = t.hx[1] + 6 * a2;
    const T* x3 = t.hx[2] + 6 * a3;
    const T vol = (T)0.125 * x1[0] * x2[0] * x3[0];  // h1 h2 h3 / 8
    const T sig = x1[5] * x2[5] * x3[5];             // sqrt(8 / (h1 h2 h3))
    tm.sync();
    for (int idx = tm.id; idx < mmm; idx += tm.n) {
      const int i1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
      s.A[idx] = vol * t.w[i1 + 1] * t.w[i2 + 1] * t.w[i3 + 1] * (T)f[interior_node(G, a1, a2, a3, idx)];
    }
    tm.sync();
    interior_forward(I, s.Sr, s.A, s.B, sig, tm);
    T* Ge = Gsave ? Gsave + e * (int64_t)mmm : nullptr;
    for (int idx = tm.id; idx < mmm; idx += tm.n) {
      const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
      const T v = s.A[idx] * inv_d(t, sc, s.lI, (T)G.lam, idx, k1, k2, k3, mmm);
      s.A[idx] = v;
      if (Ge) Ge[idx] = v;
    }
    tm.sync();
    faces_reduce(m, F.ne, s.a0, s.A, s.X, tm);
    tm.sync();
    double* Ze = Z + e * 6 * mm;
    faces_backward(F, s.Sh, s.X, s.Tt, sc, [&](int idx, T v) { Ze[idx] = (double)v; }, tm);
  }
}

// u_I = H_II^{-1} (F_I - H_IB uhat) written into the nodal array.  With Gin
// (the coefficients k_elem_condense stored for the same f) the forward
// transform of F_I is taken from there instead of being recomputed.  cs as
// for k_elem_condense; T and Gin as there, f, uh and un FP64.
template <typename T, int PC>
__global__ void __launch_bounds__(512, 1) k_elem_recover(Geo G, Tabs<T> t, const double* __restrict__ f,
                                                       const T* __restrict__ Gin,
                                                       const double* __restrict__ uh, double* __restrict__ un,
                                                       T* ws, WsPlan wp, int cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m, mmm = mm * m;
  const Team tm = team_of(cs);
  FdmSmem<T> s = fdm_layout(m, smem_raw, ws, wp, blockIdx.x / cs);
  load_tables(m, t, s.Sh, s.a0, s.lI);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) s.Sr[i] = t.Sref[i];
  const Lines F{m, m / 2, (m + 1) / 2, m, m, 6 * mm};
  const Lines I{m, m / 2, (m + 1) / 2, m, m, mmm};
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    const T* x1 = t.hx[0] + 6 * a1;
    const T* x2 = t.hx[1] + 6 * a2;
    const T* x3 = t.hx[2] + 6 * a3;
    const T vol = (T)0.125 * x1[0] * x2[0] * x3[0];  // h1 h2 h3 / 8
    const T sig = x1[5] * x2[5] * x3[5];             // sqrt(8 / (h1 h2 h3))
    tm.sync();
    if (!Gin) {
      for (int idx = tm.id; idx < mmm; idx += tm.n) {
        const int i1 = idx % m, i2 = (idx / m) % m, i3 = idx / mm;
        s.A[idx] = vol * t.w[i1 + 1] * t.w[i2 + 1] * t.w[i3 + 1] * (T)f[interior_node(G, a1, a2, a3, idx)];
      }
    }
    for (int idx = tm.id; idx < 6 * mm; idx += tm.n) {
      const int fc = idx / mm;
      s.X[idx] = (T)uh[elem_face_base(G, a1, a2, a3, fc) + (idx - fc * mm)];
    }
    tm.sync();
    if (!Gin) interior_forward(I, s.Sr, s.A, s.B, sig, tm);
    face_pairs(mm, s.X, tm);
    tm.sync();
    faces_forward(F, s.Sh, s.X, s.Tt, sc, tm);
    if (Gin) {
      const T* Ge = Gin + e * (int64_t)mmm;
      for (int idx = tm.id; idx < mmm; idx += tm.n) {
        const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
        s.A[idx] = Ge[idx] - face_expand(m, F.ne, s.a0, s.X, k1, k2, k3) *
                                 inv_d(t, sc, s.lI, (T)G.lam, idx, k1, k2, k3, mmm);
      }
    } else {
      for (int idx = tm.id; idx < mmm; idx += tm.n) {
        const int k1 = idx % m, k2 = (idx / m) % m, k3 = idx / mm;
        s.A[idx] = (s.A[idx] - face_expand(m, F.ne, s.a0, s.X, k1, k2, k3)) *
                   inv_d(t, sc, s.lI, (T)G.lam, idx, k1, k2, k3, mmm);
      }
    }
    tm.sync();
    interior_backward(I, s.Sr, s.A, s.B, tm);
    for (int idx = tm.id; idx < mmm; idx += tm.n)
      un[interior_node(G, a1, a2, a3, idx)] = (double)(sig * unfold_at(I, 0, s.B, idx));
  }
}

constexpr size_t kSmemCap = 112 * 1024;
constexpr size_t kSchurSmemCap = 200 * 1024;

}  // namespace

template <typename T>
LaunchCfg plan_elem_schur(const Geo& G, int nsm, size_t cap, int block, int wide) {
  const size_t m = G.m, mm = m * m;
  LaunchCfg c;
  if (cap == 0) cap = kSchurSmemCap;
  // levels of the face-parallel form run the kernel in eigenbasis mode, which has no
  // face transforms and so no transform scratch (region 2)
  const size_t sizes[4] = {mm + 2 * m, 6 * mm, face_form(G) ? 0 : 6 * mm, mm * m};
  c.ws = plan_regions(sizes, 4, sizeof(T), cap, &c.smem);
  c.ok = plan_ok(c.ws, sizes, 4, sizeof(T), c.smem);
  c.block = block ? block : (c.smem > 100 * 1024 ? 512 : 256);
  const int64_t grid = (int64_t)nsm * resident_blocks(c, wide);
  c.grid = (int)(G.nelem < grid ? G.nelem : grid);
  if (c.grid < 1) c.grid = 1;
  // eigenbasis mode with the eigenspace array W in global memory: two CTAs per element (a
  // cluster) when halving the work units shortens a partial last wave.  Each CTA keeps its
  // own tables and face data X (transformed in place), so both must be in shared memory.
  // Rounds are counted per SM (CTAs sharing an SM share its throughput).
  if (face_form(G) && c.ws.in_smem[0] && c.ws.in_smem[1] && !c.ws.in_smem[3] && grid >= 2) {
    const int64_t r1 = (G.nelem + nsm - 1) / nsm, r2 = (2 * G.nelem + nsm - 1) / nsm;
    if (r2 < 2 * r1) {
      c.cluster = 2;
      const int64_t nc = G.nelem < grid / 2 ? G.nelem : grid / 2;
      c.grid = (int)(2 * nc);
    }
  }
  return c;
}

template <typename T, int NB>
void launch_elem_schur_nb(const Geo& G, const Tabs<T>& t, const T* u, T* Z, T* ws, const LaunchCfg& c,
                          cudaStream_t st, int pre) {
  switch (G.p) {
    case 2: launch_clustered(k_elem_schur<T, 2, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    case 4: launch_clustered(k_elem_schur<T, 4, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    case 8: launch_clustered(k_elem_schur<T, 8, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    case 16: launch_clustered(k_elem_schur<T, 16, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    case 32: launch_clustered(k_elem_schur<T, 32, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    case 48: launch_clustered(k_elem_schur<T, 48, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
    default: launch_clustered(k_elem_schur<T, 0, NB>, c, st, G, t, u, Z, ws, c.ws, pre, c.cluster); break;
  }
}

template <typename T>
void launch_elem_schur(const Geo& G, const Tabs<T>& t, const T* u, T* Z, T* ws, const LaunchCfg& c,
                       cudaStream_t st, int pre) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  if (c.wide)
    launch_elem_schur_nb<T, 1>(G, t, u, Z, ws, c, st, pre);
  else
    launch_elem_schur_nb<T, 2>(G, t, u, Z, ws, c, st, pre);
}

template <typename T, int NB>
static int schur_attrs_nb() {
  int bad = cudaFuncSetAttribute(k_elem_schur<T, 0, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 2, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 4, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 8, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 16, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 32, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_elem_schur<T, 48, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

template <typename T>
static int schur_attrs() {
  return schur_attrs_nb<T, 1>() | schur_attrs_nb<T, 2>();
}

}  // namespace semmg
