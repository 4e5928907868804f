// Per-node pieces of the assembled skeleton block H_BB, shared by the
// skeleton-parallel assembly and the face-parallel form of the operator.
//
// On the tensor-product mesh the assembled operator is the Kronecker sum of
// the assembled 1D matrices (Sec. 2.1 and 3.2), so H_BB at a skeleton node is
// the product of three assembled 1D masses times lam plus three line sums of
// the assembled 1D stiffness, each weighted by the masses of the other axes.
#pragma once
#include "semmg_internal.h"

namespace semmg {

namespace {

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

// H_BB u at skeleton node s (global coordinates g, entity group `type`).
template <typename T>
__device__ __forceinline__ T node_hbb(const Geo& G, const Tabs<T>& t, const T* __restrict__ u, int64_t s, int type,
                                      const int* g) {
  const int nd[3] = {G.n1, G.n2, G.n3};
  bool on[3];
  for (int d = 0; d < 3; ++d) on[d] = (g[d] - divp(G, g[d]) * G.p) == 0;
  T M[3], L[3];
  for (int d = 0; d < 3; ++d) {
    M[d] = mass1d(G, t, d, g[d], nd[d]);
    const bool other = on[(d + 1) % 3] || on[(d + 2) % 3];
    L[d] = line_sum(G, t, u, s, type, g, d, other);
  }
  return (T)G.lam * M[0] * M[1] * M[2] * u[s] + M[1] * M[2] * L[0] + M[0] * M[2] * L[1] + M[0] * M[1] * L[2];
}

}  // namespace

}  // namespace semmg
