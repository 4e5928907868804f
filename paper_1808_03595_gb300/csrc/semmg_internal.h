// Internal declarations of the semmg CUDA library: level geometry, device
// tables, skeleton indexing and kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "semmg.h"
#include "ff.cuh"

namespace semmg {

#define SEMMG_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------- geometry
// One level of the hierarchy on the tensor-product mesh: degree p, m = p-1
// interior nodes per element edge, n_S = 2p-1 star points per direction
// (Sec. 2.3), and the offsets of the entity groups of a condensed vector
// (layout documented in semmg.h).
struct Geo {
  int p, m, nS;
  int n1, n2, n3;
  int nv1, nv2, nv3;
  int64_t oF1, oF2, oF3, oE1, oE2, oE3, oV, size;
  int64_t nelem, nstar;
  uint64_t pinv;  // ceil(2^32 / p): exact division g / p for 0 <= g < 2^20
  double lam;
  unsigned char dir[6];  // faces -x1, +x1, -x2, +x2, -x3, +x3: 1 = Dirichlet, 0 = Neumann or periodic
  unsigned char per[3];  // periodic axes: vertex plane n_d is the image of plane 0 (its slots unused)
};

SEMMG_HD int ncount(const Geo& G, int d) { return d == 0 ? G.n1 : (d == 1 ? G.n2 : G.n3); }

// Whether vertex plane c along axis d holds no unknowns: a Dirichlet face, or
// the image plane of a periodic axis.
SEMMG_HD bool dir_plane(const Geo& G, int d, int c) {
  const int nd = ncount(G, d);
  return (c == 0 && G.dir[2 * d]) || (c == nd && (G.dir[2 * d + 1] || G.per[d]));
}

// Global node index along a periodic axis mapped onto [0, n_d p) (offsets of
// at most one period); unchanged on other axes.
SEMMG_HD int wrapg(const Geo& G, int d, int g) {
  if (!G.per[d]) return g;
  const int L = ncount(G, d) * G.p;
  return g < 0 ? g + L : (g >= L ? g - L : g);
}

// Element index along a periodic axis mapped onto [0, n_d).
SEMMG_HD int wrape(const Geo& G, int d, int a) {
  if (!G.per[d]) return a;
  const int nd = ncount(G, d);
  return a < 0 ? a + nd : (a >= nd ? a - nd : a);
}

enum EntityType { ENT_F1 = 0, ENT_F2, ENT_F3, ENT_E1, ENT_E2, ENT_E3, ENT_V, ENT_NONE };

// Star kernel constants shared with the host-side operation count: k3-planes of
// the eigenspace held at once, and outputs per thread in the grouped transforms.
SEMMG_HD int star_slab_thickness(int nS) { return nS <= 16 ? 8 : (nS <= 32 ? 4 : 2); }
constexpr int kStarGroup = 4;

SEMMG_HD int divp(const Geo& G, int g) {
  return (int)(((unsigned long long)(unsigned)g * G.pinv) >> 32);
}

// Skeleton slot of the global GLL node (g1, g2, g3), or -1 for an element
// interior node; periodic images and offsets past a periodic end map to the
// unknown they repeat.  `type` receives the entity group.
SEMMG_HD int64_t skel_index(const Geo& G, int g1, int g2, int g3, int* type = nullptr) {
  g1 = wrapg(G, 0, g1);
  g2 = wrapg(G, 1, g2);
  g3 = wrapg(G, 2, g3);
  const int a1 = divp(G, g1), a2 = divp(G, g2), a3 = divp(G, g3);
  const int q1 = g1 - a1 * G.p, q2 = g2 - a2 * G.p, q3 = g3 - a3 * G.p;
  const int m = G.m;
  const int64_t mm = (int64_t)m * m;
  const int v1 = (q1 == 0), v2 = (q2 == 0), v3 = (q3 == 0);
  const int cnt = v1 + v2 + v3;
  int t = ENT_NONE;
  int64_t s = -1;
  if (cnt == 3) {
    t = ENT_V;
    s = G.oV + ((int64_t)a3 * G.nv2 + a2) * G.nv1 + a1;
  } else if (cnt == 2) {
    if (!v1) {
      t = ENT_E1;
      s = G.oE1 + (((int64_t)a3 * G.nv2 + a2) * G.n1 + a1) * m + (q1 - 1);
    } else if (!v2) {
      t = ENT_E2;
      s = G.oE2 + (((int64_t)a3 * G.n2 + a2) * G.nv1 + a1) * m + (q2 - 1);
    } else {
      t = ENT_E3;
      s = G.oE3 + (((int64_t)a3 * G.nv2 + a2) * G.nv1 + a1) * m + (q3 - 1);
    }
  } else if (cnt == 1) {
    if (v1) {
      t = ENT_F1;
      s = G.oF1 + (((int64_t)a3 * G.n2 + a2) * G.nv1 + a1) * mm + (int64_t)(q3 - 1) * m + (q2 - 1);
    } else if (v2) {
      t = ENT_F2;
      s = G.oF2 + (((int64_t)a3 * G.nv2 + a2) * G.n1 + a1) * mm + (int64_t)(q3 - 1) * m + (q1 - 1);
    } else {
      t = ENT_F3;
      s = G.oF3 + (((int64_t)a3 * G.n2 + a2) * G.n1 + a1) * mm + (int64_t)(q2 - 1) * m + (q1 - 1);
    }
  }
  if (type) *type = t;
  return s;
}

// Skeleton slot of the node at in-plane offsets (ja, jb), -m <= ja, jb <= m, from
// vertex (c1, c2, c3) on the star plane normal to axis dd (ja along the fast
// in-plane axis: x2 for dd = 0, else x1; jb along the slow one: x3 for dd < 2,
// else x2): skel_index of that node, from the entity it lies on (a face
// quadrant, a half edge or the vertex) without decoding global coordinates.
// The vertex must not lie on the image plane of a periodic axis.
SEMMG_HD int64_t star_plane_slot(const Geo& G, int dd, int c1, int c2, int c3, int ja, int jb) {
  const int m = G.m;
  const int64_t mm = (int64_t)m * m;
  const int ia = ja > 0 ? ja - 1 : m + ja, ib = jb > 0 ? jb - 1 : m + jb;  // interior indices
  if (dd == 0) {  // plane c1: x2 (ja), x3 (jb)
    const int a2 = ja > 0 ? c2 : wrape(G, 1, c2 - 1), a3 = jb > 0 ? c3 : wrape(G, 2, c3 - 1);
    if (ja != 0 && jb != 0) return G.oF1 + (((int64_t)a3 * G.n2 + a2) * G.nv1 + c1) * mm + (int64_t)ib * m + ia;
    if (jb != 0) return G.oE3 + (((int64_t)a3 * G.nv2 + c2) * G.nv1 + c1) * m + ib;
    if (ja != 0) return G.oE2 + (((int64_t)c3 * G.n2 + a2) * G.nv1 + c1) * m + ia;
  } else if (dd == 1) {  // plane c2: x1 (ja), x3 (jb)
    const int a1 = ja > 0 ? c1 : wrape(G, 0, c1 - 1), a3 = jb > 0 ? c3 : wrape(G, 2, c3 - 1);
    if (ja != 0 && jb != 0) return G.oF2 + (((int64_t)a3 * G.nv2 + c2) * G.n1 + a1) * mm + (int64_t)ib * m + ia;
    if (jb != 0) return G.oE3 + (((int64_t)a3 * G.nv2 + c2) * G.nv1 + c1) * m + ib;
    if (ja != 0) return G.oE1 + (((int64_t)c3 * G.nv2 + c2) * G.n1 + a1) * m + ia;
  } else {  // plane c3: x1 (ja), x2 (jb)
    const int a1 = ja > 0 ? c1 : wrape(G, 0, c1 - 1), a2 = jb > 0 ? c2 : wrape(G, 1, c2 - 1);
    if (ja != 0 && jb != 0) return G.oF3 + (((int64_t)c3 * G.n2 + a2) * G.n1 + a1) * mm + (int64_t)ib * m + ia;
    if (jb != 0) return G.oE2 + (((int64_t)c3 * G.n2 + a2) * G.nv1 + c1) * m + ib;
    if (ja != 0) return G.oE1 + (((int64_t)c3 * G.nv2 + c2) * G.n1 + a1) * m + ia;
  }
  return G.oV + ((int64_t)c3 * G.nv2 + c2) * G.nv1 + c1;
}

// Index stride of a run of nodes along axis d (0-based) inside one entity.
SEMMG_HD int run_stride(const Geo& G, int type, int d) {
  switch (type) {
    case ENT_F1: return d == 1 ? 1 : G.m;
    case ENT_F2: return d == 0 ? 1 : G.m;
    case ENT_F3: return d == 0 ? 1 : G.m;
    default: return 1;
  }
}

// Decode a skeleton slot into its global node coordinates; returns the entity
// type and whether the node lies on a Dirichlet face.
SEMMG_HD int skel_decode(const Geo& G, int64_t s, int* g, bool* bdry) {
  const int p = G.p, m = G.m;
  const int64_t mm = (int64_t)m * m;
  int t;
  int c1 = 0, c2 = 0, c3 = 0;  // plane / element coordinates
  if (s < G.oF2) {
    t = ENT_F1;
    int64_t r = s - G.oF1;
    const int64_t f = r / mm, w = r - f * mm;
    const int i3 = (int)(w / m), i2 = (int)(w - (int64_t)i3 * m);
    c1 = (int)(f % G.nv1);
    const int64_t f2 = f / G.nv1;
    const int a2 = (int)(f2 % G.n2), a3 = (int)(f2 / G.n2);
    g[0] = c1 * p; g[1] = a2 * p + i2 + 1; g[2] = a3 * p + i3 + 1;
    *bdry = dir_plane(G, 0, c1);
  } else if (s < G.oF3) {
    t = ENT_F2;
    int64_t r = s - G.oF2;
    const int64_t f = r / mm, w = r - f * mm;
    const int i3 = (int)(w / m), i1 = (int)(w - (int64_t)i3 * m);
    const int a1 = (int)(f % G.n1);
    const int64_t f2 = f / G.n1;
    c2 = (int)(f2 % G.nv2);
    const int a3 = (int)(f2 / G.nv2);
    g[0] = a1 * p + i1 + 1; g[1] = c2 * p; g[2] = a3 * p + i3 + 1;
    *bdry = dir_plane(G, 1, c2);
  } else if (s < G.oE1) {
    t = ENT_F3;
    int64_t r = s - G.oF3;
    const int64_t f = r / mm, w = r - f * mm;
    const int i2 = (int)(w / m), i1 = (int)(w - (int64_t)i2 * m);
    const int a1 = (int)(f % G.n1);
    const int64_t f2 = f / G.n1;
    const int a2 = (int)(f2 % G.n2);
    c3 = (int)(f2 / G.n2);
    g[0] = a1 * p + i1 + 1; g[1] = a2 * p + i2 + 1; g[2] = c3 * p;
    *bdry = dir_plane(G, 2, c3);
  } else if (s < G.oE2) {
    t = ENT_E1;
    int64_t r = s - G.oE1;
    const int64_t e = r / m;
    const int i1 = (int)(r - e * m);
    const int a1 = (int)(e % G.n1);
    const int64_t e2 = e / G.n1;
    c2 = (int)(e2 % G.nv2);
    c3 = (int)(e2 / G.nv2);
    g[0] = a1 * p + i1 + 1; g[1] = c2 * p; g[2] = c3 * p;
    *bdry = dir_plane(G, 1, c2) || dir_plane(G, 2, c3);
  } else if (s < G.oE3) {
    t = ENT_E2;
    int64_t r = s - G.oE2;
    const int64_t e = r / m;
    const int i2 = (int)(r - e * m);
    c1 = (int)(e % G.nv1);
    const int64_t e2 = e / G.nv1;
    const int a2 = (int)(e2 % G.n2);
    c3 = (int)(e2 / G.n2);
    g[0] = c1 * p; g[1] = a2 * p + i2 + 1; g[2] = c3 * p;
    *bdry = dir_plane(G, 0, c1) || dir_plane(G, 2, c3);
  } else if (s < G.oV) {
    t = ENT_E3;
    int64_t r = s - G.oE3;
    const int64_t e = r / m;
    const int i3 = (int)(r - e * m);
    c1 = (int)(e % G.nv1);
    const int64_t e2 = e / G.nv1;
    c2 = (int)(e2 % G.nv2);
    const int a3 = (int)(e2 / G.nv2);
    g[0] = c1 * p; g[1] = c2 * p; g[2] = a3 * p + i3 + 1;
    *bdry = dir_plane(G, 0, c1) || dir_plane(G, 1, c2);
  } else {
    t = ENT_V;
    int64_t r = s - G.oV;
    c1 = (int)(r % G.nv1);
    const int64_t r2 = r / G.nv1;
    c2 = (int)(r2 % G.nv2);
    c3 = (int)(r2 / G.nv2);
    g[0] = c1 * p; g[1] = c2 * p; g[2] = c3 * p;
    *bdry = dir_plane(G, 0, c1) || dir_plane(G, 1, c2) || dir_plane(G, 2, c3);
  }
  return t;
}

// Base slot of a face of element (a1,a2,a3); f = 2d + side, side 0 at local
// index 0, side 1 at local index p along axis d.
SEMMG_HD int64_t elem_face_base(const Geo& G, int a1, int a2, int a3, int f) {
  const int64_t mm = (int64_t)G.m * G.m;
  const int side = f & 1;
  // the far face of the last element of a periodic axis is plane 0
  switch (f >> 1) {
    case 0: {
      const int c = (side && G.per[0] && a1 + 1 == G.n1) ? 0 : a1 + side;
      return G.oF1 + (((int64_t)a3 * G.n2 + a2) * G.nv1 + c) * mm;
    }
    case 1: {
      const int c = (side && G.per[1] && a2 + 1 == G.n2) ? 0 : a2 + side;
      return G.oF2 + (((int64_t)a3 * G.nv2 + c) * G.n1 + a1) * mm;
    }
    default: {
      const int c = (side && G.per[2] && a3 + 1 == G.n3) ? 0 : a3 + side;
      return G.oF3 + (((int64_t)c * G.n2 + a2) * G.n1 + a1) * mm;
    }
  }
}

// ---------------------------------------------------------------- tables
// One face of the face groups (F1, F2, F3 in slot order) for the face-parallel
// form of the operator (face_kernel.cuh), built on the host at setup.  The face
// has normal axis d and in-plane axes a (fast) and b (slow); Md is the
// assembled normal mass on its plane, cd0 / cdL / cdR the normal stiffness
// line sum (cd0 u + cdL u(plane below) + cdR u(plane above)).
template <typename T>
struct FaceRec {
  int64_t base;                // slot of the face's first node
  int64_t zm, zp;              // Z offsets of the face as side 2d+1 of the element below / 2d of the one above, or -1
  int64_t eA0, eAp, eB0, eBp;  // first slots of the edges at q_a = 0, q_a = p, q_b = 0, q_b = p
  int64_t nbL, nbR;            // first slots of the parallel faces on the planes below / above, or -1
  int dir;                     // no unknowns (Dirichlet plane or periodic image plane)
  int pad;
  T cf;                        // sqrt(h_a h_b) / 2
  T e0, ea, eb;                // face part of H_BB in the face eigenbasis / c_f: e0 + ea Lam[k_a] + eb Lam[k_b]
  T cdL, cdR;
  T edA, edB;                  // edge couplings: Md (h_b/2)(2/h_a), Md (h_a/2)(2/h_b)
};

// Levels that run the face-parallel form of the operator: from p = 12 on, where
// the saved element work outweighs the extra launch (at p = 8 the element-face
// form is faster on GB300).
inline bool face_form(const Geo& G) { return G.m >= 11; }

// Device tables of one level in one precision.
template <typename T>
struct Tabs {
  const T* w;      // GLL weights, p+1
  const T* Ls;     // standard-element stiffness, (p+1)^2 row-major
  const T* Sh;     // m x m: Sh[i][k] = w[i+1] Sref[i][k]
  const T* Sref;   // m x m: interior generalised eigenvectors, Sref^T M_II Sref = I, columns even then odd
  const T* a0;     // m: sum_i Sref[i][k] Ls[i+1][0]
  const T* ap;     // m: sum_i Sref[i][k] Ls[i+1][p]
  const T* lamI;   // m: interior eigenvalues
  const int* hcls[3];  // per axis: width class of every element
  int nhcls[3];        // width classes per axis
  const T* Relem;      // per width-class triple: m^3 values 1/(lam + sum 4/h^2 Lam), or null
  const T* h[3];   // element widths per axis
  // per axis, 6 derived values per element width h (computed on the host in
  // FP64): h, 2/h, 4/h^2, sqrt(h), (2/h)^(3/2), sqrt(2/h)
  const T* hx[3];
  const T* starS[3];    // per axis: nv_d blocks of nS x nS, S[j][k], row j <-> offset j-m
  const T* starLam[3];  // per axis: nv_d x nS
  const unsigned char* act[3];  // per axis: nv_d x nS active flags
  const unsigned char* starSym[3];  // per axis: nv_d flags, centrosymmetric line (columns: even, then odd)
  const int* starCls[3];           // per axis: nv_d line classes
  int ncls[3];                     // classes per axis
  const T* Rtab;   // per star class (c1*ncls2 + c2)*ncls3 + c3: nS^3 values 1/(lam+Lam1+Lam2+Lam3), or null
  const T* w1d;    // m+1: smoother weight at offset |j| (Sec. 3.2, weights)
  const int* order;  // nstar star indices, most operations first (longest-first hand-out), or null
  const T* J;      // (p+1) x (pc+1) interpolation from level-1, row-major; null on level 0
  int pc;
  // tensor-core star tables (FP32 levels of the tensor-core forms, else null): per
  // axis and line class, T(S)[e][j] = S[j][e] and N(S)[j][e] = S[j][e] as K-major
  // operands (core matrices of 8 rows x 16 bytes), n_S rounded up to 16 and
  // zero-padded: TF32 (tcT, tcN) or BF16 bit patterns (bfT, bfN)
  const T* tcT[3];
  const T* tcN[3];
  const unsigned short* bfT[3];
  const unsigned short* bfN[3];
  // element-centred blocks (Sec. 3.4), when that smoother is selected (else null): per axis
  // n_d block lines of nE x nE eigenvectors S[j][k], nE eigenvalues and nE weight factors
  // (nE = 3p - 1)
  const T* ebS[3];
  const T* ebST[3];      // transposes: ST[k][j] = S[j][k]
  const T* ebLam[3];
  const T* ebW[3];
  const int* ebCls[3];   // line class of every block line
  int ebNcls[3];
  const T* ebR;          // per class triple: nE^3 values 1/(lam + Lam1 + Lam2 + Lam3) [k3][k2][k1], or null
  const FaceRec<T>* faces;  // face-parallel operator levels (face_form), else null
};

// Coarse fast-diagonalisation tables (level 0, FP64): K_d = n_d p0 - 1
// interior grid points per axis.
struct CoarseTabs {
  int K[3];
  int g0[3];  // global node index of coarse grid point 0 along each axis (1 after a Dirichlet face, else 0)
  const double* S[3];    // K_d x K_d, S[g][k]
  const double* lam[3];  // K_d
};

// ---------------------------------------------------------------- launchers
// Per-CTA working arrays of a kernel, each placed in shared memory when it
// fits under the cap (in the given priority order) and otherwise in a
// per-CTA slice of a global workspace (L2-resident for the sizes used).
constexpr int kMaxRegions = 6;
struct WsPlan {
  int64_t off[kMaxRegions];      // offset in elements of T (smem base or CTA slice)
  int in_smem[kMaxRegions];
  int64_t gstride;               // elements of T per CTA in the global workspace
};

struct LaunchCfg {
  int grid = 0;
  int block = 256;
  size_t smem = 0;               // dynamic shared memory bytes
  WsPlan ws{};
  bool ok = false;               // plan_ok() passed
  // register budget of the kernel build: 0 = at most 64 registers per thread
  // (1024 resident threads per SM), 1 = at most 128 (512 resident threads)
  int wide = 0;
  int depth = 0;                 // element-block kernel: k3-planes of the eigenspace slab
  int bf16 = 0;                  // tensor-core star kernel: BF16 operands (else TF32)
  int cluster = 1;               // CTAs per cluster sharing one work item (element kernels: 1 or 2)
  size_t ws_elems() const {
    return (size_t)ws.gstride * (size_t)grid;
  }
};

// Greedy placement: regions visited in `order` (all regions when order is
// null), placed in shared memory while the running total stays under
// cap_bytes, otherwise in the per-CTA global slice.  sizes are in elements of
// `esize` bytes.  Every region gets a disjoint range; plan_ok() re-checks that.
inline WsPlan plan_regions(const size_t* sizes, int n, size_t esize, size_t cap_bytes, size_t* smem_bytes,
                           const int* order = nullptr) {
  WsPlan w{};
  size_t sm = 0, gl = 0;
  for (int k = 0; k < n; ++k) {
    const int i = order ? order[k] : k;
    const size_t sz = (sizes[i] + 3) & ~size_t(3);  // keep 32-byte alignment for doubles
    if ((sm + sz) * esize <= cap_bytes) {
      w.in_smem[i] = 1;
      w.off[i] = (int64_t)sm;
      sm += sz;
    } else {
      w.in_smem[i] = 0;
      w.off[i] = (int64_t)gl;
      gl += sz;
    }
  }
  w.gstride = (int64_t)((gl + 31) & ~size_t(31));
  *smem_bytes = sm * esize;
  return w;
}

// Host check that the regions are pairwise disjoint and inside their memory.
inline bool plan_ok(const WsPlan& w, const size_t* sizes, int n, size_t esize, size_t smem_bytes) {
  for (int i = 0; i < n; ++i) {
    const int64_t lim = w.in_smem[i] ? (int64_t)(smem_bytes / esize) : w.gstride;
    if (w.off[i] < 0 || w.off[i] + (int64_t)sizes[i] > lim) return false;
    for (int j = 0; j < i; ++j) {
      if (w.in_smem[i] != w.in_smem[j]) continue;
      const bool disjoint = w.off[i] + (int64_t)sizes[i] <= w.off[j] || w.off[j] + (int64_t)sizes[j] <= w.off[i];
      if (!disjoint) return false;
    }
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T* ws_ptr(const WsPlan& w, int i, unsigned char* smem, T* gws) {
  return w.in_smem[i] ? reinterpret_cast<T*>(smem) + w.off[i]
                      : gws + (int64_t)blockIdx.x * w.gstride + w.off[i];
}

// Launch with clusters of c.cluster CTAs along x (c.cluster = 1: a plain launch).
template <typename... Exp, typename... Act>
void launch_clustered(void (*kernel)(Exp...), const LaunchCfg& c, cudaStream_t st, Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c.grid);
  cfg.blockDim = dim3((unsigned)c.block);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c.cluster > 1 ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Act&&>(args)...);
}

inline int blocks_per_sm(size_t smem) {
  int b = (int)((228 * 1024) / (smem + 1024));
  if (b > 8) b = 8;
  if (b < 1) b = 1;
  return b;
}

// Resident CTAs per SM of c (block and smem set) under the shared-memory,
// thread and register-file limits; sets c.wide (the register budget) from
// `wide` (0 / 1), or, when wide < 0, to 1 exactly when the wider budget
// costs no resident threads.
inline int resident_blocks(LaunchCfg& c, int wide) {
  int bps = blocks_per_sm(c.smem);
  if (bps * c.block > 2048) bps = 2048 / c.block;
  c.wide = wide >= 0 ? wide : (bps * c.block <= 512 ? 1 : 0);
  const int reg_threads = c.wide ? 512 : 1024;  // 64K registers / (128 or 64) per thread
  if (bps * c.block > reg_threads) bps = reg_threads / c.block;
  return bps < 1 ? 1 : bps;
}

template <typename T> LaunchCfg plan_elem_schur(const Geo& G, int nsm, size_t cap = 0, int block = 0,
                                                int wide = -1);
// pre = 1 (fused form only): u holds the faces transformed by launch_face_fwd and Z
// receives the element terms in the face eigenbasis, for launch_face_bwd_assemble
template <typename T> void launch_elem_schur(const Geo& G, const Tabs<T>& t, const T* u, T* Z, T* ws,
                                             const LaunchCfg& c, cudaStream_t st, int pre = 0);
// Face-parallel form of the condensed operator (face_kernel.cuh), for levels
// with face interiors (m >= 1):
//   launch_face_fwd: Ut[s] = c_f (Sh^T U_f Sh) on every face f (slots of the
//     face groups, same indexing as u; Ut holds at least G.oE1 values);
//   launch_face_bwd_assemble: per face, the two elements' eigenbasis terms
//     and the face part of H_BB u (from Ut) combined and transformed back once,
//     then out = F - Hhat u (mode 0) or Hhat u (mode 1) on the face slots;
//     edges and vertices as launch_assemble.
template <typename T> void launch_face_fwd(const Geo& G, const Tabs<T>& t, const T* u, T* Ut, cudaStream_t st);
template <typename T, typename TF>
void launch_face_bwd_assemble(const Geo& G, const Tabs<T>& t, const TF* F, const T* u, const T* Ut, const T* Zh,
                              TF* out, int mode, cudaStream_t st);
int set_face_smem_limits();
// Float-float instantiations (kernels_ff.cu): the face-parallel form only (levels with m >= 11).
int set_ff_smem_limits();
// Condensation and recovery with the interior transforms staged through shared memory
// (fdm_stream.cuh), instantiated for float-float; recovery from the saved coefficients only.
template <typename T> LaunchCfg plan_fs(const Geo& G, int nsm);
template <typename T> void launch_fs_condense(const Geo& G, const Tabs<T>& t, const double* f_nodal, double* Z,
                                              T* Gsave, T* ws, const LaunchCfg& c, cudaStream_t st);
template <typename T> void launch_fs_recover(const Geo& G, const Tabs<T>& t, const T* Gin, const double* uhat,
                                             double* u_nodal, T* ws, const LaunchCfg& c, cudaStream_t st);
// Element Schur term in the face eigenbasis with the eigenspace streamed plane by plane
// (schur_eb.cuh): the float-float element kernel of the face-parallel levels.
template <typename T> LaunchCfg plan_schur_eb(const Geo& G, int nsm);
template <typename T> void launch_schur_eb(const Geo& G, const Tabs<T>& t, const T* Ut, T* Z, T* ws,
                                           const LaunchCfg& c, cudaStream_t st);
LaunchCfg plan_elem_fdm(const Geo& G, int nsm);
// Arithmetic T: double, or ff (float-float) where the work arrays fit in shared memory (larger
// elements take launch_fs_condense / launch_fs_recover).
// Gsave (optional): scaled interior eigen-coefficients D^{-1} S^T F_I per element, m^3 each
template <typename T>
void launch_elem_condense(const Geo& G, const Tabs<T>& t, const double* f_nodal, double* Z, T* Gsave, T* ws,
                          const LaunchCfg& c, cudaStream_t st);
// Gin (optional): the coefficients saved by launch_elem_condense for the same f_nodal
template <typename T>
void launch_elem_recover(const Geo& G, const Tabs<T>& t, const double* f_nodal, const T* Gin, const double* uhat,
                         double* u_nodal, T* ws, const LaunchCfg& c, cudaStream_t st);
template <typename T> void launch_assemble(const Geo& G, const Tabs<T>& t, const T* F, const T* u,
                                           const T* Z, T* out, int mode, cudaStream_t st);
// out = F - Hhat u (mode 0) / Hhat u (mode 1) in FP64 arithmetic with FP32 F and out
void launch_assemble_mixed(const Geo& G, const Tabs<double>& t, const float* F, const double* u, const double* Z,
                           float* out, int mode, cudaStream_t st);
void launch_assemble_rhs(const Geo& G, const Tabs<double>& t, const double* f_nodal, const double* Z,
                         double* Fhat, cudaStream_t st);
void launch_pack(const Geo& G, const double* nodal, double* hat, cudaStream_t st);
void launch_unpack(const Geo& G, const double* hat, double* nodal, cudaStream_t st);
void launch_pack_dirichlet(const Geo& G, const double* nodal, double* hat, cudaStream_t st);

// element-centred block smoother (kernels_eblock.cu)
template <typename T>
LaunchCfg plan_eblock(const Geo& G, int nsm);
template <typename T>
void launch_eblock(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws, const LaunchCfg& c, cudaStream_t st);
template <typename T>
void launch_eblock_gather(const Geo& G, const T* Ob, T* du, int accumulate, cudaStream_t st);
int set_eblock_smem_limits();
template <typename T> LaunchCfg plan_star(const Geo& G, int nsm, size_t cap = 0, int block = 0, int wide = -1);
template <typename T> void launch_star(const Geo& G, const Tabs<T>& t, const T* r, T* Ob, T* ws,
                                       const LaunchCfg& c, int* counter, cudaStream_t st);
// Star smoother with tensor-core transforms (FP32 data, TF32 or BF16 operands,
// 31 <= n_S <= 95); err is set to 1 when a tensor-core completion wait runs out
// (wait_budget clock cycles per wait); the kernel then drains its products and
// returns.
LaunchCfg plan_star_tc(const Geo& G, int nsm, int bf16);
void launch_star_tc(const Geo& G, const Tabs<float>& t, const float* r, float* Ob, const LaunchCfg& c, int* counter,
                    int* err, long long wait_budget, cudaStream_t st);
// default budget of a tensor-core completion wait: about 2 s at 2 GHz
constexpr long long kTcWaitDefault = 4000000000LL;
int set_star_tc_smem_limits();
template <typename T> void launch_star_gather(const Geo& G, const T* Ob, T* du, int accumulate,
                                              cudaStream_t st);
template <typename T> void launch_prolong_add(const Geo& Gc, const Geo& Gf, const Tabs<T>& tf,
                                              const T* uc, T* uf, cudaStream_t st);
template <typename T> void launch_restrict(const Geo& Gf, const Geo& Gc, const Tabs<T>& tf, const T* rf,
                                           T* rc, T* FB, T* EB, cudaStream_t st);
void launch_coarse_solve(const Geo& G0, const CoarseTabs& ct, const double* F0, double* U0, double* X,
                         double* Y, cudaStream_t st);
template <typename T> void launch_norm2(const T* x, int64_t n, double* partial, int npart, double* out,
                                        cudaStream_t st);
template <typename TY, typename TX> void launch_axpy(TY* y, const TX* x, double a, int64_t n,
                                                     cudaStream_t st);
template <typename TO, typename TI> void launch_copy(TO* y, const TI* x, int64_t n, cudaStream_t st);

// Device-resident scalars of Algorithm 5.
struct KrylovScal {
  double gamma, gamma0, delta, beta, alpha, qp;
};
void launch_krylov_init(KrylovScal* k, cudaStream_t st);
// gamma = z.r, gamma0 = z.s, beta = (gamma - gamma0) / delta, delta = gamma; p = beta p + z
template <typename T> void launch_krylov_beta_dir(const T* z, const double* r, const double* s, double* p,
                                                  int64_t n, double* part, int npart, KrylovScal* k,
                                                  cudaStream_t st);
// alpha = gamma / (q.p)
void launch_krylov_alpha(const double* q, const double* p, int64_t n, double* part, int npart, KrylovScal* k,
                         cudaStream_t st);
// s = r; u += alpha p; r -= alpha q; *rnorm2 = ||r||^2
void launch_krylov_update(double* u, double* r, double* s, const double* p, const double* q, int64_t n,
                          double* part, int npart, const KrylovScal* k, double* rnorm2, cudaStream_t st);

int set_kernel_smem_limits();
int smooth_with_scratch(semmg_ctx* c, int level, int dtype, const void* r, void* du, void* scratch,
                        size_t scratch_bytes, cudaStream_t st);

}  // namespace semmg
