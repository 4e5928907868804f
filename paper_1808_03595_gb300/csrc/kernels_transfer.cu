// Inter-level transfers of the p-multigrid (Sec. 4.1).
//
// Prolongation from degree pc to pf is the embedded interpolation, the tensor
// product of the 1D matrices J[I][i] = l^c_i(xi^f_I), restricted to the
// condensed system.  GLL includes the element end points, so a fine face
// interior depends only on the full coarse face (its interior, four edges and
// four corners): 2D interpolation per face, 1D per edge, a copy per vertex.
// Restriction is the exact transpose: every fine skeleton value is spread
// back over the coarse nodes of its face (2D), edge (1D) or vertex, and the
// pieces that land on coarse edges and corners are gathered per coarse node.
#include "semmg_internal.h"

namespace semmg {

namespace {

constexpr int kThreads = 256;

struct FaceRef {
  int d;        // normal axis
  int c;        // vertex plane along d
  int ea, eb;   // element indices along the tangential axes a < b
  int ax_a, ax_b;
};

SEMMG_HD int64_t face_count(const Geo& G, int d) {
  if (d == 0) return (int64_t)G.n3 * G.n2 * G.nv1;
  if (d == 1) return (int64_t)G.n3 * G.nv2 * G.n1;
  return (int64_t)G.nv3 * G.n2 * G.n1;
}

SEMMG_HD int64_t edge_count(const Geo& G, int d) {
  if (d == 0) return (int64_t)G.nv3 * G.nv2 * G.n1;
  if (d == 1) return (int64_t)G.nv3 * G.n2 * G.nv1;
  return (int64_t)G.n3 * G.nv2 * G.nv1;
}

// Face number (within its group) -> geometry; same order as the face groups of a condensed vector.
SEMMG_HD FaceRef face_ref(const Geo& G, int d, int64_t f) {
  FaceRef r;
  r.d = d;
  if (d == 0) {  // [a3][a2][c1]
    r.c = (int)(f % G.nv1);
    r.ea = (int)((f / G.nv1) % G.n2);
    r.eb = (int)(f / ((int64_t)G.nv1 * G.n2));
    r.ax_a = 1; r.ax_b = 2;
  } else if (d == 1) {  // [a3][c2][a1]
    r.ea = (int)(f % G.n1);
    r.c = (int)((f / G.n1) % G.nv2);
    r.eb = (int)(f / ((int64_t)G.n1 * G.nv2));
    r.ax_a = 0; r.ax_b = 2;
  } else {  // [c3][a2][a1]
    r.ea = (int)(f % G.n1);
    r.eb = (int)((f / G.n1) % G.n2);
    r.c = (int)(f / ((int64_t)G.n1 * G.n2));
    r.ax_a = 0; r.ax_b = 1;
  }
  return r;
}

SEMMG_HD int64_t face_number(const Geo& G, int d, int c, int ea, int eb) {
  if (d == 0) return ((int64_t)eb * G.n2 + ea) * G.nv1 + c;
  if (d == 1) return ((int64_t)eb * G.nv2 + c) * G.n1 + ea;
  return ((int64_t)c * G.n2 + eb) * G.n1 + ea;
}

SEMMG_HD int plane_count(const Geo& G, int d) { return d == 0 ? G.nv1 : (d == 1 ? G.nv2 : G.nv3); }
SEMMG_HD int elem_count(const Geo& G, int d) { return d == 0 ? G.n1 : (d == 1 ? G.n2 : G.n3); }

// Edge number (within its group) along axis d at vertex planes (ca, cb) of the
// other two axes a < b, element e along d.
SEMMG_HD int64_t edge_number(const Geo& G, int d, int ca, int cb, int e) {
  if (d == 0) return ((int64_t)cb * G.nv2 + ca) * G.n1 + e;   // [c3][c2][a1]
  if (d == 1) return ((int64_t)cb * G.n2 + e) * G.nv1 + ca;   // [c3][a2][c1]
  return ((int64_t)e * G.nv2 + cb) * G.nv1 + ca;               // [a3][c2][c1]
}

SEMMG_HD void edge_ref(const Geo& G, int d, int64_t k, int* ca, int* cb, int* e) {
  if (d == 0) { *e = (int)(k % G.n1); *ca = (int)((k / G.n1) % G.nv2); *cb = (int)(k / ((int64_t)G.n1 * G.nv2)); }
  else if (d == 1) { *ca = (int)(k % G.nv1); *e = (int)((k / G.nv1) % G.n2); *cb = (int)(k / ((int64_t)G.nv1 * G.n2)); }
  else { *ca = (int)(k % G.nv1); *cb = (int)((k / G.nv1) % G.nv2); *e = (int)(k / ((int64_t)G.nv1 * G.nv2)); }
}

SEMMG_HD int64_t face_group_offset(const Geo& G, int d) {
  return d == 0 ? G.oF1 : (d == 1 ? G.oF2 : G.oF3);
}
SEMMG_HD int64_t edge_group_offset(const Geo& G, int d) {
  return d == 0 ? G.oE1 : (d == 1 ? G.oE2 : G.oE3);
}

// ------------------------------------------------------------ prolongation

template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong_faces(Geo Gc, Geo Gf, const T* __restrict__ J,
                                                             const T* __restrict__ uc, T* __restrict__ uf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* C = reinterpret_cast<T*>(smem_raw);
  const int pc = Gc.p, pf = Gf.p, mf = Gf.m, P1 = pc + 1;
  T* T1 = C + P1 * P1;
  const int64_t n0 = face_count(Gf, 0), n1 = face_count(Gf, 1);
  int64_t f = blockIdx.x;
  const int d = f < n0 ? 0 : (f < n0 + n1 ? 1 : 2);
  f -= d == 0 ? 0 : (d == 1 ? n0 : n0 + n1);
  const FaceRef fr = face_ref(Gf, d, f);
  if (dir_plane(Gf, d, fr.c)) return;  // Dirichlet face
  for (int idx = threadIdx.x; idx < P1 * P1; idx += blockDim.x) {
    const int ib = idx / P1, ia = idx - ib * P1;
    int g[3];
    g[d] = fr.c * pc;
    g[fr.ax_a] = fr.ea * pc + ia;
    g[fr.ax_b] = fr.eb * pc + ib;
    C[idx] = uc[skel_index(Gc, g[0], g[1], g[2])];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P1 * mf; idx += blockDim.x) {
    const int ib = idx / mf, Ia = idx - ib * mf;
    const T* jr = J + (Ia + 1) * P1;
    const T* cr = C + ib * P1;
    T s = 0;
    for (int ia = 0; ia < P1; ++ia) s += jr[ia] * cr[ia];
    T1[idx] = s;
  }
  __syncthreads();
  T* out = uf + face_group_offset(Gf, d) + f * (int64_t)mf * mf;
  for (int idx = threadIdx.x; idx < mf * mf; idx += blockDim.x) {
    const int Ib = idx / mf, Ia = idx - Ib * mf;
    const T* jr = J + (Ib + 1) * P1;
    T s = 0;
    for (int ib = 0; ib < P1; ++ib) s += jr[ib] * T1[ib * mf + Ia];
    out[idx] += s;
  }
}

template <typename T>
__global__ void k_prolong_edges(Geo Gc, Geo Gf, const T* __restrict__ J, const T* __restrict__ uc,
                                T* __restrict__ uf) {
  const int pc = Gc.p, mf = Gf.m, P1 = pc + 1;
  const int64_t total = (edge_count(Gf, 0) + edge_count(Gf, 1) + edge_count(Gf, 2)) * mf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(t % mf);
    int64_t k = t / mf;
    int d = 0;
    while (k >= edge_count(Gf, d)) { k -= edge_count(Gf, d); ++d; }
    int ca, cb, e;
    edge_ref(Gf, d, k, &ca, &cb, &e);
    const int ax_a = d == 0 ? 1 : 0, ax_b = d == 2 ? 1 : 2;
    if (dir_plane(Gf, ax_a, ca) || dir_plane(Gf, ax_b, cb)) continue;  // on a Dirichlet face
    int g[3];
    g[ax_a] = ca * pc;
    g[ax_b] = cb * pc;
    const T* jr = J + (I + 1) * P1;
    T s = 0;
    for (int i = 0; i < P1; ++i) {
      g[d] = e * pc + i;
      s += jr[i] * uc[skel_index(Gc, g[0], g[1], g[2])];
    }
    uf[edge_group_offset(Gf, d) + k * mf + I] += s;
  }
}

template <typename T>
__global__ void k_prolong_vertices(Geo Gc, Geo Gf, const T* __restrict__ uc, T* __restrict__ uf) {
  const int64_t nv = (int64_t)Gf.nv1 * Gf.nv2 * Gf.nv3;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x)
    uf[Gf.oV + v] += uc[Gc.oV + v];
}

// ------------------------------------------------------------ restriction

// Per fine face: Full = J^T R J over the whole coarse face ((pc+1)^2, into FB);
// its interior is the coarse face interior (unique owner).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_restrict_faces(Geo Gf, Geo Gc, const T* __restrict__ J,
                                                              const T* __restrict__ rf, T* __restrict__ rc,
                                                              T* __restrict__ FB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pc = Gc.p, mc = Gc.m, mf = Gf.m, P1 = pc + 1;
  T* R = reinterpret_cast<T*>(smem_raw);
  T* T1 = R + mf * mf;
  const int64_t n0 = face_count(Gf, 0), n1 = face_count(Gf, 1);
  int64_t f = blockIdx.x;
  const int d = f < n0 ? 0 : (f < n0 + n1 ? 1 : 2);
  f -= d == 0 ? 0 : (d == 1 ? n0 : n0 + n1);
  const FaceRef fr = face_ref(Gf, d, f);
  const int64_t fnum = blockIdx.x;  // FB face numbers follow the concatenated groups
  T* fb = FB + fnum * (int64_t)P1 * P1;
  T* rcf = rc + face_group_offset(Gc, d) + f * (int64_t)mc * mc;
  if (dir_plane(Gf, d, fr.c)) {
    for (int idx = threadIdx.x; idx < P1 * P1; idx += blockDim.x) fb[idx] = 0;
    for (int idx = threadIdx.x; idx < mc * mc; idx += blockDim.x) rcf[idx] = 0;
    return;
  }
  const T* src = rf + face_group_offset(Gf, d) + f * (int64_t)mf * mf;
  for (int idx = threadIdx.x; idx < mf * mf; idx += blockDim.x) R[idx] = src[idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < mf * P1; idx += blockDim.x) {  // T1[Ib][ia] = sum_Ia R[Ib][Ia] J[Ia+1][ia]
    const int Ib = idx / P1, ia = idx - Ib * P1;
    const T* rr = R + Ib * mf;
    T s = 0;
    for (int Ia = 0; Ia < mf; ++Ia) s += rr[Ia] * J[(Ia + 1) * P1 + ia];
    T1[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P1 * P1; idx += blockDim.x) {  // Full[ib][ia] = sum_Ib J[Ib+1][ib] T1[Ib][ia]
    const int ib = idx / P1, ia = idx - ib * P1;
    T s = 0;
    for (int Ib = 0; Ib < mf; ++Ib) s += J[(Ib + 1) * P1 + ib] * T1[Ib * P1 + ia];
    fb[idx] = s;
    if (ib >= 1 && ib < pc && ia >= 1 && ia < pc) rcf[(ib - 1) * mc + (ia - 1)] = s;
  }
}

// Per fine edge and coarse index i: EB[edge][i] = sum_I J[I+1][i] r_edge[I]
template <typename T>
__global__ void k_restrict_edges(Geo Gf, Geo Gc, const T* __restrict__ J, const T* __restrict__ rf,
                                 T* __restrict__ EB) {
  const int pc = Gc.p, mf = Gf.m, P1 = pc + 1;
  const int64_t total = (edge_count(Gf, 0) + edge_count(Gf, 1) + edge_count(Gf, 2)) * P1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % P1);
    const int64_t kk = t / P1;
    int64_t k = kk;
    int d = 0;
    while (k >= edge_count(Gf, d)) { k -= edge_count(Gf, d); ++d; }
    const T* re = rf + edge_group_offset(Gf, d) + k * mf;
    T s = 0;
    for (int I = 0; I < mf; ++I) s += J[(I + 1) * P1 + i] * re[I];
    EB[kk * P1 + i] = s;  // edges on Dirichlet faces hold zero residual, so their entries are zero
  }
}

// Coarse edge interiors and vertices: gather the pieces from EB and FB.
template <typename T>
__global__ void k_restrict_gather(Geo Gf, Geo Gc, const T* __restrict__ rf, T* __restrict__ rc,
                                  const T* __restrict__ FB, const T* __restrict__ EB) {
  const int pc = Gc.p, mc = Gc.m, P1 = pc + 1;
  const int64_t nE = (edge_count(Gc, 0) + edge_count(Gc, 1) + edge_count(Gc, 2)) * mc;
  const int64_t nV = (int64_t)Gc.nv1 * Gc.nv2 * Gc.nv3;
  const int64_t eoff[3] = {0, edge_count(Gc, 0), edge_count(Gc, 0) + edge_count(Gc, 1)};
  const int64_t foff[3] = {0, face_count(Gc, 0), face_count(Gc, 0) + face_count(Gc, 1)};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nE + nV; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nE) {
      const int ic = (int)(t % mc) + 1;  // coarse local index along the edge
      int64_t k = t / mc;
      int d = 0;
      while (k >= edge_count(Gc, d)) { k -= edge_count(Gc, d); ++d; }
      int ca, cb, e;
      edge_ref(Gc, d, k, &ca, &cb, &e);
      const int ax_a = d == 0 ? 1 : 0, ax_b = d == 2 ? 1 : 2;
      T* out = rc + edge_group_offset(Gc, d) + k * mc + (ic - 1);
      if (dir_plane(Gc, ax_a, ca) || dir_plane(Gc, ax_b, cb)) {
        *out = 0;
        continue;
      }
      T s = EB[(eoff[d] + k) * P1 + ic];
      // faces normal to ax_a at plane ca: tangential axes {d, ax_b}
      // faces normal to ax_b at plane cb: tangential axes {d, ax_a}
      for (int side = 0; side < 2; ++side) {
        for (int which = 0; which < 2; ++which) {
          const int nrm = which == 0 ? ax_a : ax_b;
          const int oth = which == 0 ? ax_b : ax_a;
          const int cn = which == 0 ? ca : cb;
          const int co = which == 0 ? cb : ca;
          const int eo = wrape(Gc, oth, co - 1 + side);  // element along oth (periodic: wrapped)
          if (eo < 0 || eo >= elem_count(Gc, oth)) continue;
          const int lo = side == 1 ? 0 : pc;  // local index along oth
          // tangential ordering: a' < b'
          const int ta = d < oth ? d : oth, tb = d < oth ? oth : d;
          const int ea = ta == d ? e : eo, eb = tb == d ? e : eo;
          const int la = ta == d ? ic : lo, lb = tb == d ? ic : lo;
          const int64_t fn = foff[nrm] + face_number(Gc, nrm, cn, ea, eb);
          s += FB[fn * P1 * P1 + lb * P1 + la];
        }
      }
      *out = s;
    } else {
      const int64_t v = t - nE;
      const int c[3] = {(int)(v % Gc.nv1), (int)((v / Gc.nv1) % Gc.nv2), (int)(v / ((int64_t)Gc.nv1 * Gc.nv2))};
      T* out = rc + Gc.oV + v;
      if (dir_plane(Gc, 0, c[0]) || dir_plane(Gc, 1, c[1]) || dir_plane(Gc, 2, c[2])) {
        *out = 0;
        continue;
      }
      T s = rf[Gf.oV + v];
      for (int d = 0; d < 3; ++d) {  // six edges
        const int ax_a = d == 0 ? 1 : 0, ax_b = d == 2 ? 1 : 2;
        for (int side = 0; side < 2; ++side) {
          const int e = wrape(Gc, d, c[d] - 1 + side);
          if (e < 0 || e >= elem_count(Gc, d)) continue;
          const int64_t en = eoff[d] + edge_number(Gc, d, c[ax_a], c[ax_b], e);
          s += EB[en * P1 + (side == 1 ? 0 : pc)];
        }
      }
      for (int d = 0; d < 3; ++d) {  // twelve faces
        const int ax_a = d == 0 ? 1 : 0, ax_b = d == 2 ? 1 : 2;
        for (int sb = 0; sb < 2; ++sb)
          for (int sa = 0; sa < 2; ++sa) {
            const int ea = wrape(Gc, ax_a, c[ax_a] - 1 + sa), eb = wrape(Gc, ax_b, c[ax_b] - 1 + sb);
            if (ea < 0 || ea >= elem_count(Gc, ax_a) || eb < 0 || eb >= elem_count(Gc, ax_b)) continue;
            const int64_t fn = foff[d] + face_number(Gc, d, c[d], ea, eb);
            s += FB[fn * P1 * P1 + (sb == 1 ? 0 : pc) * P1 + (sa == 1 ? 0 : pc)];
          }
      }
      *out = s;
    }
  }
}

inline int grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
void launch_prolong_add(const Geo& Gc, const Geo& Gf, const Tabs<T>& tf, const T* uc, T* uf, cudaStream_t st) {
  const int64_t nF = face_count(Gf, 0) + face_count(Gf, 1) + face_count(Gf, 2);
  const int64_t nE = (edge_count(Gf, 0) + edge_count(Gf, 1) + edge_count(Gf, 2)) * Gf.m;
  const int64_t nV = (int64_t)Gf.nv1 * Gf.nv2 * Gf.nv3;
  const size_t smem = (size_t)((Gc.p + 1) * (Gc.p + 1) + (Gc.p + 1) * Gf.m) * sizeof(T);
  if (nF > 0 && Gf.m > 0) k_prolong_faces<T><<<(unsigned)nF, kThreads, smem, st>>>(Gc, Gf, tf.J, uc, uf);
  if (nE > 0) k_prolong_edges<T><<<grid_for(nE), kThreads, 0, st>>>(Gc, Gf, tf.J, uc, uf);
  k_prolong_vertices<T><<<grid_for(nV), kThreads, 0, st>>>(Gc, Gf, uc, uf);
}

template <typename T>
void launch_restrict(const Geo& Gf, const Geo& Gc, const Tabs<T>& tf, const T* rf, T* rc, T* FB, T* EB,
                     cudaStream_t st) {
  const int64_t nF = face_count(Gf, 0) + face_count(Gf, 1) + face_count(Gf, 2);
  const int64_t nEt = (edge_count(Gf, 0) + edge_count(Gf, 1) + edge_count(Gf, 2)) * (Gc.p + 1);
  const int64_t nG = (edge_count(Gc, 0) + edge_count(Gc, 1) + edge_count(Gc, 2)) * Gc.m +
                     (int64_t)Gc.nv1 * Gc.nv2 * Gc.nv3;
  const size_t smem = (size_t)(Gf.m * Gf.m + Gf.m * (Gc.p + 1)) * sizeof(T);
  if (nF > 0) k_restrict_faces<T><<<(unsigned)nF, kThreads, smem, st>>>(Gf, Gc, tf.J, rf, rc, FB);
  if (nEt > 0) k_restrict_edges<T><<<grid_for(nEt), kThreads, 0, st>>>(Gf, Gc, tf.J, rf, EB);
  k_restrict_gather<T><<<grid_for(nG), kThreads, 0, st>>>(Gf, Gc, rf, rc, FB, EB);
}

int64_t restrict_face_buffer(const Geo& Gf, int pc) {
  return (face_count(Gf, 0) + face_count(Gf, 1) + face_count(Gf, 2)) * (int64_t)(pc + 1) * (pc + 1);
}
int64_t restrict_edge_buffer(const Geo& Gf, int pc) {
  return (edge_count(Gf, 0) + edge_count(Gf, 1) + edge_count(Gf, 2)) * (int64_t)(pc + 1);
}

template void launch_prolong_add<double>(const Geo&, const Geo&, const Tabs<double>&, const double*, double*,
                                         cudaStream_t);
template void launch_prolong_add<float>(const Geo&, const Geo&, const Tabs<float>&, const float*, float*,
                                        cudaStream_t);
template void launch_restrict<double>(const Geo&, const Geo&, const Tabs<double>&, const double*, double*, double*,
                                      double*, cudaStream_t);
template void launch_restrict<float>(const Geo&, const Geo&, const Tabs<float>&, const float*, float*, float*,
                                     float*, cudaStream_t);

int set_transfer_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_prolong_faces<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_prolong_faces<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_restrict_faces<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_restrict_faces<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

}  // namespace semmg
