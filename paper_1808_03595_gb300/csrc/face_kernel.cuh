// Face-parallel form of the condensed operator (Sec. 2.2).
//
// An element's Schur term H_BI H_II^{-1} H_IB sees each of its faces through
// the in-plane transform c_f Sh^T U_f Sh (elem_kernel.cuh), and returns to a
// face through the transposed transform.  The two elements sharing a face have
// the same in-plane widths on a tensor-product mesh, so both transforms are
// the same for them: they run here once per face instead of once per element
// face.  k_face_fwd transforms every face of u; the element kernel (pre = 1)
// turns the six transformed faces of an element into its six face terms in the
// same basis; k_face_bwd adds the two element terms of a face to the face part
// of H_BB u, which is diagonal in that basis, transforms the sum back and adds
// the couplings to the face's edges.  Edge and vertex slots, which have no
// Schur term, are finished by k_edge_assemble.
#pragma once
#include "elem_kernel.cuh"
#include "skel_ops.cuh"

namespace semmg {

namespace {

constexpr int kFaceThreads = 320;  // upper bound; face_threads picks the launch size

// Ut = c_f Sh^T U_f Sh for nfb consecutive faces per block (face records in t.faces).
// Shared memory: Sh[m^2], X[nfb m^2], Tt[nfb m^2], cf[nfb].
template <typename T, int PC>
__global__ void __launch_bounds__(kFaceThreads) k_face_fwd(Geo G, Tabs<T> t, const T* __restrict__ u,
                                                          T* __restrict__ Ut, int nfb, int64_t nF) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m;
  T* Sh = reinterpret_cast<T*>(smem_raw);
  T* X = Sh + mm;
  T* Tt = X + nfb * mm;
  T* cf = Tt + nfb * mm;
  const int64_t F0 = (int64_t)blockIdx.x * nfb;
  const int nf = (int)(nF - F0 < nfb ? nF - F0 : nfb);
  const FaceRec<T>* rec = t.faces + F0;
  for (int i = threadIdx.x; i < mm; i += blockDim.x) Sh[i] = t.Sh[i];
  if ((int)threadIdx.x < nf) cf[threadIdx.x] = rec[threadIdx.x].cf;
  const Lines L{m, m / 2, (m + 1) / 2, m, m, nf * mm};
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm;
    X[idx] = u[rec[j].base + (idx - j * mm)];
  }
  __syncthreads();
  fold_lines(L, 0, X, Tt);
  __syncthreads();
  tx_lines_g(L, 0, Sh, Tt, X, (T)1, (const T*)nullptr);
  __syncthreads();
  fold_lines(L, 1, X, Tt);
  __syncthreads();
  tx_lines_g(L, 1, Sh, Tt, X, (T)1, (const T*)cf);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm;
    Ut[rec[j].base + (idx - j * mm)] = X[idx];
  }
}

// The face slots of H_BB u in the face eigenbasis.  On a face (normal d,
// in-plane axes a, b; U the m x m face values, U_L / U_R the parallel faces on
// the planes below and above, W = diag(w_1..w_m)), H_BB u restricted to the
// face interior is
//   Md (M_b (x) L_a + M_a (x) L_b) U + M_a (x) M_b (lam Md U + cd0 U + cdL U_L + cdR U_R)
// plus the couplings of the in-plane lines to the face's four edges.  With
// M_a = (h_a/2) W, L_a = (2/h_a) Ls, Ls_II Sref = W Sref Lam and
// U = Sref Uh Sref^T (Uh = Sh^T U Sh, Sh = W Sref) every interior term is
// Sh (Uh scaled entrywise) Sh^T:
//   W U W -> Uh,   W U Ls_II -> Uh Lam (columns k_a),   Ls_II U W -> Lam Uh (rows k_b).
// k_face_fwd stores Ut = c_f Uh for every face, c_f^2 = (h_a/2)(h_b/2), and the
// element terms arrive as c_f Sh Zh Sh^T, so one back transform gives
//   Sh Y Sh^T,  Y = (D / c_f) Ut + c_f (cdL Ut_L + cdR Ut_R - Zh_below - Zh_above) entrywise,
//   D(k_a, k_b) = c_f^2 (lam Md + cd0) + Md ((h_b/2)(2/h_a) Lam[k_a] + (h_a/2)(2/h_b) Lam[k_b]),
// and the edge couplings are added node by node:
//   Md ((h_b/2) w_{q_b} (2/h_a) (Ls[q_a][0] U(0, q_b) + Ls[q_a][p] U(p, q_b)) + (a <-> b)).

// Edge and vertex slots (no Schur term).  Their H_BB rows are three line sums
// of about 2p terms each, so three threads share a slot (one axis each) and
// the block combines them: kEdgeSlots slots per block.
constexpr int kEdgeSlots = 64;

template <typename T, typename TF>
__global__ void __launch_bounds__(3 * kEdgeSlots) k_edge_assemble(Geo G, Tabs<T> t, const TF* __restrict__ F,
                                                                 const T* __restrict__ u, TF* __restrict__ out,
                                                                 int mode) {
  __shared__ T Ms[3][kEdgeSlots], Lsum[3][kEdgeSlots];
  const int d = threadIdx.x / kEdgeSlots, k = threadIdx.x - d * kEdgeSlots;
  const int64_t s = G.oE1 + (int64_t)blockIdx.x * kEdgeSlots + k;
  int g[3];
  bool bd = true;
  int type = 0;
  if (s < G.size) type = skel_decode(G, s, g, &bd);
  if (!bd) {
    const int nd[3] = {G.n1, G.n2, G.n3};
    bool on[3];
    for (int e = 0; e < 3; ++e) on[e] = (g[e] - divp(G, g[e]) * G.p) == 0;
    Ms[d][k] = mass1d(G, t, d, g[d], nd[d]);
    Lsum[d][k] = line_sum(G, t, u, s, type, g, d, on[(d + 1) % 3] || on[(d + 2) % 3]);
  }
  __syncthreads();
  if (d != 0 || s >= G.size) return;
  if (bd) {
    out[s] = 0;
    return;
  }
  const T M0 = Ms[0][k], M1 = Ms[1][k], M2 = Ms[2][k];
  const T Hu = (T)G.lam * M0 * M1 * M2 * u[s] + M1 * M2 * Lsum[0][k] + M0 * M2 * Lsum[1][k] + M0 * M1 * Lsum[2][k];
  out[s] = (TF)(mode == 0 ? (T)F[s] - Hu : Hu);
}

// nfb faces per block (face records in t.faces).
// Shared memory (see face_bwd_smem): FaceRec[nfb], then in T: Sh[m^2], X[nfb m^2],
// Tt[nfb m^2], lam[m], Ls[.][0][m], Ls[.][p][m], w[p+1].
template <typename T, typename TF, int PC>
__global__ void __launch_bounds__(kFaceThreads) k_face_bwd(Geo G, Tabs<T> t, const TF* __restrict__ F,
                                                          const T* __restrict__ u, const T* __restrict__ Ut,
                                                          const T* __restrict__ Zh, TF* __restrict__ out, int mode,
                                                          int nfb, int64_t nF) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = PC ? PC : G.p, m = p - 1, mm = m * m, P1 = p + 1;
  FaceRec<T>* fr = reinterpret_cast<FaceRec<T>*>(smem_raw);
  T* Sh = reinterpret_cast<T*>(fr + nfb);
  T* X = Sh + mm;
  T* Tt = X + nfb * mm;
  T* lam = Tt + nfb * mm;
  T* L0 = lam + m;
  T* Lp = L0 + m;
  T* wq = Lp + m;
  const int64_t F0 = (int64_t)blockIdx.x * nfb;
  const int nf = (int)(nF - F0 < nfb ? nF - F0 : nfb);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) Sh[i] = t.Sh[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    lam[i] = t.lamI[i];
    L0[i] = t.Ls[(i + 1) * P1];
    Lp[i] = t.Ls[(i + 1) * P1 + p];
  }
  for (int i = threadIdx.x; i < P1; i += blockDim.x) wq[i] = t.w[i];
  if ((int)threadIdx.x < nf) fr[threadIdx.x] = t.faces[F0 + threadIdx.x];
  __syncthreads();
  // Y in the face eigenbasis ([k_b][k_a], the layout of the face slots)
  const Lines L{m, m / 2, (m + 1) / 2, m, m, nf * mm};
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm, r = idx - j * mm, kb = r / m, ka = r - kb * m;
    const FaceRec<T>& f = fr[j];
    T side = 0;
    if (f.zm >= 0) side -= Zh[f.zm + r];
    if (f.zp >= 0) side -= Zh[f.zp + r];
    if (f.nbL >= 0) side += f.cdL * Ut[f.nbL + r];
    if (f.nbR >= 0) side += f.cdR * Ut[f.nbR + r];
    const T D = f.e0 + f.ea * lam[ka] + f.eb * lam[kb];
    X[idx] = D * Ut[f.base + r] + f.cf * side;
  }
  __syncthreads();
  txT_lines_g(L, 0, Sh, X, Tt);
  __syncthreads();
  unfold_lines(L, 0, Tt, X);
  __syncthreads();
  txT_lines_g(L, 1, Sh, X, Tt);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm, r = idx - j * mm, qb = r / m + 1, qa = r - (qb - 1) * m + 1;
    const FaceRec<T>& f = fr[j];
    const int64_t s = f.base + r;
    if (f.dir) {
      out[s] = 0;
      continue;
    }
    const T la = L0[qa - 1] * u[f.eA0 + (qb - 1)] + Lp[qa - 1] * u[f.eAp + (qb - 1)];
    const T lb = L0[qb - 1] * u[f.eB0 + (qa - 1)] + Lp[qb - 1] * u[f.eBp + (qa - 1)];
    const T Hu = unfold_at(L, 1, Tt, idx) + f.edA * wq[qb] * la + f.edB * wq[qa] * lb;
    out[s] = (TF)(mode == 0 ? (T)F[s] - Hu : Hu);
  }
}

// Threads of a face block: the grouped line transforms of its faces (m lines per face,
// groups of 4 outputs) in as few rounds of at most kFaceThreads as they need, the
// rounds filled evenly (m = 47: 564 work items, 2 rounds of 288 threads instead of 3 of
// 256 with the last one a fifth full).
inline int face_threads(int m, int nfb) {
  if (m < 32) return 256;  // smaller faces fill 256 threads in one or two rounds already
  const int ne = (m + 1) / 2, groups = (ne + 3) / 4 + (m - ne + 3) / 4;
  const int items = nfb * m * groups;
  const int rounds = (items + kFaceThreads - 1) / kFaceThreads;
  const int per = (items + rounds - 1) / rounds;
  const int t = (per + 31) / 32 * 32;
  return t < 64 ? 64 : t;
}

// faces per block: about 1024 face nodes, at most 32 faces
inline int face_nfb(int m) {
  const int n = 1024 / (m * m);
  return n < 1 ? 1 : (n > 32 ? 32 : n);
}

constexpr size_t kFaceSmemLimit = 200 * 1024;

template <typename T>
size_t face_fwd_smem(int m, int nfb) {
  const size_t mm = (size_t)m * m;
  return (mm + 2 * nfb * mm + nfb) * sizeof(T);
}

template <typename T>
size_t face_bwd_smem(int m, int nfb) {
  const size_t mm = (size_t)m * m;
  return nfb * sizeof(FaceRec<T>) + (mm + 2 * nfb * mm + 3 * (size_t)m + (m + 2)) * sizeof(T);
}

int64_t face_count(const Geo& G) { return (G.oE1 - G.oF1) / ((int64_t)G.m * G.m); }

template <typename T, int PC>
void face_fwd_pc(const Geo& G, const Tabs<T>& t, const T* u, T* Ut, cudaStream_t st) {
  const int64_t nF = face_count(G);
  const int nfb = face_nfb(G.m);
  const int64_t blocks = (nF + nfb - 1) / nfb;
  k_face_fwd<T, PC><<<(unsigned)blocks, face_threads(G.m, nfb), face_fwd_smem<T>(G.m, nfb), st>>>(G, t, u, Ut, nfb,
                                                                                               nF);
}

template <typename T, typename TF, int PC>
void face_bwd_pc(const Geo& G, const Tabs<T>& t, const TF* F, const T* u, const T* Ut, const T* Zh, TF* out,
                 int mode, cudaStream_t st) {
  const int64_t nF = face_count(G);
  const int nfb = face_nfb(G.m);
  const int64_t fblocks = (nF + nfb - 1) / nfb;
  const int64_t eblocks = (G.size - G.oE1 + kEdgeSlots - 1) / kEdgeSlots;
  const int nt = face_threads(G.m, nfb);
  k_face_bwd<T, TF, PC><<<(unsigned)fblocks, nt, face_bwd_smem<T>(G.m, nfb), st>>>(G, t, F, u, Ut, Zh, out, mode, nfb,
                                                                                  nF);
  if (eblocks > 0) k_edge_assemble<T, TF><<<(unsigned)eblocks, 3 * kEdgeSlots, 0, st>>>(G, t, F, u, out, mode);
}

template <typename T, typename TF, int PC>
int face_attrs_pc() {
  int bad = cudaFuncSetAttribute(k_face_bwd<T, TF, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kFaceSmemLimit);
  if (std::is_same<T, TF>::value)
    bad |= cudaFuncSetAttribute(k_face_fwd<T, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFaceSmemLimit);
  return bad;
}

template <typename T, typename TF>
int face_attrs() {
  return face_attrs_pc<T, TF, 0>() | face_attrs_pc<T, TF, 8>() | face_attrs_pc<T, TF, 16>() |
         face_attrs_pc<T, TF, 32>() | face_attrs_pc<T, TF, 48>();
}

}  // namespace

template <typename T>
void launch_face_fwd(const Geo& G, const Tabs<T>& t, const T* u, T* Ut, cudaStream_t st) {
  if (G.m == 0) return;
  switch (G.p) {
    case 8: face_fwd_pc<T, 8>(G, t, u, Ut, st); break;
    case 16: face_fwd_pc<T, 16>(G, t, u, Ut, st); break;
    case 32: face_fwd_pc<T, 32>(G, t, u, Ut, st); break;
    case 48: face_fwd_pc<T, 48>(G, t, u, Ut, st); break;
    default: face_fwd_pc<T, 0>(G, t, u, Ut, st); break;
  }
}

template <typename T, typename TF>
void launch_face_bwd_assemble(const Geo& G, const Tabs<T>& t, const TF* F, const T* u, const T* Ut, const T* Zh,
                              TF* out, int mode, cudaStream_t st) {
  switch (G.p) {
    case 8: face_bwd_pc<T, TF, 8>(G, t, F, u, Ut, Zh, out, mode, st); break;
    case 16: face_bwd_pc<T, TF, 16>(G, t, F, u, Ut, Zh, out, mode, st); break;
    case 32: face_bwd_pc<T, TF, 32>(G, t, F, u, Ut, Zh, out, mode, st); break;
    case 48: face_bwd_pc<T, TF, 48>(G, t, F, u, Ut, Zh, out, mode, st); break;
    default: face_bwd_pc<T, TF, 0>(G, t, F, u, Ut, Zh, out, mode, st); break;
  }
}

}  // namespace semmg
