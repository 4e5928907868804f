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
// Schur term, are finished by the last blocks of the same launch.
#include "elem_kernel.cuh"
#include "skel_ops.cuh"

namespace semmg {

namespace {

constexpr int kFaceThreads = 256;

// Face F of the face groups (F1, F2, F3 in slot order).
struct FaceRef {
  int64_t base;    // slot of the face's first node
  int64_t zm, zp;  // offsets in Z of the face as side 2d+1 of the element below / side 2d of the one above, or -1
  int d, c;        // normal axis and vertex plane
  int aa, ab;      // element coordinates along the in-plane axes (fast, slow)
  int dir;         // no unknowns: a Dirichlet plane or the image plane of a periodic axis
};

__device__ FaceRef face_ref(const Geo& G, int64_t F, int64_t nF1, int64_t nF2) {
  const int64_t mm = (int64_t)G.m * G.m;
  FaceRef r;
  int a[3];
  if (F < nF1) {
    const int f = (int)F, q = f / G.nv1;
    r.d = 0;
    r.c = f - q * G.nv1;
    a[1] = q % G.n2;
    a[2] = q / G.n2;
    r.base = G.oF1 + F * mm;
  } else if (F < nF1 + nF2) {
    const int f = (int)(F - nF1), q = f / G.n1;
    r.d = 1;
    a[0] = f - q * G.n1;
    r.c = q % G.nv2;
    a[2] = q / G.nv2;
    r.base = G.oF2 + (int64_t)f * mm;
  } else {
    const int f = (int)(F - nF1 - nF2), q = f / G.n1;
    r.d = 2;
    a[0] = f - q * G.n1;
    a[1] = q % G.n2;
    r.c = q / G.n2;
    r.base = G.oF3 + (int64_t)f * mm;
  }
  const int d = r.d, ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
  r.aa = a[ia];
  r.ab = a[ib];
  r.dir = dir_plane(G, d, r.c);
  // the element below the plane is absent at a low non-periodic face (on a periodic axis
  // plane 0 is the far face of the last element), the one above at the high face
  r.zm = r.zp = -1;
  if (r.c > 0 || G.per[d]) {
    a[d] = wrape(G, d, r.c - 1);
    r.zm = ((((int64_t)a[2] * G.n2 + a[1]) * G.n1 + a[0]) * 6 + 2 * d + 1) * mm;
  }
  if (r.c < ncount(G, d)) {
    a[d] = r.c;
    r.zp = ((((int64_t)a[2] * G.n2 + a[1]) * G.n1 + a[0]) * 6 + 2 * d) * mm;
  }
  return r;
}

// c_f = sqrt(h_a h_b) / 2 of a face from the per-width tables
template <typename T>
__device__ __forceinline__ T face_cf(const Tabs<T>& t, const FaceRef& r) {
  const int ia = r.d == 0 ? 1 : 0, ib = r.d == 2 ? 1 : 2;
  return (T)0.5 * t.hx[ia][6 * r.aa + 3] * t.hx[ib][6 * r.ab + 3];
}

// Ut = c_f Sh^T U_f Sh for nfb consecutive faces per block.
// Shared memory: base[nfb] (int64), Sh[m^2], X[nfb m^2], Tt[nfb m^2], cf[nfb].
template <typename T, int PC>
__global__ void __launch_bounds__(kFaceThreads) k_face_fwd(Geo G, Tabs<T> t, const T* __restrict__ u,
                                                          T* __restrict__ Ut, int nfb, int64_t nF, int64_t nF1,
                                                          int64_t nF2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = PC ? PC - 1 : G.m, mm = m * m;
  int64_t* base = reinterpret_cast<int64_t*>(smem_raw);
  T* Sh = reinterpret_cast<T*>(base + nfb);
  T* X = Sh + mm;
  T* Tt = X + nfb * mm;
  T* cf = Tt + nfb * mm;
  const int64_t F0 = (int64_t)blockIdx.x * nfb;
  const int nf = (int)(nF - F0 < nfb ? nF - F0 : nfb);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) Sh[i] = t.Sh[i];
  if ((int)threadIdx.x < nf) {
    const FaceRef r = face_ref(G, F0 + threadIdx.x, nF1, nF2);
    base[threadIdx.x] = r.base;
    cf[threadIdx.x] = face_cf(t, r);
  }
  __syncthreads();
  const Lines L{m, m / 2, (m + 1) / 2, m, m, nf * mm};
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm;
    X[idx] = u[base[j] + (idx - j * mm)];
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
    Ut[base[j] + (idx - j * mm)] = X[idx];
  }
}

// Per-face constants of the skeleton assembly on a face (normal axis d, plane
// c, in-plane axes a (fast) and b (slow)): masses, stiffness scales and the
// slots of the face's four edges and of the two parallel faces across the
// element below and above.
template <typename T>
struct FaceAsm {
  T cA, cB;         // h_a / 2, h_b / 2 (in-plane masses are these times the GLL weight)
  T kA, kB;         // 2 / h_a, 2 / h_b
  T Md, lamMd;      // assembled normal mass on the plane, lam times it
  T cd0, cdL, cdR;  // normal line sum: cd0 u + cdL u(plane c-1) + cdR u(plane c+1)
  int64_t eA0, eAp, eB0, eBp;  // first slots of the edges at q_a = 0, q_a = p, q_b = 0, q_b = p
  int64_t nbL, nbR;            // first slots of the parallel faces on planes c-1, c+1, or -1
};

template <typename T>
__device__ FaceAsm<T> face_asm(const Geo& G, const Tabs<T>& t, const FaceRef& r) {
  const int p = G.p, d = r.d, ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
  const bool hasL = r.c > 0 || G.per[d], hasR = r.c < ncount(G, d);
  FaceAsm<T> f;
  f.cA = (T)0.5 * t.h[ia][r.aa];
  f.cB = (T)0.5 * t.h[ib][r.ab];
  f.kA = t.hx[ia][6 * r.aa + 1];
  f.kB = t.hx[ib][6 * r.ab + 1];
  const int eL = hasL ? wrape(G, d, r.c - 1) : 0;
  const T kL = hasL ? t.hx[d][6 * eL + 1] : (T)0, kR = hasR ? t.hx[d][6 * r.c + 1] : (T)0;
  T Md = 0;
  if (hasL) Md += (T)0.5 * t.h[d][eL] * t.w[p];
  if (hasR) Md += (T)0.5 * t.h[d][r.c] * t.w[0];
  f.Md = Md;
  f.lamMd = (T)G.lam * Md;
  f.cd0 = kL * t.Ls[p * (p + 1) + p] + kR * t.Ls[0];
  f.cdL = kL * t.Ls[p * (p + 1)];
  f.cdR = kR * t.Ls[p];
  int g[3];
  g[d] = r.c * p;
  g[ia] = r.aa * p;
  g[ib] = r.ab * p + 1;
  f.eA0 = skel_index(G, g[0], g[1], g[2]);
  g[ia] = r.aa * p + p;
  f.eAp = skel_index(G, g[0], g[1], g[2]);
  g[ia] = r.aa * p + 1;
  g[ib] = r.ab * p;
  f.eB0 = skel_index(G, g[0], g[1], g[2]);
  g[ib] = r.ab * p + p;
  f.eBp = skel_index(G, g[0], g[1], g[2]);
  g[ib] = r.ab * p + 1;
  g[d] = (r.c - 1) * p;  // wraps on a periodic axis
  f.nbL = hasL ? skel_index(G, g[0], g[1], g[2]) : -1;
  g[d] = (r.c + 1) * p;
  f.nbR = hasR ? skel_index(G, g[0], g[1], g[2]) : -1;
  return f;
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

// Blocks [0, nfblocks): nfb faces each; the rest: one edge or vertex slot per thread.
// Shared memory (see face_bwd_smem): FaceRef[nfb], FaceAsm[nfb], then in T: Sh[m^2],
// X[nfb m^2], Tt[nfb m^2], lam[m], Ls[.][0][m], Ls[.][p][m], w[p+1], cf, e0, ea, eb [nfb each].
template <typename T, typename TF, int PC>
__global__ void __launch_bounds__(kFaceThreads) k_face_bwd(Geo G, Tabs<T> t, const TF* __restrict__ F,
                                                          const T* __restrict__ u, const T* __restrict__ Ut,
                                                          const T* __restrict__ Zh, TF* __restrict__ out, int mode,
                                                          int nfb, int64_t nF, int64_t nF1, int64_t nF2,
                                                          int nfblocks) {
  if ((int)blockIdx.x >= nfblocks) {
    const int64_t s = G.oE1 + (int64_t)(blockIdx.x - nfblocks) * blockDim.x + threadIdx.x;
    if (s >= G.size) return;
    int g[3];
    bool bd;
    const int type = skel_decode(G, s, g, &bd);
    if (bd) {
      out[s] = 0;
      return;
    }
    const T Hu = node_hbb(G, t, u, s, type, g);
    out[s] = (TF)(mode == 0 ? (T)F[s] - Hu : Hu);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = PC ? PC : G.p, m = p - 1, mm = m * m, P1 = p + 1;
  FaceRef* fr = reinterpret_cast<FaceRef*>(smem_raw);
  FaceAsm<T>* fa = reinterpret_cast<FaceAsm<T>*>(fr + nfb);
  T* Sh = reinterpret_cast<T*>(fa + nfb);
  T* X = Sh + mm;
  T* Tt = X + nfb * mm;
  T* lam = Tt + nfb * mm;
  T* L0 = lam + m;
  T* Lp = L0 + m;
  T* wq = Lp + m;
  T* cf = wq + P1;
  T* e0 = cf + nfb;
  T* ea = e0 + nfb;
  T* eb = ea + nfb;
  const int64_t F0 = (int64_t)blockIdx.x * nfb;
  const int nf = (int)(nF - F0 < nfb ? nF - F0 : nfb);
  for (int i = threadIdx.x; i < mm; i += blockDim.x) Sh[i] = t.Sh[i];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    lam[i] = t.lamI[i];
    L0[i] = t.Ls[(i + 1) * P1];
    Lp[i] = t.Ls[(i + 1) * P1 + p];
  }
  for (int i = threadIdx.x; i < P1; i += blockDim.x) wq[i] = t.w[i];
  if ((int)threadIdx.x < nf) {
    const FaceRef r = face_ref(G, F0 + threadIdx.x, nF1, nF2);
    const FaceAsm<T> f = face_asm(G, t, r);
    const T c = face_cf(t, r);
    fr[threadIdx.x] = r;
    fa[threadIdx.x] = f;
    cf[threadIdx.x] = c;
    e0[threadIdx.x] = c * (f.lamMd + f.cd0);
    ea[threadIdx.x] = f.Md * f.cB * f.kA / c;
    eb[threadIdx.x] = f.Md * f.cA * f.kB / c;
  }
  __syncthreads();
  // Y in the face eigenbasis ([k_b][k_a], the layout of the face slots)
  const Lines L{m, m / 2, (m + 1) / 2, m, m, nf * mm};
  for (int idx = threadIdx.x; idx < nf * mm; idx += blockDim.x) {
    const int j = idx / mm, r = idx - j * mm, kb = r / m, ka = r - kb * m;
    const FaceRef& fj = fr[j];
    const FaceAsm<T>& f = fa[j];
    T side = 0;
    if (fj.zm >= 0) side -= Zh[fj.zm + r];
    if (fj.zp >= 0) side -= Zh[fj.zp + r];
    if (f.nbL >= 0) side += f.cdL * Ut[f.nbL + r];
    if (f.nbR >= 0) side += f.cdR * Ut[f.nbR + r];
    const T D = e0[j] + ea[j] * lam[ka] + eb[j] * lam[kb];
    X[idx] = D * Ut[fj.base + r] + cf[j] * side;
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
    const FaceRef& fj = fr[j];
    const int64_t s = fj.base + r;
    if (fj.dir) {
      out[s] = 0;
      continue;
    }
    const FaceAsm<T>& f = fa[j];
    const T la = L0[qa - 1] * u[f.eA0 + (qb - 1)] + Lp[qa - 1] * u[f.eAp + (qb - 1)];
    const T lb = L0[qb - 1] * u[f.eB0 + (qa - 1)] + Lp[qb - 1] * u[f.eBp + (qa - 1)];
    const T Hu = unfold_at(L, 1, Tt, idx) + f.Md * (f.cB * wq[qb] * f.kA * la + f.cA * wq[qa] * f.kB * lb);
    out[s] = (TF)(mode == 0 ? (T)F[s] - Hu : Hu);
  }
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
  return nfb * sizeof(int64_t) + (mm + 2 * nfb * mm + nfb) * sizeof(T);
}

template <typename T>
size_t face_bwd_smem(int m, int nfb) {
  const size_t mm = (size_t)m * m;
  const size_t elems = mm + 2 * nfb * mm + 3 * (size_t)m + (m + 2) + 4 * (size_t)nfb;
  return nfb * (sizeof(FaceRef) + sizeof(FaceAsm<T>)) + elems * sizeof(T);
}

void face_counts(const Geo& G, int64_t* nF1, int64_t* nF2, int64_t* nF) {
  const int64_t mm = (int64_t)G.m * G.m;
  *nF1 = (G.oF2 - G.oF1) / mm;
  *nF2 = (G.oF3 - G.oF2) / mm;
  *nF = (G.oE1 - G.oF1) / mm;
}

template <typename T, int PC>
void face_fwd_pc(const Geo& G, const Tabs<T>& t, const T* u, T* Ut, cudaStream_t st) {
  int64_t nF1, nF2, nF;
  face_counts(G, &nF1, &nF2, &nF);
  const int nfb = face_nfb(G.m);
  const int64_t blocks = (nF + nfb - 1) / nfb;
  k_face_fwd<T, PC><<<(unsigned)blocks, kFaceThreads, face_fwd_smem<T>(G.m, nfb), st>>>(G, t, u, Ut, nfb, nF, nF1,
                                                                                        nF2);
}

template <typename T, typename TF, int PC>
void face_bwd_pc(const Geo& G, const Tabs<T>& t, const TF* F, const T* u, const T* Ut, const T* Zh, TF* out,
                 int mode, cudaStream_t st) {
  int64_t nF1, nF2, nF;
  face_counts(G, &nF1, &nF2, &nF);
  const int nfb = face_nfb(G.m);
  const int64_t fblocks = (nF + nfb - 1) / nfb;
  const int64_t eblocks = (G.size - G.oE1 + kFaceThreads - 1) / kFaceThreads;
  k_face_bwd<T, TF, PC><<<(unsigned)(fblocks + eblocks), kFaceThreads, face_bwd_smem<T>(G.m, nfb), st>>>(
      G, t, F, u, Ut, Zh, out, mode, nfb, nF, nF1, nF2, (int)fblocks);
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
         face_attrs_pc<T, TF, 32>();
}

}  // namespace

template <typename T>
void launch_face_fwd(const Geo& G, const Tabs<T>& t, const T* u, T* Ut, cudaStream_t st) {
  if (G.m == 0) return;
  switch (G.p) {
    case 8: face_fwd_pc<T, 8>(G, t, u, Ut, st); break;
    case 16: face_fwd_pc<T, 16>(G, t, u, Ut, st); break;
    case 32: face_fwd_pc<T, 32>(G, t, u, Ut, st); break;
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
    default: face_bwd_pc<T, TF, 0>(G, t, F, u, Ut, Zh, out, mode, st); break;
  }
}

// largest face-kernel shared memory at degree p (both element types), for setup checks
size_t face_smem_bytes(int p) {
  const int m = p - 1;
  if (m < 1) return 0;
  const int nfb = face_nfb(m);
  return std::max(face_fwd_smem<double>(m, nfb), face_bwd_smem<double>(m, nfb));
}

int set_face_smem_limits() {
  return face_attrs<double, double>() | face_attrs<float, float>() | face_attrs<double, float>();
}

template void launch_face_fwd<double>(const Geo&, const Tabs<double>&, const double*, double*, cudaStream_t);
template void launch_face_fwd<float>(const Geo&, const Tabs<float>&, const float*, float*, cudaStream_t);
template void launch_face_bwd_assemble<double, double>(const Geo&, const Tabs<double>&, const double*,
                                                       const double*, const double*, const double*, double*, int,
                                                       cudaStream_t);
template void launch_face_bwd_assemble<float, float>(const Geo&, const Tabs<float>&, const float*, const float*,
                                                     const float*, const float*, float*, int, cudaStream_t);
template void launch_face_bwd_assemble<double, float>(const Geo&, const Tabs<double>&, const float*, const double*,
                                                      const double*, const double*, float*, int, cudaStream_t);

}  // namespace semmg
