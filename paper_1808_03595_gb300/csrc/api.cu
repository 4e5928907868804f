// C ABI of the semmg library: context setup (level hierarchy of Sec. 4.1),
// buffer management and the orchestration of Algorithms 2-4 on one stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <new>
#include <string>
#include <vector>

#include "semmg_internal.h"
#include "setup_host.h"

namespace semmg {
int set_elem_smem_limits();
int set_star_smem_limits();
int set_transfer_smem_limits();
int set_face_smem_limits();
int64_t restrict_face_buffer(const Geo& Gf, int pc);
int64_t restrict_edge_buffer(const Geo& Gf, int pc);
}  // namespace semmg

using namespace semmg;

namespace {

// default of the divergence stop: the outer iteration ends when ||r|| exceeds
// this multiple of ||r_0|| (semmg_set_guards changes it per context)
constexpr double kDivergence = 1e3;


struct DevLevel {
  Tabs<double> td{};
  Tabs<float> tf{};
  Tabs<ff> tff{};      // float-float tables (SEMMG_MIXED_FF, _FF_TC; face-parallel levels only)
  void* Fw = nullptr;  // V-cycle vectors in the working precision
  void* Uw = nullptr;
  void* Rw = nullptr;
  LaunchCfg schur64, schur32, star64, star32;
  LaunchCfg startc;  // tensor-core star smoother (SEMMG_MIXED_TC, _FP32_TC, _BF16, _FF_TC), when the level allows it
  LaunchCfg eb64, eb32;  // element-centred block smoother (SEMMG_SMOOTHER_ELEMENT)
};

// n_S rounded up to 16, the operand size of the tensor-core star tables
int tc_pad(int nS) { return (nS + 15) / 16 * 16; }

// IEEE float rounded to TF32 (10 stored mantissa bits), nearest-even
float round_tf32(double x) {
  float f = (float)x;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  if ((b & 0x7F800000u) != 0x7F800000u) {
    b += 0xFFFu + ((b >> 13) & 1u);
    b &= ~0x1FFFu;
  }
  std::memcpy(&f, &b, 4);
  return f;
}

// IEEE float rounded to BF16 (7 stored mantissa bits), nearest-even: the bit pattern
uint16_t round_bf16_bits(double x) {
  float f = (float)x;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  if ((b & 0x7F800000u) != 0x7F800000u) b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

// element offset of (row, k) in a K-major tensor-core operand with K = np and E
// elements per 16-byte core-matrix row (4 for TF32, 8 for BF16)
size_t tc_off(int row, int k, int np, int E) {
  return ((size_t)(row >> 3) * (np / E) + (k / E)) * (8 * E) + (row & 7) * E + (k % E);
}

Geo make_geo(const int n[3], int p, double lam, const int bc[6]) {
  Geo g{};
  for (int f = 0; f < 6; ++f) g.dir[f] = bc[f] == SEMMG_BC_DIRICHLET ? 1 : 0;
  for (int d = 0; d < 3; ++d) g.per[d] = bc[2 * d] == SEMMG_BC_PERIODIC ? 1 : 0;
  g.p = p;
  g.m = p - 1;
  g.nS = 2 * p - 1;
  g.n1 = n[0]; g.n2 = n[1]; g.n3 = n[2];
  g.nv1 = n[0] + 1; g.nv2 = n[1] + 1; g.nv3 = n[2] + 1;
  const int64_t m = g.m, mm = m * m;
  g.oF1 = 0;
  g.oF2 = g.oF1 + (int64_t)g.n3 * g.n2 * g.nv1 * mm;
  g.oF3 = g.oF2 + (int64_t)g.n3 * g.nv2 * g.n1 * mm;
  g.oE1 = g.oF3 + (int64_t)g.nv3 * g.n2 * g.n1 * mm;
  g.oE2 = g.oE1 + (int64_t)g.nv3 * g.nv2 * g.n1 * m;
  g.oE3 = g.oE2 + (int64_t)g.nv3 * g.n2 * g.nv1 * m;
  g.oV = g.oE3 + (int64_t)g.n3 * g.nv2 * g.nv1 * m;
  g.size = g.oV + (int64_t)g.nv1 * g.nv2 * g.nv3;
  g.nelem = (int64_t)g.n1 * g.n2 * g.n3;
  g.nstar = (int64_t)g.nv1 * g.nv2 * g.nv3;
  g.pinv = ((1ull << 32) + (uint64_t)p - 1) / (uint64_t)p;
  g.lam = lam;
  return g;
}

}  // namespace

struct semmg_ctx {
  semmg_opts opts{};
  double lam = 0;
  int nsm = 0;
  std::vector<double> h[3];
  std::vector<Geo> geo;
  std::vector<HostLevel> hl;
  std::vector<DevLevel> dl;
  HostCoarse hc;
  CoarseTabs ct{};
  std::vector<void*> allocs;
  // shared scratch (sized in doubles for the largest level)
  void* Zs = nullptr;
  void* Obs = nullptr;
  void* FBs = nullptr;
  void* EBs = nullptr;
  void* wss = nullptr;
  size_t ws_bytes = 0;
  LaunchCfg fdm;
  LaunchCfg fsff;  // float-float condensation and recovery (fdm_stream.cuh), when the form and level allow it
  // FP64 outer iteration
  double* Fh = nullptr;
  double* Uh = nullptr;
  double* Rh = nullptr;
  // scaled interior eigen-coefficients of the right-hand side, kept from the
  // condensation to the recovery of one solve (nelem m^3 at the finest level)
  double* Gs = nullptr;
  // FP64 copy of a level's u for the FP64 level residuals of the SEMMG_MIXED cycle
  double* U64s = nullptr;
  // faces of a level's u in the interior eigenbasis (face-parallel operator form;
  // face slots of the finest level, in doubles)
  void* Uts = nullptr;
  // Algorithm 5 vectors (old residual s, search direction p, q = Hhat p) and scalars
  double* kS = nullptr;
  double* kP = nullptr;
  double* kQ = nullptr;
  KrylovScal* kscal = nullptr;
  // coarse solve
  double* cX = nullptr;
  double* cY = nullptr;
  double* F0d = nullptr;
  double* U0d = nullptr;
  // norms
  double* part = nullptr;
  int npart = 0;
  double* dnorm = nullptr;
  double* hnorm = nullptr;  // pinned
  int* star_counter = nullptr;  // work counter of the star kernel (self-resetting)
  int* dev_err = nullptr;       // set by a kernel whose bounded device wait ran out
  int* hdev_err = nullptr;      // pinned copy
  // failure-detection limits (semmg_set_guards)
  double divergence = kDivergence;
  long long tc_wait = kTcWaitDefault;
  // host-buffer solve
  double* fnod = nullptr;
  double* unod = nullptr;
  std::string err;
  // timing
  int timing = 0;
  struct Pending { int kind; int ev; double flops, bytes; int64_t launches; double xflops; };
  std::vector<cudaEvent_t> events;
  std::vector<Pending> pending;
  int ev_used = 0;
  semmg_kstat ks[SEMMG_K_COUNT] = {};
  // one outer iteration captured as a CUDA graph (replayed by semmg_solve while
  // timing is off); rebuilt after launch shapes change
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  int step_capture_failed = 0;
  // per-kernel timing inside that graph: its own events (recorded by event nodes) and
  // launch groups, read after every replay
  bool capturing = false;
  std::vector<cudaEvent_t> step_events;
  std::vector<Pending> step_pending;
  int step_ev_used = 0;
  bool step_replayed = false;

  int L() const { return (int)geo.size() - 1; }

  void drop_step_graph() {
    if (step_exec) cudaGraphExecDestroy(step_exec);
    step_exec = nullptr;
    step_capture_failed = 0;
    step_pending.clear();
    step_replayed = false;
  }

  ~semmg_ctx() {
    drop_step_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t e : step_events) cudaEventDestroy(e);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    if (hnorm) cudaFreeHost(hnorm);
    if (hdev_err) cudaFreeHost(hdev_err);
    cudaGetLastError();
  }
};

namespace {

int fail(semmg_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int check_cuda(semmg_ctx* c, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, SEMMG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
  return SEMMG_OK;
}

void* dalloc(semmg_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->allocs.push_back(p);
  return p;
}

template <typename T>
const T* upload(semmg_ctx* c, const std::vector<double>& v, bool* ok) {
  std::vector<T> tmp(v.begin(), v.end());
  T* d = (T*)dalloc(c, tmp.size() * sizeof(T));
  if (!d) {
    *ok = false;
    return nullptr;
  }
  if (!tmp.empty() && cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    *ok = false;
  return d;
}

const unsigned char* upload_u8(semmg_ctx* c, const std::vector<unsigned char>& v, bool* ok) {
  unsigned char* d = (unsigned char*)dalloc(c, v.size());
  if (!d) {
    *ok = false;
    return nullptr;
  }
  if (!v.empty() && cudaMemcpy(d, v.data(), v.size(), cudaMemcpyHostToDevice) != cudaSuccess) *ok = false;
  return d;
}

// The face records of a face-parallel level (FaceRec), in face order.
template <typename T>
std::vector<FaceRec<T>> build_face_recs(const Geo& G, const HostLevel& H, const std::vector<double>* h) {
  const int p = G.p, P1 = p + 1;
  const int64_t mm = (int64_t)G.m * G.m;
  const int nd[3] = {G.n1, G.n2, G.n3}, nv[3] = {G.nv1, G.nv2, G.nv3};
  std::vector<FaceRec<T>> out;
  out.reserve((size_t)((G.oE1 - G.oF1) / mm));
  for (int d = 0; d < 3; ++d) {
    const int ia = d == 0 ? 1 : 0, ib = d == 2 ? 1 : 2;
    // slot order of the group: F1 [a3][a2][c1], F2 [a3][c2][a1], F3 [c3][a2][a1]
    int ext[3];
    for (int e = 0; e < 3; ++e) ext[e] = e == d ? nv[e] : nd[e];
    for (int i2 = 0; i2 < ext[2]; ++i2)
      for (int i1 = 0; i1 < ext[1]; ++i1)
        for (int i0 = 0; i0 < ext[0]; ++i0) {
          int a[3] = {i0, i1, i2};
          const int c = a[d];
          FaceRec<T> r{};
          const int64_t f = (int64_t)out.size() - (d == 0 ? 0 : (d == 1 ? (G.oF2 - G.oF1) / mm : (G.oF3 - G.oF1) / mm));
          r.base = (d == 0 ? G.oF1 : (d == 1 ? G.oF2 : G.oF3)) + f * mm;
          r.dir = dir_plane(G, d, c);
          const bool hasL = c > 0 || G.per[d], hasR = c < nd[d];
          const int eL = hasL ? wrape(G, d, c - 1) : 0;
          r.zm = r.zp = r.nbL = r.nbR = -1;
          if (hasL) {
            int e[3] = {a[0], a[1], a[2]};
            e[d] = eL;
            r.zm = ((((int64_t)e[2] * G.n2 + e[1]) * G.n1 + e[0]) * 6 + 2 * d + 1) * mm;
          }
          if (hasR) r.zp = ((((int64_t)a[2] * G.n2 + a[1]) * G.n1 + a[0]) * 6 + 2 * d) * mm;
          const double ha = h[ia][a[ia]], hb = h[ib][a[ib]];
          const double cA = 0.5 * ha, cB = 0.5 * hb, kA = 2.0 / ha, kB = 2.0 / hb;
          const double kL = hasL ? 2.0 / h[d][eL] : 0.0, kR = hasR ? 2.0 / h[d][c] : 0.0;
          double Md = 0.0;
          if (hasL) Md += 0.5 * h[d][eL] * H.w[p];
          if (hasR) Md += 0.5 * h[d][c] * H.w[0];
          const double cd0 = kL * H.Ls[(size_t)p * P1 + p] + kR * H.Ls[0];
          const double cf = 0.5 * std::sqrt(ha) * std::sqrt(hb);
          r.cf = (T)cf;
          r.e0 = (T)(cf * (G.lam * Md + cd0));
          r.ea = (T)(Md * cB * kA / cf);
          r.eb = (T)(Md * cA * kB / cf);
          r.cdL = (T)(kL * H.Ls[(size_t)p * P1]);
          r.cdR = (T)(kR * H.Ls[p]);
          r.edA = (T)(Md * cB * kA);
          r.edB = (T)(Md * cA * kB);
          int g[3];
          g[d] = c * p;
          g[ia] = a[ia] * p;
          g[ib] = a[ib] * p + 1;
          r.eA0 = skel_index(G, g[0], g[1], g[2]);
          g[ia] = a[ia] * p + p;
          r.eAp = skel_index(G, g[0], g[1], g[2]);
          g[ia] = a[ia] * p + 1;
          g[ib] = a[ib] * p;
          r.eB0 = skel_index(G, g[0], g[1], g[2]);
          g[ib] = a[ib] * p + p;
          r.eBp = skel_index(G, g[0], g[1], g[2]);
          g[ib] = a[ib] * p + 1;
          g[d] = (c - 1) * p;  // wraps on a periodic axis
          if (hasL) r.nbL = skel_index(G, g[0], g[1], g[2]);
          g[d] = (c + 1) * p;
          if (hasR) r.nbR = skel_index(G, g[0], g[1], g[2]);
          out.push_back(r);
        }
  }
  return out;
}

template <typename T>
Tabs<T> upload_tabs(semmg_ctx* c, const Geo& G, const HostLevel& H, const std::vector<double>* h, bool* ok) {
  Tabs<T> t{};
  t.faces = nullptr;
  if (face_form(G)) {
    const std::vector<FaceRec<T>> fr = build_face_recs<T>(G, H, h);
    void* d = dalloc(c, fr.size() * sizeof(FaceRec<T>));
    if (!d || cudaMemcpy(d, fr.data(), fr.size() * sizeof(FaceRec<T>), cudaMemcpyHostToDevice) != cudaSuccess)
      *ok = false;
    t.faces = (const FaceRec<T>*)d;
  }
  t.w = upload<T>(c, H.w, ok);
  t.Ls = upload<T>(c, H.Ls, ok);
  t.Sh = upload<T>(c, H.Sh, ok);
  t.Sref = upload<T>(c, H.Sref, ok);
  t.a0 = upload<T>(c, H.a0, ok);
  t.ap = upload<T>(c, H.ap, ok);
  t.lamI = upload<T>(c, H.lamI, ok);
  for (int d = 0; d < 3; ++d) {
    t.h[d] = upload<T>(c, h[d], ok);
    std::vector<double> hx(6 * h[d].size());
    for (size_t a = 0; a < h[d].size(); ++a) {
      const double ha = h[d][a];
      hx[6 * a + 0] = ha;
      hx[6 * a + 1] = 2.0 / ha;
      hx[6 * a + 2] = 4.0 / (ha * ha);
      hx[6 * a + 3] = std::sqrt(ha);
      hx[6 * a + 4] = std::pow(2.0 / ha, 1.5);
      hx[6 * a + 5] = std::sqrt(2.0 / ha);
    }
    t.hx[d] = upload<T>(c, hx, ok);
    t.starS[d] = upload<T>(c, H.starS[d], ok);
    t.starLam[d] = upload<T>(c, H.starLam[d], ok);
    t.act[d] = upload_u8(c, H.act[d], ok);
  }
  for (int d = 0; d < 3; ++d) {
    t.starSym[d] = upload_u8(c, H.sym[d], ok);
    std::vector<int> ci(H.cls[d].begin(), H.cls[d].end());
    int* dci = (int*)dalloc(c, ci.size() * sizeof(int));
    if (!dci || cudaMemcpy(dci, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) *ok = false;
    t.starCls[d] = dci;
    t.ncls[d] = (int)H.rep[d].size();
  }
  t.Rtab = nullptr;  // built by build_star_rtab (FP64 only)
  for (int d = 0; d < 3; ++d) {
    const std::vector<int>& hc = H.hcls[d];
    int* dhc = (int*)dalloc(c, hc.size() * sizeof(int));
    if (!dhc || cudaMemcpy(dhc, hc.data(), hc.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) *ok = false;
    t.hcls[d] = dhc;
    t.nhcls[d] = (int)H.hval[d].size();
  }
  t.Relem = H.Relem.empty() ? nullptr : upload<T>(c, H.Relem, ok);
  t.w1d = upload<T>(c, H.w1d, ok);
  for (int d = 0; d < 3; ++d) {
    t.ebS[d] = H.ebS[d].empty() ? nullptr : upload<T>(c, H.ebS[d], ok);
    t.ebST[d] = H.ebST[d].empty() ? nullptr : upload<T>(c, H.ebST[d], ok);
    t.ebLam[d] = H.ebLam[d].empty() ? nullptr : upload<T>(c, H.ebLam[d], ok);
    t.ebW[d] = H.ebW[d].empty() ? nullptr : upload<T>(c, H.ebW[d], ok);
    t.ebCls[d] = nullptr;
    t.ebNcls[d] = (int)H.ebRep[d].size();
    if (!H.ebCls[d].empty()) {
      int* dc = (int*)dalloc(c, H.ebCls[d].size() * sizeof(int));
      if (!dc || cudaMemcpy(dc, H.ebCls[d].data(), H.ebCls[d].size() * sizeof(int), cudaMemcpyHostToDevice) !=
                     cudaSuccess)
        *ok = false;
      t.ebCls[d] = dc;
    }
  }
  t.ebR = H.ebR.empty() ? nullptr : upload<T>(c, H.ebR, ok);
  t.J = H.J.empty() ? nullptr : upload<T>(c, H.J, ok);
  t.pc = H.pc;
  return t;
}

// Tensor-core operand tables T(S) and N(S) per axis and line class, TF32 or BF16.
void upload_tc_tables(semmg_ctx* c, const HostLevel& H, Tabs<float>& t, bool bf16, bool* ok) {
  const int nS = 2 * H.p - 1, np = tc_pad(nS), E = bf16 ? 8 : 4;
  const size_t tb = (size_t)np * np;
  for (int d = 0; d < 3; ++d) {
    const size_t ncls = H.rep[d].size();
    std::vector<float> T, N;
    std::vector<uint16_t> Tb, Nb;
    if (bf16) {
      Tb.assign(ncls * tb, 0);
      Nb.assign(ncls * tb, 0);
    } else {
      T.assign(ncls * tb, 0.0f);
      N.assign(ncls * tb, 0.0f);
    }
    for (size_t r = 0; r < ncls; ++r) {
      const double* S = &H.starS[d][(size_t)H.rep[d][r] * nS * nS];
      for (int j = 0; j < nS; ++j)
        for (int e = 0; e < nS; ++e) {
          if (bf16) {
            const uint16_t v = round_bf16_bits(S[j * nS + e]);
            Tb[r * tb + tc_off(e, j, np, E)] = v;
            Nb[r * tb + tc_off(j, e, np, E)] = v;
          } else {
            const float v = round_tf32(S[j * nS + e]);
            T[r * tb + tc_off(e, j, np, E)] = v;
            N[r * tb + tc_off(j, e, np, E)] = v;
          }
        }
    }
    const size_t bytes = ncls * tb * (bf16 ? 2 : 4);
    void* dT = dalloc(c, bytes);
    void* dN = dalloc(c, bytes);
    const void* hT = bf16 ? (const void*)Tb.data() : (const void*)T.data();
    const void* hN = bf16 ? (const void*)Nb.data() : (const void*)N.data();
    if (!dT || !dN || cudaMemcpy(dT, hT, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dN, hN, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      *ok = false;
    if (bf16) {
      t.bfT[d] = (const unsigned short*)dT;
      t.bfN[d] = (const unsigned short*)dN;
    } else {
      t.tcT[d] = (const float*)dT;
      t.tcN[d] = (const float*)dN;
    }
  }
}

// 1/(lam + Lam1[k1] + Lam2[k2] + Lam3[k3]) for every star class (class
// (r1 n2c + r2) n3c + r3, layout [k3][k2][k1] per class), from the eigenvalues
// of the classes' representative vertex lines; IEEE division, the sum in the
// order lam + Lam1 + Lam2 + Lam3.
__global__ void k_build_rtab(int nS, int n2c, int n3c, const int* __restrict__ rep1, const int* __restrict__ rep2,
                             const int* __restrict__ rep3, const double* __restrict__ L1,
                             const double* __restrict__ L2, const double* __restrict__ L3, double lam, int64_t total,
                             double* __restrict__ R) {
  const int64_t n3 = (int64_t)nS * nS * nS;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cls = i / n3, k = i - cls * n3;
    const int k1 = (int)(k % nS), k2 = (int)((k / nS) % nS), k3 = (int)(k / ((int64_t)nS * nS));
    const int r3 = (int)(cls % n3c), r2 = (int)((cls / n3c) % n2c), r1 = (int)(cls / ((int64_t)n3c * n2c));
    R[i] = 1.0 / (lam + L1[(int64_t)rep1[r1] * nS + k1] + L2[(int64_t)rep2[r2] * nS + k2] +
                  L3[(int64_t)rep3[r3] * nS + k3]);
  }
}

// The FP64 star kernel's 1/D tables of a level (Tabs::Rtab), built on the device
// when they have at most `cap` entries; otherwise the kernel divides.
void build_star_rtab(semmg_ctx* c, const Geo& G, const HostLevel& H, Tabs<double>& t, size_t cap, bool* ok);

int g_limits_done = 0;

template <typename T> const Tabs<T>& tabs(const semmg_ctx* c, int l);
template <> const Tabs<double>& tabs<double>(const semmg_ctx* c, int l) { return c->dl[l].td; }
template <> const Tabs<float>& tabs<float>(const semmg_ctx* c, int l) { return c->dl[l].tf; }
template <typename T> const LaunchCfg& schur_cfg(const semmg_ctx* c, int l);
template <> const LaunchCfg& schur_cfg<double>(const semmg_ctx* c, int l) { return c->dl[l].schur64; }
template <> const LaunchCfg& schur_cfg<float>(const semmg_ctx* c, int l) { return c->dl[l].schur32; }
template <typename T> const LaunchCfg& star_cfg(const semmg_ctx* c, int l);
template <> const LaunchCfg& star_cfg<double>(const semmg_ctx* c, int l) { return c->dl[l].star64; }
template <> const LaunchCfg& star_cfg<float>(const semmg_ctx* c, int l) { return c->dl[l].star32; }

struct Tic;
int ev_get(semmg_ctx* c);

// Algorithmic work per launch (see semmg.h, timing).
double star_flops(const Geo& G) { return 37.0 * G.nS * (double)G.nS * G.nS * (double)G.nstar; }
// 73 n_E^3 per element-centred block (Sec. 3.4), n_E = 3p - 1
double eblock_flops(const Geo& G) {
  const double nE = 3.0 * G.p - 1.0;
  return 73.0 * nE * nE * nE * (double)G.nelem;
}
double schur_flops(const Geo& G) { return 73.0 * G.m * (double)G.m * G.m * (double)G.nelem; }
double fdm_flops(const Geo& G) {
  const double p = G.p;
  return (12.0 * p * p * p * p + 25.0 * p * p * p) * (double)G.nelem;
}

}  // namespace
namespace {

bool valid_level(const semmg_ctx* c, int level) { return c && level >= 0 && level <= c->L(); }

// ---- timing: an event pair around each launch group of one kernel class
// Next timing event: from the context's pool, or, while the outer iteration is
// being captured, from the pool of its graph.
int ev_get(semmg_ctx* c) {
  std::vector<cudaEvent_t>& pool = c->capturing ? c->step_events : c->events;
  int& used = c->capturing ? c->step_ev_used : c->ev_used;
  if (used == (int)pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    pool.push_back(e);
  }
  return used++;
}

void ev_record(semmg_ctx* c, int ev, cudaStream_t st) {
  if (c->capturing)
    cudaEventRecordWithFlags(c->step_events[ev], st, cudaEventRecordExternal);  // an event node of the graph
  else
    cudaEventRecord(c->events[ev], st);
}

struct Tic {
  semmg_ctx* c;
  int kind;
  int ev = -1;
  cudaStream_t st;
  Tic(semmg_ctx* c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) {
    if (c->timing) {
      ev = ev_get(c);
      if (ev >= 0) ev_record(c, ev, st);
    }
  }
  void toc(double flops, double bytes, int64_t launches = 1, double xflops = 0.0) {
    if (!c->timing || ev < 0) return;
    const int e1 = ev_get(c);
    if (e1 < 0) return;
    ev_record(c, e1, st);
    (c->capturing ? c->step_pending : c->pending).push_back({kind, ev, flops, bytes, launches, xflops});
  }
};

// the launch groups of the last replay of the captured outer iteration
void collect_step_timing(semmg_ctx* c) {
  if (!c->step_replayed) return;
  c->step_replayed = false;
  if (c->step_pending.empty()) return;
  cudaEventSynchronize(c->step_events[c->step_ev_used - 1]);
  for (const auto& p : c->step_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->step_events[p.ev], c->step_events[p.ev + 1]);
    semmg_kstat& k = c->ks[p.kind];
    k.ms += ms;
    k.launches += p.launches;
    k.flops += p.flops;
    k.bytes += p.bytes;
    k.xflops += p.xflops;
  }
}

void collect_timing(semmg_ctx* c) {
  collect_step_timing(c);
  if (c->pending.empty()) return;
  cudaEventSynchronize(c->events[c->ev_used - 1]);
  for (const auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->events[p.ev], c->events[p.ev + 1]);
    semmg_kstat& k = c->ks[p.kind];
    k.ms += ms;
    k.launches += p.launches;
    k.flops += p.flops;
    k.bytes += p.bytes;
    k.xflops += p.xflops;
  }
  c->pending.clear();
  c->ev_used = 0;
}

// Operations one launch of the CUDA-core star kernel (star_kernel.cuh) executes
// on level l, from its loop trip counts: adds, multiplies and divisions count 1,
// fused multiply-adds 2, as ncu counts FP64 thread instructions (a division counts
// 1 here although the hardware runs it as several instructions).  Per star, from
// the folding flag and active range of its three vertex lines: the gather, the
// folds and unfolds, the grouped transforms (the backward ones run every lane of
// a group), the eigenspace segments of every k3-slab (1/D from the table or by
// division) with the contractions along the normals (in FP64 four lanes per
// output and two combining adds per thread and round), and the weighted output.
double star_exec_ops(const semmg_ctx* c, int l, bool fp64, int block, std::vector<double>* each = nullptr) {
  const Geo& G = c->geo[l];
  const HostLevel& H = c->hl[l];
  const int nS = G.nS, m = G.m, ts = star_slab_thickness(nS), kG = kStarGroup;
  const bool rtab = fp64 && c->dl[l].td.Rtab != nullptr;
  struct Line { int sym, lo, hi, pa; };
  std::vector<Line> ln[3];
  const int nv[3] = {G.nv1, G.nv2, G.nv3};
  for (int d = 0; d < 3; ++d) {
    ln[d].resize(nv[d]);
    for (int cc = 0; cc < nv[d]; ++cc) {
      const unsigned char* a = &H.act[d][(size_t)cc * nS];
      int lo = 0, hi = nS;
      while (lo < nS && !a[lo]) ++lo;
      while (hi > lo && !a[hi - 1]) --hi;
      ln[d][cc] = Line{H.sym[d][cc] ? 1 : 0, lo, hi, a[m] ? 1 : 0};
    }
  }
  auto fwd = [&](int sy, int w) { return sy ? (double)(m + 1) * (m + 1) + (double)m * m : (double)w * w; };
  auto bwd = [&](int sy, int w) {
    if (sy) return (double)((m + kG) / kG) * kG * (m + 1) + (double)((m + kG - 1) / kG) * kG * m;
    return (double)((w + kG - 1) / kG) * kG * w;
  };
  const double n2 = (double)nS * nS;
  double total = 0.0;
  if (each) each->assign((size_t)G.nstar, 0.0);
  for (int c3 = 0; c3 < G.nv3; ++c3)
    for (int c2 = 0; c2 < G.nv2; ++c2)
      for (int c1 = 0; c1 < G.nv1; ++c1) {
        if ((G.per[0] && c1 == G.n1) || (G.per[1] && c2 == G.n2) || (G.per[2] && c3 == G.n3)) continue;
        const Line L[3] = {ln[0][c1], ln[1][c2], ln[2][c3]};
        int w[3];
        for (int d = 0; d < 3; ++d) w[d] = L[d].hi - L[d].lo;
        double ops = 0.0;
        for (int dd = 0; dd < 3; ++dd) {
          const int a = dd == 0 ? 1 : 0, b = dd == 2 ? 1 : 2;  // fast and slow in-plane axes
          ops += 2.0 * (L[a].sym + L[b].sym) * nS * (nS - 1.0);  // folds and unfolds of all n_S^2 points
          ops += 3.0 * n2;                                        // weights and weighted output
          if (!L[dd].pa) continue;
          ops += (double)w[a] * w[b];                             // gather: residual / multiplicity
          ops += 2.0 * (w[b] * (fwd(L[a].sym, w[a]) + bwd(L[a].sym, w[a])) +
                        w[a] * (fwd(L[b].sym, w[b]) + bwd(L[b].sym, w[b])));
        }
        int nz[3];
        for (int d = 0; d < 3; ++d) nz[d] = L[d].pa ? (L[d].sym ? m + 1 : w[d]) : 0;
        const double both = (double)nz[1] * nz[0], one = (double)nz[1] * (w[0] - nz[0]) + (double)(w[1] - nz[1]) * nz[0];
        const double dead = L[2].pa ? (double)(w[1] - nz[1]) * (w[0] - nz[0]) : 0.0;
        const double vop = rtab ? 1.0 : 4.0;  // E / D: the table's product, or the sum of D and a division
        for (int k3s = L[2].lo; k3s < L[2].hi; k3s += ts) {
          const int tn = std::min(ts, L[2].hi - k3s);
          const int kl = std::min(std::max(L[2].lo + nz[2] - k3s, 0), tn);  // k3 with s3[k3] live
          const double tail = nz[2] ? 1.0 : 0.0;
          ops += both * (tn * (3.0 + vop) + kl * 4.0 + tail);
          ops += one * (tn * (1.0 + vop) + kl * 4.0 + tail);
          ops += dead * (kl * (rtab ? 2.0 : 5.0) + 2.0);
          const double nb1 = L[0].pa ? (double)tn * w[1] : 0.0, nb2 = L[1].pa ? (double)tn * w[0] : 0.0;
          ops += 2.0 * (nb1 * nz[0] + nb2 * nz[1]);
          if (fp64) {
            const double rounds = std::ceil(4.0 * (nb1 + nb2) / block);
            ops += 2.0 * block * rounds;
          } else {
            ops += 3.0 * (nb1 + nb2);
          }
        }
        total += ops;
        if (each) (*each)[((size_t)c3 * G.nv2 + c2) * G.nv1 + c1] = ops;
      }
  return total;
}

// Star order of level l for the star kernels: most operations first (per-star counts of
// star_exec_ops), so the long stars start first and the short ones fill the tail.
bool upload_star_order(semmg_ctx* c, int l) {
  std::vector<double> cost;
  star_exec_ops(c, l, true, 512, &cost);
  std::vector<int> order(cost.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  int* d = (int*)dalloc(c, order.size() * sizeof(int));
  if (!d || cudaMemcpy(d, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return false;
  c->dl[l].td.order = d;
  c->dl[l].tf.order = d;
  return true;
}

// V-cycle in FP32 (the mixed forms)
bool cycle32(const semmg_ctx* c) { return c->opts.precision != SEMMG_FP64; }
// FP32 V-cycle whose level residuals are formed in float-float on the face-parallel
// levels (FP64 on the others)
bool residff(const semmg_ctx* c) {
  return c->opts.precision == SEMMG_MIXED_FF || c->opts.precision == SEMMG_MIXED_FF_TC;
}
// FP32 V-cycle whose level residuals are formed in FP64 (all levels, or the levels
// without the float-float form)
bool resid64(const semmg_ctx* c) {
  return c->opts.precision == SEMMG_MIXED || c->opts.precision == SEMMG_MIXED_TC ||
         c->opts.precision == SEMMG_MIXED_BF16 || residff(c);
}
// The star smoother on the tensor cores where a level allows it
bool tc_form(int precision) {
  return precision == SEMMG_MIXED_TC || precision == SEMMG_MIXED_FP32_TC || precision == SEMMG_MIXED_BF16 ||
         precision == SEMMG_MIXED_FF_TC;
}

// out = F - Hhat u (mode 0) or Hhat u (mode 1) on level l with arithmetic in T
// (u, Schur terms) and F, out of type TF; cfg: the Schur kernel's launch shape.
template <typename T, typename TF>
void apply_op(semmg_ctx* c, int l, const Tabs<T>& tb, const LaunchCfg& cfg, const TF* F, const T* u, TF* out,
              int mode, cudaStream_t st) {
  const Geo& G = c->geo[l];
  const double vec = (double)G.size * sizeof(TF), uvec = (double)G.size * sizeof(T);
  const double zb = (double)G.nelem * 6 * G.m * G.m * sizeof(T);
  const double fb = (double)G.oE1 * sizeof(T);
  if (face_form(G) || std::is_same<T, ff>::value) {
    {
      Tic t(c, SEMMG_K_ELEM_SCHUR, st);
      launch_face_fwd<T>(G, tb, u, (T*)c->Uts, st);
      // the element terms in the face eigenbasis: float-float streams the eigenspace through
      // registers (its arithmetic is issue-bound, the stored form memory-bound); FP64 and FP32
      // keep the stored form, whose FP64 work fits the narrow FP64 pipe as well
      if constexpr (std::is_same<T, ff>::value)
        launch_schur_eb<T>(G, tb, (const T*)c->Uts, (T*)c->Zs, (T*)c->wss, plan_schur_eb<T>(G, c->nsm), st);
      else
        launch_elem_schur<T>(G, tb, (const T*)c->Uts, (T*)c->Zs, (T*)c->wss, cfg, st, 1);
      t.toc(schur_flops(G), 3 * fb + zb, 2);
    }
    Tic t(c, SEMMG_K_ASSEMBLE, st);
    launch_face_bwd_assemble<T, TF>(G, tb, F, u, (const T*)c->Uts, (const T*)c->Zs, out, mode, st);
    t.toc(0.0, vec * (mode == 0 ? 2 : 1) + uvec + zb, 2);  // face back transforms, edge and vertex slots
    return;
  }
  if constexpr (!std::is_same<T, ff>::value) {
    {
      Tic t(c, SEMMG_K_ELEM_SCHUR, st);
      launch_elem_schur<T>(G, tb, u, (T*)c->Zs, (T*)c->wss, cfg, st);
      t.toc(schur_flops(G), zb * 2, G.m > 0 ? 1 : 0);
    }
    Tic t(c, SEMMG_K_ASSEMBLE, st);
    if constexpr (std::is_same<T, TF>::value)
      launch_assemble<T>(G, tb, F, u, (T*)c->Zs, out, mode, st);
    else
      launch_assemble_mixed(G, tb, F, u, (const double*)c->Zs, out, mode, st);
    t.toc(0.0, vec * (mode == 0 ? 2 : 1) + uvec + zb);
  }
}

// out = F - Hhat u (mode 0) or Hhat u (mode 1) on level l.  FP32 vectors of
// the SEMMG_MIXED form get FP64 arithmetic (FP64 face terms Z, FP64 sums).
template <typename T>
void op_residual(semmg_ctx* c, int l, const T* F, const T* u, T* out, int mode, cudaStream_t st) {
  const Geo& G = c->geo[l];
  if constexpr (std::is_same<T, float>::value) {
    if (residff(c) && face_form(G)) {
      // u widened to float-float (exactly), then the float-float kernels
      {
        Tic t(c, SEMMG_K_VECTOR, st);
        launch_copy<ff, float>((ff*)c->U64s, u, G.size, st);
        t.toc(0.0, (double)G.size * 12);
      }
      apply_op<ff, float>(c, l, c->dl[l].tff, c->dl[l].schur64, F, (const ff*)c->U64s, out, mode, st);
      return;
    }
    if (resid64(c)) {
      // u widened to FP64 once, then the FP64 kernels; F and the result stay FP32
      {
        Tic t(c, SEMMG_K_VECTOR, st);
        launch_copy<double, float>(c->U64s, u, G.size, st);
        t.toc(0.0, (double)G.size * 12);
      }
      apply_op<double, float>(c, l, c->dl[l].td, c->dl[l].schur64, F, c->U64s, out, mode, st);
      return;
    }
  }
  apply_op<T, T>(c, l, tabs<T>(c, l), schur_cfg<T>(c, l), F, u, out, mode, st);
}

// du = Smoother(r) (accumulate: du += Smoother(r)) on level l >= 1
template <typename T>
void op_smooth(semmg_ctx* c, int l, const T* r, T* du, int accumulate, cudaStream_t st) {
  const Geo& G = c->geo[l];
  const double vec = (double)G.size * sizeof(T);
  if (c->opts.smoother != SEMMG_SMOOTHER_STAR) {
    const double nE = 3.0 * G.p - 1.0;
    const double obe = (double)G.nelem * 6 * nE * nE * sizeof(T);
    {
      Tic t(c, SEMMG_K_STAR, st);
      const LaunchCfg& cfg = std::is_same<T, double>::value ? c->dl[l].eb64 : c->dl[l].eb32;
      launch_eblock<T>(G, tabs<T>(c, l), r, (T*)c->Obs, (T*)c->wss, cfg, st);
      t.toc(eblock_flops(G), vec + obe);
    }
    Tic t(c, SEMMG_K_STAR_GATHER, st);
    launch_eblock_gather<T>(G, (const T*)c->Obs, du, accumulate, st);
    t.toc(0.0, obe + vec * (accumulate ? 2 : 1));
    return;
  }
  const double ob = (double)G.nstar * 3 * G.nS * G.nS * sizeof(T);
  {
    Tic t(c, SEMMG_K_STAR, st);
    bool done = false;
    double xf = 0.0;
    if constexpr (std::is_same<T, float>::value) {
      if (c->dl[l].startc.ok) {
        launch_star_tc(G, c->dl[l].tf, r, (float*)c->Obs, c->dl[l].startc, c->star_counter, c->dev_err,
                       c->tc_wait, st);
        done = true;
      }
    }
    if (!done) {
      launch_star<T>(G, tabs<T>(c, l), r, (T*)c->Obs, (T*)c->wss, star_cfg<T>(c, l), c->star_counter, st);
      if (c->timing) xf = star_exec_ops(c, l, std::is_same<T, double>::value, star_cfg<T>(c, l).block);
    }
    t.toc(star_flops(G), vec + ob, 1, xf);
  }
  Tic t(c, SEMMG_K_STAR_GATHER, st);
  launch_star_gather<T>(G, (const T*)c->Obs, du, accumulate, st);
  t.toc(0.0, ob + vec * (accumulate ? 2 : 1));
}

template <typename T>
void op_restrict(semmg_ctx* c, int l, const T* fine, T* coarse, cudaStream_t st) {
  Tic t(c, SEMMG_K_TRANSFER, st);
  launch_restrict<T>(c->geo[l], c->geo[l - 1], tabs<T>(c, l), fine, coarse, (T*)c->FBs, (T*)c->EBs, st);
  t.toc(0.0, (double)(c->geo[l].size + c->geo[l - 1].size) * sizeof(T), 3);
}

template <typename T>
void op_prolong_add(semmg_ctx* c, int l, const T* coarse, T* fine, cudaStream_t st) {
  Tic t(c, SEMMG_K_TRANSFER, st);
  launch_prolong_add<T>(c->geo[l - 1], c->geo[l], tabs<T>(c, l), coarse, fine, st);
  t.toc(0.0, (double)(2 * c->geo[l].size + c->geo[l - 1].size) * sizeof(T), 3);
}

template <typename T> void op_coarse(semmg_ctx* c, const T* F0, T* U0, cudaStream_t st);
template <>
void op_coarse<double>(semmg_ctx* c, const double* F0, double* U0, cudaStream_t st) {
  Tic t(c, SEMMG_K_COARSE, st);
  launch_coarse_solve(c->geo[0], c->ct, F0, U0, c->cX, c->cY, st);
  t.toc(0.0, 2.0 * c->geo[0].size * sizeof(double), 8);
}
template <>
void op_coarse<float>(semmg_ctx* c, const float* F0, float* U0, cudaStream_t st) {
  const int64_t n = c->geo[0].size;
  Tic t(c, SEMMG_K_COARSE, st);
  launch_copy<double, float>(c->F0d, F0, n, st);
  launch_coarse_solve(c->geo[0], c->ct, c->F0d, c->U0d, c->cX, c->cY, st);
  launch_copy<float, double>(U0, c->U0d, n, st);
  t.toc(0.0, 2.0 * n * sizeof(float), 10);
}

// Smoothing steps on level l: the base count, or base 2^(L-l) when varied (Sec. 4.1).
int nu_at(const semmg_ctx* c, int l, int base) { return c->opts.nu_vary ? base << (c->L() - l) : base; }

// Algorithm 3 with u_L = 0 on the residual held in Fw[L]: Uw[L] <- MultigridCycle(0, Fw[L]).
template <typename T>
void vcycle0(semmg_ctx* c, cudaStream_t st) {
  const int L = c->L();
  for (int l = L; l >= 1; --l) {
    T* F = (T*)c->dl[l].Fw;
    T* U = (T*)c->dl[l].Uw;
    T* R = (T*)c->dl[l].Rw;
    const int64_t n = c->geo[l].size;
    const int nu_pre = nu_at(c, l, c->opts.nu_pre);
    if (nu_pre >= 1) {
      op_smooth<T>(c, l, F, U, 0, st);  // u_l = 0 + Smoother(F_l - H_l 0)
      for (int i = 1; i < nu_pre; ++i) {
        op_residual<T>(c, l, F, U, R, 0, st);
        op_smooth<T>(c, l, R, U, 1, st);
      }
    } else {
      cudaMemsetAsync(U, 0, n * sizeof(T), st);
    }
    op_residual<T>(c, l, F, U, R, 0, st);
    op_restrict<T>(c, l, R, (T*)c->dl[l - 1].Fw, st);
  }
  op_coarse<T>(c, (const T*)c->dl[0].Fw, (T*)c->dl[0].Uw, st);
  for (int l = 1; l <= L; ++l) {
    T* F = (T*)c->dl[l].Fw;
    T* U = (T*)c->dl[l].Uw;
    T* R = (T*)c->dl[l].Rw;
    op_prolong_add<T>(c, l, (const T*)c->dl[l - 1].Uw, U, st);
    const int nu_post = nu_at(c, l, c->opts.nu_post);
    for (int i = 0; i < nu_post; ++i) {
      op_residual<T>(c, l, F, U, R, 0, st);
      op_smooth<T>(c, l, R, U, 1, st);
    }
  }
}

// z = MultigridCycle(0, r) into Uw[L] for r in FP64; the cycle runs in the context precision.
void precondition(semmg_ctx* c, const double* r, cudaStream_t st) {
  const int L = c->L();
  const int64_t n = c->geo[L].size;
  const size_t es = cycle32(c) ? sizeof(float) : sizeof(double);
  {
    Tic t(c, SEMMG_K_VECTOR, st);
    if (cycle32(c))
      launch_copy<float, double>((float*)c->dl[L].Fw, r, n, st);
    else
      launch_copy<double, double>((double*)c->dl[L].Fw, r, n, st);
    t.toc(0.0, (double)n * (8 + es));
  }
  if (cycle32(c))
    vcycle0<float>(c, st);
  else
    vcycle0<double>(c, st);
}

// u += MultigridCycle(0, r) with r in FP64.
void correction(semmg_ctx* c, double* u, const double* r, cudaStream_t st) {
  const int L = c->L();
  const int64_t n = c->geo[L].size;
  const size_t es = cycle32(c) ? sizeof(float) : sizeof(double);
  precondition(c, r, st);
  Tic t(c, SEMMG_K_VECTOR, st);
  if (cycle32(c))
    launch_axpy<double, float>(u, (const float*)c->dl[L].Uw, 1.0, n, st);
  else
    launch_axpy<double, double>(u, (const double*)c->dl[L].Uw, 1.0, n, st);
  t.toc(0.0, (double)n * (16 + es));
}

// F_hat = F_B - H_BI H_II^{-1} F_I; with `save`, the scaled interior
// eigen-coefficients of F_I are kept in Gs for recover_impl(..., use_saved).
// The solve of a float-float form condenses and recovers in float-float where the finest
// level has its tables (the face-parallel levels); the public entry points stay FP64.
bool ff_fdm(const semmg_ctx* c) { return residff(c) && c->dl[c->L()].tff.Sh != nullptr; }
// the shared-memory-staged form pays where the stored form's m^3 work arrays live in global memory
bool ff_staged(const semmg_ctx* c) { return c->fsff.ok && !c->fdm.ws.in_smem[3]; }

void condense_impl(semmg_ctx* c, const double* f, double* fh, bool save, cudaStream_t st, bool ffok = false) {
  const int L = c->L();
  const Geo& G = c->geo[L];
  const double nn = (double)(G.n1 * G.p + 1) * (G.n2 * G.p + 1) * (G.n3 * G.p + 1);
  Tic t(c, SEMMG_K_CONDENSE, st);
  if (ffok && ff_fdm(c) && ff_staged(c))
    launch_fs_condense<ff>(G, c->dl[L].tff, f, (double*)c->Zs, save ? (ff*)c->Gs : nullptr, (ff*)c->wss, c->fsff, st);
  else if (ffok && ff_fdm(c))
    launch_elem_condense<ff>(G, c->dl[L].tff, f, (double*)c->Zs, save ? (ff*)c->Gs : nullptr, (ff*)c->wss, c->fdm,
                             st);
  else
    launch_elem_condense<double>(G, c->dl[L].td, f, (double*)c->Zs, save ? c->Gs : nullptr, (double*)c->wss,
                                 c->fdm, st);
  launch_assemble_rhs(G, c->dl[L].td, f, (const double*)c->Zs, fh, st);
  t.toc(G.m > 0 ? fdm_flops(G) : 0.0, 8.0 * (nn + G.size), 2);
}

// u = (u_hat, H_II^{-1}(F_I - H_IB u_hat)); use_saved: F_I's coefficients from
// the preceding condense_impl(..., save = true) on the same f.
void recover_impl(semmg_ctx* c, const double* f, const double* uh, double* u, bool use_saved, cudaStream_t st,
                  bool ffok = false) {
  const int L = c->L();
  const Geo& G = c->geo[L];
  const double nn = (double)(G.n1 * G.p + 1) * (G.n2 * G.p + 1) * (G.n3 * G.p + 1);
  Tic t(c, SEMMG_K_RECOVER, st);
  launch_unpack(G, uh, u, st);
  if (ffok && use_saved && ff_fdm(c) && ff_staged(c))
    launch_fs_recover<ff>(G, c->dl[L].tff, (const ff*)c->Gs, uh, u, (ff*)c->wss, c->fsff, st);
  else if (ffok && use_saved && ff_fdm(c))
    launch_elem_recover<ff>(G, c->dl[L].tff, f, (const ff*)c->Gs, uh, u, (ff*)c->wss, c->fdm, st);
  else
    launch_elem_recover<double>(G, c->dl[L].td, f, use_saved ? c->Gs : nullptr, uh, u, (double*)c->wss, c->fdm, st);
  t.toc(G.m > 0 ? fdm_flops(G) : 0.0, 8.0 * (2 * nn + G.size), 2);
}

// Start of the outer iteration from u_hat = 0 (g = NULL): r = F_hat; or, with
// Dirichlet data g, from u_hat = E g: r = F_hat - Hhat E g (lifting).  ||r||^2
// into dnorm, and for Algorithm 5 s = r, p = 0, delta = 1.
void iter_start(semmg_ctx* c, cudaStream_t st, const double* g = nullptr) {
  const int L = c->L();
  const int64_t n = c->geo[L].size;
  if (g) {
    {
      Tic t(c, SEMMG_K_VECTOR, st);
      launch_pack_dirichlet(c->geo[L], g, c->Uh, st);
      t.toc(0.0, 16.0 * n);
    }
    op_residual<double>(c, L, c->Fh, c->Uh, c->Rh, 0, st);
  }
  Tic t(c, SEMMG_K_VECTOR, st);
  if (!g) {
    cudaMemsetAsync(c->Uh, 0, n * sizeof(double), st);
    launch_copy<double, double>(c->Rh, c->Fh, n, st);
  }
  launch_norm2<double>(c->Rh, n, c->part, c->npart, c->dnorm, st);
  if (c->opts.solver == SEMMG_SOLVER_KMG) {
    launch_copy<double, double>(c->kS, c->Rh, n, st);
    cudaMemsetAsync(c->kP, 0, n * sizeof(double), st);
    launch_krylov_init(c->kscal, st);
  }
  t.toc(2.0 * n, 8.0 * n * (c->opts.solver == SEMMG_SOLVER_KMG ? 6 : 3), 3);
}

// One outer iteration, ||r||^2 into dnorm.  Algorithm 4: u += MultigridCycle(0, r),
// r = F - Hhat u.  Algorithm 5: z = MultigridCycle(0, r), beta, p = beta p + z,
// q = Hhat p, alpha, s = r, u += alpha p, r -= alpha q.
void iter_step(semmg_ctx* c, cudaStream_t st) {
  const int L = c->L();
  const int64_t n = c->geo[L].size;
  if (c->opts.solver == SEMMG_SOLVER_MG) {
    correction(c, c->Uh, c->Rh, st);
    op_residual<double>(c, L, c->Fh, c->Uh, c->Rh, 0, st);
    Tic t(c, SEMMG_K_VECTOR, st);
    launch_norm2<double>(c->Rh, n, c->part, c->npart, c->dnorm, st);
    t.toc(2.0 * n, 8.0 * n, 2);
    return;
  }
  precondition(c, c->Rh, st);
  const bool mixed = cycle32(c);
  {
    Tic t(c, SEMMG_K_VECTOR, st);
    if (mixed)
      launch_krylov_beta_dir<float>((const float*)c->dl[L].Uw, c->Rh, c->kS, c->kP, n, c->part, c->npart, c->kscal,
                                    st);
    else
      launch_krylov_beta_dir<double>((const double*)c->dl[L].Uw, c->Rh, c->kS, c->kP, n, c->part, c->npart,
                                     c->kscal, st);
    t.toc(6.0 * n, n * (mixed ? 4.0 + 8 + 8 + 4 + 16 : 8.0 * 6), 3);
  }
  op_residual<double>(c, L, c->Fh, c->kP, c->kQ, 1, st);  // q = Hhat p
  Tic t(c, SEMMG_K_VECTOR, st);
  launch_krylov_alpha(c->kQ, c->kP, n, c->part, c->npart, c->kscal, st);
  launch_krylov_update(c->Uh, c->Rh, c->kS, c->kP, c->kQ, n, c->part, c->npart, c->kscal, c->dnorm, st);
  t.toc(8.0 * n, 8.0 * n * 9, 4);
}

// One outer iteration on stream st: replayed from a CUDA graph captured on the
// context's own stream at the first call (one launch instead of one per kernel,
// which is what the low-degree levels are bound by); launched kernel by kernel
// while timing is on or if the capture failed.
void run_step(semmg_ctx* c, cudaStream_t st) {
  collect_step_timing(c);  // the previous replay's events are reused
  if (!c->step_exec && !c->step_capture_failed) {
    bool ok = c->cap_stream || cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    cudaGraph_t g = nullptr;
    c->step_pending.clear();
    c->step_ev_used = 0;
    if (ok && cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      c->capturing = true;
      iter_step(c, c->cap_stream);
      c->capturing = false;
      ok = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && g;
      if (ok && cudaGraphInstantiate(&c->step_exec, g, 0) != cudaSuccess) c->step_exec = nullptr;
      if (g) cudaGraphDestroy(g);
    }
    if (!c->step_exec) {
      cudaGetLastError();
      c->step_capture_failed = 1;
      c->step_pending.clear();
    }
  }
  if (c->step_exec) {
    cudaGraphLaunch(c->step_exec, st);
    c->step_replayed = true;
  } else {
    iter_step(c, st);
  }
}

// sqrt of the squared norm left in dnorm by the last iteration (one 8-byte copy + sync)
int dnorm_sync(semmg_ctx* c, cudaStream_t st, double* out) {
  cudaMemcpyAsync(c->hnorm, c->dnorm, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(c->hdev_err, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(c, "norm");
  *out = std::sqrt(*c->hnorm);
  if (*c->hdev_err) return fail(c, SEMMG_ERR_TIMEOUT, "a tensor-core completion wait ran out");
  return check_cuda(c, "norm");
}

void build_star_rtab(semmg_ctx* c, const Geo& G, const HostLevel& H, Tabs<double>& t, size_t cap, bool* ok) {
  t.Rtab = nullptr;
  const size_t nS = (size_t)G.nS, n3 = nS * nS * nS;
  const size_t n2c = H.rep[1].size(), n3c = H.rep[2].size();
  const size_t total = H.rep[0].size() * n2c * n3c * n3;
  if (total == 0 || total > cap) return;
  int* dr[3];
  for (int d = 0; d < 3; ++d) {
    dr[d] = (int*)dalloc(c, H.rep[d].size() * sizeof(int));
    if (!dr[d] || cudaMemcpy(dr[d], H.rep[d].data(), H.rep[d].size() * sizeof(int), cudaMemcpyHostToDevice) !=
                      cudaSuccess) {
      *ok = false;
      return;
    }
  }
  double* R = (double*)dalloc(c, total * sizeof(double));
  if (!R) {
    *ok = false;
    return;
  }
  k_build_rtab<<<4 * c->nsm, 256>>>(G.nS, (int)n2c, (int)n3c, dr[0], dr[1], dr[2], t.starLam[0], t.starLam[1],
                                    t.starLam[2], G.lam, (int64_t)total, R);
  // done before setup returns, whatever stream the caller orders its work on
  if (cudaStreamSynchronize(0) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    *ok = false;
    return;
  }
  t.Rtab = R;
}

int set_limits(semmg_ctx* c) {
  if (g_limits_done) return SEMMG_OK;
  if (set_elem_smem_limits() | set_star_smem_limits() | set_transfer_smem_limits() | set_star_tc_smem_limits() |
      set_eblock_smem_limits() | set_face_smem_limits() | set_ff_smem_limits())
    return fail(c, SEMMG_ERR_CUDA, "cudaFuncSetAttribute failed: %s", cudaGetErrorString(cudaGetLastError()));
  g_limits_done = 1;
  return SEMMG_OK;
}

}  // namespace


namespace semmg {

// Star smoothing of one level (semmg_smooth's work, with the same kernels:
// the tensor-core star kernel where semmg_smooth takes it, else the CUDA-core
// one) with the star output buffer and the per-block work arrays placed in
// caller-provided device memory instead of the context's scratch; the grid of
// the CUDA-core kernel shrinks until its work arrays fit.  Returns
// SEMMG_ERR_UNSUPPORTED when the level does not fit or its star launch plan is
// unusable, SEMMG_ERR_INVALID_ARG for a scratch base that is not 256-byte aligned.
int smooth_with_scratch(semmg_ctx* c, int level, int dtype, const void* r, void* du, void* scratch,
                        size_t scratch_bytes, cudaStream_t st) {
  if (!valid_level(c, level) || level < 1 || !r || !du || r == du || !scratch) return SEMMG_ERR_INVALID_ARG;
  if (dtype != SEMMG_F64 && dtype != SEMMG_F32) return SEMMG_ERR_INVALID_ARG;
  if (((uintptr_t)scratch & 255u) != 0)
    return fail(c, SEMMG_ERR_INVALID_ARG, "smooth_noalloc: scratch base is not 256-byte aligned");
  if (c->opts.smoother != SEMMG_SMOOTHER_STAR)
    return fail(c, SEMMG_ERR_UNSUPPORTED, "smooth_noalloc: vertex-star smoother only");
  const Geo& G = c->geo[level];
  const size_t es = dtype == SEMMG_F64 ? sizeof(double) : sizeof(float);
  const bool tensor = dtype == SEMMG_F32 && c->dl[level].startc.ok;  // as op_smooth<float> decides
  LaunchCfg cfg = dtype == SEMMG_F64 ? c->dl[level].star64 : (tensor ? c->dl[level].startc : c->dl[level].star32);
  if (!cfg.ok)
    return fail(c, SEMMG_ERR_UNSUPPORTED, "smooth_noalloc: no usable star launch plan on level %d", level);
  const size_t ob_bytes = ((size_t)G.nstar * 3 * G.nS * G.nS * es + 255) & ~size_t(255);
  const size_t per_cta = tensor ? 0 : (size_t)cfg.ws.gstride * es;  // the tensor-core kernel has no work arrays
  if (ob_bytes > scratch_bytes)
    return fail(c, SEMMG_ERR_UNSUPPORTED,
                "smooth_noalloc: level %d needs %zu bytes of star output buffer, more than the %zu-byte scratch",
                level, ob_bytes, scratch_bytes);
  if (per_cta > 0) {
    const size_t fit = (scratch_bytes - ob_bytes) / per_cta;
    if (fit < 1)
      return fail(c, SEMMG_ERR_UNSUPPORTED,
                  "smooth_noalloc: level %d needs %zu + %zu bytes of scratch, more than the %zu-byte scratch", level,
                  ob_bytes, per_cta, scratch_bytes);
    if ((size_t)cfg.grid > fit) cfg.grid = (int)fit;
  }
  unsigned char* base = (unsigned char*)scratch;
  if (dtype == SEMMG_F64) {
    launch_star<double>(G, c->dl[level].td, (const double*)r, (double*)base, (double*)(base + ob_bytes), cfg,
                        nullptr, st);
    launch_star_gather<double>(G, (const double*)base, (double*)du, 0, st);
  } else {
    if (tensor)
      launch_star_tc(G, c->dl[level].tf, (const float*)r, (float*)base, cfg, nullptr, c->dev_err, c->tc_wait, st);
    else
      launch_star<float>(G, c->dl[level].tf, (const float*)r, (float*)base, (float*)(base + ob_bytes), cfg, nullptr,
                         st);
    launch_star_gather<float>(G, (const float*)base, (float*)du, 0, st);
  }
  return check_cuda(c, "smooth_noalloc");
}

}  // namespace semmg

extern "C" {

void semmg_default_opts(semmg_opts* o) {
  if (!o) return;
  o->p0 = 2;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->precision = SEMMG_FP64;
  o->max_iter = 50;
  o->solver = SEMMG_SOLVER_MG;
  o->nu_vary = 0;
  o->smoother = SEMMG_SMOOTHER_STAR;
}

int semmg_setup(const semmg_mesh* mesh, int p, double lambda, const semmg_opts* opts, void* stream,
                semmg_ctx** out) {
  if (!out) return SEMMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh) return SEMMG_ERR_INVALID_ARG;
  semmg_opts o;
  semmg_default_opts(&o);
  if (opts) o = *opts;
  if (p < 1 || p > SEMMG_MAX_DEGREE) return SEMMG_ERR_UNSUPPORTED;
  if (o.p0 < 1 || o.p0 > p) return SEMMG_ERR_UNSUPPORTED;
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return SEMMG_ERR_INVALID_ARG;
  if (o.nu_pre < 0 || o.nu_post < 0 || o.max_iter < 0) return SEMMG_ERR_INVALID_ARG;
  if (o.precision < SEMMG_FP64 || o.precision > SEMMG_MIXED_FF_TC)
    return SEMMG_ERR_INVALID_ARG;
  if (o.solver != SEMMG_SOLVER_MG && o.solver != SEMMG_SOLVER_KMG) return SEMMG_ERR_INVALID_ARG;
  if (o.nu_vary != 0 && o.nu_vary != 1) return SEMMG_ERR_INVALID_ARG;
  if (o.smoother != SEMMG_SMOOTHER_STAR && o.smoother != SEMMG_SMOOTHER_ELEMENT &&
      o.smoother != SEMMG_SMOOTHER_ELEMENT_MULT)
    return SEMMG_ERR_INVALID_ARG;
  bool any_dirichlet = false;
  for (int f = 0; f < 6; ++f) {
    if (mesh->bc[f] != SEMMG_BC_DIRICHLET && mesh->bc[f] != SEMMG_BC_NEUMANN && mesh->bc[f] != SEMMG_BC_PERIODIC)
      return SEMMG_ERR_INVALID_ARG;
    any_dirichlet |= mesh->bc[f] == SEMMG_BC_DIRICHLET;
  }
  for (int d = 0; d < 3; ++d) {
    const bool plo = mesh->bc[2 * d] == SEMMG_BC_PERIODIC, phi = mesh->bc[2 * d + 1] == SEMMG_BC_PERIODIC;
    if (plo != phi) return SEMMG_ERR_INVALID_ARG;         // periodic pairs the two faces of an axis
    if (plo && mesh->n[d] < 2) return SEMMG_ERR_UNSUPPORTED;  // a star would meet itself
    // an element-centred block spans three elements along each axis, which must differ
    if (plo && o.smoother != SEMMG_SMOOTHER_STAR && mesh->n[d] < 3) return SEMMG_ERR_UNSUPPORTED;
  }
  if (!any_dirichlet && !(lambda > 0.0)) return SEMMG_ERR_UNSUPPORTED;  // singular (pure Neumann, lambda = 0)
  for (int d = 0; d < 3; ++d) {
    if (mesh->n[d] < 1 || !mesh->h[d]) return SEMMG_ERR_INVALID_ARG;
    if ((int64_t)mesh->n[d] * p + 1 >= (1 << 20)) return SEMMG_ERR_UNSUPPORTED;
    for (int a = 0; a < mesh->n[d]; ++a)
      if (!(mesh->h[d][a] > 0.0) || !std::isfinite(mesh->h[d][a])) return SEMMG_ERR_INVALID_ARG;
  }
  std::unique_ptr<semmg_ctx> c(new (std::nothrow) semmg_ctx());
  if (!c) return SEMMG_ERR_NOMEM;
  c->opts = o;
  c->lam = lambda;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  if (set_limits(c.get()) != SEMMG_OK) return SEMMG_ERR_CUDA;
  for (int d = 0; d < 3; ++d) c->h[d].assign(mesh->h[d], mesh->h[d] + mesh->n[d]);
  // level degrees (Sec. 4.1): p0 2^l while below p, then p
  std::vector<int> degs{o.p0};
  while (degs.back() * 2 < p) degs.push_back(degs.back() * 2);
  if (degs.back() != p) degs.push_back(p);
  const int nl = (int)degs.size();
  c->geo.resize(nl);
  c->hl.resize(nl);
  c->dl.resize(nl);
  for (int l = 0; l < nl; ++l) {
    c->geo[l] = make_geo(mesh->n, degs[l], lambda, mesh->bc);
    c->hl[l].p = degs[l];
    c->hl[l].lam = lambda;
    build_level_tables(c->hl[l], c->h, mesh->bc);
    if (l > 0 && o.smoother != SEMMG_SMOOTHER_STAR) build_eblock_tables(c->hl[l], c->h, mesh->bc, o.smoother);
    if (l > 0) {
      lagrange_interp(c->hl[l - 1].x, c->hl[l].x, c->hl[l].J);
      c->hl[l].pc = degs[l - 1];
    }
  }
  build_coarse_tables(degs[0], c->h, mesh->bc, c->hc);
  bool ok = true;
  for (int l = 0; l < nl; ++l) {
    c->dl[l].td = upload_tabs<double>(c.get(), c->geo[l], c->hl[l], c->h, &ok);
    c->dl[l].tf = upload_tabs<float>(c.get(), c->geo[l], c->hl[l], c->h, &ok);
    if (residff(c.get()) && face_form(c->geo[l]))
      c->dl[l].tff = upload_tabs<ff>(c.get(), c->geo[l], c->hl[l], c->h, &ok);
    // 1/D tables of the FP64 star kernel: always when small; up to kMaxStarRtabFp64 entries (GB on
    // stretched meshes, where every vertex line is its own class) for the FP64 V-cycle
    if (l >= 1 && ok && o.smoother == SEMMG_SMOOTHER_STAR)
      build_star_rtab(c.get(), c->geo[l], c->hl[l], c->dl[l].td,
                      o.precision == SEMMG_FP64 ? kMaxStarRtabFp64 : kMaxRtabEntries, &ok);
  }
  // longest-first star order per smoothing level (scheduling only: results are unchanged)
  for (int l = 1; ok && l < nl; ++l)
    if (o.smoother == SEMMG_SMOOTHER_STAR && !upload_star_order(c.get(), l)) ok = false;
  for (int d = 0; d < 3; ++d) {
    c->ct.K[d] = c->hc.K[d];
    c->ct.g0[d] = c->hc.g0[d];
    c->ct.S[d] = upload<double>(c.get(), c->hc.S[d], &ok);
    c->ct.lam[d] = upload<double>(c.get(), c->hc.lam[d], &ok);
  }
  if (!ok) return SEMMG_ERR_NOMEM;
  // launch plans and scratch sizes
  size_t zs = 0, obs = 0, fbs = 0, ebs = 0, wsb = 0;
  for (int l = 0; l < nl; ++l) {
    const Geo& G = c->geo[l];
    DevLevel& D = c->dl[l];
    D.schur64 = plan_elem_schur<double>(G, c->nsm);
    D.schur32 = plan_elem_schur<float>(G, c->nsm);
    if (residff(c.get()) && face_form(G)) {
      const LaunchCfg eb = plan_schur_eb<ff>(G, c->nsm);
      if (!eb.ok) return SEMMG_ERR_UNSUPPORTED;
      wsb = std::max(wsb, eb.ws_elems() * sizeof(ff));
    }
    wsb = std::max(wsb, D.schur64.ws_elems() * sizeof(double));
    wsb = std::max(wsb, D.schur32.ws_elems() * sizeof(float));
    zs = std::max(zs, (size_t)(G.nelem * 6 * (int64_t)G.m * G.m));
    if (l >= 1) {
      D.star64 = plan_star<double>(G, c->nsm);
      D.star32 = plan_star<float>(G, c->nsm);
      if (o.smoother != SEMMG_SMOOTHER_STAR) {
        D.eb64 = plan_eblock<double>(G, c->nsm);
        D.eb32 = plan_eblock<float>(G, c->nsm);
        if (!D.eb64.ok || !D.eb32.ok) return SEMMG_ERR_UNSUPPORTED;
        wsb = std::max(wsb, D.eb64.ws_elems() * sizeof(double));
        wsb = std::max(wsb, D.eb32.ws_elems() * sizeof(float));
        const int64_t nE = 3 * (int64_t)G.p - 1;
        obs = std::max(obs, (size_t)(G.nelem * 6 * nE * nE));
      }
      if (tc_form(o.precision) && o.smoother == SEMMG_SMOOTHER_STAR) {
        const bool bf16 = o.precision == SEMMG_MIXED_BF16;
        D.startc = plan_star_tc(G, c->nsm, bf16 ? 1 : 0);
        if (D.startc.ok) {
          upload_tc_tables(c.get(), c->hl[l], D.tf, bf16, &ok);
          if (!ok) return SEMMG_ERR_NOMEM;
        }
      }
      wsb = std::max(wsb, D.star64.ws_elems() * sizeof(double));
      wsb = std::max(wsb, D.star32.ws_elems() * sizeof(float));
      obs = std::max(obs, (size_t)(G.nstar * 3 * (int64_t)G.nS * G.nS));
      fbs = std::max(fbs, (size_t)restrict_face_buffer(G, degs[l - 1]));
      ebs = std::max(ebs, (size_t)restrict_edge_buffer(G, degs[l - 1]));
    }
  }
  c->fdm = plan_elem_fdm(c->geo[nl - 1], c->nsm);
  if (residff(c.get()) && face_form(c->geo[nl - 1]) && !c->fdm.ws.in_smem[3]) {
    c->fsff = plan_fs<ff>(c->geo[nl - 1], c->nsm);
    if (c->fsff.ok) wsb = std::max(wsb, c->fsff.ws_elems() * sizeof(ff));
  }
  for (int l = 0; l < nl; ++l) {
    const DevLevel& D = c->dl[l];
    if (!D.schur64.ok || !D.schur32.ok || (l >= 1 && (!D.star64.ok || !D.star32.ok)))
      return SEMMG_ERR_UNSUPPORTED;
  }
  if (!c->fdm.ok) return SEMMG_ERR_UNSUPPORTED;
  wsb = std::max(wsb, c->fdm.ws_elems() * sizeof(double));
  c->Zs = dalloc(c.get(), zs * sizeof(double));
  c->Obs = dalloc(c.get(), obs * sizeof(double));
  c->FBs = dalloc(c.get(), fbs * sizeof(double));
  c->EBs = dalloc(c.get(), ebs * sizeof(double));
  c->wss = dalloc(c.get(), wsb);
  c->ws_bytes = wsb;
  const size_t esz = o.precision != SEMMG_FP64 ? sizeof(float) : sizeof(double);
  for (int l = 0; l < nl; ++l) {
    const size_t n = (size_t)c->geo[l].size;
    c->dl[l].Fw = dalloc(c.get(), n * esz);
    c->dl[l].Uw = dalloc(c.get(), n * esz);
    c->dl[l].Rw = dalloc(c.get(), n * esz);
    if (!c->dl[l].Fw || !c->dl[l].Uw || !c->dl[l].Rw) return SEMMG_ERR_NOMEM;
  }
  const size_t nL = (size_t)c->geo[nl - 1].size;
  c->Fh = (double*)dalloc(c.get(), nL * sizeof(double));
  c->Uh = (double*)dalloc(c.get(), nL * sizeof(double));
  c->Rh = (double*)dalloc(c.get(), nL * sizeof(double));
  {
    const Geo& GL = c->geo[nl - 1];
    const size_t ng = (size_t)GL.nelem * GL.m * GL.m * GL.m;
    if (ng > 0) {
      c->Gs = (double*)dalloc(c.get(), ng * sizeof(double));
      if (!c->Gs) return SEMMG_ERR_NOMEM;
    }
  }
  if (c->geo[nl - 1].oE1 > 0) {
    c->Uts = dalloc(c.get(), (size_t)c->geo[nl - 1].oE1 * sizeof(double));
    if (!c->Uts) return SEMMG_ERR_NOMEM;
  }
  if (resid64(c.get())) {  // the widened copy of u (FP64, or float-float of the same size)
    static_assert(sizeof(ff) == sizeof(double), "float-float and FP64 share the widened copy");
    c->U64s = (double*)dalloc(c.get(), nL * sizeof(double));
    if (!c->U64s) return SEMMG_ERR_NOMEM;
  }
  if (o.solver == SEMMG_SOLVER_KMG) {
    c->kS = (double*)dalloc(c.get(), nL * sizeof(double));
    c->kP = (double*)dalloc(c.get(), nL * sizeof(double));
    c->kQ = (double*)dalloc(c.get(), nL * sizeof(double));
    c->kscal = (KrylovScal*)dalloc(c.get(), sizeof(KrylovScal));
    if (!c->kS || !c->kP || !c->kQ || !c->kscal) return SEMMG_ERR_NOMEM;
  }
  const size_t nK = (size_t)c->ct.K[0] * c->ct.K[1] * c->ct.K[2];
  c->cX = (double*)dalloc(c.get(), nK * sizeof(double));
  c->cY = (double*)dalloc(c.get(), nK * sizeof(double));
  c->F0d = (double*)dalloc(c.get(), (size_t)c->geo[0].size * sizeof(double));
  c->U0d = (double*)dalloc(c.get(), (size_t)c->geo[0].size * sizeof(double));
  c->npart = 512;
  c->part = (double*)dalloc(c.get(), 2 * c->npart * sizeof(double));  // two partial-sum rows (Algorithm 5)
  c->dnorm = (double*)dalloc(c.get(), sizeof(double));
  c->star_counter = (int*)dalloc(c.get(), 4 * sizeof(int));
  if (!c->star_counter || cudaMemset(c->star_counter, 0, 4 * sizeof(int)) != cudaSuccess) return SEMMG_ERR_NOMEM;
  c->dev_err = (int*)dalloc(c.get(), sizeof(int));
  if (!c->dev_err || cudaMemset(c->dev_err, 0, sizeof(int)) != cudaSuccess) return SEMMG_ERR_NOMEM;
  if (!c->Zs || !c->Obs || !c->FBs || !c->EBs || !c->wss || !c->Fh || !c->Uh || !c->Rh || !c->cX || !c->cY ||
      !c->F0d || !c->U0d || !c->part || !c->dnorm)
    return SEMMG_ERR_NOMEM;
  if (cudaMallocHost((void**)&c->hnorm, sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&c->hdev_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_NOMEM;
  }
  *c->hdev_err = 0;
  *c->hnorm = 0.0;
  for (int l = 0; l < nl; ++l) {
    const size_t n = (size_t)c->geo[l].size;
    cudaMemsetAsync(c->dl[l].Fw, 0, n * esz, st);
    cudaMemsetAsync(c->dl[l].Uw, 0, n * esz, st);
    cudaMemsetAsync(c->dl[l].Rw, 0, n * esz, st);
  }
  cudaMemsetAsync(c->Fh, 0, nL * sizeof(double), st);
  cudaMemsetAsync(c->Uh, 0, nL * sizeof(double), st);
  cudaMemsetAsync(c->Rh, 0, nL * sizeof(double), st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  *out = c.release();
  return SEMMG_OK;
}

void semmg_destroy(semmg_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  delete c;
}

int semmg_num_levels(const semmg_ctx* c, int* nl) {
  if (!c || !nl) return SEMMG_ERR_INVALID_ARG;
  *nl = (int)c->geo.size();
  return SEMMG_OK;
}

int semmg_level_degree(const semmg_ctx* c, int level, int* p) {
  if (!valid_level(c, level) || !p) return SEMMG_ERR_INVALID_ARG;
  *p = c->geo[level].p;
  return SEMMG_OK;
}

int semmg_condensed_size(const semmg_ctx* c, int level, int64_t* n) {
  if (!valid_level(c, level) || !n) return SEMMG_ERR_INVALID_ARG;
  *n = c->geo[level].size;
  return SEMMG_OK;
}

int semmg_nodal_size(const semmg_ctx* c, int level, int64_t* n) {
  if (!valid_level(c, level) || !n) return SEMMG_ERR_INVALID_ARG;
  const Geo& G = c->geo[level];
  *n = (int64_t)(G.n1 * G.p + 1) * (G.n2 * G.p + 1) * (G.n3 * G.p + 1);
  return SEMMG_OK;
}

int semmg_pack(semmg_ctx* c, int level, const double* u_nodal, double* u_hat, void* stream) {
  if (!valid_level(c, level) || !u_nodal || !u_hat) return SEMMG_ERR_INVALID_ARG;
  launch_pack(c->geo[level], u_nodal, u_hat, (cudaStream_t)stream);
  return check_cuda(c, "pack");
}

int semmg_pack_dirichlet(semmg_ctx* c, int level, const double* g_nodal, double* u_hat, void* stream) {
  if (!valid_level(c, level) || !g_nodal || !u_hat) return SEMMG_ERR_INVALID_ARG;
  launch_pack_dirichlet(c->geo[level], g_nodal, u_hat, (cudaStream_t)stream);
  return check_cuda(c, "pack_dirichlet");
}

int semmg_unpack(semmg_ctx* c, int level, const double* u_hat, double* u_nodal, void* stream) {
  if (!valid_level(c, level) || !u_nodal || !u_hat) return SEMMG_ERR_INVALID_ARG;
  launch_unpack(c->geo[level], u_hat, u_nodal, (cudaStream_t)stream);
  return check_cuda(c, "unpack");
}

int semmg_apply_condensed(semmg_ctx* c, int level, const double* u, double* y, void* stream) {
  if (!valid_level(c, level) || !u || !y || u == y) return SEMMG_ERR_INVALID_ARG;
  op_residual<double>(c, level, nullptr, u, y, 1, (cudaStream_t)stream);
  return check_cuda(c, "apply_condensed");
}

int semmg_residual(semmg_ctx* c, int level, const double* f, const double* u, double* r, void* stream) {
  if (!valid_level(c, level) || !f || !u || !r || u == r) return SEMMG_ERR_INVALID_ARG;
  op_residual<double>(c, level, f, u, r, 0, (cudaStream_t)stream);
  return check_cuda(c, "residual");
}

int semmg_residual_cycle(semmg_ctx* c, int level, const float* f, const float* u, float* r, void* stream) {
  if (!valid_level(c, level) || !f || !u || !r || u == r) return SEMMG_ERR_INVALID_ARG;
  if (!cycle32(c)) return fail(c, SEMMG_ERR_UNSUPPORTED, "residual_cycle: the context's V-cycle is FP64");
  op_residual<float>(c, level, f, u, r, 0, (cudaStream_t)stream);
  return check_cuda(c, "residual_cycle");
}

int semmg_smooth(semmg_ctx* c, int level, int dtype, const void* r, void* du, void* stream) {
  if (!valid_level(c, level) || level < 1 || !r || !du || r == du) return SEMMG_ERR_INVALID_ARG;
  if (dtype == SEMMG_F64)
    op_smooth<double>(c, level, (const double*)r, (double*)du, 0, (cudaStream_t)stream);
  else if (dtype == SEMMG_F32)
    op_smooth<float>(c, level, (const float*)r, (float*)du, 0, (cudaStream_t)stream);
  else
    return SEMMG_ERR_INVALID_ARG;
  return check_cuda(c, "smooth");
}

int semmg_restrict(semmg_ctx* c, int level, int dtype, const void* fine, void* coarse, void* stream) {
  if (!valid_level(c, level) || level < 1 || !fine || !coarse) return SEMMG_ERR_INVALID_ARG;
  if (dtype == SEMMG_F64)
    op_restrict<double>(c, level, (const double*)fine, (double*)coarse, (cudaStream_t)stream);
  else if (dtype == SEMMG_F32)
    op_restrict<float>(c, level, (const float*)fine, (float*)coarse, (cudaStream_t)stream);
  else
    return SEMMG_ERR_INVALID_ARG;
  return check_cuda(c, "restrict");
}

int semmg_prolong_add(semmg_ctx* c, int level, int dtype, const void* coarse, void* fine, void* stream) {
  if (!valid_level(c, level) || level < 1 || !fine || !coarse) return SEMMG_ERR_INVALID_ARG;
  if (dtype == SEMMG_F64)
    op_prolong_add<double>(c, level, (const double*)coarse, (double*)fine, (cudaStream_t)stream);
  else if (dtype == SEMMG_F32)
    op_prolong_add<float>(c, level, (const float*)coarse, (float*)fine, (cudaStream_t)stream);
  else
    return SEMMG_ERR_INVALID_ARG;
  return check_cuda(c, "prolong_add");
}

int semmg_coarse_solve(semmg_ctx* c, const double* f0, double* u0, void* stream) {
  if (!c || !f0 || !u0 || f0 == u0) return SEMMG_ERR_INVALID_ARG;
  op_coarse<double>(c, f0, u0, (cudaStream_t)stream);
  return check_cuda(c, "coarse_solve");
}

int semmg_vcycle(semmg_ctx* c, double* u, const double* f, void* stream) {
  if (!c || !u || !f) return SEMMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int L = c->L();
  op_residual<double>(c, L, f, u, c->Rh, 0, st);
  correction(c, u, c->Rh, st);
  return check_cuda(c, "vcycle");
}

int semmg_condense_rhs(semmg_ctx* c, const double* f, double* fh, void* stream) {
  if (!c || !f || !fh) return SEMMG_ERR_INVALID_ARG;
  condense_impl(c, f, fh, false, (cudaStream_t)stream);
  return check_cuda(c, "condense_rhs");
}

int semmg_recover(semmg_ctx* c, const double* f, const double* uh, double* u, void* stream) {
  if (!c || !f || !uh || !u) return SEMMG_ERR_INVALID_ARG;
  recover_impl(c, f, uh, u, false, (cudaStream_t)stream);
  return check_cuda(c, "recover");
}

}  // extern "C"

namespace {

// condense, Algorithm 4 or 5 from u_hat = 0 (or E g), recover
int solve_impl(semmg_ctx* c, const double* f, const double* g, double* u, double rtol, semmg_info* info,
               cudaStream_t st) {
  cudaMemsetAsync(c->dev_err, 0, sizeof(int), st);  // a wait that ran out in an earlier call is not this one's
  condense_impl(c, f, c->Fh, true, st, true);
  int rc = check_cuda(c, "condense_rhs");
  if (rc) return rc;
  iter_start(c, st, g);
  double r0 = 0.0, rn = 0.0;
  rc = dnorm_sync(c, st, &r0);  // r_0 = Fhat - Hhat u_hat_0
  if (rc) return rc;
  int it = 0;
  int status = SEMMG_OK;
  if (!std::isfinite(r0)) status = SEMMG_ERR_NONFINITE;
  rn = r0;
  while (status == SEMMG_OK && rn > rtol * r0 && it < c->opts.max_iter) {
    run_step(c, st);
    rc = dnorm_sync(c, st, &rn);
    if (rc) return rc;
    ++it;
    if (!std::isfinite(rn))
      status = SEMMG_ERR_NONFINITE;
    else if (rn > c->divergence * r0)
      status = SEMMG_ERR_DIVERGED;
  }
  if (status == SEMMG_OK && rn > rtol * r0) status = SEMMG_ERR_NOT_CONVERGED;
  recover_impl(c, f, c->Uh, u, true, st, true);
  rc = check_cuda(c, "recover");
  if (rc) return rc;
  if (info) {
    info->iters = it;
    info->res0 = r0;
    info->res_final = rn;
    info->rho = (it > 0 && r0 > 0) ? std::pow(rn / r0, 1.0 / it) : 0.0;
    info->status = status;
  }
  if (status != SEMMG_OK) fail(c, status, "solve: %s after %d cycles", semmg_strerror(status), it);
  return status;
}

}  // namespace

extern "C" {

int semmg_solve(semmg_ctx* c, const double* f, double* u, double rtol, semmg_info* info, void* stream) {
  if (!c || !f || !u || !(rtol > 0.0)) return SEMMG_ERR_INVALID_ARG;
  return solve_impl(c, f, nullptr, u, rtol, info, (cudaStream_t)stream);
}

int semmg_solve_dirichlet(semmg_ctx* c, const double* f, const double* g, double* u, double rtol,
                          semmg_info* info, void* stream) {
  if (!c || !f || !g || !u || !(rtol > 0.0)) return SEMMG_ERR_INVALID_ARG;
  return solve_impl(c, f, g, u, rtol, info, (cudaStream_t)stream);
}

int semmg_solve_host(semmg_ctx* c, const double* f_host, double* u_host, double rtol, semmg_info* info,
                     void* stream) {
  if (!c || !f_host || !u_host) return SEMMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nn = 0;
  semmg_nodal_size(c, c->L(), &nn);
  if (!c->fnod) {
    c->fnod = (double*)dalloc(c, nn * sizeof(double));
    c->unod = (double*)dalloc(c, nn * sizeof(double));
    if (!c->fnod || !c->unod) return fail(c, SEMMG_ERR_NOMEM, "solve_host: device buffers");
  }
  // u: a page-locked (registered) host buffer is written by the unpack and recovery kernels
  // through its device mapping, so the result needs no copy after the solve; any other host
  // memory gets the copy
  double* u_map = nullptr;
  {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, u_host) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
      u_map = (double*)pa.devicePointer;
    cudaGetLastError();  // an unregistered pointer is not an error here
  }
  cudaMemcpyAsync(c->fnod, f_host, nn * sizeof(double), cudaMemcpyHostToDevice, st);
  const int rc = semmg_solve(c, c->fnod, u_map ? u_map : c->unod, rtol, info, stream);
  if (rc != SEMMG_OK && rc != SEMMG_ERR_NOT_CONVERGED && rc != SEMMG_ERR_NONFINITE) return rc;
  if (!u_map) cudaMemcpyAsync(u_host, c->unod, nn * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(c, "solve_host");
  return rc;
}

const char* semmg_strerror(int code) {
  switch (code) {
    case SEMMG_OK: return "success";
    case SEMMG_ERR_INVALID_ARG: return "invalid argument";
    case SEMMG_ERR_UNSUPPORTED: return "unsupported configuration";
    case SEMMG_ERR_CUDA: return "CUDA error";
    case SEMMG_ERR_NOT_CONVERGED: return "not converged";
    case SEMMG_ERR_NONFINITE: return "non-finite residual";
    case SEMMG_ERR_TIMEOUT: return "device wait timed out";
    case SEMMG_ERR_NOMEM: return "out of memory";
    case SEMMG_ERR_DIVERGED: return "residual diverged";
    default: return "unknown error";
  }
}

const char* semmg_last_error(const semmg_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"

extern "C" {

int semmg_set_timing(semmg_ctx* c, int enable) {
  if (!c) return SEMMG_ERR_INVALID_ARG;
  collect_timing(c);
  if (c->timing != (enable ? 1 : 0)) c->drop_step_graph();  // recaptured with or without event nodes
  c->timing = enable ? 1 : 0;
  for (auto& k : c->ks) k = semmg_kstat{};
  return check_cuda(c, "set_timing");
}

int semmg_get_kstat(semmg_ctx* c, int kind, semmg_kstat* out) {
  if (!c || !out || kind < 0 || kind >= SEMMG_K_COUNT) return SEMMG_ERR_INVALID_ARG;
  collect_timing(c);
  *out = c->ks[kind];
  return check_cuda(c, "get_kstat");
}

int semmg_reset_kstats(semmg_ctx* c) {
  if (!c) return SEMMG_ERR_INVALID_ARG;
  collect_timing(c);
  for (auto& k : c->ks) k = semmg_kstat{};
  return check_cuda(c, "reset_kstats");
}

int semmg_set_guards(semmg_ctx* c, double divergence, long long tc_wait_cycles) {
  if (!c || !(divergence > 0.0) || tc_wait_cycles < 0) return SEMMG_ERR_INVALID_ARG;
  c->divergence = divergence;
  if (c->tc_wait != tc_wait_cycles) c->drop_step_graph();  // the captured launches hold the budget
  c->tc_wait = tc_wait_cycles;
  return SEMMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batched form (one CUDA graph)

namespace {

struct BatchCtl {
  double res0sq;
  double ressq;
  double rtol;
  double div;  // divergence factor of the solve's context
  int iters;
  int maxit;
  int status;
  int pad;
};

// r_0 known: start the loop unless the right-hand side is zero or not finite.
__global__ void k_batch_init(BatchCtl* ctl, const double* dnorm, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r0 = *dnorm;
  ctl->res0sq = r0;
  ctl->ressq = r0;
  ctl->iters = 0;
  const bool finite = isfinite(r0);
  const bool need = finite && r0 > ctl->rtol * ctl->rtol * r0;  // not yet converged (as semmg_solve tests it)
  ctl->status = !finite ? SEMMG_ERR_NONFINITE : ((need && ctl->maxit <= 0) ? SEMMG_ERR_NOT_CONVERGED : SEMMG_OK);
  cudaGraphSetConditional(h, (need && ctl->maxit > 0) ? 1u : 0u);
}

// after a cycle: continue while ||r||^2 > rtol^2 ||r_0||^2 and below the cycle cap
__global__ void k_batch_check(BatchCtl* ctl, const double* dnorm, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = *dnorm;
  ctl->ressq = r;
  ctl->iters += 1;
  unsigned cont = 1u;
  if (!isfinite(r)) {
    ctl->status = SEMMG_ERR_NONFINITE;
    cont = 0u;
  } else if (r <= ctl->rtol * ctl->rtol * ctl->res0sq) {
    ctl->status = SEMMG_OK;
    cont = 0u;
  } else if (r > ctl->div * ctl->div * ctl->res0sq) {
    ctl->status = SEMMG_ERR_DIVERGED;
    cont = 0u;
  } else if (ctl->iters >= ctl->maxit) {
    ctl->status = SEMMG_ERR_NOT_CONVERGED;
    cont = 0u;
  }
  cudaGraphSetConditional(h, cont);
}

}  // namespace

struct semmg_batch {
  std::vector<semmg_ctx*> ctxs;
  BatchCtl* dctl = nullptr;
  BatchCtl* hctl = nullptr;  // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t nodes = 0;
  ~semmg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (dctl) cudaFree(dctl);
    if (hctl) cudaFreeHost(hctl);
    cudaGetLastError();
  }
};

namespace {

// Enqueue one solve of context c (device nodal f -> u) into the capturing stream s.
int capture_solve(semmg_ctx* c, const double* f, const double* gdata, double* u, BatchCtl* ctl, cudaStream_t s,
                  cudaStream_t sb) {
  condense_impl(c, f, c->Fh, true, s, true);
  iter_start(c, s, gdata);
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g) != cudaSuccess || cs != cudaStreamCaptureStatusActive)
    return fail(c, SEMMG_ERR_CUDA, "batch: stream is not capturing");
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    return check_cuda(c, "batch: conditional handle");
  k_batch_init<<<1, 32, 0, s>>>(ctl, c->dnorm, h);
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps) != cudaSuccess)
    return check_cuda(c, "batch: capture info");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if (cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp) != cudaSuccess) return check_cuda(c, "batch: while node");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return check_cuda(c, "batch: body capture");
  iter_step(c, sb);
  k_batch_check<<<1, 32, 0, sb>>>(ctl, c->dnorm, h);
  cudaGraph_t got = nullptr;
  if (cudaStreamEndCapture(sb, &got) != cudaSuccess) return check_cuda(c, "batch: body end");
  if (cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return check_cuda(c, "batch: dependencies");
  recover_impl(c, f, c->Uh, u, true, s, true);
  return check_cuda(c, "batch: capture");
}

}  // namespace

extern "C" {

int semmg_batch_create(semmg_ctx* const* ctxs, int nb, const double* const* f, double* const* u, double rtol,
                       void* stream, semmg_batch** out) {
  return semmg_batch_create_dirichlet(ctxs, nb, f, nullptr, u, rtol, stream, out);
}

int semmg_batch_create_dirichlet(semmg_ctx* const* ctxs, int nb, const double* const* f, const double* const* g,
                                 double* const* u, double rtol, void* stream, semmg_batch** out) {
  if (!out) return SEMMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || !f || !u || nb < 1 || !(rtol > 0.0)) return SEMMG_ERR_INVALID_ARG;
  for (int i = 0; i < nb; ++i) {
    if (!ctxs[i] || !f[i] || !u[i]) return SEMMG_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return SEMMG_ERR_INVALID_ARG;  // one context per branch: its buffers are not shared
  }
  std::unique_ptr<semmg_batch> b(new (std::nothrow) semmg_batch());
  if (!b) return SEMMG_ERR_NOMEM;
  b->ctxs.assign(ctxs, ctxs + nb);
  if (cudaMalloc((void**)&b->dctl, nb * sizeof(BatchCtl)) != cudaSuccess ||
      cudaMallocHost((void**)&b->hctl, nb * sizeof(BatchCtl)) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_NOMEM;
  }
  for (int i = 0; i < nb; ++i) {
    b->hctl[i] = BatchCtl{0.0, 0.0, rtol, ctxs[i]->divergence, 0, ctxs[i]->opts.max_iter, 0, 0};
  }
  if (cudaMemcpy(b->dctl, b->hctl, nb * sizeof(BatchCtl), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return SEMMG_ERR_CUDA;
  }
  // timing events cannot be recorded inside the captured graph
  std::vector<int> timing(nb);
  for (int i = 0; i < nb; ++i) {
    timing[i] = ctxs[i]->timing;
    collect_timing(ctxs[i]);
    ctxs[i]->timing = 0;
  }
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> s(nb, nullptr), sb(nb, nullptr);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  int rc = SEMMG_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < nb; ++i) {
      if (s[i]) cudaStreamDestroy(s[i]);
      if (sb[i]) cudaStreamDestroy(sb[i]);
      ctxs[i]->timing = timing[i];
    }
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    if (cap) cudaStreamDestroy(cap);
  };
  bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; ok && i < nb; ++i)
    ok = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&sb[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; ok && i <= nb; ++i) ok = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cleanup();
    return SEMMG_ERR_CUDA;
  }
  cudaStreamSynchronize((cudaStream_t)stream);
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return SEMMG_ERR_CUDA;
  }
  cudaEventRecord(ev[nb], cap);
  for (int i = 0; i < nb && rc == SEMMG_OK; ++i) {
    cudaStreamWaitEvent(s[i], ev[nb], 0);
    rc = capture_solve(ctxs[i], f[i], g ? g[i] : nullptr, u[i], b->dctl + i, s[i], sb[i]);
    cudaEventRecord(ev[i], s[i]);
    cudaStreamWaitEvent(cap, ev[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
  if (rc == SEMMG_OK && (ee != cudaSuccess || !graph)) rc = SEMMG_ERR_CUDA;
  if (rc == SEMMG_OK) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    b->nodes = (int64_t)nn;
    if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = SEMMG_ERR_CUDA;
  }
  b->graph = graph;
  cudaGetLastError();
  cleanup();
  if (rc != SEMMG_OK) return rc;
  *out = b.release();
  return SEMMG_OK;
}

int semmg_batch_solve(semmg_batch* b, semmg_info* infos, void* stream) {
  if (!b || !b->exec) return SEMMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)b->ctxs.size();
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return check_cuda(b->ctxs[0], "batch_solve: launch");
  cudaMemcpyAsync(b->hctl, b->dctl, nb * sizeof(BatchCtl), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(b->ctxs[0], "batch_solve");
  int first = SEMMG_OK;
  for (int i = 0; i < nb; ++i) {
    const BatchCtl& k = b->hctl[i];
    if (infos) {
      infos[i].iters = k.iters;
      infos[i].res0 = std::sqrt(k.res0sq);
      infos[i].res_final = std::sqrt(k.ressq);
      infos[i].rho = (k.iters > 0 && k.res0sq > 0) ? std::pow(std::sqrt(k.ressq / k.res0sq), 1.0 / k.iters) : 0.0;
      infos[i].status = k.status;
    }
    if (first == SEMMG_OK && k.status != SEMMG_OK) first = k.status;
  }
  return first;
}

int semmg_batch_graph_nodes(const semmg_batch* b, int64_t* nodes) {
  if (!b || !nodes) return SEMMG_ERR_INVALID_ARG;
  *nodes = b->nodes;
  return SEMMG_OK;
}

void semmg_batch_destroy(semmg_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------- launch autotuning

namespace {

struct TuneChoice {
  size_t cap;
  int block;
  int wide;
};
std::mutex g_tune_lock;
// (kernel, element size, degree, elements) -> choice: the best shape depends on how many
// stars / elements share the SMs, so each mesh size is timed once per process
std::map<std::tuple<int, int, int, int64_t>, TuneChoice> g_tune;

const size_t kTuneCaps[3] = {48 * 1024, 100 * 1024, 200 * 1024};
const int kTuneBlocks[2] = {256, 512};
const int kTuneWide[2] = {0, 1};

template <typename T>
float time_launch(semmg_ctx* c, int l, int kernel, const LaunchCfg& cfg, const T* in, T* out, cudaStream_t st) {
  const Geo& G = c->geo[l];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the Schur kernel is timed inside the whole operator application (its face-parallel form
  // moves work between the Schur and the assembly launches); out: a level-sized scratch vector
  auto run = [&]() {
    if (kernel == 0)
      launch_star<T>(G, tabs<T>(c, l), in, (T*)c->Obs, (T*)c->wss, cfg, c->star_counter, st);
    else
      apply_op<T, T>(c, l, tabs<T>(c, l), cfg, (const T*)nullptr, in, out, 1, st);
  };
  run();
  cudaEventRecord(e0, st);
  const int reps = 3;
  for (int i = 0; i < reps; ++i) run();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

template <typename T>
void tune_one(semmg_ctx* c, int l, int kernel, LaunchCfg& slot, const T* in, T* out, cudaStream_t st) {
  const Geo& G = c->geo[l];
  const auto key = std::make_tuple(kernel, (int)sizeof(T), G.p, (int64_t)G.nelem);
  {
    std::lock_guard<std::mutex> g(g_tune_lock);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const TuneChoice& ch = it->second;
      LaunchCfg cf = kernel == 0 ? plan_star<T>(G, c->nsm, ch.cap, ch.block, ch.wide)
                                 : plan_elem_schur<T>(G, c->nsm, ch.cap, ch.block, ch.wide);
      if (cf.ok && cf.ws_elems() * sizeof(T) <= c->ws_bytes) slot = cf;
      return;
    }
  }
  float best = 1e30f;
  TuneChoice bc{0, 0, 0};
  LaunchCfg bcfg = slot;
  for (size_t cap : kTuneCaps)
    for (int blk : kTuneBlocks)
      for (int wide : kTuneWide) {
        LaunchCfg cf = kernel == 0 ? plan_star<T>(G, c->nsm, cap, blk, wide)
                                   : plan_elem_schur<T>(G, c->nsm, cap, blk, wide);
        if (!cf.ok || cf.ws_elems() * sizeof(T) > c->ws_bytes) continue;
        const float ms = time_launch<T>(c, l, kernel, cf, in, out, st);
        if (ms < best) {
          best = ms;
          bc = TuneChoice{cap, blk, wide};
          bcfg = cf;
        }
      }
  if (best < 1e30f) {
    slot = bcfg;
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune[key] = bc;
  }
}

}  // namespace

extern "C" int semmg_autotune(semmg_ctx* c, void* stream) {
  if (!c) return SEMMG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->drop_step_graph();
  collect_timing(c);
  const int saved = c->timing;
  c->timing = 0;
  const int L = c->L();
  // the star kernel in the V-cycle precision; the Schur kernel in FP64 arithmetic
  // except for the all-FP32 cycle (whose outer residual is FP64 too).  The FP64
  // timing input is Uh, which holds at least as many values as any level.
  const bool c32 = cycle32(c);
  const bool all32 = c->opts.precision == SEMMG_MIXED_FP32 || c->opts.precision == SEMMG_MIXED_FP32_TC;
  for (int l = 0; l <= L; ++l) {
    if (l >= 1 && c->opts.smoother == SEMMG_SMOOTHER_STAR) {  // the element-centred kernel has one shape
      if (c32)
        tune_one<float>(c, l, 0, c->dl[l].star32, (const float*)c->dl[l].Fw, nullptr, st);
      else
        tune_one<double>(c, l, 0, c->dl[l].star64, (const double*)c->dl[l].Fw, nullptr, st);
    }
    if (c->geo[l].m == 0) continue;
    // operator outputs: the level's FP32 work vector / the finest-level FP64 residual (scratch here)
    if (all32) tune_one<float>(c, l, 1, c->dl[l].schur32, (const float*)c->dl[l].Fw, (float*)c->dl[l].Rw, st);
    if (!all32 || l == L) tune_one<double>(c, l, 1, c->dl[l].schur64, c->Uh, c->Rh, st);
  }
  c->timing = saved;
  if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(c, "autotune");
  return check_cuda(c, "autotune");
}

extern "C" int semmg_set_launch(semmg_ctx* c, int level, int kernel, int dtype, int smem_cap, int block,
                                int max_regs) {
  if (!valid_level(c, level) || (kernel != 0 && kernel != 1) || (dtype != SEMMG_F64 && dtype != SEMMG_F32))
    return SEMMG_ERR_INVALID_ARG;
  if (smem_cap < 0 || smem_cap > 200 * 1024 || (block != 256 && block != 512) || (max_regs != 64 && max_regs != 128))
    return SEMMG_ERR_INVALID_ARG;
  if (kernel == 0 && level < 1) return SEMMG_ERR_INVALID_ARG;
  if (kernel == 1 && c->geo[level].m == 0) return SEMMG_ERR_INVALID_ARG;
  const Geo& G = c->geo[level];
  const int wide = max_regs == 128 ? 1 : 0;
  DevLevel& D = c->dl[level];
  LaunchCfg cf;
  size_t es;
  if (dtype == SEMMG_F64) {
    es = sizeof(double);
    cf = kernel == 0 ? plan_star<double>(G, c->nsm, smem_cap, block, wide)
                     : plan_elem_schur<double>(G, c->nsm, smem_cap, block, wide);
  } else {
    es = sizeof(float);
    cf = kernel == 0 ? plan_star<float>(G, c->nsm, smem_cap, block, wide)
                     : plan_elem_schur<float>(G, c->nsm, smem_cap, block, wide);
  }
  if (!cf.ok || cf.ws_elems() * es > c->ws_bytes)
    return fail(c, SEMMG_ERR_UNSUPPORTED, "set_launch: shape does not fit the work memory of the context");
  LaunchCfg& slot = kernel == 0 ? (dtype == SEMMG_F64 ? D.star64 : D.star32) : (dtype == SEMMG_F64 ? D.schur64 : D.schur32);
  slot = cf;
  c->drop_step_graph();
  return SEMMG_OK;
}

extern "C" int semmg_get_launch(const semmg_ctx* c, int level, int kernel, int dtype, int* block, int* smem,
                                int* grid, int* max_regs) {
  if (!valid_level(c, level) || !block || !smem || !grid || !max_regs || (kernel != 0 && kernel != 1))
    return SEMMG_ERR_INVALID_ARG;
  const DevLevel& D = c->dl[level];
  const LaunchCfg* cf;
  if (kernel == 0) cf = dtype == SEMMG_F32 ? (D.startc.ok ? &D.startc : &D.star32) : &D.star64;
  else cf = dtype == SEMMG_F32 ? &D.schur32 : &D.schur64;
  *block = cf->block;
  *smem = (int)cf->smem;
  *grid = cf->grid;
  *max_regs = cf->wide ? 128 : 64;
  return SEMMG_OK;
}
