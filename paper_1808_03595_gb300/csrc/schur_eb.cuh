// Element Schur term in the face eigenbasis, streamed plane by plane (Sec. 2.2).
//
// On the levels of the face-parallel operator every face arrives transformed
// into its in-plane eigenbasis (k_face_fwd).  For one element the Schur term
// H_BI H_II^{-1} H_IB u on its six faces is then, in the interior eigenbasis
// k = (k1, k2, k3),
//   W(k) = D(k)^{-1} (a0[k1] X_{0|1}(k3,k2) + a0[k2] X_{2|3}(k3,k1) + a0[k3] X_{4|5}(k2,k1)),
//   X'_{0|1}(k3,k2) = sum_k1 a0[k1] W(k),  X'_{2|3}(k3,k1) = sum_k2 a0[k2] W(k),
//   X'_{4|5}(k2,k1) = sum_k3 a0[k3] W(k),
// where X_{2d}, X_{2d+1} are alpha_d times the sum and the difference of the two
// faces normal to axis d, the one used at k being picked by the parity class of
// k_d (eigenvector columns 0..ne-1 even, ne..m-1 odd), and the sums over k_d run
// over that class.  The element's face terms are
//   Z_{2d} = alpha_d (X'_{2d} + X'_{2d+1}),  Z_{2d+1} = alpha_d (X'_{2d} - X'_{2d+1})
// (elem_kernel.cuh derives the same terms with W stored; here W is never
// stored: each k3-plane is formed in registers and consumed at once).
//
// Thread mapping (512 threads, 16 warps; one element per CTA, or per cluster of two
// CTAs that take alternate blocks of planes, at a time):
//  - warp w owns the rows k2 = w + 16 i (i < NI) of every plane; a row's parity
//    class is uniform over the warp;
//  - lane l owns NJ column slots: lanes 0..15 the even columns k1 = 16 j + l,
//    lanes 16..31 the odd columns k1 = ne + 16 j + (l - 16), so all columns of a
//    lane are of one class.
// Per plane, the sums over k1 are reduced within each half-warp by one
// butterfly reduce-scatter over the warp's rows (X'_0 in the lower half, X'_1
// in the upper); the sums over k2 are per-warp partials in shared memory, added
// in warp order every KB planes; the sums over k3 accumulate in registers, the
// even planes first (X'_4), then the odd ones (X'_5).  Every output has a fixed
// summation order.
#pragma once
#include "elem_kernel.cuh"

namespace semmg {

namespace {

constexpr int kEbWarps = 16;  // 512 threads
// planes per shared-memory round of the k2 sums: 4, or 2 with two column slots (whose wider
// partial-sum rows would not leave room for the table staging)
__host__ __device__ constexpr int eb_kb(int nj) { return nj > 1 ? 2 : 4; }
constexpr int kEbSmemMax = 224 * 1024;

__device__ __forceinline__ float eb_shx(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double eb_shx(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ ff eb_shx(ff v, int off) {
  return ff(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// Reduce-scatter over the 16 lanes of a half-warp: R values per lane (R a power of
// two) -> the sum over the half-warp of value rs16_index<R>(lane).  Partners add in
// either order, which gives the same bits (addition commutes).
template <int R, typename T>
__device__ __forceinline__ T rs16_reduce(T* v, int lane) {
  int off = 8;
#pragma unroll
  for (int n = R; n > 1; n >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const T send = hi ? v[k] : v[k + n / 2];
      const T keep = hi ? v[k + n / 2] : v[k];
      v[k] = keep + eb_shx(send, off);
    }
  }
  T t = v[0];
#pragma unroll
  for (; off > 0; off >>= 1) t = t + eb_shx(t, off);
  return t;
}

template <int R>
__device__ __forceinline__ int rs16_index(int lane) {
  int idx = 0, off = 8;
#pragma unroll
  for (int n = R; n > 1; n >>= 1, off >>= 1)
    if (lane & off) idx += n / 2;
  return idx;
}

__host__ __device__ constexpr int eb_pow2(int n) { return n <= 1 ? 1 : (n <= 2 ? 2 : (n <= 4 ? 4 : 8)); }

// Shared memory of the kernel, in elements of T: X (6 m^2), Y (k2 partial sums:
// 16 warps x KB planes x 2 classes x NJ*32 slots), a0 (m), lI (m), and with the
// 1/D table the staging of each thread's table values for two planes
// (2 x NI*NJ slots x 512 threads, thread index fastest).
__host__ __device__ constexpr size_t eb_smem_elems(int m, int ni, int nj, bool tab) {
  return (size_t)6 * m * m + (size_t)kEbWarps * eb_kb(nj) * 2 * nj * 32 + 2 * (size_t)m +
         (tab ? (size_t)2 * ni * nj * 512 : 0);
}

// Asynchronous copy of one 8-byte table value into shared memory (cp.async, sm_80+);
// copies complete in commit-group order, and a thread reads only its own copies.
__device__ __forceinline__ void eb_cp8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void eb_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void eb_cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// 1/D at one point: the element class's table, or the sum of the scaled eigenvalues inverted
__device__ __forceinline__ double eb_inv(double d) { return 1.0 / d; }
__device__ __forceinline__ float eb_inv(float d) { return rcp_approx(d); }
__device__ __forceinline__ ff eb_inv(ff d) { return ff_recip(d); }

// TAB: 1/D from the element class's table (t.Relem), else computed per point; a
// template parameter so that neither form carries the other's work.
template <typename T, int NI, int NJ, bool TAB>
__global__ void __launch_bounds__(512, 1) k_schur_eb(Geo G, Tabs<T> t, const T* __restrict__ Ut, T* __restrict__ Z,
                                                     T* ws, int cs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kEbKB = eb_kb(NJ);
  const int m = G.m, mm = m * m, ne = (m + 1) / 2;
  const int64_t n3 = (int64_t)mm * m;
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Y = X + 6 * mm;
  T* a0 = Y + kEbWarps * kEbKB * 2 * NJ * 32;
  T* lI = a0 + m;
  T* Rs = lI + m;  // [step & 1][i NJ + j][thread] (TAB only)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = lane >> 4, hl = lane & 15;
  // cs = 2: the two CTAs of a cluster share an element, taking alternate blocks of KB planes of
  // each parity class; the second CTA's sums over k3 (faces 4, 5) go through ws to the first,
  // which adds them after its own
  const Team tm = team_of(cs);
  const int rank = tm.id / (int)blockDim.x;
  T* wsT = ws + (int64_t)(blockIdx.x / cs) * 2 * NI * NJ * 512;
  // this CTA's plane after k3 (k3 < 0: its first plane), or -1
  auto next_plane = [&](int k3) -> int {
    if (k3 >= 0) {
      const int q = k3 >= ne ? 1 : 0, lo = q ? ne : 0, hi = q ? m : ne, off = k3 - lo;
      if ((off + 1) % kEbKB != 0 && k3 + 1 < hi) return k3 + 1;
      const int nb = lo + (off / kEbKB + cs) * kEbKB;
      if (nb < hi) return nb;
      if (q == 1) return -1;
    } else if (rank * kEbKB < ne) {
      return rank * kEbKB;
    }
    return ne + rank * kEbKB < m ? ne + rank * kEbKB : -1;
  };
  for (int i = tid; i < m; i += blockDim.x) {
    a0[i] = t.a0[i];
    lI[i] = t.lamI[i];
  }
  const T lam = (T)G.lam;
  constexpr int R = eb_pow2(NI);
  const int me = rs16_index<R>(lane);                 // the row whose k1 sum this lane receives
  const bool wr = (hl & (16 / R - 1)) == 0 && me < NI;  // one writer lane per row and half
  // columns and rows of this lane (invalid ones point at index 0 and carry zero weights)
  int k1v[NJ], k2v[NI];
  bool ok1[NJ], ok2[NI], odd2[NI];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const int c = half ? ne + 16 * j + hl : 16 * j + hl;
    ok1[j] = half ? c < m : c < ne;
    k1v[j] = ok1[j] ? c : 0;
  }
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int r = warp + kEbWarps * i;
    ok2[i] = r < m;
    odd2[i] = r >= ne;  // uniform over the warp
    k2v[i] = ok2[i] ? r : 0;
  }
  for (int64_t e = blockIdx.x / cs; e < G.nelem; e += gridDim.x / cs) {
    int a1, a2, a3;
    elem_coords(G, e, &a1, &a2, &a3);
    const ElemScal<T> sc = elem_scalars(t, a1, a2, a3);
    const T* Rt = TAB ? t.Relem + sc.cls * n3 : nullptr;
    // stage this thread's table values of plane k3 into buffer b (one commit group per plane)
    auto stage = [&](int k3, int b) {
      if constexpr (TAB) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j)
            if (ok2[i] && ok1[j])
              eb_cp8(Rs + ((size_t)(b * NI * NJ + i * NJ + j) * blockDim.x + tid),
                     Rt + ((int64_t)k3 * m + k2v[i]) * m + k1v[j]);
        eb_cp_commit();
      }
    };
    tm.sync();  // X and Y of the previous element are consumed, and the team's ws slice
    for (int idx = tid; idx < 3 * mm; idx += blockDim.x) {
      const int d = idx / mm, r = idx - d * mm;
      const T a = Ut[elem_face_base(G, a1, a2, a3, 2 * d) + r];
      const T b = Ut[elem_face_base(G, a1, a2, a3, 2 * d + 1) + r];
      X[(2 * d) * mm + r] = sc.ald(d) * (a + b);
      X[(2 * d + 1) * mm + r] = sc.ald(d) * (a - b);
    }
    __syncthreads();
    T a1r[NJ], a2r[NI];
#pragma unroll
    for (int j = 0; j < NJ; ++j) a1r[j] = ok1[j] ? a0[k1v[j]] : (T)0;
#pragma unroll
    for (int i = 0; i < NI; ++i) a2r[i] = ok2[i] ? a0[k2v[i]] : (T)0;
    T* Ze = Z + e * 6 * mm;
    const T al0 = sc.al[0], al1 = sc.al[1], al2 = sc.al[2];
    int step = 0;  // planes this CTA has done in this element (staging buffer step & 1)
    {
      const int f = next_plane(-1);
      if (f >= 0) stage(f, 0);
    }
    for (int q3 = 0; q3 < 2; ++q3) {
      const int lo3 = q3 ? ne : 0, hi3 = q3 ? m : ne;
      T x45[NI][NJ], b3[NI][NJ];
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          x45[i][j] = (ok2[i] && ok1[j]) ? X[(4 + q3) * mm + k2v[i] * m + k1v[j]] : (T)0;
          b3[i][j] = (T)0;
        }
      for (int k3b = lo3 + rank * kEbKB; k3b < hi3; k3b += cs * kEbKB) {
        const int nb = hi3 - k3b < kEbKB ? hi3 - k3b : kEbKB;
        for (int kb = 0; kb < nb; ++kb, ++step) {
          const int k3 = k3b + kb;
          const T a3 = a0[k3];
          const int buf = step & 1;
          if constexpr (TAB) {  // the next plane's values on their way, this plane's in place
            const int nk = next_plane(k3);
            if (nk >= 0) {
              stage(nk, buf ^ 1);
              eb_cp_wait<1>();
            } else {
              eb_cp_wait<0>();
            }
          }
          T x01[NI], x23e[NJ], x23o[NJ], b1[R], b2e[NJ], b2o[NJ];
#pragma unroll
          for (int i = 0; i < NI; ++i) x01[i] = X[half * mm + k3 * m + k2v[i]];
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            x23e[j] = X[2 * mm + k3 * m + k1v[j]];
            x23o[j] = X[3 * mm + k3 * m + k1v[j]];
            b2e[j] = (T)0;
            b2o[j] = (T)0;
          }
#pragma unroll
          for (int i = 0; i < R; ++i) b1[i] = (T)0;
#pragma unroll
          for (int i = 0; i < NI; ++i) {
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              const bool ok = ok2[i] && ok1[j];
              const T x23 = odd2[i] ? x23o[j] : x23e[j];
              T E = a1r[j] * x01[i];
              E = madd(a2r[i], x23, E);
              E = madd(a3, x45[i][j], E);
              // 1/D: the class table, or lam + sum_d (4/h_d^2) Lam[k_d] summed in that order and inverted
              T rinv;
              if constexpr (TAB)
                rinv = Rs[(size_t)(buf * NI * NJ + i * NJ + j) * blockDim.x + tid];
              else
                rinv = eb_inv(lam + sc.e[0] * lI[k1v[j]] + sc.e[1] * lI[k2v[i]] + sc.e[2] * lI[k3]);
              const T V = ok ? E * rinv : (T)0;
              b1[i] = madd(a1r[j], V, b1[i]);
              if (odd2[i])
                b2o[j] = madd(a2r[i], V, b2o[j]);
              else
                b2e[j] = madd(a2r[i], V, b2e[j]);
              b3[i][j] = madd(a3, V, b3[i][j]);
            }
          }
          // faces 0 / 1 at (k3, k2): the half-warp sums, even class below, odd above
          const T s1 = rs16_reduce<R>(b1, lane);
          const T other = eb_shx(s1, 16);
#pragma unroll
          for (int i = 0; i < NI; ++i)
            if (wr && me == i && ok2[i]) {
              const int r = k3 * m + k2v[i];
              if (half == 0)
                Ze[0 * mm + r] = al0 * (s1 + other);
              else
                Ze[1 * mm + r] = al0 * (other - s1);
            }
          // faces 2 / 3: this warp's partial sums over its rows
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            Y[((warp * kEbKB + kb) * 2 + 0) * (NJ * 32) + j * 32 + lane] = b2e[j];
            Y[((warp * kEbKB + kb) * 2 + 1) * (NJ * 32) + j * 32 + lane] = b2o[j];
          }
        }
        __syncthreads();
        // faces 2 / 3 at (k3, k1): the 16 warps' partial sums in warp order
        for (int o = tid; o < nb * NJ * 32; o += blockDim.x) {
          const int kb = o / (NJ * 32), s = o - kb * (NJ * 32), j = s >> 5, ln = s & 31;
          const int c = (ln >> 4) ? ne + 16 * j + (ln & 15) : 16 * j + (ln & 15);
          const bool okc = (ln >> 4) ? c < m : c < ne;
          if (!okc) continue;
          T se = Y[((0 * kEbKB + kb) * 2 + 0) * (NJ * 32) + s];
          T so = Y[((0 * kEbKB + kb) * 2 + 1) * (NJ * 32) + s];
#pragma unroll
          for (int w = 1; w < kEbWarps; ++w) {
            se = se + Y[((w * kEbKB + kb) * 2 + 0) * (NJ * 32) + s];
            so = so + Y[((w * kEbKB + kb) * 2 + 1) * (NJ * 32) + s];
          }
          const int r = (k3b + kb) * m + c;
          Ze[2 * mm + r] = al1 * (se + so);
          Ze[3 * mm + r] = al1 * (se - so);
        }
        __syncthreads();
      }
      // faces 4 / 5 at (k2, k1): the even planes' sums wait in X_4 (read into registers at
      // the start and owned by this thread); with a second CTA its sums come through ws
      if (cs > 1 && rank == 1) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j) wsT[(size_t)(q3 * NI * NJ + i * NJ + j) * 512 + tid] = b3[i][j];
      }
      if (q3 == 0) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j)
            if (ok2[i] && ok1[j]) X[4 * mm + k2v[i] * m + k1v[j]] = b3[i][j];
      } else {
        tm.sync();  // the second CTA's sums are in ws
        if (rank == 0) {
#pragma unroll
          for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
              if (!(ok2[i] && ok1[j])) continue;
              const int r = k2v[i] * m + k1v[j];
              T ev = X[4 * mm + r], od = b3[i][j];
              if (cs > 1) {
                ev = ev + wsT[(size_t)(0 * NI * NJ + i * NJ + j) * 512 + tid];
                od = od + wsT[(size_t)(1 * NI * NJ + i * NJ + j) * 512 + tid];
              }
              Ze[4 * mm + r] = al2 * (ev + od);
              Ze[5 * mm + r] = al2 * (ev - od);
            }
        }
      }
    }
  }
}

}  // namespace

// Launch shape of the streamed eigenbasis Schur kernel for the level (block 512).
template <typename T>
LaunchCfg plan_schur_eb(const Geo& G, int nsm) {
  LaunchCfg c;
  const int m = G.m, nj = m > 32 ? 2 : 1, ni = m <= 16 ? 1 : (m <= 32 ? 2 : 3);
  c.block = 512;
  c.smem = eb_smem_elems(m, ni, nj, true) * sizeof(T);  // the table-staging size covers both forms
  c.ok = m >= 1 && m < SEMMG_MAX_DEGREE && c.smem <= (size_t)kEbSmemMax;
  // one CTA per SM: the kernel takes 70 to 122 registers a thread (FP32 to FP64 tiles); two
  // per element (a cluster) when halving the work units shortens the rounds per SM
  // (elements with m >= 32 only: on smaller ones the split's exchange costs more than it saves)
  const int64_t r1 = (G.nelem + nsm - 1) / nsm, r2 = (2 * G.nelem + nsm - 1) / nsm;
  c.cluster = (m >= 32 && nsm >= 2 && r2 < 2 * r1) ? 2 : 1;
  const int64_t teams = nsm / c.cluster, nt = G.nelem < teams ? G.nelem : teams;
  c.grid = (int)((nt < 1 ? 1 : nt) * c.cluster);
  c.ws.gstride = (int64_t)2 * ni * nj * 512;  // per CTA: covers the team's slice
  if (c.grid < 1) c.grid = 1;
  return c;
}

template <typename T, bool TAB>
void launch_schur_eb_tab(const Geo& G, const Tabs<T>& t, const T* Ut, T* Z, T* ws, const LaunchCfg& c,
                         cudaStream_t st) {
  if (G.m <= 16)
    launch_clustered(k_schur_eb<T, 1, 1, TAB>, c, st, G, t, Ut, Z, ws, c.cluster);
  else if (G.m <= 32)
    launch_clustered(k_schur_eb<T, 2, 1, TAB>, c, st, G, t, Ut, Z, ws, c.cluster);
  else
    launch_clustered(k_schur_eb<T, 3, 2, TAB>, c, st, G, t, Ut, Z, ws, c.cluster);
}

template <typename T>
void launch_schur_eb(const Geo& G, const Tabs<T>& t, const T* Ut, T* Z, T* ws, const LaunchCfg& c, cudaStream_t st) {
  if (G.m == 0 || G.nelem == 0 || !c.ok) return;
  if (t.Relem)
    launch_schur_eb_tab<T, true>(G, t, Ut, Z, ws, c, st);
  else
    launch_schur_eb_tab<T, false>(G, t, Ut, Z, ws, c, st);
}

template <typename T, bool TAB>
int schur_eb_attrs_tab() {
  int bad = cudaFuncSetAttribute(k_schur_eb<T, 1, 1, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEbSmemMax);
  bad |= cudaFuncSetAttribute(k_schur_eb<T, 2, 1, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEbSmemMax);
  bad |= cudaFuncSetAttribute(k_schur_eb<T, 3, 2, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEbSmemMax);
  return bad;
}

template <typename T>
int schur_eb_attrs() {
  return schur_eb_attrs_tab<T, true>() | schur_eb_attrs_tab<T, false>();
}

}  // namespace semmg
