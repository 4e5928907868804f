// Star smoother with the in-plane 1D transforms on the 5th-generation tensor
// cores (tcgen05, TF32 operands, FP32 accumulators in tensor memory); the
// eigenspace step (expansion along the normals, 1/D, contractions back) stays
// on the FP32 cores.  Same mathematics as k_star (Algorithm 1 inside
// Algorithm 2, Sec. 3.2); used by the SEMMG_MIXED_TC form for 31 <= 2p-1 <= 64.
//
// A plane transform S_b^T X S_a is two dense products per plane, run as
// D[M=128][N] += A[M][K] B[N][K] (K-major operands in shared memory, 8 rows x
// 16 bytes core matrices, no swizzle), with K = N = NP = n_S rounded up to 16:
//   forward, along the slow axis:  W  = T(S_b) . P^T     (planes 0 and 1 share
//                                   the x3 tables and are stacked along N)
//   forward, along the fast axis:  Z  = W . T(S_a)
//   backward, slow axis:           O  = N(S_b) . B^T     (B: eigenspace result)
//   backward, fast axis:           Y  = O . N(S_a)
// with T(S)[e][j] = S[j][e] and N(S)[j][e] = S[j][e] prepared at setup, rounded
// to TF32.  Rows 64..127 of every M = 128 product are padding (their input rows
// are other data in shared memory; their outputs are not read).
#pragma once
#include <cstdint>

#include "star_kernel.cuh"

namespace semmg {

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// K-major operand, no swizzle: lbo = byte step between core matrices along K,
// sbo = byte step between 8-row groups; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// non-blocking probe: has the phase with the given parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase with the given parity, at most `budget` clock cycles: one
// non-blocking probe, then potentially blocking probes while the budget lasts (a
// try_wait may suspend the thread until the phase completes, so a budget of a
// few cycles still ends after the first probe when the products are in flight)
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  if (mbar_test_wait(mbar, parity)) return true;
  while (clock64() - t0 <= budget)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// tensor-memory load: thread l of the warp reads lane (quadrant base + l), 16 consecutive columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// round a finite float to TF32 (10 stored mantissa bits), nearest-even, with
// integer operations (the conversion instruction issues on a slow pipe)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0xFFFu + ((b >> 13) & 1u);
  return __uint_as_float(b & ~0x1FFFu);
}

// float offset of element (row, k) in a K-major operand with K = np columns
__device__ __forceinline__ int coff(int row, int k, int np) {
  return ((row >> 3) * (np >> 2) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

}  // namespace tc

namespace {

// bound of the wait for products still in flight after an abort (about 2 s at
// 2 GHz); the completion waits of the normal rounds take the caller's budget
constexpr long long kTcWaitCycles = 4000000000LL;

__host__ __device__ __forceinline__ int tc_np(int nS) { return (nS + 15) / 16 * 16; }
__host__ __device__ __forceinline__ int tc_ld(int np) { return np + 4; }  // row stride of the eigenspace planes
__host__ __device__ __forceinline__ int tc_cols(int np) {
  int c = 32;
  while (c < 3 * np) c *= 2;
  return c;
}

// Shared-memory layout in floats: tables 3 NP^2 | operands 3 NP^2 | planes
// 3 NP LD | V slab ts nS^2 | Lam 3 nS | s 3 nS | s3^2 nS (tables and operands
// first: an M = 128 product over the last table or operand reads the next
// region as padding rows).
__host__ __device__ __forceinline__ size_t tc_smem_floats(int nS) {
  const int np = tc_np(nS);
  return (size_t)6 * np * np + (size_t)3 * np * tc_ld(np) + (size_t)slab_thickness(nS) * nS * nS + 7 * nS + 8;
}

// D columns [col, col + N) += A (M = 128, K = np) B^T over the whole K extent.
__device__ __forceinline__ void tc_product(uint32_t tmem, int col, const float* A, const float* B, int N, int np) {
  const uint32_t sbo = (uint32_t)np * 32;  // bytes per 8-row group
  const uint32_t idesc = tc::idesc_tf32(128, N);
  for (int s = 0; s < np / 8; ++s)
    tc::mma_tf32(tmem + col, tc::smem_desc(A + 64 * s, 128, sbo), tc::smem_desc(B + 64 * s, 128, sbo), idesc, s > 0);
}

template <int PC>
__global__ void __launch_bounds__(512, 1) k_star_tc(Geo G, Tabs<float> t, const float* __restrict__ r,
                                                     float* __restrict__ Ob, int* counter, int* err,
                                                     long long wait_budget) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_next, s_abort;
  __shared__ int s_sym[3];
  __shared__ Ranges s_rg;
  __shared__ int Ac[3 * (2 * SEMMG_MAX_DEGREE - 1)];
  const int p = PC ? PC : G.p, m = p - 1, nS = 2 * p - 1, n2 = nS * nS;
  const int np = tc_np(nS), tb = np * np, ld = tc_ld(np);
  float* Tb = reinterpret_cast<float*>(smem_raw);  // tables T(S_d) or N(S_d), d = 0..2
  float* R1 = Tb + 3 * tb;                          // operands of the current product
  float* P = R1 + 3 * tb;                           // eigenspace planes [dd][k_b][k_a], row stride ld
  float* V = P + 3 * np * ld;
  float* Lm = V + slab_thickness(nS) * n2;
  float* Sv = Lm + 3 * nS;  // vertex rows s_d
  float* s3sq = Sv + 3 * nS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float lam = (float)G.lam;
  const float rcp_mult[3] = {1.0f, 0.5f, 1.0f / 3.0f};
  const uint32_t ncols = (uint32_t)tc_cols(np);
  if (tid == 0) {
    tc::mbar_init(&s_mbar, 1);
    s_abort = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  uint32_t phase = 0;
  // one tensor-core round: operands written -> products issued -> completion awaited
  auto round = [&](auto issue) -> bool {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      issue();
      tc::mma_commit(&s_mbar);
    }
    const bool ok = tc::mbar_wait(&s_mbar, phase, wait_budget);
    phase ^= 1u;
    if (!ok) {
      s_abort = 1;
      if (lane == 0) atomicExch(err, 1);
    }
    tc::fence_after();
    __syncthreads();
    return s_abort == 0;
  };
  // TMEM lanes [0, np) x columns [c0, c0 + 16 * nchunk): 16-column chunks spread
  // over the warps of quadrants 0 and 1 (lanes 0..63); f(row, col, v[16])
  auto readout = [&](int c0, int ncol, auto f) {
    const int q = warp & 3;
    if (q < 2 && q * 32 < np) {
      const int nchunk = ncol / 16, wq = warp >> 2;  // 4 warps per quadrant
      for (int ch = wq; ch < nchunk; ch += 4) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c0 + 16 * ch), v);
        const int row = q * 32 + lane;
        if (row < np) f(row, 16 * ch, v);
      }
    }
  };
  auto load_tables = [&](const float* const* src, const int* c) {
    for (int d = 0; d < 3; ++d) {
      const float4* s4 = reinterpret_cast<const float4*>(src[d] + (int64_t)t.starCls[d][c[d]] * tb);
      float4* d4 = reinterpret_cast<float4*>(Tb + d * tb);
      for (int i = tid; i < tb / 4; i += blockDim.x) d4[i] = s4[i];
    }
  };
  int64_t st = blockIdx.x;
  while (st < G.nstar) {
    const int c[3] = {(int)(st % G.nv1), (int)((st / G.nv1) % G.nv2), (int)(st / ((int64_t)G.nv1 * G.nv2))};
    // the last vertex plane of a periodic axis repeats plane 0: its stars are never read
    const bool alias = (G.per[0] && c[0] == G.n1) || (G.per[1] && c[1] == G.n2) || (G.per[2] && c[2] == G.n3);
    if (!alias) {
    __syncthreads();
    if (tid < 3) s_sym[tid] = t.starSym[tid][c[tid]];
    for (int d = 0; d < 3; ++d)
      for (int i = tid; i < nS; i += blockDim.x) {
        Lm[d * nS + i] = t.starLam[d][(int64_t)c[d] * nS + i];
        Ac[d * nS + i] = t.act[d][(int64_t)c[d] * nS + i];
        Sv[d * nS + i] = t.starS[d][(int64_t)c[d] * n2 + m * nS + i];
      }
    load_tables(t.tcT, c);
    __syncthreads();
    for (int i = tid; i < nS; i += blockDim.x) s3sq[i] = Sv[2 * nS + i] * Sv[2 * nS + i];
    if (tid < 3) {
      const int d = tid;
      int lo = 0, hi = nS;
      while (lo < nS && !Ac[d * nS + lo]) ++lo;
      while (hi > lo && !Ac[d * nS + hi - 1]) --hi;
      s_rg.lo[d] = lo;
      s_rg.hi[d] = hi;
      s_rg.pa[d] = Ac[d * nS + m];
    }
    // 1. gather the planes divided by the multiplicity, as B operands P_dd^T:
    //    row n = dd np + ja, column k = jb (zero outside the star and in the padding)
    for (int idx = tid; idx < 3 * tb; idx += blockDim.x) {
      const int dd = idx / tb, rr = idx - dd * tb, jbp = rr / np, jap = rr - jbp * np;
      float v = 0.0f;
      if (jap < nS && jbp < nS) {
        const int ja = jap - m, jb = jbp - m;
        const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
        if (Ac[dd * nS + m] && Ac[ax_a * nS + jap] && Ac[ax_b * nS + jbp]) {
          int g[3];
          g[dd] = c[dd] * p;
          g[ax_a] = c[ax_a] * p + ja;
          g[ax_b] = c[ax_b] * p + jb;
          v = tc::to_tf32(r[skel_index(G, g[0], g[1], g[2])] * rcp_mult[(ja == 0) + (jb == 0)]);
        }
      }
      R1[tc::coff(dd * np + jap, jbp, np)] = v;
    }
    // 2. forward, slow axis: W = T(S_b) P^T (planes 0, 1: x3 tables; plane 2: x2 tables)
    if (!round([&] {
          tc_product(tmem, 0, Tb + 2 * tb, R1, 2 * np, np);
          tc_product(tmem, 2 * np, Tb + 1 * tb, R1 + 2 * tb, np, np);
        }))
      break;
    // W (lanes k_b, columns dd np + ja) -> A operands (row k_b, k = ja)
    readout(0, 3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np;
      float* a = R1 + dd * tb;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 w4 = make_float4(tc::to_tf32(v[q]), tc::to_tf32(v[q + 1]), tc::to_tf32(v[q + 2]),
                                      tc::to_tf32(v[q + 3]));
        *reinterpret_cast<float4*>(a + tc::coff(row, k0 + q, np)) = w4;
      }
    });
    // 3. forward, fast axis: Z_dd = W_dd T(S_a) (plane 0: x2 tables; planes 1, 2: x1 tables)
    if (!round([&] {
          tc_product(tmem, 0, R1, Tb + 1 * tb, np, np);
          tc_product(tmem, np, R1 + tb, Tb, np, np);
          tc_product(tmem, 2 * np, R1 + 2 * tb, Tb, np, np);
        }))
      break;
    readout(0, 3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np;
      float* dst = P + (dd * np + row) * ld + k0;
#pragma unroll
      for (int q = 0; q < 16; q += 4) *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    });
    __syncthreads();
    // the backward tables replace the forward ones while the eigenspace step runs
    load_tables(t.tcN, c);
    const int* sym = s_sym;
    const Ranges rg = s_rg;
    // 4. eigenspace: E = sum_d s_d (x) P_d, V = E / D, B_d = contraction of V with s_d;
    //    results as the B operands of the backward slow-axis product:
    //    plane 0: B1[k3][k2] at (n = k2, k = k3), plane 1: B2[k3][k1] at (np + k1, k3),
    //    plane 2: B3[k2][k1] at (2 np + k1, k2)
    const float* s1 = Sv;
    const float* s2 = Sv + nS;
    const float* s3 = Sv + 2 * nS;
    const float* P0 = P;
    const float* P1 = P + np * ld;
    const float* P2 = P + 2 * np * ld;
    const int lo1 = rg.lo[0], w1 = rg.hi[0] - rg.lo[0], lo2 = rg.lo[1], w2 = rg.hi[1] - rg.lo[1];
    const int lo3 = rg.lo[2], w3 = rg.hi[2] - rg.lo[2];
    const int nz1 = rg.pa[0] ? (sym[0] ? m + 1 : w1) : 0;
    const int nz2 = rg.pa[1] ? (sym[1] ? m + 1 : w2) : 0;
    const int nz3 = rg.pa[2] ? (sym[2] ? m + 1 : w3) : 0;
    const int seg1 = nz2 * w1, seg2 = (w2 - nz2) * nz1, nlive = seg1 + seg2;
    const int npair = nlive + (rg.pa[2] ? (w2 - nz2) * (w1 - nz1) : 0);
    const int ts = slab_thickness(nS);
    // the pair segments, the same for every slab of the star
    const PairSeg sg_live1 = pair_seg(seg1, w1, lo1, lo2);
    const PairSeg sg_live2 = pair_seg(seg2, nz1, lo1, lo2 + nz2);
    const PairSeg sg_dead = pair_seg(rg.pa[2] ? npair - nlive : 0, w1 - nz1, lo1 + nz1, lo2 + nz2);
    float* B3 = R1 + 2 * tb;
    for (int i = tid; i < tb; i += blockDim.x) B3[i] = 0.0f;
    for (int k3s = rg.lo[2]; k3s < rg.hi[2]; k3s += ts) {
      const int tn = rg.hi[2] - k3s < ts ? rg.hi[2] - k3s : ts;
      __syncthreads();
      auto live = [&](int k1, int k2) {
        const int pr = k2 * nS + k1;
        const float a3 = rg.pa[2] ? P2[k2 * ld + k1] : 0.0f;
        float* b3p = B3 + tc::coff(k1, k2, np);
        {
          const float c1 = k1 - lo1 < nz1 ? s1[k1] : 0.0f, c2 = k2 - lo2 < nz2 ? s2[k2] : 0.0f;
          // loop invariants of the k3 run (as in k_star): the (k1, k2) part of D and the rows
          // where s3 may be non-zero
          const float d12 = lam + Lm[k1] + Lm[nS + k2];
          const float* p0 = P0 + k3s * ld + k2;
          const float* p1 = P1 + k3s * ld + k1;
          const int kl = min(max(lo3 + nz3 - k3s, 0), tn);
          float b3 = 0.0f;
          // unrolled: four independent load - divide - store chains in flight per thread
#pragma unroll 4
          for (int kk = 0; kk < kl; ++kk) {
            const int k3 = k3s + kk;
            float E = c1 * p0[kk * ld] + c2 * p1[kk * ld];
            E += s3[k3] * a3;
            const float v = fast_div(E, d12 + Lm[2 * nS + k3]);
            V[kk * n2 + pr] = v;
            b3 += s3[k3] * v;
          }
#pragma unroll 4
          for (int kk = kl; kk < tn; ++kk) {
            const float E = c1 * p0[kk * ld] + c2 * p1[kk * ld];
            V[kk * n2 + pr] = fast_div(E, d12 + Lm[2 * nS + k3s + kk]);
          }
          if (nz3) *b3p += b3;
        }
      };
      auto dead = [&](int k1, int k2) {
        const int pr = k2 * nS + k1;
        const float a3 = rg.pa[2] ? P2[k2 * ld + k1] : 0.0f;
        float* b3p = B3 + tc::coff(k1, k2, np);
        (void)pr;
        {
          float b3 = 0.0f;
          for (int kk = 0; kk < tn; ++kk) {
            const int k3 = k3s + kk;
            if (k3 - lo3 >= nz3) break;
            b3 += fast_div(s3sq[k3], lam + Lm[k1] + Lm[nS + k2] + Lm[2 * nS + k3]);
          }
          *b3p += a3 * b3;
        }
      };
      for_pairs(sg_live1, live);
      for_pairs(sg_live2, live);
      for_pairs(sg_dead, dead);
      __syncthreads();
      const int nb1 = rg.pa[0] ? tn * w2 : 0, nb2 = rg.pa[1] ? tn * w1 : 0;
      for (int o = tid; o < nb1 + nb2; o += blockDim.x) {
        const bool first = o < nb1;
        const int wx = first ? w2 : w1;
        int rr = first ? o : o - nb1, kk = 0;
        while (rr >= wx) {  // rr / wx < tn <= slab depth: subtract instead of dividing
          rr -= wx;
          ++kk;
        }
        const int kx = (first ? lo2 : lo1) + rr;
        const float* vs = V + kk * n2;
        float s = 0.0f, s_1 = 0.0f, s_2 = 0.0f, s_3 = 0.0f;
        if (first) {
          const float* v = vs + kx * nS + lo1;
          const float* sv = s1 + lo1;
          int k = 0;
          for (; k + 3 < nz1; k += 4) {
            s += sv[k] * v[k];
            s_1 += sv[k + 1] * v[k + 1];
            s_2 += sv[k + 2] * v[k + 2];
            s_3 += sv[k + 3] * v[k + 3];
          }
          for (; k < nz1; ++k) s += sv[k] * v[k];
          R1[tc::coff(kx, k3s + kk, np)] = (s + s_1) + (s_2 + s_3);
        } else {
          const float* v = vs + kx + lo2 * nS;
          const float* sv = s2 + lo2;
          int k = 0;
          for (; k + 3 < nz2; k += 4) {
            s += sv[k] * v[k * nS];
            s_1 += sv[k + 1] * v[(k + 1) * nS];
            s_2 += sv[k + 2] * v[(k + 2) * nS];
            s_3 += sv[k + 3] * v[(k + 3) * nS];
          }
          for (; k < nz2; ++k) s += sv[k] * v[k * nS];
          R1[tc::coff(np + kx, k3s + kk, np)] = (s + s_1) + (s_2 + s_3);
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < 3 * tb; i += blockDim.x) R1[i] = tc::to_tf32(R1[i]);
    // 5. backward, slow axis: O = N(S_b) B^T
    if (!round([&] {
          tc_product(tmem, 0, Tb + 2 * tb, R1, 2 * np, np);
          tc_product(tmem, 2 * np, Tb + 1 * tb, R1 + 2 * tb, np, np);
        }))
      break;
    readout(0, 3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np;
      float* a = R1 + dd * tb;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 w4 = make_float4(tc::to_tf32(v[q]), tc::to_tf32(v[q + 1]), tc::to_tf32(v[q + 2]),
                                      tc::to_tf32(v[q + 3]));
        *reinterpret_cast<float4*>(a + tc::coff(row, k0 + q, np)) = w4;
      }
    });
    // 6. backward, fast axis: Y_dd = O_dd N(S_a)
    if (!round([&] {
          tc_product(tmem, 0, R1, Tb + 1 * tb, np, np);
          tc_product(tmem, np, R1 + tb, Tb, np, np);
          tc_product(tmem, 2 * np, R1 + 2 * tb, Tb, np, np);
        }))
      break;
    // 7. weights, multiplicity and mask -> per-star output planes
    float* ob = Ob + st * 3 * (int64_t)n2;
    readout(0, 3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np, jb = row;
      if (jb >= nS) return;
      const int ax_a = ax_fast(dd), ax_b = ax_slow(dd);
      const int obb = jb - m;
      const bool rowact = Ac[dd * nS + m] && Ac[ax_b * nS + jb];
      for (int q = 0; q < 16; ++q) {
        const int ja = k0 + q;
        if (ja >= nS) break;
        const int oa = ja - m;
        const bool active = rowact && Ac[ax_a * nS + ja];
        const float wgt = t.w1d[oa < 0 ? -oa : oa] * t.w1d[obb < 0 ? -obb : obb] * rcp_mult[(oa == 0) + (obb == 0)];
        ob[dd * n2 + jb * nS + ja] = active ? wgt * v[q] : 0.0f;
      }
    });
    }  // !alias
    // next star
    if (counter) {
      __syncthreads();
      if (tid == 0) s_next = atomicAdd(&counter[0], 1) + (int)gridDim.x;
      __syncthreads();
      st = s_next;
    } else {
      st += gridDim.x;
    }
  }
  if (s_abort) tc::mbar_wait(&s_mbar, phase ^ 1u, kTcWaitCycles);  // products still in flight
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
  if (counter) {
    if (tid == 0) {
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

}  // namespace

LaunchCfg plan_star_tc(const Geo& G, int nsm) {
  LaunchCfg c;
  // np <= 64: the stacked products fit N <= 128 and M = 128; below n_S = 31 the
  // CUDA-core kernel is as fast (measured: p = 8 slower on the tensor cores)
  if (G.nS > 64 || G.nS < 31) return c;
  c.smem = tc_smem_floats(G.nS) * sizeof(float);
  if (c.smem > 200 * 1024) return c;
  c.block = 512;
  c.wide = 1;
  c.ws = WsPlan{};
  c.grid = (int)(G.nstar < nsm ? G.nstar : nsm);
  if (c.grid < 1) c.grid = 1;
  c.ok = true;
  return c;
}

void launch_star_tc(const Geo& G, const Tabs<float>& t, const float* r, float* Ob, const LaunchCfg& c, int* counter,
                    int* err, long long wait_budget, cudaStream_t st) {
  if (G.nstar == 0 || !c.ok) return;
  switch (G.p) {
    case 16: k_star_tc<16><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
    case 32: k_star_tc<32><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
    default: k_star_tc<0><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
  }
}

int set_star_tc_smem_limits() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_star_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  bad |= cudaFuncSetAttribute(k_star_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return bad;
}

}  // namespace semmg
