// Star smoother with the in-plane 1D transforms on the 5th-generation tensor
// cores (tcgen05, FP32 accumulators in tensor memory), TF32 or BF16 operands;
// the eigenspace step (expansion along the normals, 1/D, contractions back)
// stays on the FP32 cores.  Same mathematics as k_star (Algorithm 1 inside
// Algorithm 2, Sec. 3.2); used by the tensor-core mixed forms for
// 31 <= n_S = 2p-1 <= 95 (16 <= p <= 48).
//
// A plane transform S_b^T X S_a is two dense products per plane, each run as
// D[M=128][N] += A[M][K] B[N][K] (K-major operands in shared memory, core
// matrices of 8 rows x 16 bytes, no swizzle) with K = N = NP = n_S rounded up
// to 16; rows NP..127 of every product are padding (they read whatever shared
// memory follows the A operand; their outputs are never read):
//   forward, slow axis:  W  = T(S_b) . P^T     (planes 0 and 1 share the x3
//                                              tables and are stacked along N)
//   forward, fast axis:  Z  = W . T(S_a)
//   backward, slow axis: O  = N(S_b) . B^T     (B: eigenspace result; one
//                                              plane at a time)
//   backward, fast axis: Y  = O . N(S_a)
// with T(S)[e][j] = S[j][e] and N(S)[j][e] = S[j][e] prepared at setup in the
// operand type.
//
// Shared memory (bytes, regions in this order): X, the three planes in turn as
// gathered operands, slow-axis results, FP32 eigenspace planes [dd][row][LD]
// and the eigenspace results B written in place; T0 and T1, two table slots;
// Y, one plane's B operand for the backward slow-axis product, or the partial
// sums of the x2 contraction during the eigenspace step; then Lam_d and the
// vertex rows s_d.  The allocation extends at least 128 operand rows past the
// start of every A operand (the three planes in X and the two table slots),
// so the padding rows of every product stay inside it.
//
// The eigenspace step holds V in registers: warp w owns the k2 rows
// lo2 + w + 16 i, its lanes the k1 columns lo1 + lane + 32 j.  Per k3 it forms
// E = s1 P0 + s2 P1 + s3 P2 and V = E / D for its (k2, k1) points, and reduces
// B1[k3][k2] = sum_k1 s1 V over its lanes (shuffle tree), keeps the partial
// B2[k3][k1] = sum over its k2 of s2 V and accumulates B3[k2][k1] = sum_k3 s3 V
// in registers.  The B2 partials of the 16 warps are summed in warp order
// after every block of kTcKB k3-planes.  Every sum runs in a fixed order, so
// results are bitwise reproducible.
#pragma once
#include <cstdint>

#include "semmg_internal.h"

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

// instruction descriptors, FP32 accumulator, A and B K-major: kind::tf32 with
// TF32 operands (format 2), kind::f16 with BF16 operands (format 1)
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
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

// One-dimensional bulk copy (TMA) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on mbar's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// arrive on mbar expecting `bytes` of transactions in the current phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
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

// a finite float rounded to BF16 (7 stored mantissa bits), nearest-even: the bit pattern
__device__ __forceinline__ uint16_t to_bf16(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

}  // namespace tc

// Operand types of the tensor-core star kernel.  E: elements per 16-byte core
// matrix row.
struct TcTf32 {
  using S = float;
  static constexpr int E = 4;
  __device__ static S cvt(float x) { return tc::to_tf32(x); }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_tf32(d, a, b, id, acc);
  }
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) { return tc::idesc_tf32(M, N); }
  __device__ static const S* tabT(const Tabs<float>& t, int d) { return t.tcT[d]; }
  __device__ static const S* tabN(const Tabs<float>& t, int d) { return t.tcN[d]; }
};

struct TcBf16 {
  using S = uint16_t;
  static constexpr int E = 8;
  __device__ static S cvt(float x) { return tc::to_bf16(x); }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    tc::mma_bf16(d, a, b, id, acc);
  }
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) { return tc::idesc_bf16(M, N); }
  __device__ static const S* tabT(const Tabs<float>& t, int d) { return t.bfT[d]; }
  __device__ static const S* tabN(const Tabs<float>& t, int d) { return t.bfN[d]; }
};

// element offset of (row, k) in a K-major operand with K = np columns
template <int E>
__host__ __device__ __forceinline__ int tc_opoff(int row, int k, int np) {
  return ((row >> 3) * (np / E) + k / E) * (8 * E) + (row & 7) * E + (k % E);
}

namespace {

// bound of the wait for products still in flight after an abort (about 2 s at
// 2 GHz); the completion waits of the normal rounds take the caller's budget
constexpr long long kTcWaitCycles = 4000000000LL;
constexpr int kTcWarps = 16;  // 512 threads
constexpr int kTcKB = 4;      // k3-planes per block of the x2-contraction sums
#ifndef SEMMG_TC_MIN_STAR
#define SEMMG_TC_MIN_STAR 31
#endif
constexpr int kTcMinStar = SEMMG_TC_MIN_STAR;  // smallest n_S on the tensor cores

__host__ __device__ __forceinline__ int tc_np(int nS) { return (nS + 15) / 16 * 16; }
__host__ __device__ __forceinline__ size_t tc_al(size_t b) { return (b + 127) & ~size_t(127); }

// byte offsets of the shared-memory regions (see the file comment)
struct TcLayout {
  int np, ld;
  size_t x, t0, t1, y, lm, sv, wt, total;
};

__host__ __device__ __forceinline__ TcLayout tc_layout(int nS, int esize) {
  TcLayout L;
  L.np = tc_np(nS);
  L.ld = L.np + 4;
  const size_t tb = (size_t)L.np * L.np * esize;
  const size_t xb = (size_t)3 * L.np * L.ld * 4 > 3 * tb ? (size_t)3 * L.np * L.ld * 4 : 3 * tb;
  const size_t yb = (size_t)kTcWarps * kTcKB * L.np * 4 > tb ? (size_t)kTcWarps * kTcKB * L.np * 4 : tb;
  L.x = 0;
  L.t0 = tc_al(xb);
  L.t1 = L.t0 + tc_al(tb);
  L.y = L.t1 + tc_al(tb);
  L.lm = L.y + tc_al(yb);
  L.sv = L.lm + tc_al((size_t)3 * nS * 4);
  L.wt = L.sv + tc_al((size_t)3 * nS * 4);
  L.total = L.wt + tc_al((size_t)(nS + 1) / 2 * 4);
  // an M = 128 product reads 128 operand rows from the start of its A operand (rows np..127 are
  // padding): the allocation reaches 128 rows past the last A operand, the table in slot T1
  const size_t a_end = L.t1 + (size_t)128 * L.np * esize;
  if (L.total < a_end) L.total = a_end;
  return L;
}

// TMEM columns [col, col + N) = A (M = 128 rows, K = np) B^T (N rows, K = np), whole K extent
template <typename OP>
__device__ __forceinline__ void tc_product(uint32_t tmem, int col, const typename OP::S* A,
                                           const typename OP::S* B, int N, int np) {
  constexpr int esz = (int)sizeof(typename OP::S);
  const uint32_t sbo = (uint32_t)(np / OP::E) * 128;  // bytes per 8-row group
  const uint32_t idesc = OP::idesc(128, N);
  const unsigned char* a = reinterpret_cast<const unsigned char*>(A);
  const unsigned char* b = reinterpret_cast<const unsigned char*>(B);
  const int steps = np * esz / 32;  // 32 bytes of K per instruction
  for (int s = 0; s < steps; ++s)
    OP::mma(tmem + col, tc::smem_desc(a + 256 * s, 128, sbo), tc::smem_desc(b + 256 * s, 128, sbo), idesc, s > 0);
}

// 16 consecutive K entries k0..k0+15 of operand row `row` (k0 a multiple of 16), rounded to the operand type
template <typename OP>
__device__ __forceinline__ void tc_store16(typename OP::S* dst, int row, int k0, const float* v, int np) {
  constexpr int E = OP::E;
  union Pack {
    uint4 u;
    typename OP::S s[E];
  };
#pragma unroll
  for (int g = 0; g < 16; g += E) {
    Pack w;
#pragma unroll
    for (int e = 0; e < E; ++e) w.s[e] = OP::cvt(v[g + e]);
    *reinterpret_cast<uint4*>(dst + tc_opoff<E>(row, k0 + g, np)) = w.u;
  }
}

__device__ __forceinline__ int tc_ax_fast(int dd) { return dd == 0 ? 1 : 0; }
__device__ __forceinline__ int tc_ax_slow(int dd) { return dd == 2 ? 1 : 2; }

struct TcRanges {
  int lo[3], hi[3], pa[3];
};

// Sums over the 32 lanes of R values per lane (R a power of two, at most 8), all at
// once: R - 1 shuffles halve the values each lane holds while doubling the lanes
// they sum, then a butterfly over the remaining lane bits.  Returns the total of
// value rs_index<R>(lane) (every lane of a group returns the same bits: a + b is
// exact-commutative).  A fixed order of additions: bitwise reproducible.
template <int R>
__device__ __forceinline__ float rs_reduce(float* v, int lane) {
  int off = 16;
#pragma unroll
  for (int n = R; n > 1; n >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      const float send = hi ? v[k] : v[k + n / 2];
      const float keep = hi ? v[k + n / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float t = v[0];
#pragma unroll
  for (; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

template <int R>
__device__ __forceinline__ int rs_index(int lane) {
  int idx = 0, off = 16;
#pragma unroll
  for (int n = R; n > 1; n >>= 1, off >>= 1)
    if (lane & off) idx += n / 2;
  return idx;
}

__host__ __device__ constexpr int tc_pow2(int n) { return n <= 1 ? 1 : (n <= 2 ? 2 : (n <= 4 ? 4 : 8)); }

// The eigenspace step of one star (see the file comment) on register tiles of NI rows (k2)
// per warp and NJ 32-lane columns (k1): B1, B2, B3 replace P0, P1, P2 in X.  Rows and columns
// outside the active ranges carry zeros (s = 0, P = 0, D = 1), so the loops have no branches;
// only the stores are guarded.  The caller picks the smallest tiles that cover the ranges.
template <int NI, int NJ>
__device__ __forceinline__ void tc_eigen(float* X, int np, int ld, int nS, float lam, const float* Lm, const float* Sv,
                                         float* Yf, const TcRanges& rg, int warp, int lane, int tid) {
  const int lo1 = rg.lo[0], hi1 = rg.hi[0], lo2 = rg.lo[1], hi2 = rg.hi[1], lo3 = rg.lo[2], hi3 = rg.hi[2];
  float* P0 = X;
  float* P1 = X + np * ld;
  float* P2 = X + 2 * np * ld;
  const float* s1 = Sv;
  const float* s2 = Sv + nS;
  const float* s3 = Sv + 2 * nS;
  constexpr int R = tc_pow2(NI);
  int k1v[NJ], k2v[NI];
  bool ok1[NJ], ok2[NI];
  float s1r[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    k1v[j] = lo1 + lane + 32 * j;
    ok1[j] = k1v[j] < hi1;
    s1r[j] = ok1[j] ? s1[k1v[j]] : 0.0f;
  }
  float p2r[NI][NJ], b3[NI][NJ], d12[NI][NJ], s2r[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    k2v[i] = lo2 + warp + kTcWarps * i;
    ok2[i] = k2v[i] < hi2;
    s2r[i] = ok2[i] ? s2[k2v[i]] : 0.0f;
    if (!ok2[i]) k2v[i] = lo2;  // a valid row to read from; its contributions are zero or unused
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const bool ok = ok2[i] && ok1[j];
      p2r[i][j] = ok ? P2[k2v[i] * ld + k1v[j]] : 0.0f;
      d12[i][j] = ok ? lam + Lm[k1v[j]] + Lm[nS + k2v[i]] : 1.0f;
      b3[i][j] = 0.0f;
    }
  }
  const int me = rs_index<R>(lane);  // the row whose B1 this lane receives
  const bool wr1 = (lane & (32 / R - 1)) == 0 && me < NI;
  const int w1 = hi1 - lo1;
  for (int k3b = lo3; k3b < hi3; k3b += kTcKB) {
    const int nb = hi3 - k3b < kTcKB ? hi3 - k3b : kTcKB;
    for (int kb = 0; kb < nb; ++kb) {
      const int k3 = k3b + kb;
      const float s3k = s3[k3], l3 = Lm[2 * nS + k3];
      float p1r[NJ], b2[NJ], p0[NI], b1[R];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        p1r[j] = ok1[j] ? P1[k3 * ld + k1v[j]] : 0.0f;
        b2[j] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) p0[i] = P0[k3 * ld + k2v[i]];
#pragma unroll
      for (int i = 0; i < R; ++i) b1[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          float e = s1r[j] * p0[i];
          e += s2r[i] * p1r[j];
          e += s3k * p2r[i][j];
          const float v = e * rcp_approx(d12[i][j] + l3);
          b1[i] += s1r[j] * v;
          b2[j] += s2r[i] * v;
          b3[i][j] += s3k * v;
        }
      }
      const float t1 = rs_reduce<R>(b1, lane);
      // this warp alone reads P0[k3][k2] of its rows (all read above): B1 takes their place
#pragma unroll
      for (int i = 0; i < NI; ++i)
        if (wr1 && me == i && ok2[i]) P0[k3 * ld + k2v[i]] = rg.pa[0] ? t1 : 0.0f;
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        if (ok1[j]) Yf[(warp * kTcKB + kb) * np + k1v[j]] = b2[j];
    }
    __syncthreads();
    // B2 rows of the block: the 16 warps' partial sums in warp order, in place of P1's rows
    for (int o = tid; o < nb * w1; o += blockDim.x) {
      const int kb = o / w1, k1 = lo1 + (o - kb * w1);
      float sum = 0.0f;
#pragma unroll
      for (int w = 0; w < kTcWarps; ++w) sum += Yf[(w * kTcKB + kb) * np + k1];
      P1[(k3b + kb) * ld + k1] = rg.pa[1] ? sum : 0.0f;
    }
    __syncthreads();
  }
  // B3 in place of P2 (the rows this warp owns and alone has read)
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    if (ok2[i]) {
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        if (ok1[j]) P2[k2v[i] * ld + k1v[j]] = rg.pa[2] ? b3[i][j] : 0.0f;
    }
  }
}

template <typename OP, int PC>
__global__ void __launch_bounds__(512, 1) k_star_tc(Geo G, Tabs<float> t, const float* __restrict__ r,
                                                     float* __restrict__ Ob, int* counter, int* err,
                                                     long long wait_budget) {
  using S = typename OP::S;
  constexpr int E = OP::E;
  // compile-time bounds of the eigenspace registers: k1 chunks of 32 lanes, k2 rows per warp
  constexpr int NJ = PC ? (2 * PC - 1 + 31) / 32 : 3;
  constexpr int NI = PC ? (2 * PC - 1 + kTcWarps - 1) / kTcWarps : 6;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t s_mbar;
  __shared__ uint64_t s_tbar;  // table copies (TMA)
  __shared__ uint32_t s_tmem;
  __shared__ int s_next, s_abort;
  __shared__ TcRanges s_rg;
  __shared__ int Ac[3 * (2 * SEMMG_MAX_DEGREE - 1)];
  const int p = PC ? PC : G.p, m = p - 1, nS = 2 * p - 1, n2 = nS * nS;
  const TcLayout lay = tc_layout(nS, (int)sizeof(S));
  const int np = lay.np, ld = lay.ld, tb = np * np;
  float* X = reinterpret_cast<float*>(smem_raw + lay.x);  // FP32 planes [dd][row][ld]
  S* Xo = reinterpret_cast<S*>(smem_raw + lay.x);         // operands, tb elements per plane
  S* T0 = reinterpret_cast<S*>(smem_raw + lay.t0);
  S* T1 = reinterpret_cast<S*>(smem_raw + lay.t1);
  S* Yo = reinterpret_cast<S*>(smem_raw + lay.y);
  float* Yf = reinterpret_cast<float*>(smem_raw + lay.y);  // x2-contraction partials [warp][kb][np]
  float* Lm = reinterpret_cast<float*>(smem_raw + lay.lm);
  float* Sv = reinterpret_cast<float*>(smem_raw + lay.sv);  // vertex rows s_d
  float* Wt = reinterpret_cast<float*>(smem_raw + lay.wt);  // smoother weights at offsets 0..m
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float lam = (float)G.lam;
  // 1 / (number of planes a node lies on) for 0, 1 or 2 zero in-plane offsets
  auto rcp_mult = [](int zeros) { return zeros == 0 ? 1.0f : (zeros == 1 ? 0.5f : 1.0f / 3.0f); };
  const uint32_t ncols = 3 * np <= 256 ? 256u : 512u;
  if (tid == 0) {
    tc::mbar_init(&s_mbar, 1);
    tc::mbar_init(&s_tbar, 1);
    s_abort = 0;
  }
  for (int i = tid; i <= m; i += blockDim.x) Wt[i] = t.w1d[i];
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  uint32_t phase = 0, tphase = 0;
  bool tpending = false;  // table copies in flight (issued, not yet awaited)
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
  // TMEM lanes [0, np) x columns [0, ncol): 16-column chunks spread over the four warps of
  // each lane quadrant; f(row, col, v[16])
  auto readout = [&](int ncol, auto f) {
    const int q = warp & 3;
    if (q * 32 < np) {
      const int nchunk = ncol / 16, wq = warp >> 2;
      for (int ch = wq; ch < nchunk; ch += kTcWarps / 4) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * ch), v);
        const int row = q * 32 + lane;
        if (row < np) f(row, 16 * ch, v);
      }
    }
  };
  // Table copies by TMA: thread 0 issues one bulk copy per table on s_tbar (the slot's
  // previous products have completed: every caller comes after the round that read it);
  // tables_ready() waits for them, bounded like the product waits.
  const uint32_t tbytes = (uint32_t)(tb * sizeof(S));
  auto load_tables = [&](S* d0, const S* s0, int c0, S* d1, const S* s1, int c1) {
    if (tid == 0) {
      tc::mbar_expect_tx(&s_tbar, tbytes * (d1 ? 2u : 1u));
      tc::bulk_g2s(d0, s0 + (int64_t)c0 * tb, tbytes, &s_tbar);
      if (d1) tc::bulk_g2s(d1, s1 + (int64_t)c1 * tb, tbytes, &s_tbar);
    }
    tpending = true;
  };
  // A thread whose wait ran out keeps its copy marked in flight (drained at exit); the
  // outcome is made uniform over the CTA before anyone issues products on the tables.
  auto tables_ready = [&]() -> bool {
    const bool ok = tc::mbar_wait(&s_tbar, tphase, wait_budget);
    if (ok) {
      tphase ^= 1u;
      tpending = false;
    } else {
      s_abort = 1;
      if (lane == 0) atomicExch(err, 1);
    }
    __syncthreads();
    return s_abort == 0;
  };
  // position in the star order (most work first when the level has an order table)
  int64_t it = blockIdx.x;
  while (it < G.nstar) {
    const int64_t st = t.order ? (int64_t)t.order[it] : it;
    const int c[3] = {(int)(st % G.nv1), (int)((st / G.nv1) % G.nv2), (int)(st / ((int64_t)G.nv1 * G.nv2))};
    // the last vertex plane of a periodic axis repeats plane 0: its stars are never read
    const bool alias = (G.per[0] && c[0] == G.n1) || (G.per[1] && c[1] == G.n2) || (G.per[2] && c[2] == G.n3);
    if (!alias) {
    __syncthreads();
    for (int d = 0; d < 3; ++d)
      for (int i = tid; i < nS; i += blockDim.x) {
        Lm[d * nS + i] = t.starLam[d][(int64_t)c[d] * nS + i];
        Ac[d * nS + i] = t.act[d][(int64_t)c[d] * nS + i];
        Sv[d * nS + i] = t.starS[d][(int64_t)c[d] * n2 + m * nS + i];
      }
    // forward slow-axis tables: x3 for planes 0 and 1, x2 for plane 2 (arriving during the gather)
    load_tables(T0, OP::tabT(t, 2), t.starCls[2][c[2]], T1, OP::tabT(t, 1), t.starCls[1][c[1]]);
    __syncthreads();
    if (tid < 3) {
      const int d = tid;
      int lo = 0, hi = nS;
      while (lo < nS && !Ac[d * nS + lo]) ++lo;
      while (hi > lo && !Ac[d * nS + hi - 1]) --hi;
      s_rg.lo[d] = lo;
      s_rg.hi[d] = hi;
      s_rg.pa[d] = Ac[d * nS + m];
    }
    // 1. the planes divided by the multiplicity, as B operands P_dd^T: row n = ja, K index jb
    //    (zero outside the star and in the padding).  The operands are filled in their memory
    //    order (a warp writes whole core matrices: no bank conflicts), eight independent loads in
    //    flight per thread.
    for (int base = tid; base < 3 * tb; base += 8 * (int)blockDim.x) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * (int)blockDim.x;
        v[u] = 0.0f;
        if (idx < 3 * tb) {
          const int dd = idx / tb, w = idx - dd * tb, cm = w / (8 * E), e = w - cm * (8 * E);
          const int jap = (cm / (np / E)) * 8 + e / E, jbp = (cm % (np / E)) * E + e % E;
          if (jap < nS && jbp < nS) {
            const int ja = jap - m, jb = jbp - m;
            const int ax_a = tc_ax_fast(dd), ax_b = tc_ax_slow(dd);
            if (Ac[dd * nS + m] && Ac[ax_a * nS + jap] && Ac[ax_b * nS + jbp])
              v[u] = __ldg(r + star_plane_slot(G, dd, c[0], c[1], c[2], ja, jb)) * rcp_mult((ja == 0) + (jb == 0));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * (int)blockDim.x;
        if (idx < 3 * tb) Xo[idx] = OP::cvt(v[u]);
      }
    }
    // 2. forward, slow axis: W = T(S_b) P^T
    if (!tables_ready()) break;
    if (!round([&] {
          tc_product<OP>(tmem, 0, T0, Xo, 2 * np, np);
          tc_product<OP>(tmem, 2 * np, T1, Xo + 2 * tb, np, np);
        }))
      break;
    // W (lanes k_b, columns dd np + ja) -> A operands (row k_b, K index ja); x1 tables into slot 0
    readout(3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np;
      tc_store16<OP>(Xo + dd * tb, row, col - dd * np, v, np);
    });
    load_tables(T0, OP::tabT(t, 0), t.starCls[0][c[0]], nullptr, nullptr, 0);
    // 3. forward, fast axis: Z_dd = W_dd T(S_a) (plane 0: x2 tables; planes 1, 2: x1 tables)
    if (!tables_ready()) break;
    if (!round([&] {
          tc_product<OP>(tmem, 0, Xo, T1, np, np);
          tc_product<OP>(tmem, np, Xo + tb, T0, np, np);
          tc_product<OP>(tmem, 2 * np, Xo + 2 * tb, T0, np, np);
        }))
      break;
    readout(3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np;
      float* dst = X + (dd * np + row) * ld + k0;
#pragma unroll
      for (int q = 0; q < 16; q += 4) *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    });
    // backward slow-axis tables (x3, x2) arrive while the eigenspace step runs
    load_tables(T0, OP::tabN(t, 2), t.starCls[2][c[2]], T1, OP::tabN(t, 1), t.starCls[1][c[1]]);
    __syncthreads();
    // 4. eigenspace step (see the file comment): B1, B2, B3 replace P0, P1, P2 in X, built for
    //    the rows and columns this star's active ranges need (half or all of the register tiles)
    {
      const TcRanges rg = s_rg;
      const bool fi = rg.hi[1] - rg.lo[1] > kTcWarps * ((NI + 1) / 2);  // k2 rows beyond the half tile
      const bool fj = rg.hi[0] - rg.lo[0] > 32 * ((NJ + 1) / 2);         // k1 columns beyond the half tile
      if (fi && fj)
        tc_eigen<NI, NJ>(X, np, ld, nS, lam, Lm, Sv, Yf, rg, warp, lane, tid);
      else if (fi)
        tc_eigen<NI, (NJ + 1) / 2>(X, np, ld, nS, lam, Lm, Sv, Yf, rg, warp, lane, tid);
      else if (fj)
        tc_eigen<(NI + 1) / 2, NJ>(X, np, ld, nS, lam, Lm, Sv, Yf, rg, warp, lane, tid);
      else
        tc_eigen<(NI + 1) / 2, (NJ + 1) / 2>(X, np, ld, nS, lam, Lm, Sv, Yf, rg, warp, lane, tid);
    }
    // 5. backward, slow axis, one plane at a time: O_dd = N(S_b) B_dd^T with B_dd (rows k_b,
    //    columns k_a in X) staged in Y as the B operand (row n = k_a, K index k_b)
    bool aborted = !tables_ready();
    for (int dd = 0; dd < 3 && !aborted; ++dd) {
      if (dd > 0) __syncthreads();  // the previous round's operand is consumed (round() waited)
      const float* B = X + dd * np * ld;
      for (int idx = tid; idx < tb; idx += blockDim.x) {  // operand memory order: whole core matrices
        const int cm = idx / (8 * E), e = idx - cm * (8 * E);
        const int ka = (cm / (np / E)) * 8 + e / E, kb = (cm % (np / E)) * E + e % E;
        Yo[idx] = OP::cvt(B[kb * ld + ka]);
      }
      aborted = !round([&] { tc_product<OP>(tmem, dd * np, dd == 2 ? T1 : T0, Yo, np, np); });
    }
    if (aborted) break;
    // O (lanes j_b, columns dd np + k_a) -> A operands (row j_b, K index k_a) in X, whose B planes
    // are consumed; the x1 tables replace the x3 ones (the x2 ones stay for plane 0)
    readout(3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np;
      tc_store16<OP>(Xo + dd * tb, row, col - dd * np, v, np);
    });
    load_tables(T0, OP::tabN(t, 0), t.starCls[0][c[0]], nullptr, nullptr, 0);
    // 6. backward, fast axis: Y_dd = O_dd N(S_a) (plane 0: x2 tables; planes 1, 2: x1 tables)
    if (!tables_ready()) break;
    if (!round([&] {
          tc_product<OP>(tmem, 0, Xo, T1, np, np);
          tc_product<OP>(tmem, np, Xo + tb, T0, np, np);
          tc_product<OP>(tmem, 2 * np, Xo + 2 * tb, T0, np, np);
        }))
      break;
    // 7. weights, multiplicity and mask -> X rows [dd][jb][ja] (the O operands there are
    //    consumed), then coalesced copies to the star's output planes
    readout(3 * np, [&](int row, int col, const float* v) {
      const int dd = col / np, k0 = col - dd * np, jb = row;
      const int ax_a = tc_ax_fast(dd), ax_b = tc_ax_slow(dd);
      const int obb = jb - m;
      const bool rowact = jb < nS && Ac[dd * nS + m] && Ac[ax_b * nS + jb];
      const float wb = rowact ? Wt[obb < 0 ? -obb : obb] : 0.0f;
      float w[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int ja = k0 + q, oa = ja - m;
        const bool active = rowact && ja < nS && Ac[ax_a * nS + ja];
        w[q] = active ? Wt[oa < 0 ? -oa : oa] * wb * rcp_mult((oa == 0) + (obb == 0)) * v[q] : 0.0f;
      }
      float* dst = X + (dd * np + row) * ld + k0;
#pragma unroll
      for (int q = 0; q < 16; q += 4) *reinterpret_cast<float4*>(dst + q) = make_float4(w[q], w[q + 1], w[q + 2], w[q + 3]);
    });
    __syncthreads();
    {
      float* ob = Ob + st * 3 * (int64_t)n2;
      for (int idx = tid; idx < 3 * n2; idx += blockDim.x) {
        const int dd = idx / n2, rr = idx - dd * n2, jb = rr / nS, ja = rr - jb * nS;
        ob[idx] = X[(dd * np + jb) * ld + ja];
      }
    }
    }  // !alias
    // next star
    if (counter) {
      __syncthreads();
      if (tid == 0) s_next = atomicAdd(&counter[0], 1) + (int)gridDim.x;
      __syncthreads();
      it = s_next;
    } else {
      it += gridDim.x;
    }
  }
  if (s_abort) tc::mbar_wait(&s_mbar, phase ^ 1u, kTcWaitCycles);  // products still in flight
  if (tpending) tc::mbar_wait(&s_tbar, tphase, kTcWaitCycles);      // table copies still in flight
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

// dynamic shared memory of the kernel, bytes; the launch also holds about 1.3 KB of static shared memory
size_t tc_smem_bytes(int nS, int bf16) { return tc_layout(nS, bf16 ? 2 : 4).total; }

constexpr size_t kTcSmemMax = 225 * 1024;  // the opt-in limit less the kernel's 2 KB of static shared memory

template <typename OP>
void launch_tc(const Geo& G, const Tabs<float>& t, const float* r, float* Ob, const LaunchCfg& c, int* counter,
               int* err, long long wait_budget, cudaStream_t st) {
  switch (G.p) {
    case 16: k_star_tc<OP, 16><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
    case 32: k_star_tc<OP, 32><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
    case 48: k_star_tc<OP, 48><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
    default: k_star_tc<OP, 0><<<c.grid, c.block, c.smem, st>>>(G, t, r, Ob, counter, err, wait_budget); break;
  }
}

template <typename OP>
int tc_attrs() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_star_tc<OP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
  bad |= cudaFuncSetAttribute(k_star_tc<OP, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
  bad |= cudaFuncSetAttribute(k_star_tc<OP, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
  bad |= cudaFuncSetAttribute(k_star_tc<OP, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
  return bad;
}

}  // namespace

LaunchCfg plan_star_tc(const Geo& G, int nsm, int bf16) {
  LaunchCfg c;
  // 31 <= n_S <= 95 (np <= 96: the stacked products fit N <= 256 and the tensor memory 512
  // columns); below n_S = 31 the CUDA-core kernel is as fast
  if (G.nS > 95 || G.nS < kTcMinStar) return c;
  c.smem = tc_smem_bytes(G.nS, bf16);
  if (c.smem > kTcSmemMax) return c;
  c.block = 32 * kTcWarps;
  c.wide = 1;
  c.bf16 = bf16 ? 1 : 0;
  c.ws = WsPlan{};
  c.grid = (int)(G.nstar < nsm ? G.nstar : nsm);
  if (c.grid < 1) c.grid = 1;
  c.ok = true;
  return c;
}

void launch_star_tc(const Geo& G, const Tabs<float>& t, const float* r, float* Ob, const LaunchCfg& c, int* counter,
                    int* err, long long wait_budget, cudaStream_t st) {
  if (G.nstar == 0 || !c.ok) return;
  if (c.bf16)
    launch_tc<TcBf16>(G, t, r, Ob, c, counter, err, wait_budget, st);
  else
    launch_tc<TcTf32>(G, t, r, Ob, c, counter, err, wait_budget, st);
}

int set_star_tc_smem_limits() { return tc_attrs<TcTf32>() | tc_attrs<TcBf16>(); }

}  // namespace semmg
