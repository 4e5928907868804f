// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  The GB300 runs
// FP32 at 63 times its FP64 rate, so the operator kernels instantiated with
// this type evaluate a residual to about 1e-14 relative accuracy on the FP32
// pipes, where FP64 would occupy the narrow FP64 pipe.
//
// The building blocks are the error-free transformations of Knuth (TwoSum:
// s + e = a + b exactly) and of the fused multiply-add (TwoProd: p + e = a b
// exactly, e = fma(a, b, -p)), combined as in Dekker's double-length
// arithmetic.  Every step uses the _rn intrinsics so the compiler cannot fuse
// or reassociate the roundings the error terms depend on.
#pragma once
#include <cuda_runtime.h>

namespace semmg {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr ff(float v) : hi(v), lo(0.0f) {}
  // nearest FP32 of v, then the nearest FP32 of the remainder (exact in FP64)
  __host__ __device__ ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth's TwoSum, no ordering assumption)
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// hi + lo = a + b exactly for |a| >= |b| (or a = 0)
__device__ __forceinline__ ff ff_fast_norm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// a + b (the sum of the high words exactly, the low words added once)
__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  ff_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_fast_norm(s, e);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

// a b (the product of the high words exactly, the cross terms once)
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_norm(p, e);
}

// acc + a b in one step: the product's error term joins the sum's
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  ff_two_sum(acc.hi, p, s, t);
  t = __fadd_rn(t, __fadd_rn(e, acc.lo));
  return ff_fast_norm(s, t);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

// c + a b in the kernels' multiply-add loops: one fused step for float-float;
// for FP32 and FP64 the expression the compiler contracts into one FMA, as
// `c += a * b` is
template <typename T>
__device__ __forceinline__ T madd(T a, T b, T c) { return c + a * b; }
__device__ __forceinline__ ff madd(ff a, ff b, ff c) { return ff_fma(a, b, c); }

// Sums of products in the kernels' long multiply-add chains: for float-float the
// running sum keeps an exact high word (TwoSum) and gathers every rounding error
// (the sums' and the products') in one FP32 word, normalised once at the end
// (the compensated dot product of Ogita, Rump and Oishi); for FP32 and FP64 a
// plain accumulator that the compiler contracts into FMAs.
template <typename T>
struct Acc {
  T v;
  __device__ __forceinline__ static Acc zero() { return Acc{(T)0}; }
  __device__ __forceinline__ void add(T a, T b) { v = v + a * b; }
  __device__ __forceinline__ T value() const { return v; }
};

template <>
struct Acc<ff> {
  float s, c;
  __device__ __forceinline__ static Acc zero() { return Acc{0.0f, 0.0f}; }
  __device__ __forceinline__ void add(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float t;
    ff_two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
  __device__ __forceinline__ ff value() const {
    float h, l;
    ff_two_sum(s, c, h, l);
    return ff(h, l);
  }
};

// 1/d by the hardware's approximate reciprocal (PTX rcp.approx.ftz.f32, about one ulp),
// for the FP32 eigenvalue sums D = lam + sum_d (4/h_d^2) Lam[k_d] > 0 of the FP32 kernels,
// which lie in the normal range where no special case applies
__device__ __forceinline__ float rcp_approx(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// 1 / d: the FP32 reciprocal refined by one Newton step in float-float,
// y + y (1 - d y), which doubles its correct bits
__device__ __forceinline__ ff ff_recip(ff d) {
  const ff y(__frcp_rn(d.hi), 0.0f);
  const ff r = ff(1.0f) - d * y;
  return ff_fma(y, r, y);
}
#endif

}  // namespace semmg
