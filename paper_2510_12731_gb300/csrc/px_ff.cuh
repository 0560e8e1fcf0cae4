// Double-FP32 ("float-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits.  Products use TwoProduct through the FMA (the exact error of
// fl(a*b) is fma(a, b, -fl(a*b))); sums use Knuth's TwoSum, so every accumulation keeps
// the rounding error of the FP32 addition.  GB300 runs FP32 at ~62x its FP64 rate,
// which makes this the fast route to FP64-class sums and products.
#pragma once
#include <cuda_runtime.h>

namespace px {
namespace ff {

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// (s, c) += (ah + al)(bh + bl): the exact product of the hi parts is split into
// fl(ah bh) + its error; the error, the two cross terms and the TwoSum error of the
// running sum go to the compensation c (the lo*lo term, < 2^-48 relative, is dropped).
// c is not renormalised here; call renorm() every few dozen steps.
__device__ __forceinline__ void mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) -> the normalised pair of the same value
__device__ __forceinline__ void renorm(float& s, float& c) {
  float t, e;
  fast_two_sum(s, c, t, e);
  s = t;
  c = e;
}

// (sh, sl) += (bh, bl), both double-FP32
__device__ __forceinline__ void add(float& sh, float& sl, float bh, float bl) {
  float t, e;
  two_sum(sh, bh, t, e);
  e = __fadd_rn(e, __fadd_rn(sl, bl));
  fast_two_sum(t, e, sh, sl);
}

__device__ __forceinline__ float2 split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double join(float h, float l) { return (double)h + (double)l; }
__device__ __forceinline__ double join(float2 v) { return (double)v.x + (double)v.y; }

}  // namespace ff
}  // namespace px
