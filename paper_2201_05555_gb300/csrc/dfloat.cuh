// Double-float arithmetic: a value hi + lo (|lo| <= half an ulp of hi, two
// FP32 numbers) carries about 48 significant bits; its operations run on the
// FP32 pipes, which issue 64 times the FP64 rate of this part.  Shared by the
// small dense kernels (dense.cu) and the symmetric Jacobi (deim.cu).
#pragma once

namespace vpk {

struct DFv {
  float h, l;
};
__device__ __forceinline__ DFv dfv(float h, float l) { return DFv{h, l}; }
__device__ __forceinline__ DFv dfv_from(double x) {
  const float h = (float)x;
  return DFv{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dfv_to(DFv a) { return (double)a.h + (double)a.l; }
// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ DFv two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return DFv{s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly for |a| >= |b| (Dekker's FastTwoSum)
__device__ __forceinline__ DFv fast_two_sum(float a, float b) {
  const float s = a + b;
  return DFv{s, b - (s - a)};
}
__device__ __forceinline__ DFv dfv_add(DFv a, DFv b) {
  const DFv s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ DFv dfv_neg(DFv a) { return DFv{-a.h, -a.l}; }
__device__ __forceinline__ DFv dfv_mul(DFv a, DFv b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
}  // namespace vpk
