// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 significand bits), computed with FP32 instructions only.  GB300 runs
// FP64 at 1/64 of its FP32 rate, so the passes that need more than FP32 accuracy
// (right-hand side, refinement residual, outputs) can use this type instead.
//
// Error-free transformations (Knuth's two-sum, Dekker's fast two-sum, the FMA
// two-product) as in the double-double literature (Dekker 1971; Hida, Li & Bailey
// 2001).  Additions use the cheaper "sloppy" form: its error is bounded by about
// 2^-44 (|a| + |b|), which is what the pair sums need (an absolute error small
// compared with the summed magnitudes).
#pragma once

#include <cuda_runtime.h>

namespace gbi {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // from a double constant (folded at compile time for literals)
  __host__ __device__ constexpr df(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ constexpr df(int i) : hi(float(i)), lo(0.f) {}
  __host__ __device__ explicit operator float() const { return hi; }
};

__host__ __device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  const float e = (a - (s - v)) + (b - v);
  return df(s, e);
}

__host__ __device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}

__host__ __device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = a * b;
  return df(p, fmaf(a, b, -p));
}

// Sums and fused products leave the result unnormalised (lo is not folded back into
// hi): the exact two-sum of the high parts keeps hi + lo accurate, lo only collects
// rounding errors far below hi, and every consumer (products, sums, the conversion to
// double) uses hi and lo separately -- 3 FP32 operations fewer per operation.
__host__ __device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df(s.hi, s.lo + (a.lo + b.lo));
}

__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ df& operator+=(df& a, df b) {
  a = a + b;
  return a;
}

// a * b + c: the product's rounding error terms are folded into the sum (12 FP32
// operations instead of 15 for a separate * and +)
__host__ __device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df s = df_two_sum(p, c.hi);
  return df(s.hi, s.lo + (e + c.lo));
}

__host__ __device__ __forceinline__ bool operator>(df a, df b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

__host__ __device__ __forceinline__ double df_to_double(df a) { return double(a.hi) + double(a.lo); }

// 1/sqrt(a): FP32 estimate, then one Newton step y + y (1 - a y^2) / 2 in double-float.
__host__ __device__ __forceinline__ df df_rsqrt(df a) {
#ifdef __CUDA_ARCH__
  const float y = rsqrtf(a.hi);
#else
  const float y = 1.0f / sqrtf(a.hi);
#endif
  const df yy = df_two_prod(y, y);
  const df r = df(1.0f, 0.0f) - a * yy;
  const df hy = df(0.5f * y, 0.0f);
  return df(y, 0.0f) + hy * r;
}

#ifdef __CUDACC__
__device__ __forceinline__ df df_shfl_xor(df v, int o) {
  return df(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}
#endif

}  // namespace gbi

// a * b + c in the arithmetic of T (fused where the type has a fused form); the
// generated pair-frame code chains its sums of products through this
__host__ __device__ __forceinline__ float gbi_fmac(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double gbi_fmac(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ gbi::df gbi_fmac(gbi::df a, gbi::df b, gbi::df c) { return gbi::df_fma(a, b, c); }
