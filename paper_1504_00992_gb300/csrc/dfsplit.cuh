// Double-float (FP32 pair) arithmetic of the mixed-precision kernels and the
// double-float GEMMs (sm_103a): the split of a double without FP64
// arithmetic, TwoSum, products accumulated into a pair, renormalisation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tg {

// x -> hi + lo with integer and FP32 operations only (GB300 runs FP64
// arithmetic and double<->float conversions on its 1/64-rate FP64 pipe):
// hi = x truncated to 24 significant bits, lo = the remaining 29 mantissa
// bits rounded to FP32, so hi + lo = x to 2^-48 relative (lo may be an FP32
// subnormal).  |x| below 2^-126 flushes to zero; non-finite x gives a
// non-finite hi.
__device__ __forceinline__ void split_bits(double x, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  const int ef = e - 1023 + 127;  // FP32 biased exponent of hi
  if (e == 0x7FF || ef >= 255) {   // Inf / NaN / beyond FP32: non-finite hi
    hi = __uint_as_float(sign | 0x7F800000u | (unsigned int)(mant >> 29) | (mant ? 1u : 0u));
    lo = 0.f;
    return;
  }
  if (ef <= 0) {
    hi = __uint_as_float(sign);
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)(mant >> 29));
  // weight of mantissa bit 0: 2^(e - 1075) = 2^(e - 1011) * 2^-64, both factors normal FP32 numbers for e >= 897
  const float r = __uint2float_rn((unsigned int)(mant & 0x1FFFFFFFull));
  const float l = (r * __uint_as_float((unsigned int)(e - 1011 + 127) << 23)) * 5.421010862427522e-20f;  // 2^-64
  lo = sign ? -l : l;
}

// (s, e) with s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// acc += (xh, xl) (yh, yl)
__device__ __forceinline__ void dfx_dd(float& h, float& lo, float xh, float xl, float yh, float yl) {
  const float ph = xh * yh;
  const float pe = fmaf(xh, yh, -ph);
  const float pc = fmaf(xh, yl, xl * yh);
  float t, e;
  two_sum(h, ph, t, e);
  h = t;
  lo += (e + pe) + pc;
}
// acc += x (yh, yl), x a single float
__device__ __forceinline__ void dfx_sd(float& h, float& lo, float x, float yh, float yl) {
  const float ph = x * yh;
  const float pe = fmaf(x, yh, -ph);
  float t, e;
  two_sum(h, ph, t, e);
  h = t;
  lo += (e + pe) + x * yl;
}
__device__ __forceinline__ void fast2(float& h, float& lo) {
  const float s = h + lo;
  lo = lo - (s - h);
  h = s;
}

// Double-float scalars (value h + l, |l| <= ulp(h) / 2) with FP32
// arithmetic only: normalised sums and products by TwoSum and FMA splitting,
// square root and reciprocal as one Newton step from the correctly rounded
// FP32 operation (relative error ~2^-47).
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl dnorm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ dfl dadd(dfl a, dfl b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return dnorm(s, e + (a.l + b.l));
}
__device__ __forceinline__ dfl dmul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dnorm(p, e);
}
__device__ __forceinline__ dfl dmulf(dfl a, float b) {  // a * b, b a single float
  const float p = a.h * b;
  const float e = fmaf(a.h, b, -p);
  return dnorm(p, fmaf(a.l, b, e));
}
__device__ __forceinline__ dfl dneg(dfl a) { return {-a.h, -a.l}; }
// sqrt(a), a > 0: the correctly rounded FP32 root y and one Newton step,
// y + (a - y^2) / (2 y), the residual by FMA
__device__ __forceinline__ dfl dsqrt(dfl a) {
  const float y = sqrtf(a.h);
  const float r = fmaf(-y, y, a.h) + a.l;
  return dnorm(y, r / (2.0f * y));
}
// 1 / b: the correctly rounded FP32 reciprocal y and one Newton step,
// y + y (1 - b y)
__device__ __forceinline__ dfl drecip(dfl b) {
  const float y = 1.0f / b.h;
  const float r = fmaf(-b.h, y, 1.0f) - b.l * y;
  return dnorm(y, y * r);
}

}  // namespace tg
