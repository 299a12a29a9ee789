// Shared device helpers of the TEBD / RRSVD kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tg {

typedef double2 cplx;  // (re, im), interleaved like C99 double _Complex

__host__ __device__ __forceinline__ cplx cmk(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
// acc += a * b
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ double cabs2(cplx a) { return fma(a.x, a.x, a.y * a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Block-wide sum of one double; `red` is shared scratch of >= 32 doubles.
// Every thread of the block must call it; all get the result.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0) {
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: per round, with key (k0, k1),
//   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2   (128-bit products)
//   c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
// and the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u64x4 { uint64_t v[4]; };

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  u64x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// 64-bit word -> double in (0, 1): ((w >> 12) + 0.5) * 2^-52, exact.
__device__ __forceinline__ double u01(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 2.220446049250313080847263336181640625e-16;
}

// Complex standard Gaussian (Re, Im iid N(0,1)) for sketch element `idx`.
__device__ __forceinline__ cplx gauss_c(uint64_t idx, uint64_t bond, uint64_t sweep, uint64_t chain, uint64_t seed,
                                        uint64_t stream) {
  u64x4 w = philox4x64_10(idx, bond, sweep, chain, seed, stream);
  const double u1 = u01(w.v[0]), u2 = u01(w.v[1]);
  const double rho = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return cmk(rho * c, rho * s);
}

// Complex standard Gaussian of sketch element `idx` from the same Philox
// words as the FP64 path, by Box-Muller in FP32 (24-bit uniforms): the
// mixed form rounds Omega to TF32, and its refinement pass needs it to FP32.
__device__ __forceinline__ float2 gauss_c_f32(uint64_t idx, uint64_t bond, uint64_t sweep, uint64_t chain,
                                              uint64_t seed) {
  const u64x4 w = philox4x64_10(idx, bond, sweep, chain, seed, 0);
  const float u1 = ((float)(unsigned int)(w.v[0] >> 40) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
  const float u2 = ((float)(unsigned int)(w.v[1] >> 40) + 0.5f) * 5.9604644775390625e-8f;
  const float rho = sqrtf(-2.f * logf(u1));
  float sn, cs;
  sincospif(2.f * u2, &sn, &cs);
  return make_float2(rho * cs, rho * sn);
}

}  // namespace tg
