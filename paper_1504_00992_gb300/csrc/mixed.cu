// Mixed-precision RRSVD (sm_103a): Alg. 1 with its products on the tensor
// cores, then the FP64 projection and small SVD of Section IV.
//
//   Y0 = A Omega and power rounds 1..q-1  : TF32 tensor-core products (FP32
//                                           accumulation), FP32 Householder QR
//                                           (blocked when it fits in shared memory);
//   power round q (Y0 if q = 0)            : the refinement pass, 3xTF32 split
//                                           products (FP32-level accuracy);
//   last QR                                : FP32 blocked Householder and an
//                                           FP64-accurate re-orthonormalisation
//                                           (qr_blocked.cu; l <= 512);
//   B^H = A^H Q, U = Q J_k, V = Qb W_k      : double-float products on the FP32
//                                           pipes (df_proj.cu for B^H, k_zgemm_df
//                                           for U and V; ~1e-14 relative);
//   QR of B^H, Jacobi SVD                   : FP64 (the existing kernels).
//
// Complex products use the real embedding: A (M x K complex) becomes the
// M x 2K real matrix of interleaved (Re, Im) entries, and X (K x l complex)
// becomes Bt (2l x 2K real, K-major) with rows
//   2c   : ( Re X[j][c], -Im X[j][c] )  and  2c+1 : ( Im X[j][c], Re X[j][c] ),
// so that real column 2c / 2c+1 of A Bt^T is Re / Im of (A X)[:, c].  A^H is
// stored once as its own N x 2M copy with the conjugate folded in.  Rows of
// every real operand are zero-padded to a multiple of 32 floats (128 bytes:
// one TMA box, aligned x coordinates).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "internal.cuh"
#include "mixed.cuh"
#include "dfsplit.cuh"
#include "profiler.cuh"
#include "tc_gemm.cuh"
#include "workspace.cuh"
#include "../../include/tebd_gb300.h"

namespace tg {

// FP32 -> BF16 bits, round to nearest even (finite inputs)
__device__ __forceinline__ unsigned bf16_rn(float x) {
  const unsigned u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------------------
// theta (FP64, m x n row-major, per instance), read once per 32 x 32 tile:
//   forward copy thf (m x K1): TF32-rounded (Re, Im) and, when requested,
//     the TF32 remainder thf_lo;
//   adjoint copy tha (n x K2), transposed through shared memory:
//     tha[c][2r] = Re theta[r][c], tha[c][2r+1] = -Im theta[r][c], and its
//     remainder;
//   BF16 copies of both (the BF16 form's products before the refinement
//     round), when thf_b / tha_b are set;
//   the tile partial sums of ||theta||_F^2 (double-float, then FP64).
// The tiles cover the zero padding of every copy.
// ---------------------------------------------------------------------------
// double-float pair sum (Knuth's TwoSum on the high words)
__device__ __forceinline__ void df_add2(float& h, float& l, float oh, float ol) {
  const float s = h + oh;
  const float v = s - h;
  float e = (h - (s - v)) + (oh - v);
  e += l + ol;
  h = s + e;
  l = e - (h - s);
}

__global__ void __launch_bounds__(256) k_conv_theta(const MixedPtrs mp, const Dims* __restrict__ dims,
                                                    const ProbPtr* __restrict__ ptrs, int mc, int nc, int K1, int K2,
                                                    int want_lo, int K1b, int K2b) {
  __shared__ float2 tile[32][33];  // TF32 hi and remainder computed once per element
  __shared__ float2 tlo[32][33];
  __shared__ unsigned tb16[32][33];  // BF16 (Re, Im) pairs of the BF16 copies
  __shared__ float red[16];
  const int z = blockIdx.z;
  const Dims D = dims[z];
  if (!D.active) return;
  const int m = D.m, n = D.n;  // this instance (theta is compact m x n); copies at capacity mc x nc
  const cplx* th = ptrs[z].theta;
  const int half1 = K1 / 2, half2 = K2 / 2;  // complex columns of thf / tha incl. padding
  float2* fh = reinterpret_cast<float2*>(mp.thf_hi + (size_t)z * mc * K1);
  float2* fl = reinterpret_cast<float2*>(mp.thf_lo + (size_t)z * mc * K1);
  float2* ah = reinterpret_cast<float2*>(mp.tha_hi + (size_t)z * nc * K2);
  float2* al = reinterpret_cast<float2*>(mp.tha_lo + (size_t)z * nc * K2);
  unsigned* fb = mp.thf_b ? reinterpret_cast<unsigned*>(mp.thf_b + (size_t)z * mc * K1b) : nullptr;
  unsigned* ab = mp.tha_b ? reinterpret_cast<unsigned*>(mp.tha_b + (size_t)z * nc * K2b) : nullptr;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float sh = 0.f, sl = 0.f;  // double-float sum of |theta|^2 over this thread's elements
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    const cplx v = (r < m && c < n) ? th[(int64_t)r * n + c] : cmk(0.0, 0.0);
    float xh, xl, yh, yl;
    split_bits(v.x, xh, xl);
    split_bits(v.y, yh, yl);
    const float hr = tf32_rna(xh), hm = tf32_rna(yh);
    const float lr = tf32_rna((xh - hr) + xl), lm = tf32_rna((yh - hm) + yl);
    tile[i][tx] = make_float2(hr, hm);
    tlo[i][tx] = make_float2(lr, lm);
    if (fb) {
      tb16[i][tx] = bf16_rn(xh) | (bf16_rn(-yh) << 16);  // adjoint entry conj(theta), read transposed below
      if (r < mc && c < K1b / 2) fb[(int64_t)r * (K1b / 2) + c] = bf16_rn(xh) | (bf16_rn(yh) << 16);
    }
    if (r < mc && c < half1) {
      fh[(int64_t)r * half1 + c] = make_float2(hr, hm);
      if (want_lo) fl[(int64_t)r * half1 + c] = make_float2(lr, lm);
    }
    // |v|^2 = xh^2 + yh^2 + 2 (xh xl + yh yl) + O(2^-48)
    const float p1 = xh * xh, e1 = fmaf(xh, xh, -p1);
    const float p2 = yh * yh, e2 = fmaf(yh, yh, -p2);
    df_add2(sh, sl, p1, e1 + 2.f * xh * xl);
    df_add2(sh, sl, p2, e2 + 2.f * yh * yl);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    df_add2(sh, sl, oh, ol);
  }
  if (tx == 0) {
    red[2 * ty] = sh;
    red[2 * ty + 1] = sl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float h = red[0], l = red[1];
    for (int w = 1; w < 8; ++w) df_add2(h, l, red[2 * w], red[2 * w + 1]);
    mp.tpart[(size_t)z * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = (double)h + (double)l;
  }
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;  // output row c, complex column r: conj of element (r, c)
    if (c < nc && r < half2) {
      const float2 h = tile[tx][i], l = tlo[tx][i];
      ah[(int64_t)c * half2 + r] = make_float2(h.x, -h.y);
      if (want_lo) al[(int64_t)c * half2 + r] = make_float2(l.x, -l.y);
    }
    if (ab && c < nc && r < K2b / 2) ab[(int64_t)c * (K2b / 2) + r] = tb16[tx][i];
  }
}

// ||theta||_F^2 of each instance: its tile partials summed into the NPART
// fixed partial sums the epilogue reads (deterministic order).
__global__ void k_part_reduce(const double* __restrict__ tpart, int ntile, const Dims* __restrict__ dims,
                              const ProbPtr* __restrict__ ptrs) {
  const int z = blockIdx.x;
  if (!dims[z].active) return;
  const int i = threadIdx.x;  // < NPART
  double s = 0.0;
  for (int t = i; t < ntile; t += NPART) s += tpart[(size_t)z * ntile + t];
  ptrs[z].part[i] = s;
}

// Omega (the Philox words of the FP64 path, FP32 Box-Muller) written directly as Bt (Np x K1), and
// its TF32 remainder when the sketch itself is the refinement pass (q = 0).
// Instance z: chain chain0 + z chain_stride and the given sweep, or (chain_stride
// < 0) its own chain index and *sweep_dev, like k_omega.
__global__ void k_omega_bt(const MixedPtrs mp, const Dims* __restrict__ dims, int Np, int K1, uint64_t seed,
                           uint64_t sweep, int64_t chain0, int chain_stride, int want_lo,
                           const uint64_t* __restrict__ sweep_dev) {
  const int z = blockIdx.y;
  const Dims D = dims[z];
  if (!D.active) return;
  const int n = D.n, l = D.l;
  float* bt = mp.bt_hi + (size_t)z * Np * K1;
  float* btl = mp.bt_lo + (size_t)z * Np * K1;
  const int half = K1 / 2;
  const int64_t total = (int64_t)(Np / 2) * half;  // (row pair c, complex column j)
  const uint64_t chain = chain_stride >= 0 ? (uint64_t)(chain0 + (int64_t)z * chain_stride) : (uint64_t)D.chain;
  if (sweep_dev) sweep = *sweep_dev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / half), j = (int)(e % half);
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f), al = a, bl = a;
    if (c < l && j < n) {
      const float2 w = gauss_c_f32((uint64_t)j * l + c, (uint64_t)D.bond, sweep, chain, seed);
      const float re = tf32_rna(w.x), im = tf32_rna(w.y);
      a = make_float2(re, -im);
      b = make_float2(im, re);
      const float rl = tf32_rna(w.x - re), il = tf32_rna(w.y - im);
      al = make_float2(rl, -il);
      bl = make_float2(il, rl);
    }
    reinterpret_cast<float2*>(bt + (size_t)(2 * c) * K1)[j] = a;
    reinterpret_cast<float2*>(bt + (size_t)(2 * c + 1) * K1)[j] = b;
    if (want_lo) {
      reinterpret_cast<float2*>(btl + (size_t)(2 * c) * K1)[j] = al;
      reinterpret_cast<float2*>(btl + (size_t)(2 * c + 1) * K1)[j] = bl;
    }
  }
}

// X (complex FP32, column-major Kc x l, instance stride Kc*l) -> Bt (Np x Kp)
// and optionally its TF32 remainder.
// Columns past the instance's own l (the junk basis vectors of a padded QR)
// become zero rows of Bt.
__global__ void k_conv_bt(const float2* __restrict__ X, const Dims* __restrict__ dims, float* bt_hi, float* bt_lo,
                          int Kc, int lc, int Np, int Kp, int want_lo) {
  const int z = blockIdx.y;
  const Dims D = dims[z];
  if (!D.active) return;
  const int l = D.l;
  const float2* x = X + (size_t)z * Kc * lc;
  float* bh = bt_hi + (size_t)z * Np * Kp;
  float* bl = bt_lo + (size_t)z * Np * Kp;
  const int half = Kp / 2;
  const int64_t total = (int64_t)(Np / 2) * half;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / half), j = (int)(e % half);
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f), al = a, bl2 = a;
    if (c < l && j < Kc) {
      const float2 v = x[(int64_t)c * Kc + j];
      const float re = tf32_rna(v.x), im = tf32_rna(v.y);
      a = make_float2(re, -im);
      b = make_float2(im, re);
      const float rl = tf32_rna(v.x - re), il = tf32_rna(v.y - im);
      al = make_float2(rl, -il);
      bl2 = make_float2(il, rl);
    }
    reinterpret_cast<float2*>(bh + (size_t)(2 * c) * Kp)[j] = a;
    reinterpret_cast<float2*>(bh + (size_t)(2 * c + 1) * Kp)[j] = b;
    if (want_lo) {
      reinterpret_cast<float2*>(bl + (size_t)(2 * c) * Kp)[j] = al;
      reinterpret_cast<float2*>(bl + (size_t)(2 * c + 1) * Kp)[j] = bl2;
    }
  }
}

// BF16 forms of k_omega_bt and k_conv_bt (the products before the refinement
// round of TEBD_PREC_BF16): Bt (Np x Kp BF16) from Omega or from X.
__global__ void k_omega_bt_bf16(uint16_t* bt_b, const Dims* __restrict__ dims, int Np, int Kp, uint64_t seed,
                                uint64_t sweep, int64_t chain0, int chain_stride, const uint64_t* __restrict__ sweep_dev) {
  const int z = blockIdx.y;
  const Dims D = dims[z];
  if (!D.active) return;
  const int n = D.n, l = D.l;
  unsigned* bt = reinterpret_cast<unsigned*>(bt_b + (size_t)z * Np * Kp);
  const int half = Kp / 2;
  const int64_t total = (int64_t)(Np / 2) * half;
  const uint64_t chain = chain_stride >= 0 ? (uint64_t)(chain0 + (int64_t)z * chain_stride) : (uint64_t)D.chain;
  if (sweep_dev) sweep = *sweep_dev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / half), j = (int)(e % half);
    unsigned a = 0, b = 0;
    if (c < l && j < n) {
      const float2 w = gauss_c_f32((uint64_t)j * l + c, (uint64_t)D.bond, sweep, chain, seed);
      a = bf16_rn(w.x) | (bf16_rn(-w.y) << 16);
      b = bf16_rn(w.y) | (bf16_rn(w.x) << 16);
    }
    bt[(size_t)(2 * c) * half + j] = a;
    bt[(size_t)(2 * c + 1) * half + j] = b;
  }
}

__global__ void k_conv_bt_bf16(const float2* __restrict__ X, const Dims* __restrict__ dims, uint16_t* bt_b, int Kc,
                               int lc, int Np, int Kp) {
  const int z = blockIdx.y;
  const Dims D = dims[z];
  if (!D.active) return;
  const int l = D.l;
  const float2* x = X + (size_t)z * Kc * lc;
  unsigned* bt = reinterpret_cast<unsigned*>(bt_b + (size_t)z * Np * Kp);
  const int half = Kp / 2;
  const int64_t total = (int64_t)(Np / 2) * half;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / half), j = (int)(e % half);
    unsigned a = 0, b = 0;
    if (c < l && j < Kc) {
      const float2 v = x[(int64_t)c * Kc + j];
      a = bf16_rn(v.x) | (bf16_rn(-v.y) << 16);
      b = bf16_rn(v.y) | (bf16_rn(v.x) << 16);
    }
    bt[(size_t)(2 * c) * half + j] = a;
    bt[(size_t)(2 * c + 1) * half + j] = b;
  }
}

// ---------------------------------------------------------------------------
// Householder QR with explicit Q in FP32: alpha = -e^{i arg x0} ||x||,
// normalised reflector v = x / (x0 - alpha) (v_0 = 1), tau = 1 + |x0| / ||x||
// (Golub & Van Loan 5.1.2; the unnormalised form of the FP64 kernel would
// overflow FP32 for columns of norm below ~1e-19).  Input M x L
// column-major (overwritten), output Q M x L column-major.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 fmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ void ffma_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float fwarp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(1024) k_qr_f32(float2* Abase, float2* Qbase, int M, int L) {
  __shared__ float red[32];
  __shared__ float2 vscale;
  __shared__ float vnorm;
  __shared__ float tau[512];
  const int z = blockIdx.x;
  float2* A = Abase + (size_t)z * M * L;
  float2* Qo = Qbase + (size_t)z * M * L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < L; ++j) {
    float2* aj = A + (int64_t)j * M;
    float s = 0.f;
    for (int r = j + tid; r < M; r += blockDim.x) s += aj[r].x * aj[r].x + aj[r].y * aj[r].y;
    s = fwarp_sum(s);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t += red[w];
      vnorm = sqrtf(t);
    }
    __syncthreads();
    if (vnorm < 1e-12f) {
      // squares in the FP32 subnormal range would make the reflector
      // non-unitary: norm of x / max|x|
      float mx = 0.f;
      for (int r = j + tid; r < M; r += blockDim.x) mx = fmaxf(mx, fmaxf(fabsf(aj[r].x), fabsf(aj[r].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) red[warp] = mx;
      __syncthreads();
      float amax = 0.f;
      for (int w = 0; w < nw; ++w) amax = fmaxf(amax, red[w]);
      __syncthreads();
      float s2 = 0.f;
      if (amax > 0.f) {
        const float ia = 1.f / amax;
        for (int r = j + tid; r < M; r += blockDim.x) {
          const float a = aj[r].x * ia, b = aj[r].y * ia;
          s2 = fmaf(a, a, fmaf(b, b, s2));
        }
      }
      s2 = fwarp_sum(s2);
      if (lane == 0) red[warp] = s2;
      __syncthreads();
      if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w];
        vnorm = amax * sqrtf(t);
      }
      __syncthreads();
    }
    if (tid == 0) {
      const float2 x0 = aj[j];
      // |x0| without squaring; see k_qr_blk_f32 for the rules on tiny columns and entries
      const float ax0 = hypotf(x0.x, x0.y);
      const float nx = vnorm;
      if (!(nx >= 1e-30f)) {  // zero column, or one below any meaningful scale: no reflection
        tau[j] = 0.f;
        vscale = make_float2(1.f, 0.f);
      } else {
        const float2 ph = (ax0 > 1e-7f * nx) ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
        const float ri = 1.f / (ax0 + nx);
        vscale = make_float2(ph.x * ri, -ph.y * ri);  // 1 / (x0 - alpha)
        aj[j] = make_float2(1.f, 0.f);
        tau[j] = 1.f + ax0 / nx;
      }
    }
    __syncthreads();
    const float t = tau[j];
    if (t != 0.f) {
      const float2 sc = vscale;
      for (int r = j + 1 + tid; r < M; r += blockDim.x) {
        const float2 v = aj[r];
        aj[r] = make_float2(v.x * sc.x - v.y * sc.y, v.x * sc.y + v.y * sc.x);
      }
      __syncthreads();
    }
    if (t != 0.f) {
      for (int c = j + 1 + warp; c < L; c += nw) {
        float2* ac = A + (int64_t)c * M;
        float2 sd = make_float2(0.f, 0.f);
        for (int r = j + lane; r < M; r += 32) ffma_conj(sd, aj[r], ac[r]);
        sd.x = fwarp_sum(sd.x) * t;
        sd.y = fwarp_sum(sd.y) * t;
        for (int r = j + lane; r < M; r += 32) {
          const float2 p = fmul(aj[r], sd);
          ac[r] = make_float2(ac[r].x - p.x, ac[r].y - p.y);
        }
      }
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)M * L; e += blockDim.x) {
    const int c = (int)(e / M), r = (int)(e % M);
    Qo[e] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int j = L - 1; j >= 0; --j) {
    const float t = tau[j];
    if (t == 0.f) continue;
    const float2* aj = A + (int64_t)j * M;
    for (int c = j + warp; c < L; c += nw) {
      float2* qc = Qo + (int64_t)c * M;
      float2 sd = make_float2(0.f, 0.f);
      for (int r = j + lane; r < M; r += 32) ffma_conj(sd, aj[r], qc[r]);
      sd.x = fwarp_sum(sd.x) * t;
      sd.y = fwarp_sum(sd.y) * t;
      for (int r = j + lane; r < M; r += 32) {
        const float2 p = fmul(aj[r], sd);
        qc[r] = make_float2(qc[r].x - p.x, qc[r].y - p.y);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 3-D map over (K-padded row, row, instance) of FP32 (or BF16) data with a
// box of one 128-byte row segment x box_rows x 1 and 128-byte swizzle.
static bool make_map(CUtensorMap* m, const void* base, int Kp, int rows, int batch, int box_rows, bool bf16 = false) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t es_b = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * es_b, (cuuint64_t)rows * Kp * es_b};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es_b), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims,
             strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

MixedSizes mixed_sizes(int m, int n, int k, int l, int bf16, const Caps* gate) {
  MixedSizes s;
  s.bf16 = bf16 ? 1 : 0;
  s.K1 = ((2 * n + TC_BK - 1) / TC_BK) * TC_BK;
  s.K2 = ((2 * m + TC_BK - 1) / TC_BK) * TC_BK;
  s.K1b = ((2 * n + 63) / 64) * 64;
  s.K2b = ((2 * m + 63) / 64) * 64;
  s.Np = ((2 * l + 15) / 16) * 16;
  s.BN = s.Np <= TC_MAXBN ? s.Np : TC_MAXBN;
  const int Kmax = s.K1 > s.K2 ? s.K1 : s.K2;
  const size_t f = sizeof(float);
  s.thf = (size_t)m * s.K1 * f;
  s.tha = (size_t)n * s.K2 * f;
  s.bt = (size_t)s.Np * Kmax * f;
  s.yf = (size_t)m * l * sizeof(float2);
  s.ytf = (size_t)n * l * sizeof(float2);
  s.df = (size_t)l * l * sizeof(float2);
  // the projection runs on the tensor cores from BF16 digits (oz_proj.cu)
  s.bd = oz_digits_bytes(n, m);
  s.bsc = oz_scales_bytes(n, m);
  s.ad = oz_digits_bytes(l, m);
  s.asc = oz_scales_bytes(l, m);
  s.thfb = s.bf16 ? (size_t)m * s.K1b * 2 : 0;
  s.thab = s.bf16 ? (size_t)n * s.K2b * 2 : 0;
  s.btb = s.bf16 ? (size_t)s.Np * (s.K1b > s.K2b ? s.K1b : s.K2b) * 2 : 0;
  {
    const OzStageBytes ob = oz_stage_bytes(m, n, k, l, gate);
    s.gad = ob.ad;
    s.gas = ob.as;
    s.gbd = ob.bd;
    s.gbs = ob.bs;
  }
  const int mx = m > n ? m : n;
  s.qs = ((!qr_blk_f32_fits(m, l) && qr_multi_f32_fits(m, l)) || (!qr_blk_f32_fits(n, l) && qr_multi_f32_fits(n, l)))
             ? qr_multi_f32_scratch(mx, l) * sizeof(float2)
             : 0;
  {
    const int c1 = s.bf16 && s.K1b > s.K1 ? s.K1b : s.K1, c2 = s.bf16 && s.K2b > s.K2 ? s.K2b : s.K2;
    s.ntile = ((c1 / 2 + 31) / 32) * ((c2 / 2 + 31) / 32);
  }
  (void)k;
  return s;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t mixed_bytes(const MixedSizes& s, int batch) {
  return 2 * up256(s.thf * batch) + 2 * up256(s.tha * batch) + 2 * up256(s.bt * batch) + 2 * up256(s.yf * batch) +
         2 * up256(s.ytf * batch) + up256(s.df * batch) +
         up256((size_t)s.ntile * sizeof(double) * batch) + up256(s.qs * batch) + up256(s.bd * batch) +
         up256(s.bsc * batch) + up256(s.ad * batch) + up256(s.asc * batch) + up256(s.thfb * batch) +
         up256(s.thab * batch) + up256(s.btb * batch) + up256(s.gad * batch) + up256(s.gas * batch) +
         up256(s.gbd * batch) + up256(s.gbs * batch);
}

MixedPtrs mixed_carve(char* base, const MixedSizes& s, int batch) {
  MixedPtrs p;
  size_t o = 0;
  p.thf_hi = (float*)(base + o); o += up256(s.thf * batch);
  p.thf_lo = (float*)(base + o); o += up256(s.thf * batch);
  p.tha_hi = (float*)(base + o); o += up256(s.tha * batch);
  p.tha_lo = (float*)(base + o); o += up256(s.tha * batch);
  p.bt_hi = (float*)(base + o); o += up256(s.bt * batch);
  p.bt_lo = (float*)(base + o); o += up256(s.bt * batch);
  p.Yf = (float2*)(base + o); o += up256(s.yf * batch);
  p.Qf = (float2*)(base + o); o += up256(s.yf * batch);
  p.Ytf = (float2*)(base + o); o += up256(s.ytf * batch);
  p.Qtf = (float2*)(base + o); o += up256(s.ytf * batch);
  p.Df = (float2*)(base + o); o += up256(s.df * batch);
  p.tpart = (double*)(base + o);
  o += up256((size_t)s.ntile * sizeof(double) * batch);
  p.qscr = s.qs ? (float2*)(base + o) : nullptr;
  o += up256(s.qs * batch);
  p.bd = (uint16_t*)(base + o); o += up256(s.bd * batch);
  p.bsc = (float*)(base + o); o += up256(s.bsc * batch);
  p.ad = (uint16_t*)(base + o); o += up256(s.ad * batch);
  p.asc = (float*)(base + o); o += up256(s.asc * batch);
  p.thf_b = s.bf16 ? (uint16_t*)(base + o) : nullptr; o += up256(s.thfb * batch);
  p.tha_b = s.bf16 ? (uint16_t*)(base + o) : nullptr; o += up256(s.thab * batch);
  p.bt_b = s.bf16 ? (uint16_t*)(base + o) : nullptr; o += up256(s.btb * batch);
  p.gad = (uint16_t*)(base + o); o += up256(s.gad * batch);
  p.gas = (float*)(base + o); o += up256(s.gas * batch);
  p.gbd = (uint16_t*)(base + o); o += up256(s.gbd * batch);
  p.gbs = (float*)(base + o); o += up256(s.gbs * batch);
  return p;
}

MixedPtrs mixed_offset(const MixedPtrs& p, const MixedSizes& s, int z0) {
  MixedPtrs o = p;
  const size_t z = (size_t)z0;
  auto adv = [z](auto* ptr, size_t bytes) { return ptr ? (decltype(ptr))((char*)ptr + z * bytes) : ptr; };
  o.thf_hi = adv(p.thf_hi, s.thf);
  o.thf_lo = adv(p.thf_lo, s.thf);
  o.tha_hi = adv(p.tha_hi, s.tha);
  o.tha_lo = adv(p.tha_lo, s.tha);
  o.bt_hi = adv(p.bt_hi, s.bt);
  o.bt_lo = adv(p.bt_lo, s.bt);
  o.Yf = adv(p.Yf, s.yf);
  o.Qf = adv(p.Qf, s.yf);
  o.Ytf = adv(p.Ytf, s.ytf);
  o.Qtf = adv(p.Qtf, s.ytf);
  o.Df = adv(p.Df, s.df);
  o.tpart = adv(p.tpart, (size_t)s.ntile * sizeof(double));
  o.qscr = adv(p.qscr, s.qs);
  o.bd = adv(p.bd, s.bd);
  o.bsc = adv(p.bsc, s.bsc);
  o.ad = adv(p.ad, s.ad);
  o.asc = adv(p.asc, s.asc);
  o.thf_b = adv(p.thf_b, s.thfb);
  o.tha_b = adv(p.tha_b, s.thab);
  o.bt_b = adv(p.bt_b, s.btb);
  o.gad = adv(p.gad, s.gad);
  o.gas = adv(p.gas, s.gas);
  o.gbd = adv(p.gbd, s.gbd);
  o.gbs = adv(p.gbs, s.gbs);
  return o;
}

#define MX_TRY(x)                     \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// the tensor-core kernels' shared memory limit, set once for the largest tile
static cudaError_t tc_attrs() {
  static int done = 0;
  if (!done) {
    MX_TRY(cudaFuncSetAttribute(k_tc_gemm<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes(TC_MAXBN)));
    MX_TRY(cudaFuncSetAttribute(k_tc_gemm<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem_bytes(TC_MAXBN)));
    done = 1;
  }
  return cudaSuccess;
}

static int grid1d(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 1024) b = 1024;
  return (int)(b < 1 ? 1 : b);
}

// One tensor-core product: out (rows x l complex, per instance) from
// A (rows x Kp) and Bt (Np x Kp); npass 1 or 3.
// bf16: A0, B0 hold BF16 copies (one pass; A1, B1 unused) and Kp counts BF16
// values; otherwise FP32 arrays of TF32-rounded values.
static cudaError_t tc_product(const void* A0, const void* A1, const void* B0, const void* B1, int rows, int Kp,
                              const MixedSizes& s0, int l, int npass, float2* out, int batch, int* err,
                              cudaStream_t st, int half, bool bf16 = false) {
  // half: the columns of the product split over two CTAs (tile width rounded to 16)
  MixedSizes s = s0;
  if (half && s.BN > 16) s.BN = ((s.BN / 2 + 15) / 16) * 16;
  CUtensorMap ma0, ma1, mb0, mb1;
  if (!make_map(&ma0, A0, Kp, rows, batch, TC_BM, bf16) || !make_map(&ma1, bf16 ? A0 : A1, Kp, rows, batch, TC_BM, bf16) ||
      !make_map(&mb0, B0, Kp, s.Np, batch, s.BN, bf16) || !make_map(&mb1, bf16 ? B0 : B1, Kp, s.Np, batch, s.BN, bf16))
    return cudaErrorInvalidValue;
  TcArgs a;
  a.M = rows;
  a.Kp = Kp;
  a.BN = s.BN;
  a.l = l;
  a.npass = npass;
  a.out = out;
  a.out_stride = (int64_t)rows * l;
  a.err = err;
  // an injected pipeline stall (test hook): no operand copies, short waits
  // (never inside a stream capture, where it would stall every replay)
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap_st) != cudaSuccess) cap_st = cudaStreamCaptureStatusActive;
  const bool stall = cap_st == cudaStreamCaptureStatusNone && fault_take(TEBD_FAULT_TC_STALL);
  a.poll_limit = stall ? (1u << 12) : (1u << 24);
  a.stall = stall ? 1 : 0;
  const size_t sm = tc_smem_bytes(s.BN);
  MX_TRY(tc_attrs());
  dim3 grid((rows + TC_BM - 1) / TC_BM, (s.Np + s.BN - 1) / s.BN, batch);
  if (bf16) {
    ProfScope ps("k_tc_gemm[bf16]", st);
    k_tc_gemm<TC_BF16><<<grid, 128, sm, st>>>(ma0, ma1, mb0, mb1, a);
  } else {
    ProfScope ps(npass == 1 ? "k_tc_gemm[tf32]" : "k_tc_gemm[3xtf32]", st);
    k_tc_gemm<TC_TF32><<<grid, 128, sm, st>>>(ma0, ma1, mb0, mb1, a);
  }
  return cudaGetLastError();
}

static cudaError_t qr_f32(float2* A, float2* Q, int M, int L, int batch, const MixedPtrs& mp, const MixedSizes& s,
                          const Dims* dims, int use_n, cudaStream_t st, int threads) {
  if (!qr_blk_f32_fits(M, L) && mp.qscr && qr_multi_f32_fits(M, L))
    return launch_qr_multi_f32(A, Q, mp.qscr, s.qs / sizeof(float2), M, L, batch, st, dims, use_n);
  ProfScope ps("k_qr_f32", st);
  if (qr_blk_f32_fits(M, L)) return launch_qr_blk_f32(A, Q, M, L, batch, st, dims, use_n, threads);
  k_qr_f32<<<batch, 1024, 0, st>>>(A, Q, M, L);
  return cudaGetLastError();
}

static cudaError_t conv_bt(const float2* X, const Dims* dims, const MixedPtrs& mp, int Kc, int l, int Kp,
                           const MixedSizes& s, int lo, int batch, cudaStream_t st) {
  ProfScope ps("k_conv_bt", st);
  k_conv_bt<<<dim3(grid1d((int64_t)(s.Np / 2) * (Kp / 2)), batch), 256, 0, st>>>(X, dims, mp.bt_hi, mp.bt_lo, Kc, l,
                                                                                   s.Np, Kp, lo);
  return cudaGetLastError();
}

static cudaError_t conv_bt_bf16(const float2* X, const Dims* dims, const MixedPtrs& mp, int Kc, int l, int Kp,
                                const MixedSizes& s, int batch, cudaStream_t st) {
  ProfScope ps("k_conv_bt", st);
  k_conv_bt_bf16<<<dim3(grid1d((int64_t)(s.Np / 2) * (Kp / 2)), batch), 256, 0, st>>>(X, dims, mp.bt_b, Kc, l, s.Np,
                                                                                      Kp);
  return cudaGetLastError();
}

cudaError_t mixed_prepare(const Caps& cap) {
  if (!encode_fn()) return cudaErrorNotSupported;
  MX_TRY(oz_prepare());
  MX_TRY(jacobi_df_prepare());
  MX_TRY(cholqr_prepare());
  MX_TRY(tc_attrs());
  return qr_blocked_prepare(cap.m, cap.n, cap.l);
}

cudaError_t run_rrsvd_mixed(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, const MixedPtrs& mp,
                            int q, uint64_t seed, uint64_t sweep, int64_t chain0, int chain_stride, int* status,
                            int* err, cudaStream_t st, const uint64_t* sweep_dev, const MixedKnobs* knobs,
                            int bf16_form) {
  const MixedKnobs kn = knobs ? *knobs : MixedKnobs{0, 0, 0, 0, 0};
  // capacities: every FP32 array is laid out at these sizes, zero-padded past
  // each instance's own (m, n, l) from dims
  const int m = cap.m, n = cap.n, k = cap.k, l = cap.l;
  const MixedSizes s = mixed_sizes(m, n, k, l, bf16_form);
  // BF16 products: every one before the refinement round (the last power
  // round; Y0 itself when q = 0, which then stays 3xTF32)
  const bool bf = bf16_form && mp.thf_b && q > 0;
  {
    ProfScope ps("k_conv_theta", st);
    // padded extents (>= n, >= m) of every copy written
    const int cext = (bf && s.K1b > s.K1 ? s.K1b : s.K1) / 2, rext = (bf && s.K2b > s.K2 ? s.K2b : s.K2) / 2;
    MixedPtrs mq = mp;
    if (!bf) mq.thf_b = mq.tha_b = nullptr;
    const dim3 grid((cext + 31) / 32, (rext + 31) / 32, batch);  // grid.x * grid.y <= s.ntile
    k_conv_theta<<<grid, 256, 0, st>>>(mq, dims, ptrs, m, n, s.K1, s.K2, 1, s.K1b, s.K2b);
    MX_TRY(cudaGetLastError());
    k_part_reduce<<<batch, NPART, 0, st>>>(mp.tpart, (int)(grid.x * grid.y), dims, ptrs);
    MX_TRY(cudaGetLastError());
  }
  MX_TRY(launch_oz_digits_theta(dims, ptrs, mp.bd, mp.bsc, m, n, batch, st));
  {
    ProfScope ps("k_omega_bt", st);
    if (bf)
      k_omega_bt_bf16<<<dim3(grid1d((int64_t)(s.Np / 2) * (s.K1b / 2)), batch), 256, 0, st>>>(
          mp.bt_b, dims, s.Np, s.K1b, seed, sweep, chain0, chain_stride, sweep_dev);
    else
      k_omega_bt<<<dim3(grid1d((int64_t)(s.Np / 2) * (s.K1 / 2)), batch), 256, 0, st>>>(
          mp, dims, s.Np, s.K1, seed, sweep, chain0, chain_stride, q == 0 ? 1 : 0, sweep_dev);
    MX_TRY(cudaGetLastError());
  }
  // Y0 = A Omega: TF32, or the refinement pass when q == 0
  const int p0 = (q == 0) ? 3 : 1;
  if (bf)
    MX_TRY(tc_product(mp.thf_b, nullptr, mp.bt_b, nullptr, m, s.K1b, s, l, 1, mp.Yf, batch, err, st, kn.tc_half, true));
  else
    MX_TRY(tc_product(mp.thf_hi, mp.thf_lo, mp.bt_hi, mp.bt_lo, m, s.K1, s, l, p0, mp.Yf, batch, err, st,
                      kn.tc_half));
  for (int j = 1; j <= q; ++j) {
    const int np = (j == q) ? 3 : 1;
    const bool b16 = bf && np == 1;  // BF16 for the rounds before the refinement round
    MX_TRY(qr_f32(mp.Yf, mp.Qf, m, l, batch, mp, s, dims, 0, st, kn.qr_threads));    // Y = Q R
    if (b16) {
      MX_TRY(conv_bt_bf16(mp.Qf, dims, mp, m, l, s.K2b, s, batch, st));
      MX_TRY(tc_product(mp.tha_b, nullptr, mp.bt_b, nullptr, n, s.K2b, s, l, 1, mp.Ytf, batch, err, st, kn.tc_half,
                        true));  // A^H Q
    } else {
      MX_TRY(conv_bt(mp.Qf, dims, mp, m, l, s.K2, s, np == 3, batch, st));
      MX_TRY(tc_product(mp.tha_hi, mp.tha_lo, mp.bt_hi, mp.bt_lo, n, s.K2, s, l, np, mp.Ytf, batch, err, st,
                        kn.tc_half));  // A^H Q
    }
    MX_TRY(qr_f32(mp.Ytf, mp.Qtf, n, l, batch, mp, s, dims, 1, st, kn.qr_threads));  // = Q~ R~
    if (b16) {
      MX_TRY(conv_bt_bf16(mp.Qtf, dims, mp, n, l, s.K1b, s, batch, st));
      MX_TRY(tc_product(mp.thf_b, nullptr, mp.bt_b, nullptr, m, s.K1b, s, l, 1, mp.Yf, batch, err, st, kn.tc_half,
                        true));  // A Q~
    } else {
      MX_TRY(conv_bt(mp.Qtf, dims, mp, n, l, s.K1, s, np == 3, batch, st));
      MX_TRY(tc_product(mp.thf_hi, mp.thf_lo, mp.bt_hi, mp.bt_lo, m, s.K1, s, l, np, mp.Yf, batch, err, st,
                        kn.tc_half));  // A Q~
    }
  }
  // last QR: FP32 Householder, then the FP64-accurate re-orthonormalisation.
  // Plans and handles refuse sketches wider than 512 columns, and l <= m, so
  // every basis they pass fits it.
  if (!reorth_fits(m, l)) return cudaErrorInvalidValue;
  MX_TRY(qr_f32(mp.Yf, mp.Qf, m, l, batch, mp, s, dims, 0, st, kn.qr_threads));
  // digits of Q_f once: the Gram of the re-orthonormalisation and the
  // projection B^H = A^H Q both take them
  MX_TRY(launch_oz_digits_qf(dims, mp.Qf, mp.ad, mp.asc, m, l, batch, st));
  MX_TRY(launch_oz_gram(dims, ptrs, mp.ad, mp.asc, m, l, batch, err, st));
  MX_TRY(launch_reorth(mp.Qf, mp.Df, dims, ptrs, m, l, batch, status, st));
  MX_TRY(launch_proj_oz(dims, ptrs, mp.Qf, mp.Df, mp.ad, mp.asc, mp.bd, mp.bsc, m, n, l, batch, err, st,
                        true));  // B^H = A^H Q
  // QR of B^H: Cholesky QR where the one-CTA Householder would run (it falls
  // back to Householder per ill-conditioned instance), else the size rule
  // the FP64-accurate products after the projection: tensor cores from digit
  // splits, or double-float GEMMs on the CUDA cores
  const bool tc = kn.dfg == 1 || (kn.dfg == 0 && oz_stage_rule(cap));
  const OzScratch oz{mp.gad, mp.gas, mp.gbd, mp.gbs};
  if (kn.qrbh == 3 || (kn.qrbh == 0 && !qr_multi_chosen(QR_BH, cap, batch, 0)))
    MX_TRY(run_cholqr_bh(const_cast<Dims*>(dims), ptrs, batch, cap, st, tc ? &oz : nullptr, err));
  else
    MX_TRY(launch_qr_sized(QR_BH, dims, ptrs, batch, cap, st, kn.qrbh));
  // Jacobi SVD: double-float one-CTA kernel unless the cluster form is chosen
  if (kn.jac == 3 || (kn.jac == 0 && !jacobi_cluster_chosen(cap, batch, 0)))
    MX_TRY(launch_jacobi_df(dims, ptrs, batch, cap.l, status, st));
  else
    MX_TRY(launch_jacobi_sized(dims, ptrs, batch, cap, status, st, kn.jac));
  for (int stage : {G_U, G_V})
    MX_TRY(tc ? launch_oz_stage(stage, dims, ptrs, batch, cap, oz, err, st)
              : launch_zgemm_df(stage, dims, ptrs, batch, cap, st));
  return cudaSuccess;
}

}  // namespace tg
