// Double-float projection of the mixed-precision RRSVD (sm_103a): the step
// B = Q^H A of Section IV, formed as its adjoint B^H = A^H Q with the
// re-orthonormalised basis Q = Q_f (I + D) of qr_blocked.cu.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"
#include "dfsplit.cuh"

namespace tg {

// ---------------------------------------------------------------------------
// Projection B^H = A^H Q with Q = Q_f (I + D) (the re-orthonormalised basis):
// X = A^H Q_f in double-float arithmetic, A^H from the double-float copy of
// conj(A) and the FP32 Q_f used as it is (its entries are exact single
// floats), then B^H = X + X D.
// Complex products by Gauss's three multiplications: for alpha = a + ib
// (from A^H) and beta = c + id (from Q_f),
//   t1 = a (c + d),  t2 = d (a + b),  t3 = c (b - a),
//   Re = t1 - t2,  Im = t1 + t3,
// three double-float products instead of four; a, a + b, b - a are
// double-float, c, d single floats, c + d a TwoSum pair.  64 x 32 output tile
// per CTA, 4 x 2 outputs per thread, K in slices of 16 each closed by a
// renormalising Fast2Sum of the accumulators.
// ---------------------------------------------------------------------------
enum { PJ_TM = 64, PJ_TN = 32, PJ_TK = 16 };

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

// thd and Q_f at capacity mc x nc and mc x lc per instance; the instance's
// own (m, n, l) from dims bound the sum and the output (D.n x D.l, compact).
__global__ void __launch_bounds__(256) k_proj_df(const float4* __restrict__ thd, const float2* __restrict__ Qf,
                                                 const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                 int mc, int nc, int lc) {
  __shared__ float4 Aab[PJ_TK][PJ_TM];  // (a_h, a_l, b_h, b_l)
  __shared__ float4 Asd[PJ_TK][PJ_TM];  // (a+b)_h, (a+b)_l, (b-a)_h, (b-a)_l
  __shared__ float4 Bs[PJ_TK][PJ_TN + 1];  // (c, d, (c+d)_h, (c+d)_l); padded against bank conflicts
                                          // of the k-fastest stores
  const int z = blockIdx.z;
  const Dims Dm = dims[z];
  if (!Dm.active) return;
  const int m = Dm.m, n = Dm.n, l = Dm.l;
  const int tm = blockIdx.y * PJ_TM, tn = blockIdx.x * PJ_TN;
  if (tm >= n || tn >= l) return;
  const float4* th = thd + (size_t)z * mc * nc;
  const float2* q = Qf + (size_t)z * mc * lc;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float h1[4][2], l1[4][2], h2[4][2], l2[4][2], h3[4][2], l3[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) h1[i][j] = l1[i][j] = h2[i][j] = l2[i][j] = h3[i][j] = l3[i][j] = 0.f;
  for (int k0 = 0; k0 < m; k0 += PJ_TK) {
    // A^H tile: element (r, k) = conj(theta[k][r]), pre-split; consecutive
    // threads read consecutive r
    for (int e = tid; e < PJ_TM * PJ_TK; e += 256) {
      const int r = e % PJ_TM, kk = e / PJ_TM;
      const int gr = tm + r, gk = k0 + kk;
      const float4 f = (gr < n && gk < m) ? th[(size_t)gk * nc + gr] : make_float4(0.f, 0.f, 0.f, 0.f);
      float sh, se, dh, de;
      two_sum(f.x, f.z, sh, se);
      two_sum(f.z, -f.x, dh, de);
      Aab[kk][r] = f;
      Asd[kk][r] = make_float4(sh, se + (f.y + f.w), dh, de + (f.w - f.y));
    }
    // Q_f tile: element (k, c) at q[c * m + k]
    for (int e = tid; e < PJ_TK * PJ_TN; e += 256) {
      const int kk = e % PJ_TK, c = e / PJ_TK;
      const int gk = k0 + kk, gc = tn + c;
      float2 v = make_float2(0.f, 0.f);
      if (gk < m && gc < l) v = q[(size_t)gc * mc + gk];
      float sh, se;
      two_sum(v.x, v.y, sh, se);
      Bs[kk][c] = make_float4(v.x, v.y, sh, se);
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < PJ_TK; ++kk) {
      float4 b[2];
      b[0] = Bs[kk][tx];
      b[1] = Bs[kk][tx + 16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 ab = Aab[kk][ty + 16 * i];
        const float4 sd = Asd[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          dfx_dd(h1[i][j], l1[i][j], ab.x, ab.y, b[j].z, b[j].w);  // a (c + d)
          dfx_sd(h2[i][j], l2[i][j], b[j].y, sd.x, sd.y);          // d (a + b)
          dfx_sd(h3[i][j], l3[i][j], b[j].x, sd.z, sd.w);          // c (b - a)
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        fast2(h1[i][j], l1[i][j]);
        fast2(h2[i][j], l2[i][j]);
        fast2(h3[i][j], l3[i][j]);
      }
    __syncthreads();
  }
  cplx* X = ptrs[z].Yt;  // n x l column-major
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = tm + ty + 16 * i, c = tn + tx + 16 * j;
      if (r < n && c < l) {
        const double t1 = (double)h1[i][j] + (double)l1[i][j];
        const double t2 = (double)h2[i][j] + (double)l2[i][j];
        const double t3 = (double)h3[i][j] + (double)l3[i][j];
        X[(size_t)c * n + r] = cmk(t1 - t2, t1 + t3);
      }
    }
}

cudaError_t launch_proj_df(const float4* thd, const Dims* dims, const ProbPtr* ptrs, const float2* Qf,
                           const float2* Dbuf, int m, int n, int l, int batch, cudaStream_t st) {
  {
    ProfScope ps("k_zgemm_df[project]", st);
    k_proj_df<<<dim3((l + PJ_TN - 1) / PJ_TN, (n + PJ_TM - 1) / PJ_TM, batch), 256, 0, st>>>(thd, Qf, dims, ptrs, m,
                                                                                             n, l);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_fold_bh(Dbuf, dims, ptrs, n, l, batch, st);
}


// ---------------------------------------------------------------------------
// Gate of large local dimensions as a double-float GEMM (the TF32 form's
// counterpart of k_gate_gemm): theta~ = G C over the physical indices,
// FP64-accurate on the FP32 pipes.  G and the pre-gate theta C are split at
// staging into FP32 pairs (integer bit operations), products by Gauss's rule
// with three double-float products (t1 = a (c+d), t2 = d (a+b), t3 = c (b-a)),
// 64 x 32 output tiles (rows (i, j) of G, columns (alpha, beta) with beta
// fastest), 4 x 2 outputs per thread, K = d_l d_r in slices of 16 closed by a
// renormalising Fast2Sum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gate_gemm_df(const Dims* __restrict__ dims,
                                                      const ProbPtr* __restrict__ ptrs) {
  __shared__ float4 Aab[PJ_TK][PJ_TM];      // (a_h, a_l, b_h, b_l) of G
  __shared__ float4 Asd[PJ_TK][PJ_TM];      // (a+b)_h, (a+b)_l, (b-a)_h, (b-a)_l
  __shared__ float4 Bcd[PJ_TK][PJ_TN + 1];  // (c_h, c_l, d_h, d_l) of C
  __shared__ float2 Bsum[PJ_TK][PJ_TN + 1]; // (c+d)_h, (c+d)_l
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  if (!P.Cpre) return;
  const int dl = D.dl, dr = D.dr, cl = D.cl, cr = D.cr;
  const int M = dl * dr, N = cl * cr, K = M, n_ = D.n;
  const int tm = blockIdx.y * PJ_TM, tn = blockIdx.x * PJ_TN;
  if (tm >= M || tn >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float h1[4][2], l1[4][2], h2[4][2], l2[4][2], h3[4][2], l3[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) h1[i][j] = l1[i][j] = h2[i][j] = l2[i][j] = h3[i][j] = l3[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += PJ_TK) {
    for (int e = tid; e < PJ_TM * PJ_TK; e += 256) {  // G tile: consecutive threads along k
      const int kk = e % PJ_TK, r = e / PJ_TK;
      const int gr = tm + r, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gr < M && gk < K) v = P.gate[(int64_t)gr * K + gk];
      float ah, al, bh, bl;
      split_bits(v.x, ah, al);
      split_bits(v.y, bh, bl);
      float sh, se, dh, de;
      two_sum(ah, bh, sh, se);
      two_sum(bh, -ah, dh, de);
      Aab[kk][r] = make_float4(ah, al, bh, bl);
      Asd[kk][r] = make_float4(sh, se + (al + bl), dh, de + (bl - al));
    }
    for (int e = tid; e < PJ_TK * PJ_TN; e += 256) {  // C tile: consecutive threads along (alpha, beta)
      const int c = e % PJ_TN, kk = e / PJ_TN;
      const int gn = tn + c, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gn < N && gk < K) {
        const int ip = gk / dr, jp = gk % dr, a = gn / cr, cc = gn % cr;
        v = P.Cpre[(int64_t)(ip * cl + a) * n_ + jp * cr + cc];
      }
      float ch, clo, dh, dlo;
      split_bits(v.x, ch, clo);
      split_bits(v.y, dh, dlo);
      float sh, se;
      two_sum(ch, dh, sh, se);
      Bcd[kk][c] = make_float4(ch, clo, dh, dlo);
      Bsum[kk][c] = make_float2(sh, se + (clo + dlo));
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < PJ_TK; ++kk) {
      float4 b[2];
      float2 bs[2];
      b[0] = Bcd[kk][tx]; b[1] = Bcd[kk][tx + 16];
      bs[0] = Bsum[kk][tx]; bs[1] = Bsum[kk][tx + 16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 ab = Aab[kk][ty + 16 * i];
        const float4 sd = Asd[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          dfx_dd(h1[i][j], l1[i][j], ab.x, ab.y, bs[j].x, bs[j].y);  // a (c + d)
          dfx_dd(h2[i][j], l2[i][j], b[j].z, b[j].w, sd.x, sd.y);    // d (a + b)
          dfx_dd(h3[i][j], l3[i][j], b[j].x, b[j].y, sd.z, sd.w);    // c (b - a)
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        fast2(h1[i][j], l1[i][j]);
        fast2(h2[i][j], l2[i][j]);
        fast2(h3[i][j], l3[i][j]);
      }
    __syncthreads();
  }
  cplx* th = const_cast<cplx*>(P.theta);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = tm + ty + 16 * i, c = tn + tx + 16 * j;
      if (r < M && c < N) {
        const int ii = r / dr, jj = r % dr, a = c / cr, cc = c % cr;
        const double t1 = (double)h1[i][j] + (double)l1[i][j];
        const double t2 = (double)h2[i][j] + (double)l2[i][j];
        const double t3 = (double)h3[i][j] + (double)l3[i][j];
        th[(int64_t)(ii * cl + a) * n_ + jj * cr + cc] = cmk(t1 - t2, t1 + t3);
      }
    }
}

cudaError_t launch_gate_gemm_df(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st) {
  const int M = cap.dl * cap.dr, N = cap.cl * cap.cr;
  if (M < GATE_GEMM_MIN) return cudaSuccess;
  ProfScope ps("k_gate_gemm_df", st);
  dim3 grid((N + PJ_TN - 1) / PJ_TN, (M + PJ_TM - 1) / PJ_TM, batch);
  k_gate_gemm_df<<<grid, 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

}  // namespace tg
