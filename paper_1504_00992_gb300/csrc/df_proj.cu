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
// double-float, c, d single floats, c + d a TwoSum pair.  K in slices of 16
// each closed by a renormalising Fast2Sum of the accumulators.
// Tiles: 64 rows x 8 CT columns per CTA of 128 threads, 4 x CT outputs per
// thread (CT = 4 or 5, whichever pads l less: 40-column tiles fit l = 120
// exactly); the wide per-thread tile halves the shared-memory loads per
// product against 4 x 2, and two CTAs share an SM (~254 registers each).
// ---------------------------------------------------------------------------
enum { PJ_TM = 64, PJ_TK = 16, PJ_BX = 8, PJ_BY = 16, PJ_NT = PJ_BX * PJ_BY, PJ_RT = PJ_TM / PJ_BY };

// thd and Q_f at capacity mc x nc and mc x lc per instance; the instance's
// own (m, n, l) from dims bound the sum and the output (D.n x D.l, compact).
template <int CT>
__global__ void __launch_bounds__(PJ_NT, 2) k_proj_df(const float4* __restrict__ thd, const float2* __restrict__ Qf,
                                                     const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                     int mc, int nc, int lc) {
  constexpr int TN = PJ_BX * CT;
  __shared__ float4 Aab[PJ_TK][PJ_TM];  // (a_h, a_l, b_h, b_l)
  __shared__ float4 Asd[PJ_TK][PJ_TM];  // (a+b)_h, (a+b)_l, (b-a)_h, (b-a)_l
  __shared__ float4 Bs[PJ_TK][TN + 1];  // (c, d, (c+d)_h, (c+d)_l); padded against bank conflicts
                                        // of the k-fastest stores
  const int z = blockIdx.z;
  const Dims Dm = dims[z];
  if (!Dm.active) return;
  const int m = Dm.m, n = Dm.n, l = Dm.l;
  const int tm = blockIdx.y * PJ_TM, tn = blockIdx.x * TN;
  if (tm >= n || tn >= l) return;
  const float4* th = thd + (size_t)z * mc * nc;
  const float2* q = Qf + (size_t)z * mc * lc;
  const int tid = threadIdx.x, tx = tid % PJ_BX, ty = tid / PJ_BX;
  float h1[PJ_RT][CT], l1[PJ_RT][CT], h2[PJ_RT][CT], l2[PJ_RT][CT], h3[PJ_RT][CT], l3[PJ_RT][CT];
#pragma unroll
  for (int i = 0; i < PJ_RT; ++i)
#pragma unroll
    for (int j = 0; j < CT; ++j) h1[i][j] = l1[i][j] = h2[i][j] = l2[i][j] = h3[i][j] = l3[i][j] = 0.f;
  for (int k0 = 0; k0 < m; k0 += PJ_TK) {
    // A^H tile: element (r, k) = conj(theta[k][r]), pre-split; consecutive
    // threads read consecutive r
    for (int e = tid; e < PJ_TM * PJ_TK; e += PJ_NT) {
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
    for (int e = tid; e < PJ_TK * TN; e += PJ_NT) {
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
      float4 b[CT];
#pragma unroll
      for (int j = 0; j < CT; ++j) b[j] = Bs[kk][tx + PJ_BX * j];
#pragma unroll
      for (int i = 0; i < PJ_RT; ++i) {
        const float4 ab = Aab[kk][ty + PJ_BY * i];
        const float4 sd = Asd[kk][ty + PJ_BY * i];
#pragma unroll
        for (int j = 0; j < CT; ++j) {
          dfx_dd(h1[i][j], l1[i][j], ab.x, ab.y, b[j].z, b[j].w);  // a (c + d)
          dfx_sd(h2[i][j], l2[i][j], b[j].y, sd.x, sd.y);          // d (a + b)
          dfx_sd(h3[i][j], l3[i][j], b[j].x, sd.z, sd.w);          // c (b - a)
        }
      }
    }
#pragma unroll
    for (int i = 0; i < PJ_RT; ++i)
#pragma unroll
      for (int j = 0; j < CT; ++j) {
        fast2(h1[i][j], l1[i][j]);
        fast2(h2[i][j], l2[i][j]);
        fast2(h3[i][j], l3[i][j]);
      }
    __syncthreads();
  }
  cplx* X = ptrs[z].Yt;  // n x l column-major
#pragma unroll
  for (int i = 0; i < PJ_RT; ++i)
#pragma unroll
    for (int j = 0; j < CT; ++j) {
      const int r = tm + ty + PJ_BY * i, c = tn + tx + PJ_BX * j;
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
    const int t32 = (l + 31) / 32, t40 = (l + 39) / 40;  // column tiles of 32 or 40: the smaller padding
    if (40 * t40 < 32 * t32)
      k_proj_df<5><<<dim3(t40, (n + PJ_TM - 1) / PJ_TM, batch), PJ_NT, 0, st>>>(thd, Qf, dims, ptrs, m, n, l);
    else
      k_proj_df<4><<<dim3(t32, (n + PJ_TM - 1) / PJ_TM, batch), PJ_NT, 0, st>>>(thd, Qf, dims, ptrs, m, n, l);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_fold_bh(Dbuf, dims, ptrs, n, l, batch, st);
}

}  // namespace tg
