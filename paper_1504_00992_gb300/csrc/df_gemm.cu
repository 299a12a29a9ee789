// Complex GEMMs of the bond update in double-float arithmetic on the FP32
// pipes (the TF32 form's counterparts of the FP64 kernels; sm_103a).
//
//   theta contraction (Eq. of the two-site wave function): for a bond whose
//     gate is applied as a GEMM, C = L R with
//       L[(i cl + a), g] = lam_l[a] Gamma_l[i][a][g] lam_m[g],
//       R[g, (j cr + c)] = Gamma_r[j][g][c] lam_r[c],
//     written to the pre-gate buffer Cpre (row-major, n = d_r cr columns);
//   gate: theta~[(i cl + a), (j cr + c)] =
//       sum_{i'j'} G[(i dr + j), (i' dr + j')] C[(i' cl + a), (j' cr + c)],
//     rows (i, j) of G times the (d_l d_r) x (cl cr) gather of C.
// Both: operands split at staging into FP32 pairs (integer bit operations;
// lam_m multiplies Gamma_r in FP64 first, lam_l lam_r scale the FP64 result
// in the epilogue), complex products by Gauss's
// rule with three double-float products (for alpha = a + ib, beta = c + id:
// t1 = a (c + d), t2 = d (a + b), t3 = c (b - a), Re = t1 - t2,
// Im = t1 + t3), 64 x 32 output tiles, 4 x 2 outputs per thread, K in slices
// of 16 closed by a renormalising Fast2Sum.  FP64-accurate (relative 2^-44
// per product), about 4x the FP64 pipe's rate.
#include <cuda_runtime.h>

#include "dfsplit.cuh"
#include "internal.cuh"
#include "profiler.cuh"

namespace tg {

enum { DG_TM = 64, DG_TN = 32, DG_TK = 16 };

// Operand access.  Each thread stages the same rows of A and the same column
// of B in every K slice, so the index arithmetic of a row or column is done
// once: A rows are contiguous in k (a_row), B columns are addressed from a
// per-column base (b_col) plus a per-k offset (b_at).

// Operands of the gate GEMM (bonds with Cpre set).
struct DgGate {
  __device__ static int rows(const Dims& D) { return D.dl * D.dr; }
  __device__ static int cols(const Dims& D) { return D.cl * D.cr; }
  __device__ static int depth(const Dims& D) { return D.dl * D.dr; }
  __device__ static const cplx* a_row(const Dims& D, const ProbPtr& P, int r) {
    return P.gate + (int64_t)r * (D.dl * D.dr);
  }
  __device__ static int64_t b_col(const Dims& D, const ProbPtr& P, int c) {
    return (int64_t)(c / D.cr) * D.n + c % D.cr;  // (alpha, beta) -> alpha n + beta
  }
  __device__ static cplx b_at(const Dims& D, const ProbPtr& P, int64_t cb, int k) {
    const int ip = k / D.dr, jp = k - ip * D.dr;  // k = (i', j')
    return P.Cpre[cb + (int64_t)ip * D.cl * D.n + jp * D.cr];
  }
  __device__ static void store(const Dims& D, const ProbPtr& P, int r, int c, cplx v) {
    const int i = r / D.dr, j = r % D.dr, al = c / D.cr, be = c % D.cr;
    const_cast<cplx*>(P.theta)[(int64_t)(i * D.cl + al) * D.n + j * D.cr + be] = v;
  }
};

// Operands of the theta contraction into Cpre: A = Gamma_l (rows (i, alpha)),
// B = lam_m Gamma_r (columns (j, beta)); lam_l[alpha] lam_r[beta] scale the
// result in the epilogue.
struct DgTheta {
  __device__ static int rows(const Dims& D) { return D.dl * D.cl; }
  __device__ static int cols(const Dims& D) { return D.dr * D.cr; }
  __device__ static int depth(const Dims& D) { return D.cm; }
  __device__ static const cplx* a_row(const Dims& D, const ProbPtr& P, int r) {
    const int i = r / D.cl, al = r - i * D.cl;
    return P.gl + ((int64_t)i * P.cap_l + al) * P.cap_m;
  }
  __device__ static int64_t b_col(const Dims& D, const ProbPtr& P, int c) {
    const int j = c / D.cr, be = c - j * D.cr;
    return (int64_t)j * P.cap_m * P.cap_r + be;
  }
  __device__ static cplx b_at(const Dims& D, const ProbPtr& P, int64_t cb, int g) {
    return cscale(P.gr[cb + (int64_t)g * P.cap_r], P.lamm[g]);
  }
  __device__ static void store(const Dims& D, const ProbPtr& P, int r, int c, cplx v) {
    P.Cpre[(int64_t)r * D.n + c] = cscale(v, P.laml[r % D.cl] * P.lamr[c % D.cr]);
  }
};

template <class Op>
__global__ void __launch_bounds__(256) k_cgemm_df(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  __shared__ float4 Aab[DG_TK][DG_TM];      // (a_h, a_l, b_h, b_l)
  __shared__ float4 Asd[DG_TK][DG_TM];      // (a+b)_h, (a+b)_l, (b-a)_h, (b-a)_l
  __shared__ float4 Bcd[DG_TK][DG_TN + 1];  // (c_h, c_l, d_h, d_l)
  __shared__ float2 Bsum[DG_TK][DG_TN + 1]; // (c+d)_h, (c+d)_l
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  if (!P.Cpre) return;
  const int M = Op::rows(D), N = Op::cols(D), K = Op::depth(D);
  const int tm = blockIdx.y * DG_TM, tn = blockIdx.x * DG_TN;
  if (tm >= M || tn >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // staging assignment: A elements (kk = tid % 16, rows tid / 16 + 16 t),
  // B elements (column tid % 32, kk = tid / 32 + 8 t)
  constexpr int AT = DG_TM * DG_TK / 256, BT = DG_TK * DG_TN / 256;
  const int akk = tid % DG_TK, bc = tid % DG_TN;
  const cplx* arow[AT];
#pragma unroll
  for (int t = 0; t < AT; ++t) {
    const int gr = tm + tid / DG_TK + (256 / DG_TK) * t;
    arow[t] = (gr < M) ? Op::a_row(D, P, gr) : nullptr;
  }
  const int gn = tn + bc;
  const int64_t bcol = (gn < N) ? Op::b_col(D, P, gn) : 0;
  float h1[4][2], l1[4][2], h2[4][2], l2[4][2], h3[4][2], l3[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) h1[i][j] = l1[i][j] = h2[i][j] = l2[i][j] = h3[i][j] = l3[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += DG_TK) {
#pragma unroll
    for (int t = 0; t < AT; ++t) {  // A tile: consecutive threads along k
      const int r = tid / DG_TK + (256 / DG_TK) * t, gk = k0 + akk;
      cplx v = cmk(0.0, 0.0);
      if (arow[t] && gk < K) v = arow[t][gk];
      float ah, al, bh, bl;
      split_bits(v.x, ah, al);
      split_bits(v.y, bh, bl);
      float sh, se, dh, de;
      two_sum(ah, bh, sh, se);
      two_sum(bh, -ah, dh, de);
      Aab[akk][r] = make_float4(ah, al, bh, bl);
      Asd[akk][r] = make_float4(sh, se + (al + bl), dh, de + (bl - al));
    }
#pragma unroll
    for (int t = 0; t < BT; ++t) {  // B tile: consecutive threads along the columns
      const int kk = tid / DG_TN + (256 / DG_TN) * t, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gn < N && gk < K) v = Op::b_at(D, P, bcol, gk);
      float ch, clo, dh, dlo;
      split_bits(v.x, ch, clo);
      split_bits(v.y, dh, dlo);
      float sh, se;
      two_sum(ch, dh, sh, se);
      Bcd[kk][bc] = make_float4(ch, clo, dh, dlo);
      Bsum[kk][bc] = make_float2(sh, se + (clo + dlo));
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < DG_TK; ++kk) {
      float4 b[2];
      float2 bs[2];
      b[0] = Bcd[kk][tx];
      b[1] = Bcd[kk][tx + 16];
      bs[0] = Bsum[kk][tx];
      bs[1] = Bsum[kk][tx + 16];
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
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = tm + ty + 16 * i, c = tn + tx + 16 * j;
      if (r < M && c < N) {
        const double t1 = (double)h1[i][j] + (double)l1[i][j];
        const double t2 = (double)h2[i][j] + (double)l2[i][j];
        const double t3 = (double)h3[i][j] + (double)l3[i][j];
        Op::store(D, P, r, c, cmk(t1 - t2, t1 + t3));
      }
    }
}

cudaError_t launch_gate_gemm_df(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st) {
  const int M = cap.dl * cap.dr, N = cap.cl * cap.cr;
  if (M < GATE_GEMM_MIN) return cudaSuccess;
  ProfScope ps("k_gate_gemm_df", st);
  dim3 grid((N + DG_TN - 1) / DG_TN, (M + DG_TM - 1) / DG_TM, batch);
  k_cgemm_df<DgGate><<<grid, 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

cudaError_t launch_theta_df(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st) {
  if (cap.dl * cap.dr < GATE_GEMM_MIN) return cudaSuccess;
  const int M = cap.dl * cap.cl, N = cap.dr * cap.cr;
  ProfScope ps("k_theta_df", st);
  dim3 grid((N + DG_TN - 1) / DG_TN, (M + DG_TM - 1) / DG_TM, batch);
  k_cgemm_df<DgTheta><<<grid, 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

}  // namespace tg
