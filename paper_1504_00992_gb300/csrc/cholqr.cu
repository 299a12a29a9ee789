// Cholesky QR of B^H for the mixed form (sm_103a): the QR factorisation the
// small-B SVD of Section IV's step ii starts from (B^H = Qb Rb, then the
// one-sided Jacobi SVD of Rb^H), for well-conditioned B.
//
// CholeskyQR2 (Yamamoto, Nakatsukasa, Yanagisawa, Fukaya, ETNA 44, 2015):
//   G1 = B B^H = R1^H R1,  Q1 = B^H R1^-1,
//   G2 = Q1^H Q1 = R2^H R2, Qb = Q1 R2^-1,
// with the Gram matrices and the triangular products FP64-accurate (on the
// tensor cores from exact digit splits, k_oz_gemm, or in double-float
// arithmetic, k_zgemm_df; stages G_G1 .. G_X) and the Cholesky
// factorisations and triangular inverses in FP64 here.  For kappa(B) below
// ~1e8 the two passes give an orthonormal Qb and a backward-stable
// factorisation (residual and orthogonality at the unit-roundoff level), so
// the singular values of Rb are those of B to ~eps ||B||.  Rb^H is formed as
// X = B Qb.  An instance whose first Gram matrix is too ill-conditioned for
// that (a Cholesky pivot below CQ_PIVOT times the largest diagonal entry,
// i.e. kappa(B) above ~1e5) is flagged (Dims::qflag) and factored by the
// Householder QR instead; its Cholesky output is replaced by the identity so
// that the products in between stay finite.
#include <cuda_runtime.h>
#include <math.h>

#include "dfsplit.cuh"
#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"

namespace tg {

static const double CQ_PIVOT = 1e-10;

// Cholesky G = R^H R of the l x l Hermitian matrix in P.R (upper triangle,
// column-major, in place), then J = R^-1 (upper triangular, zero below).  One
// CTA per instance.  pass 0 sets dims[p].qflag to 0 or 1; pass 1 skips the
// instances already flagged and flags those whose second Gram fails.
__global__ void __launch_bounds__(256) k_chol_inv(Dims* dims, const ProbPtr* __restrict__ ptrs, int pass) {
  __shared__ double red[32];
  __shared__ double s_inv;
  __shared__ int s_fail;
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  if (pass == 1 && D.qflag) return;
  const ProbPtr P = ptrs[p];
  const int L = D.l, tid = threadIdx.x;
  cplx* G = P.R;
  cplx* J = P.J;
  double dm = 0.0;
  for (int j = tid; j < L; j += blockDim.x) dm = fmax(dm, G[(size_t)j * L + j].x);
  // block maximum through the sum helper's pattern
  {
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) red[warp] = dm;
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
      red[0] = m;
      s_fail = !(m > 0.0) || !isfinite(m);
    }
    __syncthreads();
    dm = red[0];
  }
  for (int j = 0; j < L && !s_fail; ++j) {
    if (tid == 0) {
      const double d = G[(size_t)j * L + j].x;
      if (!(d > CQ_PIVOT * dm) || !isfinite(d)) {
        s_fail = 1;
      } else {
        const double r = sqrt(d);
        G[(size_t)j * L + j] = cmk(r, 0.0);
        s_inv = 1.0 / r;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double inv = s_inv;
    for (int c = j + 1 + tid; c < L; c += blockDim.x) G[(size_t)c * L + j] = cscale(G[(size_t)c * L + j], inv);
    __syncthreads();
    // trailing update of the upper triangle: G[c1][c2] -= conj(R[j][c1]) R[j][c2], j < c1 <= c2
    const int w = L - j - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int c1 = j + 1 + e % w, c2 = j + 1 + e / w;
      if (c1 > c2) continue;
      const cplx a = G[(size_t)c1 * L + j], b = G[(size_t)c2 * L + j];
      cplx& g = G[(size_t)c2 * L + c1];
      g.x -= a.x * b.x + a.y * b.y;
      g.y -= a.x * b.y - a.y * b.x;
    }
    __syncthreads();
  }
  const int fail = s_fail;
  if (tid == 0) dims[p].qflag = fail ? 1 : (pass == 0 ? 0 : D.qflag);
  if (fail) {  // identity factor: the products in between stay finite
    for (int e = tid; e < L * L; e += blockDim.x) J[e] = cmk((e / L) == (e % L) ? 1.0 : 0.0, 0.0);
    return;
  }
  // J = R^-1 by back substitution, one column per thread: R x = e_c
  for (int c = tid; c < L; c += blockDim.x) {
    cplx* x = J + (size_t)c * L;
    for (int i = c + 1; i < L; ++i) x[i] = cmk(0.0, 0.0);
    for (int i = c; i >= 0; --i) {
      cplx s = cmk(i == c ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= c; ++k) {
        const cplx r = G[(size_t)k * L + i], v = x[k];
        s.x -= r.x * v.x - r.y * v.y;
        s.y -= r.x * v.y + r.y * v.x;
      }
      const double rii = G[(size_t)i * L + i].x;  // real and positive
      x[i] = cscale(s, 1.0 / rii);
    }
  }
}

// The same factorisation in double-float arithmetic (FP32 pairs, 2^-48;
// the FP32 pipe runs 64x the FP64 one) with the Gram's upper triangle packed
// in shared memory (element (r, c), r <= c, at c (c + 1) / 2 + r) for
// l <= CS_MAXL, then R^-1 in place, column by column (R X = I):
//   X[j][j] = 1 / R[j][j],  X[0:j, j] = -X[j][j] X[0:j, 0:j] R[0:j, j],
// the leading block X[0:j, 0:j] being the columns already inverted; each
// column's j dot products run on the threads (row r: sum over k = r .. j-1),
// into scratch first (they read the column they replace).  The trailing
// updates of the factorisation enumerate the packed pairs c1 <= c2 directly,
// so every lane does work.  G is scaled by a power of four first, so that its
// largest diagonal entry lies in [0.5, 4), and R^-1 scaled back.
enum { CS_THREADS = 256, CS_MAXL = 160 };

__host__ __device__ inline size_t cs_smem_bytes(int L) { return ((size_t)L * (L + 1) / 2 + L) * sizeof(cplx); }

__device__ __forceinline__ int cs_at(int r, int c) { return c * (c + 1) / 2 + r; }

// (a, b) with a <= b from the packed index e = b (b + 1) / 2 + a
__device__ __forceinline__ void cs_pair(int e, int& a, int& b) {
  int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if ((c + 1) * (c + 2) / 2 <= e) ++c;
  if (c * (c + 1) / 2 > e) --c;
  b = c;
  a = e - c * (c + 1) / 2;
}

// Complex double-float entry: (Re hi, Re lo, Im hi, Im lo).
__device__ __forceinline__ float4 cs_split(cplx v) {
  float4 d;
  split_bits(v.x, d.x, d.y);
  split_bits(v.y, d.z, d.w);
  return d;
}

__global__ void __launch_bounds__(CS_THREADS) k_chol_inv_sm(Dims* dims, const ProbPtr* __restrict__ ptrs, int pass) {
  extern __shared__ __align__(16) unsigned char cs_raw[];
  __shared__ double red[32];
  __shared__ float2 s_inv;
  __shared__ int s_fail;
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  if (pass == 1 && D.qflag) return;
  const ProbPtr P = ptrs[p];
  const int L = D.l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = CS_THREADS / 32;
  float4* T = reinterpret_cast<float4*>(cs_raw);
  float4* tmp = T + (size_t)L * (L + 1) / 2;  // L
  const cplx* G = P.R;
  cplx* J = P.J;
  // the largest diagonal entry, then G scaled by 2^-2s (exact) to bring it
  // into [0.5, 4): FP32's range holds the factor, R^-1 is scaled back by 2^s
  double dm = 0.0;
  for (int c = tid; c < L; c += CS_THREADS) dm = fmax(dm, G[(size_t)c * L + c].x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if (lane == 0) red[warp] = dm;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
    red[0] = m;
    s_fail = !(m > 0.0) || !isfinite(m);
  }
  __syncthreads();
  dm = red[0];
  int ex = 0;
  if (!s_fail) (void)frexp(dm, &ex);  // dm = f 2^ex, f in [0.5, 1)
  const int sh = ex >> 1;             // scale G by 2^-2 sh
  const double gsc = ldexp(1.0, -2 * sh);
  for (int e = tid; e < L * L; e += CS_THREADS) {
    const int r = e % L, c = e / L;
    if (r <= c) T[cs_at(r, c)] = cs_split(cscale(G[(size_t)c * L + r], gsc));
  }
  const float piv = (float)(CQ_PIVOT * dm * gsc);
  __syncthreads();
  for (int j = 0; j < L && !s_fail; ++j) {
    if (tid == 0) {
      const float4 dd = T[cs_at(j, j)];
      const dfl d{dd.x, dd.y};
      if (!(d.h > piv) || !isfinite(d.h)) {
        s_fail = 1;
      } else {
        const dfl r = dsqrt(d);
        const dfl inv = drecip(r);
        T[cs_at(j, j)] = make_float4(r.h, r.l, 0.f, 0.f);
        s_inv = make_float2(inv.h, inv.l);
      }
    }
    __syncthreads();
    if (s_fail) break;
    const dfl inv{s_inv.x, s_inv.y};
    for (int c = j + 1 + tid; c < L; c += CS_THREADS) {
      const float4 v = T[cs_at(j, c)];
      const dfl re = dmul(dfl{v.x, v.y}, inv), im = dmul(dfl{v.z, v.w}, inv);
      T[cs_at(j, c)] = make_float4(re.h, re.l, im.h, im.l);
    }
    __syncthreads();
    // G[c1][c2] -= conj(R[j][c1]) R[j][c2], j < c1 <= c2: the packed pairs of the trailing block
    const int w = L - j - 1, j1 = j + 1;
    for (int e = tid; e < w * (w + 1) / 2; e += CS_THREADS) {
      int a, b;
      cs_pair(e, a, b);
      const int c1 = j1 + a, c2 = j1 + b;
      const float4 x = T[cs_at(j, c1)], y = T[cs_at(j, c2)];
      float4& g = T[cs_at(c1, c2)];
      // Re -= xr yr + xi yi, Im -= xr yi - xi yr
      float rh = g.x, rl = g.y, ih = g.z, il = g.w;
      dfx_dd(rh, rl, -x.x, -x.y, y.x, y.y);
      dfx_dd(rh, rl, -x.z, -x.w, y.z, y.w);
      dfx_dd(ih, il, -x.x, -x.y, y.z, y.w);
      dfx_dd(ih, il, x.z, x.w, y.x, y.y);
      fast2(rh, rl);
      fast2(ih, il);
      g = make_float4(rh, rl, ih, il);
    }
    __syncthreads();
  }
  const int fail = s_fail;
  if (tid == 0) dims[p].qflag = fail ? 1 : (pass == 0 ? 0 : D.qflag);
  if (fail) {  // identity factor: the products in between stay finite
    for (int e = tid; e < L * L; e += CS_THREADS) J[e] = cmk((e / L) == (e % L) ? 1.0 : 0.0, 0.0);
    return;
  }
  // R^-1 in place
  for (int j = 0; j < L; ++j) {
    for (int r = tid; r < j; r += CS_THREADS) {
      float sh_ = 0.f, sl = 0.f, th = 0.f, tl = 0.f;  // Re, Im of sum_k X[r][k] R[k][j]
      for (int k = r; k < j; ++k) {
        const float4 x = T[cs_at(r, k)], u = T[cs_at(k, j)];
        dfx_dd(sh_, sl, x.x, x.y, u.x, u.y);
        dfx_dd(sh_, sl, -x.z, -x.w, u.z, u.w);
        dfx_dd(th, tl, x.x, x.y, u.z, u.w);
        dfx_dd(th, tl, x.z, x.w, u.x, u.y);
      }
      fast2(sh_, sl);
      fast2(th, tl);
      tmp[r] = make_float4(sh_, sl, th, tl);
    }
    __syncthreads();
    const float4 djj = T[cs_at(j, j)];
    const dfl dj = drecip(dfl{djj.x, djj.y});
    for (int r = tid; r <= j; r += CS_THREADS) {
      if (r == j) {
        T[cs_at(j, j)] = make_float4(dj.h, dj.l, 0.f, 0.f);
      } else {
        const float4 v = tmp[r];
        const dfl re = dmul(dfl{v.x, v.y}, dneg(dj)), im = dmul(dfl{v.z, v.w}, dneg(dj));
        T[cs_at(r, j)] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
    __syncthreads();
  }
  const double back = ldexp(1.0, -sh);  // R^-1 of the unscaled G = 2^-s R'^-1
  for (int e = tid; e < L * L; e += CS_THREADS) {
    const int r = e % L, c = e / L;
    cplx v = cmk(0.0, 0.0);
    if (r <= c) {
      const float4 t = T[cs_at(r, c)];
      v = cmk(((double)t.x + (double)t.y) * back, ((double)t.z + (double)t.w) * back);
    }
    J[e] = v;
  }
}

cudaError_t cholqr_prepare() {
  static int done = 0;
  if (!done) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_chol_inv_sm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs_smem_bytes(CS_MAXL));
    if (e != cudaSuccess) return e;
    done = 1;
  }
  return cudaSuccess;
}

static cudaError_t chol_inv(Dims* dims, const ProbPtr* ptrs, int batch, int lcap, int pass, cudaStream_t st) {
  ProfScope ps("k_chol_inv", st);
  if (lcap <= CS_MAXL) {
    const cudaError_t e = cholqr_prepare();
    if (e != cudaSuccess) return e;
    k_chol_inv_sm<<<batch, CS_THREADS, cs_smem_bytes(lcap), st>>>(dims, ptrs, pass);
  } else {
    k_chol_inv<<<batch, 256, 0, st>>>(dims, ptrs, pass);
  }
  return cudaGetLastError();
}

#define CQ_TRY(x)                     \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

cudaError_t run_cholqr_bh(Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st,
                          const OzScratch* oz, int* err) {
  auto gemm = [&](int stage) {
    return oz ? launch_oz_stage(stage, dims, ptrs, batch, cap, *oz, err, st)
              : launch_zgemm_df(stage, dims, ptrs, batch, cap, st);
  };
  CQ_TRY(gemm(G_G1));                          // G1 = B B^H
  CQ_TRY(chol_inv(dims, ptrs, batch, cap.l, 0, st));  // R1, J = R1^-1
  CQ_TRY(gemm(G_Q1));                          // Q1 = B^H R1^-1
  CQ_TRY(gemm(G_G2));                          // G2 = Q1^H Q1
  CQ_TRY(chol_inv(dims, ptrs, batch, cap.l, 1, st));  // R2, J = R2^-1
  CQ_TRY(gemm(G_QB));                          // Qb = Q1 R2^-1
  CQ_TRY(gemm(G_X));                           // X = B Qb = Rb^H
  // ill-conditioned instances: Householder QR of B^H (overwrites X and Qb)
  return launch_qr(QR_BH, dims, ptrs, batch, st, 1);
}

}  // namespace tg
