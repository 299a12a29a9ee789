// RRSVD kernels, plain FP64 (sm_103a).
//
// Section IV of the paper: Alg. 1 (Gaussian sketch Y0 = A Omega, QR, and q
// power iterations A^H Q -> QR -> A Q~ -> QR) followed by B = Q^H A, the SVD
// of the small B and U = Q U~.  B is formed as its adjoint B^H = A^H Q
// (n x l); the SVD of B comes from the QR factorisation B^H = Qb Rb followed
// by a one-sided Jacobi SVD of Rb^H (Rb^H J = W S): then U~ = W and V = Qb J.
//
// On GB300 FP64 runs at about 1 TFLOP/s for the whole chip (2 FMA per clock
// per SM), so every FP64 kernel here is bound by the FP64 pipe; the designs
// spread independent work over as many SMs as possible rather than chase
// memory reuse.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "profiler.cuh"
#include "dfsplit.cuh"

namespace tg {

// ---------------------------------------------------------------------------
// Omega: n x l complex Gaussian, column-major; element (r, c) uses Philox
// counter (r*l + c, bond, sweep, chain).
// ---------------------------------------------------------------------------
__global__ void k_omega(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs, uint64_t seed,
                        uint64_t sweep, int64_t chain0, int chain_stride, const uint64_t* sweep_dev) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  cplx* om = ptrs[p].omega;
  const int64_t total = (int64_t)D.n * D.l;
  const uint64_t chain = chain_stride >= 0 ? (uint64_t)(chain0 + (int64_t)p * chain_stride) : (uint64_t)D.chain;
  if (sweep_dev) sweep = *sweep_dev;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / D.l), c = (int)(e % D.l);
    om[(int64_t)c * D.n + r] = gauss_c((uint64_t)e, (uint64_t)D.bond, sweep, chain, seed, 0);
  }
}

cudaError_t launch_omega(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, uint64_t seed,
                         uint64_t sweep, int64_t chain0, int chain_stride, cudaStream_t st,
                         const uint64_t* sweep_dev) {
  const int64_t total = (int64_t)cap.n * cap.l;
  int bx = (int)((total + 255) / 256);
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  ProfScope ps("k_omega", st);
  k_omega<<<dim3(bx, batch), 256, 0, st>>>(dims, ptrs, seed, sweep, chain0, chain_stride, sweep_dev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched complex GEMM C = op(A) op(B), FP64.
// Operands are addressed by (row stride, column stride) so the same kernel
// serves row- and column-major buffers; loads map consecutive threads onto the
// unit-stride direction.
// ---------------------------------------------------------------------------
struct GemmOp {
  int M, N, K;
  const cplx* A; int64_t ars, acs;
  const cplx* B; int64_t brs, bcs;
  cplx* C; int64_t crs, ccs;
};

template <int STAGE>
__device__ __forceinline__ GemmOp gemm_of(const Dims& D, const ProbPtr& P) {
  GemmOp g;
  if (STAGE == G_Y0 || STAGE == G_Y) {  // Y = A Omega  /  Y = A Q~   (m x l, column-major)
    g.M = D.m; g.N = D.l; g.K = D.n;
    g.A = P.theta; g.ars = D.n; g.acs = 1;
    g.B = (STAGE == G_Y0) ? P.omega : P.Qt; g.brs = 1; g.bcs = D.n;
    g.C = P.Y; g.crs = 1; g.ccs = D.m;
  } else if (STAGE == G_YT || STAGE == G_BH) {  // Y~ = A^H Q (n x l, column-major)
    g.M = D.n; g.N = D.l; g.K = D.m;
    g.A = P.theta; g.ars = 1; g.acs = D.n;       // op(A)(r, k) = conj(A[k][r])
    g.B = P.Q; g.brs = 1; g.bcs = D.m;
    g.C = P.Yt; g.crs = 1; g.ccs = D.n;
  } else if (STAGE == G_U) {  // U = Q Jk (m x k, row-major)
    g.M = D.m; g.N = D.k; g.K = D.l;
    g.A = P.Q; g.ars = 1; g.acs = D.m;
    g.B = P.Jk; g.brs = 1; g.bcs = D.l;
    g.C = P.U; g.crs = D.k; g.ccs = 1;
  } else if (STAGE == G_V) {  // V = Qb Wk, stored conjugated as Vh (k x n, row-major)
    g.M = D.n; g.N = D.k; g.K = D.l;
    g.A = P.Qt; g.ars = 1; g.acs = D.n;
    g.B = P.Wk; g.brs = 1; g.bcs = D.l;
    g.C = P.V; g.crs = 1; g.ccs = D.n;
  } else if (STAGE == G_PR) {  // Br = A Omega_r -> columns l .. l+r-1 of Y (m x r)
    g.M = D.m; g.N = D.r; g.K = D.n;
    g.A = P.theta; g.ars = D.n; g.acs = 1;
    g.B = P.omega; g.brs = 1; g.bcs = D.n;
    g.C = P.Y + (int64_t)D.l * D.m; g.crs = 1; g.ccs = D.m;
  } else if (STAGE == G_PQ) {  // C1 = Q^H Br (l x r, column-major in R)
    g.M = D.l; g.N = D.r; g.K = D.m;
    g.A = P.Q; g.ars = D.m; g.acs = 1;          // op(A)(i, k) = conj(Q[k][i])
    g.B = P.Y + (int64_t)D.l * D.m; g.brs = 1; g.bcs = D.m;
    g.C = P.R; g.crs = 1; g.ccs = D.l;
  } else {  // G_PD: Dr = Q C1 (m x r)
    g.M = D.m; g.N = D.r; g.K = D.l;
    g.A = P.Q; g.ars = 1; g.acs = D.m;
    g.B = P.R; g.brs = 1; g.bcs = D.l;
    g.C = P.Dr; g.crs = 1; g.ccs = D.m;
  }
  return g;
}

template <int STAGE>
struct StageFlags {
  static constexpr bool conjA = (STAGE == G_YT || STAGE == G_BH || STAGE == G_PQ);
  static constexpr bool conjC = (STAGE == G_V);
};

template <int T, int STAGE>
__global__ void __launch_bounds__(256) k_zgemm(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  constexpr int TK = 16;
  constexpr int S = T / 16;  // outputs per thread along each direction
  __shared__ cplx As[TK][T + 1];
  __shared__ cplx Bs[TK][T + 1];
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  if ((STAGE == G_PR || STAGE == G_PQ || STAGE == G_PD) && !D.chk) return;
  const GemmOp g = gemm_of<STAGE>(D, ptrs[p]);
  const int tm = blockIdx.y * T, tn = blockIdx.x * T;
  if (tm >= g.M || tn >= g.N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool ccol = (g.crs == 1);
  cplx acc[S][S];
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < S; ++j) acc[i][j] = cmk(0.0, 0.0);

  for (int k0 = 0; k0 < g.K; k0 += TK) {
    // A tile: op(A)(tm + r, k0 + kk) -> As[kk][r]
    for (int e = tid; e < T * TK; e += 256) {
      int r, kk;
      if (g.acs == 1) { kk = e % TK; r = e / TK; } else { r = e % T; kk = e / T; }
      const int gr = tm + r, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gr < g.M && gk < g.K) {
        v = g.A[(int64_t)gr * g.ars + (int64_t)gk * g.acs];
        if (StageFlags<STAGE>::conjA) v.y = -v.y;
      }
      As[kk][r] = v;
    }
    // B tile: B(k0 + kk, tn + c) -> Bs[kk][c]
    for (int e = tid; e < T * TK; e += 256) {
      int c, kk;
      if (g.brs == 1) { kk = e % TK; c = e / TK; } else { c = e % T; kk = e / T; }
      const int gc = tn + c, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gc < g.N && gk < g.K) v = g.B[(int64_t)gk * g.brs + (int64_t)gc * g.bcs];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      cplx a[S], b[S];
#pragma unroll
      for (int i = 0; i < S; ++i) a[i] = As[kk][(ccol ? tx : ty) + 16 * i];
#pragma unroll
      for (int j = 0; j < S; ++j) b[j] = Bs[kk][(ccol ? ty : tx) + 16 * j];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const int r = tm + (ccol ? tx : ty) + 16 * i, c = tn + (ccol ? ty : tx) + 16 * j;
      if (r < g.M && c < g.N) {
        cplx v = acc[i][j];
        if (StageFlags<STAGE>::conjC) v.y = -v.y;
        g.C[(int64_t)r * g.crs + (int64_t)c * g.ccs] = v;
      }
    }
}

template <int STAGE>
static cudaError_t launch_zgemm_stage(int rows, int cols, const Dims* dims, const ProbPtr* ptrs, int batch,
                                     cudaStream_t st, int tile = 0) {
  // Default: 32x32 tiles when they already give two CTAs per SM; otherwise
  // 16x16 tiles spread small problems over more SMs.  tile = 16 / 32 forces.
  const int t32 = ((rows + 31) / 32) * ((cols + 31) / 32) * batch;
  if (tile == 32 || (tile == 0 && t32 >= 2 * 152)) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
    k_zgemm<32, STAGE><<<grid, 256, 0, st>>>(dims, ptrs);
  } else {
    dim3 grid((cols + 15) / 16, (rows + 15) / 16, batch);
    k_zgemm<16, STAGE><<<grid, 256, 0, st>>>(dims, ptrs);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Double-float ("FP64-accurate on FP32 pipes") batched complex GEMM, same
// stages and layouts as k_zgemm.  Every FP64 input x is split at staging into
// a pair hi + lo of FP32 numbers (48 significant bits); each real product
// x y is formed error-free up to the cross terms, p = xh yh exactly split by
// FMA into (ph, pe), plus xh yl + xl yh; sums use Knuth's TwoSum on the high
// parts with the error terms gathered in a low accumulator (Dekker 1971;
// Knuth TAOCP vol. 2, 4.2.2); every 16-deep slice of the sum is accumulated
// afresh and merged with a renormalising add, which keeps the error near u^2
// (~1e-14 relative) instead of K u^2.  GB300 runs FP32 at 64x its FP64 rate,
// so this is several times faster than DFMA.
// ---------------------------------------------------------------------------
struct df2 { float h, l; };

// hi = x truncated to 24 bits, lo = the rest (integer and FP32 operations
// only: conversions through the FP64 pipe would cost half its throughput)
__device__ __forceinline__ void df_split(double x, float& h, float& l) { split_bits(x, h, l); }

// acc += x * y   (x, y double-float, acc double-float)
__device__ __forceinline__ void df_fma(df2& acc, float xh, float xl, float yh, float yl) {
  const float ph = xh * yh;
  const float pe = fmaf(xh, yh, -ph);
  const float pc = fmaf(xh, yl, xl * yh);
  const float t = acc.h + ph;
  const float z = t - acc.h;
  const float e = (acc.h - (t - z)) + (ph - z);
  acc.h = t;
  acc.l += e + pe + pc;
}

// acc += part, renormalised (Dekker's add), so the low word stays below one
// ulp of the high word over long sums.
__device__ __forceinline__ void df_merge(df2& acc, df2 part) {
  const float s = acc.h + part.h;
  const float v = s - acc.h;
  float e = (acc.h - (s - v)) + (part.h - v);
  e += acc.l + part.l;
  acc.h = s + e;
  acc.l = e - (acc.h - s);
}

template <int STAGE>
__global__ void __launch_bounds__(256) k_zgemm_df(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  constexpr int T = 32, TK = 16, S = 2;
  __shared__ float4 As[TK][T + 1];   // (re_hi, re_lo, im_hi, im_lo)
  __shared__ float4 Bs[TK][T + 1];
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  if ((STAGE == G_PR || STAGE == G_PQ || STAGE == G_PD) && !D.chk) return;
  const GemmOp g = gemm_of<STAGE>(D, ptrs[p]);
  const int tm = blockIdx.y * T, tn = blockIdx.x * T;
  if (tm >= g.M || tn >= g.N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool ccol = (g.crs == 1);
  df2 ar[S][S], ai[S][S];
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < S; ++j) { ar[i][j] = {0.f, 0.f}; ai[i][j] = {0.f, 0.f}; }
  for (int k0 = 0; k0 < g.K; k0 += TK) {
    for (int e = tid; e < T * TK; e += 256) {
      int r, kk;
      if (g.acs == 1) { kk = e % TK; r = e / TK; } else { r = e % T; kk = e / T; }
      const int gr = tm + r, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gr < g.M && gk < g.K) {
        v = g.A[(int64_t)gr * g.ars + (int64_t)gk * g.acs];
        if (StageFlags<STAGE>::conjA) v.y = -v.y;
      }
      float4 f;
      df_split(v.x, f.x, f.y);
      df_split(v.y, f.z, f.w);
      As[kk][r] = f;
    }
    for (int e = tid; e < T * TK; e += 256) {
      int c, kk;
      if (g.brs == 1) { kk = e % TK; c = e / TK; } else { c = e % T; kk = e / T; }
      const int gc = tn + c, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gc < g.N && gk < g.K) v = g.B[(int64_t)gk * g.brs + (int64_t)gc * g.bcs];
      float4 f;
      df_split(v.x, f.x, f.y);
      df_split(v.y, f.z, f.w);
      Bs[kk][c] = f;
    }
    __syncthreads();
    // each TK-deep slice is summed afresh and merged into the running sums
    df2 pr[S][S], pi[S][S];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S; ++j) { pr[i][j] = {0.f, 0.f}; pi[i][j] = {0.f, 0.f}; }
#pragma unroll 2
    for (int kk = 0; kk < TK; ++kk) {
      float4 a[S], b[S];
#pragma unroll
      for (int i = 0; i < S; ++i) a[i] = As[kk][(ccol ? tx : ty) + 16 * i];
#pragma unroll
      for (int j = 0; j < S; ++j) b[j] = Bs[kk][(ccol ? ty : tx) + 16 * j];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) {
          // re += ar br - ai bi ; im += ar bi + ai br
          df_fma(pr[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
          df_fma(pr[i][j], -a[i].z, -a[i].w, b[j].z, b[j].w);
          df_fma(pi[i][j], a[i].x, a[i].y, b[j].z, b[j].w);
          df_fma(pi[i][j], a[i].z, a[i].w, b[j].x, b[j].y);
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S; ++j) {
        df_merge(ar[i][j], pr[i][j]);
        df_merge(ai[i][j], pi[i][j]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const int r = tm + (ccol ? tx : ty) + 16 * i, c = tn + (ccol ? ty : tx) + 16 * j;
      if (r < g.M && c < g.N) {
        cplx v = cmk((double)ar[i][j].h + (double)ar[i][j].l, (double)ai[i][j].h + (double)ai[i][j].l);
        if (StageFlags<STAGE>::conjC) v.y = -v.y;
        g.C[(int64_t)r * g.crs + (int64_t)c * g.ccs] = v;
      }
    }
}

template <int STAGE>
static cudaError_t launch_zgemm_df_stage(int rows, int cols, const Dims* dims, const ProbPtr* ptrs, int batch,
                                        cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch);
  k_zgemm_df<STAGE><<<grid, 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

cudaError_t launch_zgemm_df(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                            cudaStream_t st) {
  ProfScope ps("k_zgemm_df[uv]", st);
  switch (stage) {
    case G_U: return launch_zgemm_df_stage<G_U>(cap.m, cap.k, dims, ptrs, batch, st);
    case G_V: return launch_zgemm_df_stage<G_V>(cap.n, cap.k, dims, ptrs, batch, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_zgemm_tile(int stage, int tile, const Dims* dims, const ProbPtr* ptrs, int batch,
                              const Caps& cap, cudaStream_t st) {
  ProfScope ps((stage == G_U || stage == G_V) ? "k_zgemm[uv]" : "k_zgemm[sketch]", st);
  switch (stage) {
    case G_Y0: return launch_zgemm_stage<G_Y0>(cap.m, cap.l, dims, ptrs, batch, st, tile);
    case G_YT: return launch_zgemm_stage<G_YT>(cap.n, cap.l, dims, ptrs, batch, st, tile);
    case G_Y: return launch_zgemm_stage<G_Y>(cap.m, cap.l, dims, ptrs, batch, st, tile);
    case G_BH: return launch_zgemm_stage<G_BH>(cap.n, cap.l, dims, ptrs, batch, st, tile);
    case G_U: return launch_zgemm_stage<G_U>(cap.m, cap.k, dims, ptrs, batch, st, tile);
    case G_V: return launch_zgemm_stage<G_V>(cap.n, cap.k, dims, ptrs, batch, st, tile);
    case G_PR: return launch_zgemm_stage<G_PR>(cap.m, cap.r, dims, ptrs, batch, st, tile);
    case G_PQ: return launch_zgemm_stage<G_PQ>(cap.l, cap.r, dims, ptrs, batch, st, tile);
    case G_PD: return launch_zgemm_stage<G_PD>(cap.m, cap.r, dims, ptrs, batch, st, tile);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_zgemm(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                         cudaStream_t st) {
  return launch_zgemm_tile(stage, 0, dims, ptrs, batch, cap, st);
}

// ---------------------------------------------------------------------------
// Householder QR with explicit Q (Golub & Van Loan 5.2.1 and 5.1.6).
// One CTA per problem; the M x L input is column-major and is overwritten by
// the reflectors v_j (v_j stored in column j from row j down; R above the
// diagonal, R_jj kept aside).  H_j = I - tau_j v_j v_j^H with
// alpha_j = -e^{i arg x_0} ||x||, v_0 = x_0 - alpha_j, tau_j = 1/(||x|| (||x|| + |x_0|)).
// Q = H_0 ... H_{L-1} [I; 0] is accumulated backwards into the output.
// ---------------------------------------------------------------------------
enum { QR_MAXL = 512 };

enum { QR_THREADS = 1024, JAC_THREADS = 512 };

template <int QS>
__global__ void __launch_bounds__(QR_THREADS) k_qr(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                            int only_flagged) {
  __shared__ double red[32];
  __shared__ double tau[QR_MAXL];
  __shared__ cplx alph[QR_MAXL];
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  if (only_flagged && !D.qflag) return;
  const ProbPtr P = ptrs[p];
  const int M = (QS == QR_Y) ? D.m : D.n;
  const int L = D.l;
  cplx* A = (QS == QR_Y) ? P.Y : P.Yt;
  cplx* Qo = (QS == QR_Y) ? P.Q : P.Qt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int j = 0; j < L; ++j) {
    cplx* aj = A + (int64_t)j * M;
    double s = 0.0;
    for (int r = j + tid; r < M; r += blockDim.x) s += cabs2(aj[r]);
    s = block_sum(s, red);
    if (tid == 0) {
      const cplx x0 = aj[j];
      // |x0| by hypot: the phase x0/|x0| must stay on the unit circle for H to be unitary
      const double ax0 = hypot(x0.x, x0.y);
      const double nx = sqrt(s);
      if (!(nx >= 1e-150)) {  // zero column, or one so small that tau would overflow
        tau[j] = 0.0;
        alph[j] = cmk(0.0, 0.0);
      } else {
        // the phase of a leading entry negligible against ||x|| is not used
        const cplx ph = (ax0 > 1e-15 * nx) ? cscale(x0, 1.0 / ax0) : cmk(1.0, 0.0);
        alph[j] = cscale(ph, -nx);
        aj[j] = cscale(ph, ax0 + nx);  // v_0 = x_0 - alpha
        tau[j] = 1.0 / (nx * (nx + ax0));
      }
    }
    __syncthreads();
    const double t = tau[j];
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < L; c += nw) {
        cplx* ac = A + (int64_t)c * M;
        cplx sd = cmk(0.0, 0.0);
        for (int r = j + lane; r < M; r += 32) cfma_conj(sd, aj[r], ac[r]);
        sd = cscale(warp_sum(sd), t);
        for (int r = j + lane; r < M; r += 32) {
          const cplx v = aj[r];
          ac[r] = csub(ac[r], cmul(v, sd));
        }
      }
    }
    __syncthreads();
  }
  // X = Rb^H (lower triangle, column-major L x L) for the SVD of B: element
  // (r, c) of X is conj(Rb[c][r]), Rb[i][c] = A[c M + i] above the diagonal
  // and alpha_c on it
  if (QS == QR_BH) {
    for (int e = tid; e < L * L; e += blockDim.x) {
      const int c = e / L, r = e % L;
      cplx v = cmk(0.0, 0.0);
      if (c < r) v = cconj(A[(int64_t)r * M + c]);
      else if (c == r) v = cconj(alph[c]);
      P.R[(int64_t)c * L + r] = v;
    }
  }
  // Q = [I; 0], then Q <- H_j Q for j = L-1 .. 0 (only columns c >= j change)
  for (int64_t e = tid; e < (int64_t)M * L; e += blockDim.x) {
    const int c = (int)(e / M), r = (int)(e % M);
    Qo[e] = cmk(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = L - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;  // uniform across the block
    const cplx* aj = A + (int64_t)j * M;
    for (int c = j + warp; c < L; c += nw) {
      cplx* qc = Qo + (int64_t)c * M;
      cplx sd = cmk(0.0, 0.0);
      for (int r = j + lane; r < M; r += 32) cfma_conj(sd, aj[r], qc[r]);
      sd = cscale(warp_sum(sd), t);
      for (int r = j + lane; r < M; r += 32) qc[r] = csub(qc[r], cmul(aj[r], sd));
    }
    __syncthreads();
  }
}

cudaError_t launch_qr(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st,
                      int only_flagged) {
  ProfScope ps("k_qr", st);
  // batches of four matrices per SM or more: 256-thread CTAs, four per SM,
  // so that one matrix's per-column barriers overlap with the others' work
  const int nt = batch >= 4 * 152 ? 256 : QR_THREADS;
  switch (stage) {
    case QR_Y: k_qr<QR_Y><<<batch, nt, 0, st>>>(dims, ptrs, only_flagged); break;
    case QR_YT: k_qr<QR_YT><<<batch, nt, 0, st>>>(dims, ptrs, only_flagged); break;
    case QR_BH: k_qr<QR_BH><<<batch, nt, 0, st>>>(dims, ptrs, only_flagged); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD of X = Rb^H (L x L, column-major, in place),
// where B^H = Qb Rb: columns a, b of X are rotated by the 2x2 unitary that
// diagonalises their Gram matrix [[|x_a|^2, g], [g*, |x_b|^2]], g = x_a^H x_b,
// until every pair is orthogonal to tol = 4 eps sqrt(L).  Working on Rb^H
// rather than Rb (whose rows are graded after the QR) needs 4-7 sweeps
// instead of 11-17 on decaying spectra.  Columns whose squared norm is below
// (L eps)^2 ||X||_F^2 are treated as zero: rotating them only chases rounding
// noise, and they lie far below the kept-value cutoff.  Pairs follow the
// round-robin (circle) ordering, L/2 disjoint pairs per round, one group of
// JAC_G = 8 lanes per pair (four pairs per warp): the FP64 square roots and
// divisions of each rotation are then repeated on 8 lanes rather than 32,
// which halves the FP64-pipe work of a sweep.  With X J = W S:
// Rb = J S W^H, so B = W S (Qb J)^H, i.e.
// U~ = W (normalised columns of X J) and V = Qb J.
// Output: sigma sorted descending (ties by lower index), Jk = the leading k
// columns of W (for U = Q Jk), Wk = the matching columns of J (for V = Qb Wk).
// ---------------------------------------------------------------------------
enum { JAC_MAXSWEEPS = 60, JAC_G = 8 };

// sum over the JAC_G lanes of this lane's group (the group's lanes all call it)
__device__ __forceinline__ double grp_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = JAC_G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

__global__ void __launch_bounds__(JAC_THREADS) k_jacobi(const Dims* __restrict__ dims,
                                                        const ProbPtr* __restrict__ ptrs, int* status) {
  __shared__ double sv[QR_MAXL];
  __shared__ double nrm[QR_MAXL];
  __shared__ int perm[QR_MAXL];
  __shared__ int rotated;
  __shared__ double red[32];
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  const int L = D.l, K = D.k;
  cplx* X = P.R;
  cplx* J = P.J;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gl = lane & (JAC_G - 1);                      // lane within its group
  const int grp = tid / JAC_G, ngrp = blockDim.x / JAC_G;  // group index, groups per CTA
  const unsigned gmask = ((1u << JAC_G) - 1u) << (lane & ~(JAC_G - 1));
  double f2 = 0.0;
  for (int e = tid; e < L * L; e += blockDim.x) {
    J[e] = cmk((e / L) == (e % L) ? 1.0 : 0.0, 0.0);
    f2 += cabs2(X[e]);
  }
  f2 = block_sum(f2, red);
  const int Lp = (L + 1) & ~1;
  const double eps = 2.220446049250313e-16;
  const double tol = 4.0 * eps * sqrt((double)L);
  const double small = ((double)L * eps) * ((double)L * eps) * f2;
  int sweep = 0;
  for (; sweep < JAC_MAXSWEEPS; ++sweep) {
    // exact squared column norms at the start of every sweep; within the sweep
    // they follow each rotation: |x_a'|^2 = |x_a|^2 - t|g|, |x_b'|^2 = |x_b|^2 + t|g|
    for (int c = warp; c < L; c += nw) {
      const cplx* xc = X + (int64_t)c * L;
      double s2 = 0.0;
      for (int r = lane; r < L; r += 32) s2 += cabs2(xc[r]);
      s2 = warp_sum(s2);
      if (lane == 0) nrm[c] = s2;
    }
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < Lp - 1; ++rnd) {
      for (int pi = grp; pi < Lp / 2; pi += ngrp) {
        int a, b;
        if (pi == 0) { a = Lp - 1; b = rnd; }
        else { a = (rnd + pi) % (Lp - 1); b = (rnd - pi + (Lp - 1)) % (Lp - 1); }
        if (a > b) { const int t = a; a = b; b = t; }
        if (b >= L) continue;  // uniform over the group
        cplx* xa = X + (int64_t)a * L;
        cplx* xb = X + (int64_t)b * L;
        const double aa = nrm[a], bb = nrm[b];
        if (aa <= small || bb <= small) continue;
        cplx g = cmk(0.0, 0.0);
        for (int r = gl; r < L; r += JAC_G) cfma_conj(g, xa[r], xb[r]);
        g.x = grp_sum(g.x, gmask);
        g.y = grp_sum(g.y, gmask);
        const double ag2 = cabs2(g);
        if (!(ag2 > tol * tol * (aa * bb)) || ag2 == 0.0) continue;
        const double ag = sqrt(ag2);
        // rotation: x_a' = c x_a - s e* x_b, x_b' = s e x_a + c x_b, e = g/|g|
        const cplx e = cscale(g, 1.0 / ag);
        const double zeta = (bb - aa) / (2.0 * ag);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const cplx se = cscale(e, s), sec = cconj(se);
        for (int r = gl; r < L; r += JAC_G) {
          const cplx u = xa[r], v = xb[r];
          xa[r] = csub(cscale(u, c), cmul(sec, v));
          xb[r] = cadd(cmul(se, u), cscale(v, c));
        }
        cplx* ja = J + (int64_t)a * L;
        cplx* jb = J + (int64_t)b * L;
        for (int r = gl; r < L; r += JAC_G) {
          const cplx u = ja[r], v = jb[r];
          ja[r] = csub(cscale(u, c), cmul(sec, v));
          jb[r] = cadd(cmul(se, u), cscale(v, c));
        }
        if (gl == 0) {
          nrm[a] = aa - t * ag;
          nrm[b] = bb + t * ag;
          rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (sweep == JAC_MAXSWEEPS && tid == 0) atomicOr(status, 2);  // not converged (non-fatal)
  // singular values = column norms
  for (int c = warp; c < L; c += nw) {
    const cplx* xc = X + (int64_t)c * L;
    double s = 0.0;
    for (int r = lane; r < L; r += 32) s += cabs2(xc[r]);
    s = warp_sum(s);
    if (lane == 0) sv[c] = sqrt(s);
  }
  __syncthreads();
  // rank by descending value, ties by index; a NaN value ranks below every
  // number, so perm is a permutation of 0..L-1 whatever the input
  for (int c = tid; c < L; c += blockDim.x) {
    const double s = (sv[c] == sv[c]) ? sv[c] : -1.0;
    int rk = 0;
    for (int j = 0; j < L; ++j) {
      const double t = (sv[j] == sv[j]) ? sv[j] : -1.0;
      rk += (t > s) || (t == s && j < c);
    }
    perm[rk] = c;
  }
  __syncthreads();
  for (int i = tid; i < L; i += blockDim.x) P.sigma[i] = sv[perm[i]];
  for (int e = tid; e < K * L; e += blockDim.x) {
    const int t = e / L, r = e % L;
    const int c = perm[t];
    const double s = sv[c];
    P.Jk[e] = (s > 0.0) ? cscale(X[(int64_t)c * L + r], 1.0 / s) : cmk(0.0, 0.0);
    P.Wk[e] = J[(int64_t)c * L + r];
  }
}

cudaError_t launch_jacobi(const Dims* dims, const ProbPtr* ptrs, int batch, int* status, cudaStream_t st) {
  ProfScope ps("k_jacobi", st);
  // two matrices per SM or more: 256-thread CTAs, two per SM
  k_jacobi<<<batch, batch >= 2 * 152 ? 256 : JAC_THREADS, 0, st>>>(dims, ptrs, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||theta||_F^2 in NPART fixed partial sums per problem (deterministic order).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_frob2(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  __shared__ double red[32];
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  const int64_t total = (int64_t)D.m * D.n;
  const int64_t chunk = (total + NPART - 1) / NPART;
  const int64_t lo = chunk * blockIdx.x, hi = min(total, lo + chunk);
  double s = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) s += cabs2(P.theta[e]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = s;
}

cudaError_t launch_frob2(const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st) {
  ProfScope ps("k_frob2", st);
  k_frob2<<<dim3(NPART, batch), 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Standalone epilogue: kept rank chi' = #{i < k : s_i > cutoff s_1},
// w = 1 - sum_{i < chi'} s_i^2 / ||theta||_F^2, sigma (zero past chi'),
// U columns and Vh rows past chi' zeroed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rrsvd_finalize(const Dims* __restrict__ dims,
                                                        const ProbPtr* __restrict__ ptrs, double cutoff,
                                                        double* sigma, double* w, int* rank, int* status) {
  __shared__ int s_rank;
  __shared__ double s_w;
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  const int K = D.k;
  if (threadIdx.x == 0) {
    double nf = 0.0;
    for (int i = 0; i < NPART; ++i) nf += P.part[i];
    const double s0 = P.sigma[0];
    int r = 0;
    double kept = 0.0;
    bool finite = isfinite(nf) && isfinite(s0);
    if (finite && s0 > 0.0) {
      while (r < K && P.sigma[r] > cutoff * s0) {
        kept += P.sigma[r] * P.sigma[r];
        ++r;
      }
    }
    if (!finite || r == 0) atomicOr(status, 1);
    s_rank = r;
    s_w = (nf > 0.0) ? 1.0 - kept / nf : 0.0;
    P.scal[0] = nf;
    P.scal[1] = s_w;
    P.scal[2] = (double)r;
  }
  __syncthreads();
  const int r = s_rank;
  for (int i = threadIdx.x; i < K; i += blockDim.x) sigma[(int64_t)p * K + i] = (i < r) ? P.sigma[i] : 0.0;
  if (threadIdx.x == 0) {
    if (w) w[p] = s_w;
    if (rank) rank[p] = r;
  }
  if (r < K) {
    if (P.U)
      for (int64_t e = threadIdx.x; e < (int64_t)D.m * K; e += blockDim.x)
        if ((int)(e % K) >= r) P.U[e] = cmk(0.0, 0.0);
    if (P.V)
      for (int64_t e = (int64_t)r * D.n + threadIdx.x; e < (int64_t)K * D.n; e += blockDim.x) P.V[e] = cmk(0.0, 0.0);
  }
}

cudaError_t launch_rrsvd_finalize(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, double cutoff,
                                  double* sigma, double* Vh, double* w, int* rank, int* status, cudaStream_t st) {
  (void)cap;
  (void)Vh;
  ProfScope ps("k_rrsvd_finalize", st);
  k_rrsvd_finalize<<<batch, 256, 0, st>>>(dims, ptrs, cutoff, sigma, w, rank, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The RRSVD from theta (already in place) to sigma, Jk, Wk, U, Vh.
// ---------------------------------------------------------------------------
#define TG_TRY(x)                        \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

cudaError_t run_rrsvd(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int q, uint64_t seed,
                      uint64_t sweep, int64_t chain0, int chain_stride, int* status, cudaStream_t st,
                      const uint64_t* sweep_dev, const int* tiles) {
  auto T = [&](int stage) { return tiles ? tiles[stage] : 0; };
  TG_TRY(launch_omega(dims, ptrs, batch, cap, seed, sweep, chain0, chain_stride, st, sweep_dev));
  TG_TRY(launch_zgemm_tile(G_Y0, T(G_Y0), dims, ptrs, batch, cap, st));  // Y0 = A Omega
  TG_TRY(launch_qr_sized(QR_Y, dims, ptrs, batch, cap, st));              // Y0 = Q0 R0
  for (int j = 0; j < q; ++j) {
    TG_TRY(launch_zgemm_tile(G_YT, T(G_YT), dims, ptrs, batch, cap, st)); // Y~ = A^H Q
    TG_TRY(launch_qr_sized(QR_YT, dims, ptrs, batch, cap, st));           // Y~ = Q~ R~
    TG_TRY(launch_zgemm_tile(G_Y, T(G_Y), dims, ptrs, batch, cap, st));   // Y = A Q~
    TG_TRY(launch_qr_sized(QR_Y, dims, ptrs, batch, cap, st));            // Y = Q R
  }
  TG_TRY(launch_zgemm_tile(G_BH, T(G_BH), dims, ptrs, batch, cap, st));   // B^H = A^H Q
  TG_TRY(launch_qr_sized(QR_BH, dims, ptrs, batch, cap, st));             // B^H = Qb Rb
  TG_TRY(launch_jacobi_sized(dims, ptrs, batch, cap, status, st));        // Rb^H J = W S
  TG_TRY(launch_zgemm_tile(G_U, T(G_U), dims, ptrs, batch, cap, st));     // U = Q J_k
  TG_TRY(launch_zgemm_tile(G_V, T(G_V), dims, ptrs, batch, cap, st));     // V = Qb W_k  (stored as V^H)
  TG_TRY(launch_frob2(dims, ptrs, batch, st));
  return cudaSuccess;
}

}  // namespace tg
