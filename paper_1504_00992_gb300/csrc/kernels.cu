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
#include "stages.cuh"

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
template <int T, int STAGE>
__global__ void __launch_bounds__(256) k_zgemm(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  __shared__ cplx As[ZG_TK][T + 1];
  __shared__ cplx Bs[ZG_TK][T + 1];
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  if ((STAGE == G_PR || STAGE == G_PQ || STAGE == G_PD) && !D.chk) return;
  const GemmOp g = gemm_of<STAGE>(D, ptrs[p]);
  const int tm = blockIdx.y * T, tn = blockIdx.x * T;
  if (tm >= g.M || tn >= g.N) return;
  zgemm_tile_dev<T, STAGE>(g, tm, tn, As, Bs);
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
  ProfScope ps(stage == G_U || stage == G_V ? "k_zgemm_df[uv]" : "k_zgemm_df[cholqr]", st);
  switch (stage) {
    case G_U: return launch_zgemm_df_stage<G_U>(cap.m, cap.k, dims, ptrs, batch, st);
    case G_V: return launch_zgemm_df_stage<G_V>(cap.n, cap.k, dims, ptrs, batch, st);
    case G_G1: return launch_zgemm_df_stage<G_G1>(cap.l, cap.l, dims, ptrs, batch, st);
    case G_Q1: return launch_zgemm_df_stage<G_Q1>(cap.n, cap.l, dims, ptrs, batch, st);
    case G_G2: return launch_zgemm_df_stage<G_G2>(cap.l, cap.l, dims, ptrs, batch, st);
    case G_QB: return launch_zgemm_df_stage<G_QB>(cap.n, cap.l, dims, ptrs, batch, st);
    case G_X: return launch_zgemm_df_stage<G_X>(cap.l, cap.l, dims, ptrs, batch, st);
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
  qr_dev<QS>(D, ptrs[p], red, tau, alph);
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
  jacobi_dev(D, ptrs[p], status, sv, nrm, perm, &rotated, red);
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
