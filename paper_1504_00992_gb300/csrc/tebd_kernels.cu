// TEBD two-site update kernels, plain FP64 (sm_103a): theta contraction with
// the gate fused in its epilogue, the per-sweep size plan, the Vidal-form
// rebuild after truncation, and one-site expectation values.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "profiler.cuh"
#include "stages.cuh"

namespace tg {

// ---------------------------------------------------------------------------
// Sizes of every bond of a wave from the current bond dimensions:
//   m = d_b chi_{b-1}, n = d_{b+1} chi_{b+1}, k = min(cap_b, m, n),
//   l = min(k + p, m, n)   (sketch width; exact when it reaches min(m, n)).
// Bonds of one parity share no site, so their updates are independent.
// ---------------------------------------------------------------------------
__global__ void k_plan(const ProbPtr* __restrict__ ptrs, Dims* dims, int batch, int p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= batch) return;
  dims[t] = plan_dev(ptrs[t], p);
}

cudaError_t launch_plan(const ProbPtr* ptrs, Dims* dims, int batch, int p, cudaStream_t st) {
  ProfScope ps("k_plan", st);
  k_plan<<<(batch + 127) / 128, 128, 0, st>>>(ptrs, dims, batch, p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// theta~ of each bond (Eq. deftheta then Eq. defupdatetheta):
//   C[(i',a),(j',c)] = sum_g (lam_l[a] Gl[i'][a][g] lam_m[g]) (Gr[j'][g][c] lam_r[c])
//   theta~[i*cl + a][j*cr + c] = sum_{i'j'} G[(i dr + j), (i' dr + j')] C[(i',a),(j',c)]
// A CTA owns an (alpha, beta) block with every i, j (the gate mixes only the
// physical indices), so the gate is applied from shared memory right after
// the contraction.  Tile: dl*TA <= 32 rows (TA >= 1), dr*TB <= 32 columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_theta(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                               int identity_gate, int skip_pre) {
  extern __shared__ cplx th_sm[];
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  if (skip_pre && !identity_gate && P.Cpre) return;  // contracted by launch_theta_df
  theta_tile_dev(D, P, blockIdx.y, blockIdx.x, identity_gate, th_sm);
}

// ---------------------------------------------------------------------------
// Gate as a GEMM (Eq. defupdatetheta for large local dimensions):
//   theta~[(i cl + a), (j cr + c)] = sum_{i'j'} G[(i dr + j), (i' dr + j')] C[(i' cl + a), (j' cr + c)],
// rows (i, j) of G times the (d_l d_r) x (cl cr) matrix whose column (a, c)
// gathers C over the physical indices.  32 x 32 output tiles (rows (i, j),
// columns (a, c) with c fastest), 2 x 2 outputs per thread, K = d_l d_r in
// slices of 16, FP64 (the layout of k_zgemm).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gate_gemm(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  constexpr int T = 32, TK = 16;
  __shared__ cplx As[TK][T + 1];  // G[row][k]
  __shared__ cplx Bs[TK][T + 1];  // C-gather[k][col]
  const int p = blockIdx.z;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  if (!P.Cpre) return;
  const int dl = D.dl, dr = D.dr, cl = D.cl, cr = D.cr;
  const int M = dl * dr, N = cl * cr, K = M;
  const int tm = blockIdx.y * T, tn = blockIdx.x * T;
  if (tm >= M || tn >= N) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n_ = D.n;
  cplx acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = cmk(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < T * TK; e += 256) {  // G tile: consecutive threads along k (contiguous)
      const int kk = e % TK, r = e / TK;
      const int gr = tm + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? P.gate[(int64_t)gr * K + gk] : cmk(0.0, 0.0);
    }
    for (int e = tid; e < T * TK; e += 256) {  // C tile: consecutive threads along (a, c), c fastest
      const int c = e % T, kk = e / T;
      const int gn = tn + c, gk = k0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (gn < N && gk < K) {
        const int ip = gk / dr, jp = gk % dr, a = gn / cr, cc = gn % cr;
        v = P.Cpre[(int64_t)(ip * cl + a) * n_ + jp * cr + cc];
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      const cplx a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const cplx b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  cplx* th = const_cast<cplx*>(P.theta);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = tm + ty + 16 * i, c = tn + tx + 16 * j;
      if (r < M && c < N) {
        const int ii = r / dr, jj = r % dr, a = c / cr, cc = c % cr;
        th[(int64_t)(ii * cl + a) * n_ + jj * cr + cc] = acc[i][j];
      }
    }
}

cudaError_t launch_gate_gemm(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st) {
  const int M = cap.dl * cap.dr, N = cap.cl * cap.cr;
  if (M < GATE_GEMM_MIN) return cudaSuccess;  // no bond of this wave takes the GEMM path
  ProfScope ps("k_gate_gemm", st);
  dim3 grid((N + 31) / 32, (M + 31) / 32, batch);
  k_gate_gemm<<<grid, 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

cudaError_t launch_theta(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, cudaStream_t st,
                         int identity_gate, int skip_pre) {
  const int TA = (cap.dl >= 32) ? 1 : 32 / cap.dl;
  const int TB = (cap.dr >= 32) ? 1 : 32 / cap.dr;
  dim3 grid((cap.cr + TB - 1) / TB, (cap.cl + TA - 1) / TA, batch);
  const size_t smem = sizeof(cplx) * (2 * TH_TK * TH_MAXR + TH_MAXR * TH_MAXR);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_theta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  ProfScope ps("k_theta", st);
  k_theta<<<grid, 256, smem, st>>>(dims, ptrs, identity_gate, skip_pre);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rebuild after truncation (Eq. defdiscweigt and the Vidal extraction):
//   chi' = #{i < k : s_i > cutoff s_1}, lambda'[b] = s / ||s_kept||,
//   w = 1 - sum_kept s^2 / ||theta~||_F^2,
//   Gamma'[b]^i[a][g]   = U[(i*cl + a)][g] / lam_l[a],
//   Gamma'[b+1]^j[g][c] = Vh[g][(j*cr + c)] / lam_r[c]   (divide only if lam > 0).
// One CTA per bond.  A zero or non-finite theta~ leaves the bond unchanged
// and raises status bit 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rebuild(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                 double cutoff, double* wout, int* status) {
  __shared__ int s_rank;
  __shared__ double s_inv;
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  rebuild_dev(D, ptrs[p], cutoff, wout + p, status, &s_rank, &s_inv);
}

cudaError_t launch_rebuild(const Dims* dims, const ProbPtr* ptrs, int batch, double cutoff, double* wout,
                           int* status, cudaStream_t st) {
  ProfScope ps("k_rebuild", st);
  k_rebuild<<<batch, 256, 0, st>>>(dims, ptrs, cutoff, wout, status);
  return cudaGetLastError();
}

// Adds the discarded weights of a wave, in problem order, into the per-chain
// accumulators wacc[2 slot] (sum of w) and wacc[2 slot + 1] (product of 1 - w).
__global__ void k_wacc(const Dims* dims, const ProbPtr* ptrs, const double* wout, int batch, double* wacc) {
  for (int p = 0; p < batch; ++p) {
    if (!dims[p].active) continue;
    const int s = ptrs[p].slot;
    wacc[2 * s] += wout[p];
    wacc[2 * s + 1] *= (1.0 - wout[p]);
    if (ptrs[p].wbond) *ptrs[p].wbond = wout[p];
  }
}

cudaError_t launch_wacc(const Dims* dims, const ProbPtr* ptrs, const double* wout, int batch, double* wacc,
                        cudaStream_t st) {
  k_wacc<<<1, 1, 0, st>>>(dims, ptrs, wout, batch, wacc);
  return cudaGetLastError();
}

// The sweep counter of the Philox sketch lives on the device so that a
// captured sweep can be replayed.
__global__ void k_sweep_tick(uint64_t* sweep_dev) { *sweep_dev += 1; }

cudaError_t launch_sweep_tick(uint64_t* sweep_dev, cudaStream_t st) {
  k_sweep_tick<<<1, 1, 0, st>>>(sweep_dev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// <O_site> = sum_{a,c} lam_l[a]^2 lam_r[c]^2 sum_{i,i'} conj(G^i[a][c]) O[i][i'] G^{i'}[a][c]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_expect(ChainDev ch, int site, const cplx* __restrict__ op, int d,
                                                cplx* out) {
  __shared__ double red[32];
  const int cl = ch.chi_ext[site], cr = ch.chi_ext[site + 1];
  const int capl = ch.cap_ext[site], capr = ch.cap_ext[site + 1];
  const double* ll = ch.lam_ext[site];
  const double* lr = ch.lam_ext[site + 1];
  const cplx* G = ch.gamma[site];
  double sr = 0.0, si = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)cl * cr; e += blockDim.x) {
    const int a = (int)(e / cr), c = (int)(e % cr);
    const double wgt = ll[a] * ll[a] * lr[c] * lr[c];
    for (int i = 0; i < d; ++i) {
      const cplx gi = G[((int64_t)i * capl + a) * capr + c];
      cplx og = cmk(0.0, 0.0);
      for (int ip = 0; ip < d; ++ip) cfma(og, op[i * d + ip], G[((int64_t)ip * capl + a) * capr + c]);
      cplx t = cmk(0.0, 0.0);
      cfma_conj(t, gi, og);
      sr += wgt * t.x;
      si += wgt * t.y;
    }
  }
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  if (threadIdx.x == 0) *out = cmk(sr, si);
}

cudaError_t launch_expect(const ChainDev& ch, int site, const cplx* op, int d, cplx* out, cudaStream_t st) {
  ProfScope ps("k_expect", st);
  k_expect<<<1, 256, 0, st>>>(ch, site, op, d, out);
  return cudaGetLastError();
}

}  // namespace tg
