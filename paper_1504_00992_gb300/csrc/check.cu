// Accuracy check (Alg. 2) and the fixed-precision RRSVD built on it, FP64.
//
// After the first basis of Alg. 1 (Q0 = orth(A Omega)), every round draws r Gaussian
// probes Omega_r (Philox stream 1, element (j, c) of round t at counter
// (t n + j) r + c), forms Br = A Omega_r and D = (I - Q Q^H) Br, and takes
// MAX = max_i ||d_i||.  If MAX > eps the probes' images join the basis
// ([Q | Br] is re-orthonormalised by Householder QR, l += r) and the check
// repeats while l + r stays within l_max; otherwise the check is done for
// that instance.  The rounds are a fixed launch sequence whose later rounds
// are no-ops for finished instances (per-instance flags in the device
// descriptors), so the host never waits on MAX.  The power iterations and
// steps i-iii then run on the enlarged basis, and the kept rank follows the
// basis: k = l - p.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "profiler.cuh"

namespace tg {

__global__ void k_probe_omega(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs, int t, uint64_t seed,
                              uint64_t sweep, int64_t chain0, int chain_stride) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active || !D.chk) return;
  cplx* om = ptrs[p].omega;
  const int64_t total = (int64_t)D.n * D.r;
  const uint64_t chain = chain_stride >= 0 ? (uint64_t)(chain0 + (int64_t)p * chain_stride) : (uint64_t)D.chain;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / D.r), c = (int)(e % D.r);
    om[(int64_t)c * D.n + j] = gauss_c((uint64_t)t * D.n * D.r + e, (uint64_t)D.bond, sweep, chain, seed, 1);
  }
}

// MAX of the probe residuals; on MAX > eps the basis Q is copied in front of
// Br inside Y (Y = [Q | Br]) and marked for re-orthonormalisation.
__global__ void __launch_bounds__(256) k_check_decide(Dims* dims, const ProbPtr* __restrict__ ptrs, double eps,
                                                      int l_max, int p_os) {
  __shared__ double colmax[32];
  __shared__ int extend;
  const int p = blockIdx.x;
  Dims D = dims[p];
  if (!D.active) return;
  if (!D.chk) {
    if (threadIdx.x == 0 && D.qflag) { D.qflag = 0; dims[p] = D; }
    return;
  }
  const ProbPtr P = ptrs[p];
  const int M = D.m, L = D.l, r = D.r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const cplx* Br = P.Y + (int64_t)L * M;
  double mymax = 0.0;
  for (int c = warp; c < r; c += nw) {
    double s = 0.0;
    for (int i = lane; i < M; i += 32) s += cabs2(csub(Br[(int64_t)c * M + i], P.Dr[(int64_t)c * M + i]));
    s = warp_sum(s);
    mymax = fmax(mymax, s);
  }
  if (lane == 0) colmax[warp] = mymax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m2 = 0.0;
    for (int w = 0; w < nw; ++w) m2 = fmax(m2, colmax[w]);
    extend = (sqrt(m2) > eps) ? 1 : 0;   // NaN residuals stop the check
  }
  __syncthreads();
  if (extend) {
    for (int64_t e = threadIdx.x; e < (int64_t)M * L; e += blockDim.x) P.Y[e] = P.Q[e];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (extend) {
      D.l = L + r;
      D.k = max(1, D.l - p_os);
      D.qflag = 1;
      D.chk = (D.l + r <= l_max) ? 1 : 0;
    } else {
      D.qflag = 0;
      D.chk = 0;
    }
    dims[p] = D;
  }
}

cudaError_t run_accuracy_check(const Dims* dims_mut, const ProbPtr* ptrs, int batch, const Caps& cap, int rounds,
                               double eps, int l_max, int p, uint64_t seed, uint64_t sweep, int64_t chain0,
                               int chain_stride, cudaStream_t st) {
  Dims* dims = const_cast<Dims*>(dims_mut);
  for (int t = 0; t < rounds; ++t) {
    {
      ProfScope ps("k_probe_omega", st);
      int64_t total = (int64_t)cap.n * cap.r;
      int bx = (int)((total + 255) / 256);
      bx = bx > 64 ? 64 : (bx < 1 ? 1 : bx);
      k_probe_omega<<<dim3(bx, batch), 256, 0, st>>>(dims, ptrs, t, seed, sweep, chain0, chain_stride);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    if ((e = launch_zgemm(G_PR, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;  // Br = A Omega_r
    if ((e = launch_zgemm(G_PQ, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;  // C1 = Q^H Br
    if ((e = launch_zgemm(G_PD, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;  // Dr = Q C1
    {
      ProfScope ps("k_check_decide", st);
      k_check_decide<<<batch, 256, 0, st>>>(dims, ptrs, eps, l_max, p);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_qr(QR_Y, dims, ptrs, batch, st, 1)) != cudaSuccess) return e;  // [Q | Br] = Q' R'
  }
  return cudaSuccess;
}

cudaError_t run_rrsvd_checked(Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int q, int rounds,
                              double eps, int l_max, int p, uint64_t seed, int64_t chain0, int* status,
                              cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_omega(dims, ptrs, batch, cap, seed, 0, chain0, 1, st)) != cudaSuccess) return e;
  if ((e = launch_zgemm(G_Y0, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  if ((e = launch_qr_sized(QR_Y, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  if ((e = run_accuracy_check(dims, ptrs, batch, cap, rounds, eps, l_max, p, seed, 0, chain0, 1, st)) != cudaSuccess)
    return e;
  for (int j = 0; j < q; ++j) {
    if ((e = launch_zgemm(G_YT, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
    if ((e = launch_qr_sized(QR_YT, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
    if ((e = launch_zgemm(G_Y, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
    if ((e = launch_qr_sized(QR_Y, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  }
  if ((e = launch_zgemm(G_BH, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  if ((e = launch_qr_sized(QR_BH, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  if ((e = launch_jacobi_sized(dims, ptrs, batch, cap, status, st)) != cudaSuccess) return e;
  if ((e = launch_zgemm(G_U, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  if ((e = launch_zgemm(G_V, dims, ptrs, batch, cap, st)) != cudaSuccess) return e;
  return launch_frob2(dims, ptrs, batch, st);
}

// Epilogue of a checked plan: per-instance kept rank among its own k = l - p,
// outputs at the plan's fixed stride kcap (zero past the kept rank), U copied
// from the workspace (leading dimension k) to the caller (leading dimension
// kcap), widths l reported.
__global__ void __launch_bounds__(256) k_finalize_checked(const Dims* __restrict__ dims,
                                                          const ProbPtr* __restrict__ ptrs, int kcap, double cutoff,
                                                          double* sigma, cplx* Uout, double* w, int* rank, int* lw,
                                                          int* status) {
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
    const bool finite = isfinite(nf) && isfinite(s0);
    if (finite && s0 > 0.0)
      while (r < K && P.sigma[r] > cutoff * s0) {
        kept += P.sigma[r] * P.sigma[r];
        ++r;
      }
    if (!finite || r == 0) atomicOr(status, 1);
    s_rank = r;
    s_w = (nf > 0.0) ? 1.0 - kept / nf : 0.0;
    if (w) w[p] = s_w;
    if (rank) rank[p] = r;
    if (lw) lw[p] = D.l;
  }
  __syncthreads();
  const int r = s_rank;
  for (int i = threadIdx.x; i < kcap; i += blockDim.x) sigma[(int64_t)p * kcap + i] = (i < r) ? P.sigma[i] : 0.0;
  if (Uout) {
    cplx* uo = Uout + (int64_t)p * D.m * kcap;
    for (int64_t e = threadIdx.x; e < (int64_t)D.m * kcap; e += blockDim.x) {
      const int c = (int)(e % kcap);
      const int64_t row = e / kcap;
      uo[e] = (c < r) ? P.U[row * K + c] : cmk(0.0, 0.0);
    }
  }
  if (P.V)
    for (int64_t e = (int64_t)r * D.n + threadIdx.x; e < (int64_t)kcap * D.n; e += blockDim.x) P.V[e] = cmk(0.0, 0.0);
}

cudaError_t launch_finalize_checked(const Dims* dims, const ProbPtr* ptrs, int batch, int kcap, double cutoff,
                                    double* sigma, double* Uout, double* w, int* rank, int* lw, int* status,
                                    cudaStream_t st) {
  ProfScope ps("k_rrsvd_finalize", st);
  k_finalize_checked<<<batch, 256, 0, st>>>(dims, ptrs, kcap, cutoff, sigma, (cplx*)Uout, w, rank, lw, status);
  return cudaGetLastError();
}

// Initial descriptors of a checked plan (the check rewrites l, k and flags).
__global__ void k_checked_init(Dims* dims, int batch, Dims tmpl) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < batch) dims[p] = tmpl;
}

cudaError_t launch_checked_init(Dims* dims, int batch, const Dims& tmpl, cudaStream_t st) {
  k_checked_init<<<(batch + 127) / 128, 128, 0, st>>>(dims, batch, tmpl);
  return cudaGetLastError();
}

}  // namespace tg
