// Persistent fused bond update, plain FP64 (sm_103a).
//
// One CTA carries a whole two-site update (Section II.B with the RRSVD of
// Section IV): the bond's sizes, theta~ (contraction and gate), ||theta~||_F^2,
// Omega, the sketch Y0 = theta~ Omega and the q power rounds with their QRs,
// B^H = theta~^H Q, its QR and the Jacobi SVD, U = Q J_k and V = Qb W_k, and
// the truncation, renormalisation and Gamma rebuild.  A persistent grid (as
// many CTAs as fit on the SMs) takes the bonds of a wave from an atomic work
// counter, so bonds of uneven sizes spread over the SMs with no launch
// between the stages and no grid-wide tail after each of them: the batched
// launch of all bonds of one parity of many chains (Section II.C, Eq.
// defst3rd: those bonds commute).  The counter is taken by fetch-and-add
// only: no CTA waits on another.
//
// The stages run the code of the staged kernels (stages.cuh) with the same
// per-element summation orders, so the fused and the staged paths give
// bit-identical states.  Bonds whose gate takes the GEMM path (d_l d_r >= 32)
// and sketches wider than QR_MAXL stay on the staged path (fused_fits).
#include <cuda_runtime.h>

#include "internal.cuh"
#include "profiler.cuh"
#include "stages.cuh"

namespace tg {

enum { FUSED_THREADS = 256 };

// Shared memory of one CTA: the largest stage (theta~ tiles of at most 32 x 32
// outputs: the gate's local dimensions are below 32) and the block reduction
// and broadcast slots.
struct FusedSmem {
  union {
    cplx th[2 * TH_TK * TH_MAXR + 32 * 32];
    struct {
      cplx As[ZG_TK][33];
      cplx Bs[ZG_TK][33];
    } g32;
    struct {
      cplx As[ZG_TK][17];
      cplx Bs[ZG_TK][17];
    } g16;
    struct {
      double tau[QR_MAXL];
      cplx alph[QR_MAXL];
    } qr;
    struct {
      double sv[QR_MAXL];
      double nrm[QR_MAXL];
      int perm[QR_MAXL];
    } jac;
  } u;
  double red[32];
  double s_inv;
  int item, rotated, s_rank;
};

// Every output tile of one GEMM stage, in turn, by the whole CTA (the
// per-element k order of k_zgemm, so the same result for either tile size).
template <int STAGE>
__device__ __forceinline__ void gemm_all(const Dims& D, const ProbPtr& P, FusedSmem& sm) {
  const GemmOp g = gemm_of<STAGE>(D, P);
  if (g.M <= 0 || g.N <= 0) return;
  if ((int64_t)g.M * g.N > 4 * 1024) {
    const int tn = (g.N + 31) / 32, tm = (g.M + 31) / 32;
    for (int t = 0; t < tm * tn; ++t) zgemm_tile_dev<32, STAGE>(g, (t / tn) * 32, (t % tn) * 32, sm.u.g32.As, sm.u.g32.Bs);
  } else {
    const int tn = (g.N + 15) / 16, tm = (g.M + 15) / 16;
    for (int t = 0; t < tm * tn; ++t) zgemm_tile_dev<16, STAGE>(g, (t / tn) * 16, (t % tn) * 16, sm.u.g16.As, sm.u.g16.Bs);
  }
  __syncthreads();
}

// ||theta~||_F^2 in NPART partial sums, each exactly as k_frob2 forms it (256
// per-thread partials over a contiguous chunk, then the block reduction's
// warp sums and their sum), one warp per chunk.
__device__ __forceinline__ void frob2_warps(const Dims& D, const ProbPtr& P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t total = (int64_t)D.m * D.n;
  const int64_t chunk = (total + NPART - 1) / NPART;
  for (int i = warp; i < NPART; i += nw) {
    const int64_t lo = chunk * i, hi = min(total, lo + chunk);
    double w8 = 0.0;  // lane v < 8 ends with the sum of virtual warp v
    for (int v = 0; v < 8; ++v) {
      double s = 0.0;
      for (int64_t e = lo + 32 * v + lane; e < hi; e += 256) s += cabs2(P.theta[e]);
      s = warp_sum(s);
      if (lane == v) w8 = s;
    }
    w8 = warp_sum(lane < 8 ? w8 : 0.0);
    if (lane == 0) P.part[i] = w8;
  }
}

// dims_in == nullptr: whole bond updates of TEBD bonds.  Otherwise the RRSVD
// alone (sketch to U, V) of problems with sizes dims_in[p] and theta~ already
// in place, from the counters of k_omega with chain_stride < 0: the tuner
// times it against the staged kernels on synthetic theta.
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_bond_fused(const ProbPtr* __restrict__ ptrs, Dims* dims,
                                                           const Dims* __restrict__ dims_in, int batch, int p_os,
                                                           int q, uint64_t seed,
                                                           const uint64_t* __restrict__ sweep_dev, double cutoff,
                                                           double* wout, int* status, int* queue) {
  extern __shared__ __align__(16) unsigned char fused_raw[];
  FusedSmem& sm = *reinterpret_cast<FusedSmem*>(fused_raw);
  const int tid = threadIdx.x;
  const uint64_t sweep = *sweep_dev;
  for (;;) {
    if (tid == 0) {
      const int it = atomicAdd(queue, 1);
      // the last fetch of this launch (every CTA makes exactly one fetch past
      // the end) leaves the counter at zero for the next launch
      if (it == batch + (int)gridDim.x - 1) atomicExch(queue, 0);
      sm.item = it;
    }
    __syncthreads();
    const int p = sm.item;
    __syncthreads();
    if (p >= batch) break;
    const ProbPtr& P = ptrs[p];  // read through L1 where used: not held in registers
    const bool whole = dims_in == nullptr;
    const Dims D = whole ? plan_dev(P, p_os) : dims_in[p];
    if (whole && tid == 0) dims[p] = D;  // read by the discarded-weight accumulation
    if (!D.active) continue;
    // theta~ = gate (lam Gamma lam Gamma lam), block by block
    if (whole) {
      const int TA = max(1, 32 / D.dl), TB = max(1, 32 / D.dr);
      const int na = (D.cl + TA - 1) / TA, nb = (D.cr + TB - 1) / TB;
      for (int t = 0; t < na * nb; ++t) {
        theta_tile_dev(D, P, t / nb, t % nb, 0, sm.u.th);
        __syncthreads();
      }
    }
    frob2_warps(D, P);
    // Omega: column-major n x l, element (r, c) from counter r*l + c
    {
      const int64_t total = (int64_t)D.n * D.l;
      for (int64_t e = tid; e < total; e += blockDim.x) {
        const int r = (int)(e / D.l), c = (int)(e % D.l);
        P.omega[(int64_t)c * D.n + r] = gauss_c((uint64_t)e, (uint64_t)D.bond, sweep, (uint64_t)D.chain, seed, 0);
      }
    }
    __syncthreads();
    gemm_all<G_Y0>(D, P, sm);  // Y0 = A Omega
    qr_dev<QR_Y>(D, P, sm.red, sm.u.qr.tau, sm.u.qr.alph);
    __syncthreads();
    for (int j = 0; j < q; ++j) {
      gemm_all<G_YT>(D, P, sm);  // Y~ = A^H Q
      qr_dev<QR_YT>(D, P, sm.red, sm.u.qr.tau, sm.u.qr.alph);
      __syncthreads();
      gemm_all<G_Y>(D, P, sm);  // Y = A Q~
      qr_dev<QR_Y>(D, P, sm.red, sm.u.qr.tau, sm.u.qr.alph);
      __syncthreads();
    }
    gemm_all<G_BH>(D, P, sm);  // B^H = A^H Q
    qr_dev<QR_BH>(D, P, sm.red, sm.u.qr.tau, sm.u.qr.alph);
    __syncthreads();
    jacobi_dev(D, P, status, sm.u.jac.sv, sm.u.jac.nrm, sm.u.jac.perm, &sm.rotated, sm.red);
    __syncthreads();
    gemm_all<G_U>(D, P, sm);  // U = Q J_k
    gemm_all<G_V>(D, P, sm);  // V = Qb W_k, stored as V^H
    if (whole) rebuild_dev(D, P, cutoff, wout + p, status, &sm.s_rank, &sm.s_inv);
    __syncthreads();
  }
}

bool fused_fits(const Caps& cap) {
  return cap.dl * cap.dr < GATE_GEMM_MIN && cap.l <= QR_MAXL && cap.m <= FUSED_MAXMN && cap.n <= FUSED_MAXMN;
}

static int fused_grid(int batch) {
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_bond_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FusedSmem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bond_fused, FUSED_THREADS, sizeof(FusedSmem)) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    per_sm = nb;
  }
  const int g = per_sm * (sms > 0 ? sms : 152);
  return batch < g ? batch : g;
}

cudaError_t fused_prepare() {
  fused_grid(1);
  return cudaGetLastError();
}

cudaError_t launch_bond_fused(const ProbPtr* ptrs, Dims* dims, const Dims* dims_in, int batch, int p_os, int q,
                              uint64_t seed, const uint64_t* sweep_dev, double cutoff, double* wout, int* status,
                              int* queue, cudaStream_t st) {
  if (batch < 1) return cudaSuccess;
  ProfScope ps("k_bond_fused", st);
  k_bond_fused<<<fused_grid(batch), FUSED_THREADS, sizeof(FusedSmem), st>>>(
      ptrs, dims, dims_in, batch, p_os, q, seed, sweep_dev, cutoff, wout, status, queue);
  return cudaGetLastError();
}

// Synthetic theta for the tuner: complex Gaussian entries (Philox, stream 2)
// in every problem's theta buffer at its size dims[p].
__global__ void k_tune_theta(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  cplx* th = const_cast<cplx*>(ptrs[p].theta);
  const int64_t total = (int64_t)D.m * D.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    th[e] = gauss_c((uint64_t)e, (uint64_t)p, 0, 0, 0x5eedull, 2);
}

cudaError_t launch_tune_theta(const Dims* dims, const ProbPtr* ptrs, int batch, cudaStream_t st) {
  k_tune_theta<<<dim3(64, batch), 256, 0, st>>>(dims, ptrs);
  return cudaGetLastError();
}

}  // namespace tg
