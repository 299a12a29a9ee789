// Buffers and launchers of the reverse-mode bond update (adjoint.cu).
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace tg {

// Per-bond scratch of the reverse pass (capacity sizes) and where the bond's
// cotangents live.
struct AdjPtr {
  cplx* th0;    // m x n  pre-gate theta of the recomputed update
  cplx* Mbar;   // m x n  cotangent of the blocked theta~
  cplx* Tbar;   // m x n  cotangent of theta
  cplx* Ubar;   // m x r
  cplx* Vbar;   // n x r
  cplx* T1;     // m x r
  cplx* Pv;     // n x r
  cplx* Gu;     // r x r
  cplx* Gv;     // r x r
  cplx* Cm;     // r x r
  cplx* Pbar;   // m x cm
  cplx* Rbar;   // cm x n
  double* Sbar; // r
  double* xbar; // cl
  double* ybar; // cm
  double* zbar; // cr
  cplx* Gbar;   // (dl dr)^2, accumulated over the recorded sweeps
  cplx* gbar_l; // cotangent of Gamma[b]   (capacity layout)
  cplx* gbar_r; // cotangent of Gamma[b+1]
  double* lbar;   // cotangent of lambda[b]
  double* lbar_l; // cotangent of lambda[b-1] (NULL at the left end)
  double* lbar_r; // cotangent of lambda[b+1] (NULL at the right end)
};

cudaError_t launch_adj_expect(const cplx* G, int d, int cl, int cr, int capl, int capr, const double* ll,
                              const double* lr, const cplx* op, cplx* gbar, double* llbar, double* lrbar,
                              cudaStream_t st);
cudaError_t launch_adj_keep_theta(const Dims* dims, const ProbPtr* ptrs, const AdjPtr* adj, int batch,
                                  cudaStream_t st);
cudaError_t launch_adj_bond(const Dims* dims, const ProbPtr* ptrs, const AdjPtr* adjs, int batch,
                            const char* region_lo, const char* region_hi, const char* ckpt, double cutoff,
                            double eps_f, double eps_s, cudaStream_t st);
cudaError_t launch_adj_accum(const Dims* dims, const AdjPtr* adjs, int batch, cudaStream_t st);

}  // namespace tg
