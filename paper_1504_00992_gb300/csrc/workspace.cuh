// Per-instance RRSVD workspace: one layout shared by every entry point that
// carves it (plans, TEBD handles, the no-allocation truncation).
#pragma once
#include <stddef.h>

#include "internal.cuh"

namespace tg {

// Byte offsets of one problem's buffers from the start of its block.
struct WsLayout {
  size_t omega, Y, Q, Yt, Qt, R, J, Jk, Wk, U, V, sigma, part, scal, Dr, total;
};

// Layout for sizes (m, n, k, l); U and V^H get room when own_U / own_V; r > 0
// adds the m x r block of the accuracy check.  R and J also hold the many-CTA
// QR's scratch (api.cu).
WsLayout ws_layout(int m, int n, int k, int l, bool own_U, bool own_V, int r = 0);

__host__ __device__ inline void fill_ptrs(ProbPtr& P, char* base, const WsLayout& w) {
  P.omega = (cplx*)(base + w.omega);
  P.Y = (cplx*)(base + w.Y);
  P.Q = (cplx*)(base + w.Q);
  P.Yt = (cplx*)(base + w.Yt);
  P.Qt = (cplx*)(base + w.Qt);
  P.R = (cplx*)(base + w.R);
  P.J = (cplx*)(base + w.J);
  P.Jk = (cplx*)(base + w.Jk);
  P.Wk = (cplx*)(base + w.Wk);
  P.U = (cplx*)(base + w.U);
  P.V = (cplx*)(base + w.V);
  P.sigma = (double*)(base + w.sigma);
  P.part = (double*)(base + w.part);
  P.scal = (double*)(base + w.scal);
  P.Dr = (cplx*)(base + w.Dr);
}

// Descriptors of a standalone batch (api.cu): instance p reads theta at
// theta + p * theta_stride and writes U / V^H into the caller's arrays (or its
// own block when NULL); with dims_m > 0 the Dims of every instance are also
// written (m, n, k, l, active) and *status is cleared.
__global__ void k_rrsvd_bind(ProbPtr* ptrs, int batch, char* ws, size_t per, WsLayout lay, const cplx* theta,
                             size_t theta_stride, cplx* U, size_t U_stride, cplx* Vh, size_t V_stride, Dims* dims,
                             int dims_m, int dims_n, int dims_k, int dims_l, int* status);

// Host-side fault injection (test hook, tebd_fault_inject): true once for
// each armed fault of `kind` (a one-shot flag; thread-safe).
bool fault_take(int kind);

}  // namespace tg
