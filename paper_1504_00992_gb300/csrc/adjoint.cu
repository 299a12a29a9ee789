// Reverse-mode derivative of the bond update (sm_103a, FP64).
//
// Cotangent convention: for a real loss L and complex z, z_bar = dL/dRe z +
// i dL/dIm z (dL = Re sum conj(z_bar) dz).  One CTA per bond of a recorded
// sweep, after the sweep has been recomputed from its checkpoint (so the
// workspace holds its U, S, V^H and the arena its output tensors), runs:
//   A  Vidal extraction  A' = U / x, B' = V^H / z, y' = S / ||S||:
//        U_bar = A'_bar / x, V_bar = conj(B'_bar)^T / z, x_bar, z_bar, S_bar;
//   B  Gu = U^H U_bar, Gv = V^H V_bar;
//   C  the truncated-SVD adjoint core with broadened
//        F_ab = (s_b^2 - s_a^2) / ((s_b^2 - s_a^2)^2 + eps_f),  S^-1 -> s / (s^2 + eps_s):
//        C = F o (Gu - Gu^H) S + S F o (Gv - Gv^H) + diag(S_bar)
//            + 1/2 S^-1 (I o (Gu - Gu^H))
//        T1 = U C + (U_bar - U Gu) S^-1,  Pv = (V_bar - V Gv) S^-1;
//   D  M_bar = T1 V^H + U Pv^H   (cotangent of the blocked theta~);
//   E  G_bar += sum_{a,c} theta~_bar theta^H,  theta_bar = G^H theta~_bar;
//   F  contraction theta = x A y B z:  P_bar = theta_bar R^H,
//      R_bar = P^H theta_bar, A_bar = x y P_bar, B_bar = z R_bar, and the
//      lambda cotangents.
// The truncated-SVD adjoint neglects the coupling to the discarded singular
// vectors (exact when nothing is discarded, error of order s_{k+1}/s_k).
#include <cuda_runtime.h>
#include <math.h>

#include "adjoint.cuh"
#include "profiler.cuh"

namespace tg {

// initial cotangents of L = Re <O_site> (local Vidal formula, O Hermitian)
__global__ void __launch_bounds__(256) k_adj_expect(const cplx* __restrict__ G, int d, int cl, int cr, int capl,
                                                    int capr, const double* __restrict__ ll,
                                                    const double* __restrict__ lr, const cplx* __restrict__ op,
                                                    cplx* gbar, double* llbar, double* lrbar) {
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)d * cl * cr; e += blockDim.x) {
    const int i = (int)(e / ((int64_t)cl * cr));
    const int a = (int)((e / cr) % cl), c = (int)(e % cr);
    cplx og = cmk(0.0, 0.0);
    for (int ip = 0; ip < d; ++ip) cfma(og, op[i * d + ip], G[((int64_t)ip * capl + a) * capr + c]);
    const double w = 2.0 * ll[a] * ll[a] * lr[c] * lr[c];
    const int64_t o = ((int64_t)i * capl + a) * capr + c;
    gbar[o] = cadd(gbar[o], cscale(og, w));
  }
  // dens(a, c) = Re sum_i conj(G^i) (O G)^i
  if (llbar)
    for (int a = tid; a < cl; a += blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < cr; ++c) {
        double dn = 0.0;
        for (int i = 0; i < d; ++i) {
          cplx og = cmk(0.0, 0.0);
          for (int ip = 0; ip < d; ++ip) cfma(og, op[i * d + ip], G[((int64_t)ip * capl + a) * capr + c]);
          cplx t = cmk(0.0, 0.0);
          cfma_conj(t, G[((int64_t)i * capl + a) * capr + c], og);
          dn += t.x;
        }
        s += dn * lr[c] * lr[c];
      }
      llbar[a] += 2.0 * ll[a] * s;
    }
  if (lrbar)
    for (int c = tid; c < cr; c += blockDim.x) {
      double s = 0.0;
      for (int a = 0; a < cl; ++a) {
        double dn = 0.0;
        for (int i = 0; i < d; ++i) {
          cplx og = cmk(0.0, 0.0);
          for (int ip = 0; ip < d; ++ip) cfma(og, op[i * d + ip], G[((int64_t)ip * capl + a) * capr + c]);
          cplx t = cmk(0.0, 0.0);
          cfma_conj(t, G[((int64_t)i * capl + a) * capr + c], og);
          dn += t.x;
        }
        s += dn * ll[a] * ll[a];
      }
      lrbar[c] += 2.0 * lr[c] * s;
    }
}

cudaError_t launch_adj_expect(const cplx* G, int d, int cl, int cr, int capl, int capr, const double* ll,
                              const double* lr, const cplx* op, cplx* gbar, double* llbar, double* lrbar,
                              cudaStream_t st) {
  k_adj_expect<<<1, 256, 0, st>>>(G, d, cl, cr, capl, capr, ll, lr, op, gbar, llbar, lrbar);
  return cudaGetLastError();
}

// pre-gate theta of a bond, copied out of the workspace
__global__ void k_adj_keep_theta(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                 const AdjPtr* __restrict__ adj) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  const int64_t total = (int64_t)D.m * D.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    adj[p].th0[e] = ptrs[p].theta[e];
}

cudaError_t launch_adj_keep_theta(const Dims* dims, const ProbPtr* ptrs, const AdjPtr* adj, int batch,
                                  cudaStream_t st) {
  k_adj_keep_theta<<<dim3(32, batch), 256, 0, st>>>(dims, ptrs, adj);
  return cudaGetLastError();
}

__device__ __forceinline__ const void* pre_ptr(const void* p, const char* lo, const char* hi, const char* ck) {
  const char* c = (const char*)p;
  return (c >= lo && c < hi) ? (const void*)(ck + (c - lo)) : p;
}

__global__ void __launch_bounds__(256) k_adj_bond(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                  const AdjPtr* __restrict__ adjs, const char* region_lo,
                                                  const char* region_hi, const char* ckpt, double cutoff,
                                                  double eps_f, double eps_s) {
  __shared__ int s_r;
  __shared__ double s_nrm, s_dot;
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  const AdjPtr Q = adjs[p];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int dl = D.dl, dr = D.dr, cl = D.cl, cm = D.cm, cr = D.cr, m = D.m, n = D.n, K = D.k;
  const int capl = P.cap_l, capm = P.cap_m, capr = P.cap_r;
  const cplx* A = (const cplx*)pre_ptr(P.gl, region_lo, region_hi, ckpt);
  const cplx* Bt = (const cplx*)pre_ptr(P.gr, region_lo, region_hi, ckpt);
  const double* x = (const double*)pre_ptr(P.laml, region_lo, region_hi, ckpt);
  const double* y = (const double*)pre_ptr(P.lamm, region_lo, region_hi, ckpt);
  const double* z = (const double*)pre_ptr(P.lamr, region_lo, region_hi, ckpt);
  const cplx* A2 = P.gl;   // outputs of the recomputed update
  const cplx* B2 = P.gr;
  const cplx* U = P.U;     // m x K, row-major
  const cplx* Vh = P.V;    // K x n, row-major
  const double* S = P.sigma;
  if (tid == 0) {
    int r = 0;
    double nr2 = 0.0, dot = 0.0;
    const double s0 = S[0];
    if (isfinite(s0) && s0 > 0.0)
      while (r < K && S[r] > cutoff * s0) {
        nr2 += S[r] * S[r];
        dot += Q.lbar[r] * S[r];
        ++r;
      }
    s_r = r;
    s_nrm = sqrt(nr2);
    s_dot = dot;
  }
  __syncthreads();
  const int r = s_r;
  if (r == 0) return;
  const double nrm = s_nrm, dot = s_dot;
  auto inv = [](double v) { return v > 0.0 ? 1.0 / v : 0.0; };
  auto sinv = [&](double s) { return s / (s * s + eps_s); };
  // ---- A: Vidal extraction and renormalisation
  for (int64_t e = tid; e < (int64_t)m * r; e += nt) {
    const int row = (int)(e / r), g = (int)(e % r);
    const int i = row / cl, a = row % cl;
    Q.Ubar[e] = cscale(Q.gbar_l[((int64_t)i * capl + a) * capm + g], inv(x[a]));
  }
  for (int64_t e = tid; e < (int64_t)n * r; e += nt) {
    const int row = (int)(e / r), g = (int)(e % r);
    const int j = row / cr, c = row % cr;
    Q.Vbar[e] = cscale(cconj(Q.gbar_r[((int64_t)j * capm + g) * capr + c]), inv(z[c]));
  }
  for (int a = tid; a < cl; a += nt) {
    double s = 0.0;
    for (int i = 0; i < dl; ++i)
      for (int g = 0; g < r; ++g) {
        const int64_t o = ((int64_t)i * capl + a) * capm + g;
        const cplx gb = Q.gbar_l[o], av = A2[o];
        s += gb.x * av.x + gb.y * av.y;
      }
    Q.xbar[a] = -inv(x[a]) * s;
  }
  for (int c = tid; c < cr; c += nt) {
    double s = 0.0;
    for (int j = 0; j < dr; ++j)
      for (int g = 0; g < r; ++g) {
        const int64_t o = ((int64_t)j * capm + g) * capr + c;
        const cplx gb = Q.gbar_r[o], bv = B2[o];
        s += gb.x * bv.x + gb.y * bv.y;
      }
    Q.zbar[c] = -inv(z[c]) * s;
  }
  for (int i = tid; i < r; i += nt) Q.Sbar[i] = Q.lbar[i] / nrm - dot * S[i] / (nrm * nrm * nrm);
  __syncthreads();
  // ---- B: Gu = U^H U_bar, Gv = V^H V_bar
  for (int e = tid; e < r * r; e += nt) {
    const int a = e / r, b = e % r;
    cplx gu = cmk(0.0, 0.0), gv = cmk(0.0, 0.0);
    for (int row = 0; row < m; ++row) cfma_conj(gu, U[(int64_t)row * K + a], Q.Ubar[(int64_t)row * r + b]);
    for (int row = 0; row < n; ++row) cfma(gv, Vh[(int64_t)a * n + row], Q.Vbar[(int64_t)row * r + b]);
    Q.Gu[e] = gu;
    Q.Gv[e] = gv;
  }
  __syncthreads();
  // ---- C: core matrix, then T1 and Pv
  for (int e = tid; e < r * r; e += nt) {
    const int a = e / r, b = e % r;
    cplx c = cmk(0.0, 0.0);
    if (a != b) {
      const double dsq = S[b] * S[b] - S[a] * S[a];
      const double F = dsq / (dsq * dsq + eps_f);
      const cplx ju = csub(Q.Gu[e], cconj(Q.Gu[b * r + a]));
      const cplx jv = csub(Q.Gv[e], cconj(Q.Gv[b * r + a]));
      c = cadd(cscale(ju, F * S[b]), cscale(jv, F * S[a]));
    } else {
      const cplx gd = csub(Q.Gu[e], cconj(Q.Gu[e]));   // purely imaginary
      c = cadd(cmk(Q.Sbar[a], 0.0), cscale(gd, 0.5 * sinv(S[a])));
    }
    Q.Cm[e] = c;
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)m * r; e += nt) {
    const int row = (int)(e / r), b = (int)(e % r);
    cplx t = cmk(0.0, 0.0), ug = cmk(0.0, 0.0);
    for (int a = 0; a < r; ++a) {
      const cplx u = U[(int64_t)row * K + a];
      cfma(t, u, Q.Cm[a * r + b]);
      cfma(ug, u, Q.Gu[a * r + b]);
    }
    Q.T1[e] = cadd(t, cscale(csub(Q.Ubar[e], ug), sinv(S[b])));
  }
  for (int64_t e = tid; e < (int64_t)n * r; e += nt) {
    const int row = (int)(e / r), b = (int)(e % r);
    cplx vg = cmk(0.0, 0.0);
    for (int a = 0; a < r; ++a) cfma(vg, cconj(Vh[(int64_t)a * n + row]), Q.Gv[a * r + b]);
    Q.Pv[e] = cscale(csub(Q.Vbar[e], vg), sinv(S[b]));
  }
  __syncthreads();
  // ---- D: M_bar = T1 V^H + U Pv^H
  for (int64_t e = tid; e < (int64_t)m * n; e += nt) {
    const int r1 = (int)(e / n), c1 = (int)(e % n);
    cplx t = cmk(0.0, 0.0);
    for (int b = 0; b < r; ++b) {
      cfma(t, Q.T1[(int64_t)r1 * r + b], Vh[(int64_t)b * n + c1]);
      cfma(t, U[(int64_t)r1 * K + b], cconj(Q.Pv[(int64_t)c1 * r + b]));
    }
    Q.Mbar[e] = t;
  }
  __syncthreads();
  // ---- E: gate cotangent and theta_bar = G^H theta~_bar
  const int dd = dl * dr;
  for (int e = tid; e < dd * dd; e += nt) {
    const int o = e / dd, ip = e % dd;      // G[(i j), (i' j')]
    const int i = o / dr, j = o % dr, i2 = ip / dr, j2 = ip % dr;
    cplx s = cmk(0.0, 0.0);
    for (int a = 0; a < cl; ++a)
      for (int c = 0; c < cr; ++c)
        cfma(s, Q.Mbar[(int64_t)(i * cl + a) * n + j * cr + c], cconj(Q.th0[(int64_t)(i2 * cl + a) * n + j2 * cr + c]));
    Q.Gbar[e] = cadd(Q.Gbar[e], s);
  }
  for (int64_t e = tid; e < (int64_t)m * n; e += nt) {
    const int row = (int)(e / n), col = (int)(e % n);
    const int i2 = row / cl, a = row % cl, j2 = col / cr, c = col % cr;
    cplx s = cmk(0.0, 0.0);
    for (int i = 0; i < dl; ++i)
      for (int j = 0; j < dr; ++j)
        cfma_conj(s, P.gate[(int64_t)(i * dr + j) * dd + i2 * dr + j2], Q.Mbar[(int64_t)(i * cl + a) * n + j * cr + c]);
    Q.Tbar[e] = s;
  }
  __syncthreads();
  // ---- F: contraction theta = x A y B z
  for (int64_t e = tid; e < (int64_t)m * cm; e += nt) {
    const int row = (int)(e / cm), g = (int)(e % cm);
    cplx s = cmk(0.0, 0.0);
    for (int col = 0; col < n; ++col) {
      const int j = col / cr, c = col % cr;
      const cplx rv = cscale(Bt[((int64_t)j * capm + g) * capr + c], z[c]);
      cfma(s, Q.Tbar[(int64_t)row * n + col], cconj(rv));
    }
    Q.Pbar[e] = s;
  }
  for (int64_t e = tid; e < (int64_t)cm * n; e += nt) {
    const int g = (int)(e / n), col = (int)(e % n);
    cplx s = cmk(0.0, 0.0);
    for (int row = 0; row < m; ++row) {
      const int i = row / cl, a = row % cl;
      const cplx pv = cscale(A[((int64_t)i * capl + a) * capm + g], x[a] * y[g]);
      cfma_conj(s, pv, Q.Tbar[(int64_t)row * n + col]);
    }
    Q.Rbar[e] = s;
  }
  __syncthreads();
  for (int a = tid; a < cl; a += nt) {
    double s = 0.0;
    for (int i = 0; i < dl; ++i)
      for (int g = 0; g < cm; ++g) {
        const cplx pb = Q.Pbar[(int64_t)(i * cl + a) * cm + g], av = A[((int64_t)i * capl + a) * capm + g];
        s += (pb.x * av.x + pb.y * av.y) * y[g];
      }
    Q.xbar[a] += s;
  }
  for (int g = tid; g < cm; g += nt) {
    double s = 0.0;
    for (int i = 0; i < dl; ++i)
      for (int a = 0; a < cl; ++a) {
        const cplx pb = Q.Pbar[(int64_t)(i * cl + a) * cm + g], av = A[((int64_t)i * capl + a) * capm + g];
        s += (pb.x * av.x + pb.y * av.y) * x[a];
      }
    Q.ybar[g] = s;
  }
  for (int c = tid; c < cr; c += nt) {
    double s = 0.0;
    for (int j = 0; j < dr; ++j)
      for (int g = 0; g < cm; ++g) {
        const cplx rb = Q.Rbar[(int64_t)g * n + j * cr + c], bv = Bt[((int64_t)j * capm + g) * capr + c];
        s += rb.x * bv.x + rb.y * bv.y;
      }
    Q.zbar[c] += s;
  }
  __syncthreads();
  // cotangents of the pre-update tensors replace those of the outputs
  for (int64_t e = tid; e < (int64_t)dl * cl * cm; e += nt) {
    const int g = (int)(e % cm), row = (int)(e / cm);
    const int i = row / cl, a = row % cl;
    Q.gbar_l[((int64_t)i * capl + a) * capm + g] = cscale(Q.Pbar[(int64_t)row * cm + g], x[a] * y[g]);
  }
  for (int64_t e = tid; e < (int64_t)dr * cm * cr; e += nt) {
    const int c = (int)(e % cr), rest = (int)(e / cr);
    const int g = rest % cm, j = rest / cm;
    Q.gbar_r[((int64_t)j * capm + g) * capr + c] = cscale(Q.Rbar[(int64_t)g * n + j * cr + c], z[c]);
  }
  for (int g = tid; g < capm; g += nt) Q.lbar[g] = (g < cm) ? Q.ybar[g] : 0.0;
}

cudaError_t launch_adj_bond(const Dims* dims, const ProbPtr* ptrs, const AdjPtr* adjs, int batch,
                            const char* region_lo, const char* region_hi, const char* ckpt, double cutoff,
                            double eps_f, double eps_s, cudaStream_t st) {
  ProfScope ps("k_adj_bond", st);
  k_adj_bond<<<batch, 256, 0, st>>>(dims, ptrs, adjs, region_lo, region_hi, ckpt, cutoff, eps_f, eps_s);
  return cudaGetLastError();
}

// lambda_bar[b-1] += x_bar (which = 0) or lambda_bar[b+1] += z_bar (which = 1)
__global__ void k_adj_accum(const Dims* __restrict__ dims, const AdjPtr* __restrict__ adjs, int which) {
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const AdjPtr Q = adjs[p];
  double* dst = which == 0 ? Q.lbar_l : Q.lbar_r;
  const double* src = which == 0 ? Q.xbar : Q.zbar;
  const int len = which == 0 ? D.cl : D.cr;
  if (!dst) return;
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] += src[i];
}

cudaError_t launch_adj_accum(const Dims* dims, const AdjPtr* adjs, int batch, cudaStream_t st) {
  k_adj_accum<<<batch, 128, 0, st>>>(dims, adjs, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_adj_accum<<<batch, 128, 0, st>>>(dims, adjs, 1);
  return cudaGetLastError();
}

}  // namespace tg
