// Stage bodies of the bond update as device functions executed by a whole
// CTA: the batched kernels (one problem or tile per CTA) and the fused
// per-bond kernel (fused.cu) run the same code.  Plain FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"

namespace tg {

// ---------------------------------------------------------------------------
// Batched complex GEMM C = op(A) op(B), FP64.
// Operands are addressed by (row stride, column stride) so the same code
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
  } else if (STAGE == G_PD) {  // Dr = Q C1 (m x r)
    g.M = D.m; g.N = D.r; g.K = D.l;
    g.A = P.Q; g.ars = 1; g.acs = D.m;
    g.B = P.R; g.brs = 1; g.bcs = D.l;
    g.C = P.Dr; g.crs = 1; g.ccs = D.m;
  } else if (STAGE == G_G1 || STAGE == G_G2 || STAGE == G_X) {
    // l x l Gram-type products with the n x l column-major B^H (Yt), Q1
    // (omega) or Qb (Qt): G1 = Yt^H Yt, G2 = omega^H omega, X = Yt^H Qt
    const cplx* L = (STAGE == G_G2) ? P.omega : P.Yt;
    const cplx* Rt = (STAGE == G_G1) ? P.Yt : (STAGE == G_G2 ? P.omega : P.Qt);
    g.M = D.l; g.N = D.l; g.K = D.n;
    g.A = L; g.ars = D.n; g.acs = 1;             // op(A)(i, k) = conj(L[k][i])
    g.B = Rt; g.brs = 1; g.bcs = D.n;
    g.C = P.R; g.crs = 1; g.ccs = D.l;
  } else {  // G_Q1 = Yt J, G_QB = omega J: n x l times the l x l inverse factor
    g.M = D.n; g.N = D.l; g.K = D.l;
    g.A = (STAGE == G_Q1) ? P.Yt : P.omega; g.ars = 1; g.acs = D.n;
    g.B = P.J; g.brs = 1; g.bcs = D.l;
    g.C = (STAGE == G_Q1) ? P.omega : P.Qt; g.crs = 1; g.ccs = D.n;
  }
  return g;
}

template <int STAGE>
struct StageFlags {
  static constexpr bool conjA =
      (STAGE == G_YT || STAGE == G_BH || STAGE == G_PQ || STAGE == G_G1 || STAGE == G_G2 || STAGE == G_X);
  static constexpr bool conjC = (STAGE == G_V);
};

enum { ZG_TK = 16 };

// Block-wide sums of the stages take RED_LANES per-thread partials (threads
// >= RED_LANES add zeros), so CTAs of 256, 512 or 1024 threads give
// bit-identical results.
enum { RED_LANES = 256 };

// One T x T output tile of op(A) op(B) for a CTA of 256 threads (S x S
// outputs each), K in slices of ZG_TK staged through shared memory As / Bs.
template <int T, int STAGE>
__device__ __forceinline__ void zgemm_tile_dev(const GemmOp& g, int tm, int tn, cplx (*As)[T + 1],
                                               cplx (*Bs)[T + 1]) {
  constexpr int TK = ZG_TK;
  constexpr int S = T / 16;  // outputs per thread along each direction
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

enum { QR_MAXL = 512 };

enum { QR_THREADS = 1024, JAC_THREADS = 512 };

// Householder QR with explicit Q of one problem (stage QS) by the whole CTA
// (any multiple of 32 threads); red >= 32 doubles, tau / alph >= l entries of
// shared memory.
template <int QS>
__device__ __forceinline__ void qr_dev(const Dims& D, const ProbPtr& P, double* red, double* tau, cplx* alph) {
  const int M = (QS == QR_Y) ? D.m : D.n;
  const int L = D.l;
  cplx* A = (QS == QR_Y) ? P.Y : P.Yt;
  cplx* Qo = (QS == QR_Y) ? P.Q : P.Qt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  for (int j = 0; j < L; ++j) {
    cplx* aj = A + (int64_t)j * M;
    double s = 0.0;
    // a fixed decomposition over RED_LANES partial sums, whatever the CTA
    // size: the result does not depend on the launch configuration
    if (tid < RED_LANES)
      for (int r = j + tid; r < M; r += RED_LANES) s += cabs2(aj[r]);
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

enum { JAC_MAXSWEEPS = 60, JAC_G = 8 };

// sum over the JAC_G lanes of this lane's group (the group's lanes all call it)
__device__ __forceinline__ double grp_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = JAC_G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

__device__ __forceinline__ void jacobi_finish(const Dims& D, const ProbPtr& P, double* sv, int* perm);

// One-sided Jacobi SVD of one problem by the whole CTA (any multiple of
// JAC_G threads, at least 32); sv, nrm, perm >= l entries and red >= 32
// doubles of shared memory, rotated one shared int.
__device__ __forceinline__ void jacobi_dev(const Dims& D, const ProbPtr& P, int* status, double* sv, double* nrm,
                                           int* perm, int* rotated_p, double* red) {
  int& rotated = *rotated_p;
  const int L = D.l;
  cplx* X = P.R;
  cplx* J = P.J;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gl = lane & (JAC_G - 1);                      // lane within its group
  const int grp = tid / JAC_G, ngrp = blockDim.x / JAC_G;  // group index, groups per CTA
  const unsigned gmask = ((1u << JAC_G) - 1u) << (lane & ~(JAC_G - 1));
  double f2 = 0.0;
  for (int e = tid; e < L * L; e += blockDim.x) J[e] = cmk((e / L) == (e % L) ? 1.0 : 0.0, 0.0);
  if (tid < RED_LANES)
    for (int e = tid; e < L * L; e += RED_LANES) f2 += cabs2(X[e]);
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
  jacobi_finish(D, P, sv, perm);
}

// After the sweeps (X = P.R holds X J = W S, J = P.J): singular values =
// column norms, sorted descending (ties by lower index; a NaN value ranks
// below every number, so perm is a permutation of 0..L-1 whatever the input),
// Jk = the leading k normalised columns of X J, Wk = the matching columns of J.
__device__ __forceinline__ void jacobi_finish(const Dims& D, const ProbPtr& P, double* sv, int* perm) {
  const int L = D.l, K = D.k;
  const cplx* X = P.R;
  const cplx* J = P.J;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < L; c += nw) {
    const cplx* xc = X + (int64_t)c * L;
    double s = 0.0;
    for (int r = lane; r < L; r += 32) s += cabs2(xc[r]);
    s = warp_sum(s);
    if (lane == 0) sv[c] = sqrt(s);
  }
  __syncthreads();
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

// ---------------------------------------------------------------------------
// TEBD stages: the size plan of a bond, theta~ (contraction and gate), and
// the rebuild after truncation (tebd_kernels.cu documents each).
// ---------------------------------------------------------------------------
// Sizes of one bond from its current bond dimensions (see k_plan).
__device__ __forceinline__ Dims plan_dev(const ProbPtr& P, int p) {
  Dims D;
  D.dl = P.dl_s;
  D.dr = P.dr_s;
  D.cl = *P.chi_l;
  D.cm = *P.chi_m;
  D.cr = *P.chi_r;
  D.m = D.dl * D.cl;
  D.n = D.dr * D.cr;
  const int k = min(P.chicap, min(D.m, D.n));
  D.k = k;
  D.l = min(k + p, min(D.m, D.n));
  D.bond = P.bond_s;
  D.chain = P.chain_s;
  D.active = (D.cm > 0) ? 1 : 0;
  D.r = 0;
  D.chk = 0;
  D.qflag = 0;
  return D;
}

enum { TH_TK = 16, TH_MAXR = 64 };

// One (alpha, beta) block (ablk, bblk) of theta~ by a CTA of 256 threads
// (see k_theta); th_sm holds 2 TH_TK TH_MAXR + TH_MAXR^2 complex numbers.
__device__ __forceinline__ void theta_tile_dev(const Dims& D, const ProbPtr& P, int ablk, int bblk,
                                               int identity_gate, cplx* th_sm) {
  const int dl = D.dl, dr = D.dr, cl = D.cl, cm = D.cm, cr = D.cr;
  const int TA = max(1, 32 / dl), TB = max(1, 32 / dr);
  const int a0 = ablk * TA, b0 = bblk * TB;
  if (a0 >= cl || b0 >= cr) return;
  const int ta = min(TA, cl - a0), tb = min(TB, cr - b0);
  const int rows = dl * ta, cols = dr * tb;  // <= 64 each
  cplx* Ls = th_sm;                          // [TH_TK][TH_MAXR]
  cplx* Rs = Ls + TH_TK * TH_MAXR;           // [TH_TK][TH_MAXR]
  cplx* Cs = Rs + TH_TK * TH_MAXR;           // [rows][cols]
  const int tid = threadIdx.x;
  const int nout = rows * cols;
  cplx acc[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = cmk(0.0, 0.0);
  const cplx* gl = P.gl;
  const cplx* gr = P.gr;
  for (int g0 = 0; g0 < cm; g0 += TH_TK) {
    // L rows (i', a): lam_l[a] Gl[i'][a0+a][g] lam_m[g]; g fastest
    for (int e = tid; e < TH_TK * rows; e += 256) {
      const int kk = e % TH_TK, ri = e / TH_TK;
      const int ip = ri / ta, a = ri % ta, g = g0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (g < cm) {
        v = gl[((int64_t)ip * P.cap_l + a0 + a) * P.cap_m + g];
        v = cscale(v, P.laml[a0 + a] * P.lamm[g]);
      }
      Ls[kk * TH_MAXR + ri] = v;
    }
    // R columns (j', c): Gr[j'][g][b0+c] lam_r[c]; c fastest
    for (int e = tid; e < TH_TK * cols; e += 256) {
      const int c = e % tb, rest = e / tb;
      const int jp = rest % dr, kk = rest / dr;
      const int g = g0 + kk;
      cplx v = cmk(0.0, 0.0);
      if (g < cm) {
        v = gr[((int64_t)jp * P.cap_m + g) * P.cap_r + b0 + c];
        v = cscale(v, P.lamr[b0 + c]);
      }
      Rs[kk * TH_MAXR + jp * tb + c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int o = tid + 256 * s;
      if (o < nout) {
        const int ri = o / cols, ci = o % cols;
        cplx a = acc[s];
#pragma unroll 4
        for (int kk = 0; kk < TH_TK; ++kk) cfma(a, Ls[kk * TH_MAXR + ri], Rs[kk * TH_MAXR + ci]);
        acc[s] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int o = tid + 256 * s;
    if (o < nout) Cs[o] = acc[s];
  }
  __syncthreads();
  // gate: rows of Cs are (i', a) = i'*ta + a, columns (j', c) = j'*tb + c.
  // A bond whose gate is applied as a GEMM gets its pre-gate theta in Cpre.
  const int dd = dl * dr;
  const bool pre = !identity_gate && P.Cpre != nullptr;
  cplx* th = pre ? P.Cpre : const_cast<cplx*>(P.theta);
  for (int o = tid; o < nout; o += 256) {
    const int ri = o / cols, ci = o % cols;
    const int i = ri / ta, a = ri % ta, j = ci / tb, c = ci % tb;
    const cplx* grow = P.gate + (int64_t)(i * dr + j) * dd;
    cplx v = cmk(0.0, 0.0);
    if (identity_gate || pre)
      v = Cs[(i * ta + a) * cols + j * tb + c];
    else
      for (int ip = 0; ip < dl; ++ip)
        for (int jp = 0; jp < dr; ++jp) cfma(v, grow[ip * dr + jp], Cs[(ip * ta + a) * cols + jp * tb + c]);
    th[(int64_t)(i * cl + a0 + a) * D.n + j * cr + b0 + c] = v;
  }
}

// Truncation, renormalisation and Gamma rebuild of one bond by the whole CTA
// (see k_rebuild); s_rank_p / s_inv_p point at shared scratch.
__device__ __forceinline__ void rebuild_dev(const Dims& D, const ProbPtr& P, double cutoff, double* wout_p,
                                            int* status, int* s_rank_p, double* s_inv_p) {
  if (threadIdx.x == 0) {
    double nf = 0.0;
    for (int i = 0; i < NPART; ++i) nf += P.part[i];
    const double s0 = P.sigma[0];
    int r = 0;
    double kept = 0.0;
    const bool finite = isfinite(nf) && isfinite(s0);
    if (finite && s0 > 0.0) {
      while (r < D.k && P.sigma[r] > cutoff * s0) {
        kept += P.sigma[r] * P.sigma[r];
        ++r;
      }
    }
    if (!finite || r == 0 || !isfinite(kept)) {
      atomicOr(status, 1);
      r = 0;
    }
    (*s_rank_p) = r;
    (*s_inv_p) = (r > 0) ? 1.0 / sqrt(kept) : 0.0;
    *wout_p = (r > 0 && nf > 0.0) ? 1.0 - kept / nf : 0.0;
  }
  __syncthreads();
  const int r = (*s_rank_p);
  if (r == 0) return;
  double* lam = const_cast<double*>(P.lamm);
  const int capm = P.cap_m;
  for (int i = threadIdx.x; i < capm; i += blockDim.x) lam[i] = (i < r) ? P.sigma[i] * (*s_inv_p) : 0.0;
  cplx* gl = const_cast<cplx*>(P.gl);
  cplx* gr = const_cast<cplx*>(P.gr);
  const int dl = D.dl, dr = D.dr, cl = D.cl, cr = D.cr, K = D.k;
  for (int64_t e = threadIdx.x; e < (int64_t)dl * cl * r; e += blockDim.x) {
    const int g = (int)(e % r);
    const int row = (int)(e / r);  // i*cl + a
    const int a = row % cl, i = row / cl;
    const double ll = P.laml[a];
    const cplx u = P.U[(int64_t)row * K + g];
    gl[((int64_t)i * P.cap_l + a) * capm + g] = (ll > 0.0) ? cscale(u, 1.0 / ll) : cmk(0.0, 0.0);
  }
  for (int64_t e = threadIdx.x; e < (int64_t)dr * r * cr; e += blockDim.x) {
    const int c = (int)(e % cr);
    const int rest = (int)(e / cr);
    const int g = rest % r, j = rest / r;
    const double lr = P.lamr[c];
    const cplx v = P.V[(int64_t)g * D.n + j * cr + c];
    gr[((int64_t)j * capm + g) * P.cap_r + c] = (lr > 0.0) ? cscale(v, 1.0 / lr) : cmk(0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) *P.chi_m = r;
}

}  // namespace tg
