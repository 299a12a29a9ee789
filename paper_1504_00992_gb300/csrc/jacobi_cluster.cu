// One-sided Jacobi SVD of X = Rb^H spread over a thread-block cluster per
// instance (sm_103a), for batches of a few large instances.
//
// The same method as k_jacobi (round-robin pairs, the same rotation,
// convergence test, treatment of negligible columns and ranking), with the
// L/2 disjoint pairs of each round interleaved over the JC_CL CTAs of a
// cluster instead of one CTA, one group of JC_G lanes per pair.  The columns
// of X and J stay in global memory and the squared column norms move there
// too (the instance's sigma buffer until the final values are written); the
// cluster barrier (release/acquire at cluster scope) separates the rounds,
// and columns and norms written by other CTAs are read through L2
// (ld.global.cg), JC_U rows per lane at a time so that the loads overlap.  A
// round's pairs are disjoint, so no two groups touch the same column within a
// round; the arithmetic of every pair is that of k_jacobi.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "profiler.cuh"

namespace cg = cooperative_groups;

namespace tg {

enum { JC_CL = 8, JC_THREADS = 256, JC_G = 8, JC_U = 4, JC_MAXSWEEPS = 60, JC_MAXL = 512 };
enum { JC_MIN_L = 64, JC_MAX_BATCH = 40 };

__device__ __forceinline__ double jc_grp_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = JC_G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// x_a' = c x_a - s e* x_b, x_b' = s e x_a + c x_b on the rows of this lane,
// JC_U rows loaded before any is written
__device__ __forceinline__ void jc_rotate(cplx* xa, cplx* xb, int L, int gl, double c, cplx se, cplx sec) {
  for (int r0 = gl; r0 < L; r0 += JC_G * JC_U) {
    cplx u[JC_U], v[JC_U];
#pragma unroll
    for (int q = 0; q < JC_U; ++q) {
      const int r = r0 + q * JC_G;
      u[q] = (r < L) ? __ldcg(xa + r) : cmk(0.0, 0.0);
      v[q] = (r < L) ? __ldcg(xb + r) : cmk(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < JC_U; ++q) {
      const int r = r0 + q * JC_G;
      if (r < L) {
        xa[r] = csub(cscale(u[q], c), cmul(sec, v[q]));
        xb[r] = cadd(cmul(se, u[q]), cscale(v[q], c));
      }
    }
  }
}

__global__ void __cluster_dims__(JC_CL, 1, 1) __launch_bounds__(JC_THREADS)
    k_jacobi_cl(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs, int* status) {
  __shared__ double sv[JC_MAXL];
  __shared__ int perm[JC_MAXL];
  __shared__ int rotated;
  __shared__ double red[32];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  const int p = blockIdx.x / JC_CL;
  const Dims D = dims[p];
  if (!D.active) return;  // uniform over the cluster
  const ProbPtr P = ptrs[p];
  const int L = D.l, K = D.k;
  cplx* X = P.R;
  cplx* J = P.J;
  double* nrm = P.sigma;  // squared column norms during the sweeps
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gl = lane & (JC_G - 1);
  const int ngrp = blockDim.x / JC_G;
  // group and warp indices over the cluster, interleaved over the CTAs so a
  // round's pairs (fewer than the cluster's groups) spread over all of them
  const int grp = (tid / JC_G) * JC_CL + crank, ngrp_all = JC_CL * ngrp;
  const int gwarp = warp * JC_CL + crank, nw_all = JC_CL * nw;
  const unsigned gmask = ((1u << JC_G) - 1u) << (lane & ~(JC_G - 1));
  // ||X||_F^2 in every CTA in the same order (the same value everywhere)
  double f2 = 0.0;
  for (int e = tid; e < L * L; e += blockDim.x) f2 += cabs2(X[e]);
  f2 = block_sum(f2, red);
  for (int e = crank * blockDim.x + tid; e < L * L; e += JC_CL * blockDim.x)
    J[e] = cmk((e / L) == (e % L) ? 1.0 : 0.0, 0.0);
  const int Lp = (L + 1) & ~1;
  const double eps = 2.220446049250313e-16;
  const double tol = 4.0 * eps * sqrt((double)L);
  const double small = ((double)L * eps) * ((double)L * eps) * f2;
  int sweep = 0;
  for (; sweep < JC_MAXSWEEPS; ++sweep) {
    for (int c = gwarp; c < L; c += nw_all) {
      const cplx* xc = X + (int64_t)c * L;
      double s2 = 0.0;
      for (int r = lane; r < L; r += 32) s2 += cabs2(__ldcg(xc + r));
      s2 = warp_sum(s2);
      if (lane == 0) nrm[c] = s2;
    }
    if (tid == 0) rotated = 0;
    cluster.sync();  // norms and J visible to the cluster
    for (int rnd = 0; rnd < Lp - 1; ++rnd) {
      for (int pi = grp; pi < Lp / 2; pi += ngrp_all) {
        int a, b;
        if (pi == 0) {
          a = Lp - 1;
          b = rnd;
        } else {
          a = (rnd + pi) % (Lp - 1);
          b = (rnd - pi + (Lp - 1)) % (Lp - 1);
        }
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (b >= L) continue;  // uniform over the group
        cplx* xa = X + (int64_t)a * L;
        cplx* xb = X + (int64_t)b * L;
        const double aa = __ldcg(nrm + a), bb = __ldcg(nrm + b);
        if (aa <= small || bb <= small) continue;
        cplx g = cmk(0.0, 0.0);
        for (int r0 = gl; r0 < L; r0 += JC_G * JC_U) {
          cplx u[JC_U], v[JC_U];
#pragma unroll
          for (int q = 0; q < JC_U; ++q) {
            const int r = r0 + q * JC_G;
            u[q] = (r < L) ? __ldcg(xa + r) : cmk(0.0, 0.0);
            v[q] = (r < L) ? __ldcg(xb + r) : cmk(0.0, 0.0);
          }
#pragma unroll
          for (int q = 0; q < JC_U; ++q) cfma_conj(g, u[q], v[q]);
        }
        g.x = jc_grp_sum(g.x, gmask);
        g.y = jc_grp_sum(g.y, gmask);
        const double ag2 = cabs2(g);
        if (!(ag2 > tol * tol * (aa * bb)) || ag2 == 0.0) continue;
        const double ag = sqrt(ag2);
        const cplx e = cscale(g, 1.0 / ag);
        const double zeta = (bb - aa) / (2.0 * ag);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const cplx se = cscale(e, s), sec = cconj(se);
        jc_rotate(xa, xb, L, gl, c, se, sec);
        jc_rotate(J + (int64_t)a * L, J + (int64_t)b * L, L, gl, c, se, sec);
        if (gl == 0) {
          nrm[a] = aa - t * ag;
          nrm[b] = bb + t * ag;
          rotated = 1;
        }
      }
      cluster.sync();  // the round's columns and norms visible to the cluster
    }
    // did any CTA of the cluster rotate in this sweep?
    int any = 0;
    for (int r = 0; r < JC_CL; ++r) any |= *cluster.map_shared_rank(&rotated, r);
    cluster.sync();  // every CTA has read the flags before they are reset
    if (!any) break;
  }
  if (crank != 0) return;
  if (sweep == JC_MAXSWEEPS && tid == 0) atomicOr(status, 2);  // not converged (non-fatal)
  for (int c = warp; c < L; c += nw) {
    const cplx* xc = X + (int64_t)c * L;
    double s = 0.0;
    for (int r = lane; r < L; r += 32) s += cabs2(__ldcg(xc + r));
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
    P.Jk[e] = (s > 0.0) ? cscale(__ldcg(X + (int64_t)c * L + r), 1.0 / s) : cmk(0.0, 0.0);
    P.Wk[e] = __ldcg(J + (int64_t)c * L + r);
  }
}

bool jacobi_cluster_chosen(const Caps& cap, int batch, int force) {
  const bool fits = cap.l >= JC_MIN_L && cap.l <= JC_MAXL;
  return force == 2 ? fits : (force == 0 && fits && batch <= JC_MAX_BATCH);
}

cudaError_t launch_jacobi_sized(const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap, int* status,
                                cudaStream_t st, int force) {
  if (!jacobi_cluster_chosen(cap, batch, force)) return launch_jacobi(dims, ptrs, batch, status, st);
  ProfScope ps("k_jacobi[cluster]", st);
  k_jacobi_cl<<<batch * JC_CL, JC_THREADS, 0, st>>>(dims, ptrs, status);
  return cudaGetLastError();
}

}  // namespace tg
