// Householder QR with explicit Q for few, tall instances, spread over many
// CTAs per instance (FP64 for the plain path, FP32 for the TF32 form).
//
// The one-CTA-per-instance kernels (k_qr, k_qr_f32) keep one SM busy per
// matrix: for a handful of large matrices (the long bonds of a chain with
// large local dimensions, or a small batch of big instances) the rest of the
// GPU idles.  Here the reflectors are grouped in panels of QM_NB columns
// (compact WY form: H_j0 ... H_j0+nb-1 = I - V T V^H, T upper triangular;
// Golub & Van Loan 5.2.3) and each panel is three launches:
//   qm_panel_cl  a cluster of CTAs per instance factors the panel's columns
//             (the same column steps as the one-CTA kernels, restricted to
//             the panel, with the rows split over the cluster);
//   qm_w      W = V^H C over row chunks x column blocks x instances, each
//             chunk's partial sums written to its own slot (no atomics: the
//             result does not depend on scheduling);
//   qm_upd    same grid: sums the chunks in a fixed order, forms T from
//             S = V^H V (the panel columns of W) and tau, and applies
//             C <- C - V op(T) W to its rows.
// op(T) = T^H for the trailing columns of A; Q = H_0 ... H_{L-1} [I; 0] is
// formed backwards with op(T) = T (qm_w, qm_upd per panel).  Kernel
// boundaries order the steps; within a panel the CTAs of a cluster meet at
// cluster barriers (hardware barriers of co-scheduled CTAs, no spinning).
//
// Reflector rules.  FP64 (as k_qr): alpha = -e^{i arg x0} ||x||,
// v = x - alpha e_1, tau = 1 / (||x|| (||x|| + |x0|)); columns below 1e-150
// are zero; the phase of x0 is dropped when |x0| <= 1e-15 ||x||.  FP32 (as
// k_qr_f32): normalised reflectors v0 = 1, tau = 1 + |x0| / ||x||, the norm of
// a column below 1e-12 taken from x / max|x|, columns below 1e-30 are zero,
// the phase of x0 dropped when |x0| <= 1e-7 ||x||.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"

namespace cg = cooperative_groups;

namespace tg {

enum { QM_NB = 16, QM_PT = 512, QM_AT = 256, QM_CW = QM_AT / 32, QM_MIN_RC = 512 };
enum { QM_MIN_M = 1024, QM_MIN_L = 32, QM_MAX_BATCH = 96 };

// number of row chunks of the apply kernels: rows of at least QM_MIN_RC, and
// at most L / QM_NB chunks (the partial products of the FP64 form live in the
// instance's L x L buffer R)
__host__ __device__ __forceinline__ int qm_nch(int M, int L) {
  const int a = (M + QM_MIN_RC - 1) / QM_MIN_RC;
  const int b = L / QM_NB;
  const int n = a < b ? a : b;
  return n < 1 ? 1 : n;
}

// rows [j0, M) split into nch chunks of rc rows (a multiple of 32)
__device__ __forceinline__ int qm_rc(int M, int j0, int nch) {
  const int per = (M - j0 + nch - 1) / nch;
  return ((per + 31) / 32) * 32;
}

template <typename Tc>
struct QmReal;
template <>
struct QmReal<double2> {
  typedef double R;
};
template <>
struct QmReal<float2> {
  typedef float R;
};

__device__ __forceinline__ double qm_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float qm_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double qm_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float qm_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double qm_hypot(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ float qm_hypot(float a, float b) { return hypotf(a, b); }

template <typename Tc>
__device__ __forceinline__ Tc qm_c(typename QmReal<Tc>::R x, typename QmReal<Tc>::R y) {
  Tc r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename Tc>
__device__ __forceinline__ Tc qm_mul(Tc a, Tc b) {
  return qm_c<Tc>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a b
template <typename Tc>
__device__ __forceinline__ void qm_fma_c(Tc& acc, Tc a, Tc b) {
  acc.x = qm_fma(a.x, b.x, acc.x);
  acc.x = qm_fma(-a.y, b.y, acc.x);
  acc.y = qm_fma(a.x, b.y, acc.y);
  acc.y = qm_fma(a.y, b.x, acc.y);
}
// acc += conj(a) b
template <typename Tc>
__device__ __forceinline__ void qm_fmac(Tc& acc, Tc a, Tc b) {
  acc.x = qm_fma(a.x, b.x, acc.x);
  acc.x = qm_fma(a.y, b.y, acc.x);
  acc.y = qm_fma(a.x, b.y, acc.y);
  acc.y = qm_fma(-a.y, b.x, acc.y);
}
// acc -= a b
template <typename Tc>
__device__ __forceinline__ void qm_fms(Tc& acc, Tc a, Tc b) {
  acc.x = qm_fma(-a.x, b.x, acc.x);
  acc.x = qm_fma(a.y, b.y, acc.x);
  acc.y = qm_fma(-a.x, b.y, acc.y);
  acc.y = qm_fma(-a.y, b.x, acc.y);
}
template <typename R>
__device__ __forceinline__ R qm_wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// block-wide sum and max: every thread returns the same value (same order)
template <typename R>
__device__ __forceinline__ R qm_bsum(R v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = qm_wsum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R t = 0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}
template <typename R>
__device__ __forceinline__ R qm_bmax(R v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R t = 0;
  for (int w = 0; w < nw; ++w) t = fmax(t, red[w]);
  return t;
}

// One instance as the kernels see it.
template <typename Tc>
struct QmView {
  int M, L;                      // rows and columns of this instance
  int ld, Lq;                    // column stride of A and Q, and Q's stored columns (zero past L)
  Tc* A;                         // M x L column-major (stride ld), overwritten by the reflectors
  Tc* Q;                         // M x L (stride ld)
  typename QmReal<Tc>::R* tau;   // L
  Tc* T;                         // one QM_NB x QM_NB matrix per panel, T[a][b] at a * QM_NB + b
  Tc* Wp;                        // nch x QM_NB x L partial products
  Tc* alph;                      // L: the diagonal of R (FP64 form), or null
};

// FP64 instances of the RRSVD pipeline: scratch in the instance's J
// (alpha, tau, T) and R (partial products) buffers, both free during a QR.
template <int QS>
struct QmSrc64 {
  const Dims* dims;
  const ProbPtr* ptrs;
  __device__ __forceinline__ bool get(int p, QmView<double2>& v) const {
    const Dims D = dims[p];
    if (!D.active) return false;
    const ProbPtr P = ptrs[p];
    v.M = (QS == QR_Y) ? D.m : D.n;
    v.L = D.l;
    v.ld = v.M;
    v.Lq = v.L;
    v.A = (QS == QR_Y) ? P.Y : P.Yt;
    v.Q = (QS == QR_Y) ? P.Q : P.Qt;
    v.alph = P.J;
    v.tau = reinterpret_cast<double*>(P.J + v.L);
    v.T = P.J + v.L + (v.L + 1) / 2;
    v.Wp = P.R;
    return true;
  }
};

// FP32 instances of the TF32 form: arrays laid out at the batch's capacity
// (M, L) with each instance zero-padded past its own rows (D.n when use_n,
// else D.m) and D.l columns, which it factors alone when dims is given;
// scratch in its own slot of a separate array.
struct QmSrc32 {
  float2* A;
  float2* Q;
  float2* scr;
  size_t stride;  // float2 elements of scratch per instance
  int M, L;
  const Dims* dims;
  int use_n;
  __device__ __forceinline__ bool get(int p, QmView<float2>& v) const {
    v.M = M;
    v.L = L;
    if (dims) {
      const Dims D = dims[p];
      if (!D.active) return false;
      v.M = use_n ? D.n : D.m;
      v.L = D.l;
    }
    v.ld = M;
    v.Lq = L;
    v.A = A + (size_t)p * M * L;
    v.Q = Q + (size_t)p * M * L;
    float2* s = scr + (size_t)p * stride;
    v.alph = nullptr;
    v.tau = reinterpret_cast<float*>(s);
    v.T = s + (L + 1) / 2;
    v.Wp = v.T + (size_t)((L + QM_NB - 1) / QM_NB) * QM_NB * QM_NB;
    return true;
  }
};

// The panel over a cluster of QM_PC CTAs per instance: the panel's rows
// [j0, M) are split into QM_PC contiguous blocks, one per CTA, and every
// column step's reductions (the norm, the scaled norm of tiny FP32 columns,
// the products v_j^H a_c for the panel's later columns) combine the CTAs'
// partial sums read from each other's shared memory after a cluster barrier
// (release/acquire at cluster scope), in rank order, so every CTA derives the
// same reflector.  A CTA updates only its own rows; the one element another
// CTA reads, the leading entry x0 = a_j[j] of a column, is written before the
// barrier that precedes its read (and read through L2), and its owner stores
// the reflector's v_0 there only after the next barrier, when every CTA has
// read x0.
enum { QM_PC = 8 };

template <typename Tc, class Src, bool F32>
__global__ void __cluster_dims__(QM_PC, 1, 1) __launch_bounds__(QM_PT) qm_panel_cl(Src src, int j0) {
  typedef typename QmReal<Tc>::R R;
  constexpr int NS = 3 + 2 * (QM_NB - 1);  // partial slots: norm, max, scaled norm, dot products
  __shared__ R red[32];
  __shared__ R part[NS];
  __shared__ R comb[NS];
  __shared__ R pred[QM_PT / 32][2 * (QM_NB - 1)];
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank();
  QmView<Tc> v;
  if (!src.get(blockIdx.x / QM_PC, v)) return;  // uniform over the cluster
  const int M = v.M, L = v.L;
  if (j0 >= L) return;
  const int jb = min((int)QM_NB, L - j0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int per = (M - j0 + QM_PC - 1) / QM_PC;
  const int rlo = j0 + crank * per, rhi = min(M, rlo + per);
  const R ztol = F32 ? (R)1e-30f : (R)1e-150;
  const R ptol = F32 ? (R)1e-7f : (R)1e-15;
  // sums slot s over the cluster's CTAs (in rank order) into comb[s] for s in [s0, s1)
  auto combine = [&](int s0, int s1) {
    if (tid >= s0 && tid < s1) {
      R a = 0;
      for (int c = 0; c < QM_PC; ++c) a += *cluster.map_shared_rank(&part[tid], c);
      comb[tid] = a;
    }
    __syncthreads();
  };
  Tc* pend = nullptr;  // (tid 0 of the owner) where v_0 of the previous column goes
  Tc pend_v = qm_c<Tc>(0, 0);
  for (int i = 0; i < jb; ++i) {
    const int j = j0 + i;
    Tc* aj = v.A + (int64_t)j * v.ld;
    const int r0 = max(j, rlo);
    R s = 0;
    for (int r = r0 + tid; r < rhi; r += blockDim.x) {
      const Tc x = aj[r];
      s = qm_fma(x.x, x.x, qm_fma(x.y, x.y, s));
    }
    s = qm_bsum(s, red);
    if (tid == 0) part[0] = s;
    cluster.sync();
    if (pend) {  // every CTA has read the previous column's x0
      *pend = pend_v;
      pend = nullptr;
    }
    combine(0, 1);
    R nx = qm_sqrt(comb[0]);
    if (F32 && nx < (R)1e-12f) {  // uniform over the cluster
      // squares in the FP32 subnormal range: the norm of x / max|x|
      R mx = 0;
      for (int r = r0 + tid; r < rhi; r += blockDim.x) mx = fmax(mx, fmax(fabs(aj[r].x), fabs(aj[r].y)));
      mx = qm_bmax(mx, red);
      if (tid == 0) part[1] = mx;
      cluster.sync();
      if (tid == 0) {
        R m2 = 0;
        for (int c = 0; c < QM_PC; ++c) m2 = fmax(m2, *cluster.map_shared_rank(&part[1], c));
        comb[1] = m2;
      }
      __syncthreads();
      const R amax = comb[1];
      R s2 = 0;
      if (amax > 0) {
        const R ia = (R)1 / amax;
        for (int r = r0 + tid; r < rhi; r += blockDim.x) {
          const R a = aj[r].x * ia, b = aj[r].y * ia;
          s2 = qm_fma(a, a, qm_fma(b, b, s2));
        }
      }
      s2 = qm_bsum(s2, red);
      if (tid == 0) part[2] = s2;
      cluster.sync();
      combine(2, 3);
      nx = amax * qm_sqrt(comb[2]);
    }
    // the reflector, derived identically in every CTA from x0 = a_j[j]
    const Tc x0 = __ldcg(aj + j);
    const R ax0 = qm_hypot(x0.x, x0.y);
    R t = 0;
    Tc sc = qm_c<Tc>(1, 0), v0 = x0;
    if (nx >= ztol) {
      const Tc ph = (ax0 > ptol * nx) ? qm_c<Tc>(x0.x / ax0, x0.y / ax0) : qm_c<Tc>(1, 0);
      if (F32) {
        const R ri = (R)1 / (ax0 + nx);
        sc = qm_c<Tc>(ph.x * ri, -ph.y * ri);  // 1 / (x0 - alpha)
        v0 = qm_c<Tc>(1, 0);
        t = (R)1 + ax0 / nx;
      } else {
        v0 = qm_c<Tc>(ph.x * (ax0 + nx), ph.y * (ax0 + nx));
        t = (R)1 / (nx * (nx + ax0));
      }
      if (crank == 0 && tid == 0 && !F32) v.alph[j] = qm_c<Tc>(-ph.x * nx, -ph.y * nx);
    } else if (crank == 0 && tid == 0 && !F32) {
      v.alph[j] = qm_c<Tc>(0, 0);
    }
    if (crank == 0 && tid == 0) v.tau[j] = t;
    const int nc = j0 + jb - j - 1;  // panel columns right of j (uniform)
    const bool owner = j >= rlo && j < rhi;
    if (t != 0) {
      if (tid == 0 && owner) {
        pend = aj + j;
        pend_v = v0;
      }
      if (F32) {
        for (int r = max(j + 1, rlo) + tid; r < rhi; r += blockDim.x) aj[r] = qm_mul(aj[r], sc);
        __syncthreads();
      }
    }
    if (t != 0 && nc > 0) {
      Tc* a1 = aj + v.ld;  // column j + 1
      Tc dp[QM_NB - 1];
#pragma unroll
      for (int q = 0; q < QM_NB - 1; ++q) dp[q] = qm_c<Tc>(0, 0);
      for (int r = r0 + tid; r < rhi; r += blockDim.x) {
        const Tc x = (r == j) ? v0 : aj[r];
#pragma unroll
        for (int q = 0; q < QM_NB - 1; ++q)
          if (q < nc) qm_fmac(dp[q], x, a1[(int64_t)q * v.ld + r]);
      }
#pragma unroll
      for (int q = 0; q < QM_NB - 1; ++q) {
        if (q < nc) {  // uniform
          const R sx = qm_wsum(dp[q].x), sy = qm_wsum(dp[q].y);
          if (lane == 0) {
            pred[warp][2 * q] = sx;
            pred[warp][2 * q + 1] = sy;
          }
        }
      }
      __syncthreads();
      if (tid < 2 * nc) {
        R acc = 0;
        for (int w = 0; w < nw; ++w) acc += pred[w][tid];
        part[3 + tid] = acc;
      }
      cluster.sync();
      combine(3, 3 + 2 * nc);
      Tc sd[QM_NB - 1];
#pragma unroll
      for (int q = 0; q < QM_NB - 1; ++q)
        sd[q] = (q < nc) ? qm_c<Tc>(t * comb[3 + 2 * q], t * comb[4 + 2 * q]) : qm_c<Tc>(0, 0);
      for (int r = r0 + tid; r < rhi; r += blockDim.x) {
        const Tc x = (r == j) ? v0 : aj[r];
#pragma unroll
        for (int q = 0; q < QM_NB - 1; ++q)
          if (q < nc) qm_fms(a1[(int64_t)q * v.ld + r], x, sd[q]);
      }
    }
    __syncthreads();  // the next column's loops read rows this column's loops gave other threads
  }
  cluster.sync();  // every CTA has read the last x0, and no CTA still reads another's partial sums
  if (pend) *pend = pend_v;
}

// W = V^H C over one row chunk (blockIdx.y) for QM_CW columns from j0 (one
// warp per column).  Without FORQ the panel's own columns are included: for
// column c = j0 + b, rows from c give S[a][b] = v_a^H v_b (a < b).
template <typename Tc, class Src, bool FORQ>
__global__ void __launch_bounds__(QM_AT) qm_w(Src src, int j0) {
  QmView<Tc> v;
  if (!src.get(blockIdx.z, v)) return;
  const int M = v.M, L = v.L;
  if (j0 >= L) return;
  const int jb = min((int)QM_NB, L - j0);
  const int nch = qm_nch(M, L), y = blockIdx.y;
  if (y >= nch) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = j0 + blockIdx.x * QM_CW + warp;
  if (c >= L) return;  // no block-wide synchronisation below
  const int rc = qm_rc(M, j0, nch);
  const int rlo = j0 + y * rc, rhi = min(M, rlo + rc);
  const Tc* cc = (FORQ ? v.Q : v.A) + (int64_t)c * v.ld;
  const bool pcol = !FORQ && c < j0 + jb;
  const int rstart = max(rlo, pcol ? c : j0);
  const Tc* V = v.A + (int64_t)j0 * v.ld;
  Tc acc[QM_NB];
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) acc[i] = qm_c<Tc>(0, 0);
  for (int r = rstart + lane; r < rhi; r += 32) {
    const Tc x = cc[r];
#pragma unroll
    for (int i = 0; i < QM_NB; ++i)
      if (i < jb && r >= j0 + i) qm_fmac(acc[i], V[(int64_t)i * v.ld + r], x);
  }
  Tc mine = qm_c<Tc>(0, 0);
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) {
    Tc s;
    s.x = qm_wsum(acc[i].x);
    s.y = qm_wsum(acc[i].y);
    if (lane == i) mine = s;
  }
  if (lane < QM_NB) v.Wp[((int64_t)y * QM_NB + lane) * L + c] = mine;
}

// C <- C - V op(T) W on one row chunk for QM_CW columns (one warp per column):
// op(T) = T^H on the trailing columns of A (T formed here from S and tau;
// block (0, 0) stores it for the Q formation), T on the columns from j0 of
// Q (FORQ).
template <typename Tc, class Src, bool FORQ>
__global__ void __launch_bounds__(QM_AT) qm_upd(Src src, int j0) {
  typedef typename QmReal<Tc>::R R;
  __shared__ Tc Ts[QM_NB][QM_NB + 1];
  __shared__ Tc Ss[QM_NB][QM_NB + 1];
  __shared__ Tc Wsh[QM_NB][QM_CW];
  QmView<Tc> v;
  if (!src.get(blockIdx.z, v)) return;
  const int M = v.M, L = v.L;
  if (j0 >= L) return;
  const int jb = min((int)QM_NB, L - j0);
  const int nch = qm_nch(M, L), y = blockIdx.y;
  if (y >= nch) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = (FORQ ? j0 : j0 + jb) + blockIdx.x * QM_CW;
  const bool store_t = !FORQ && blockIdx.x == 0 && y == 0;
  if (c0 >= L && !store_t) return;
  const int pan = j0 / QM_NB;
  if (FORQ) {
    if (tid < QM_NB * QM_NB) Ts[tid / QM_NB][tid % QM_NB] = v.T[(int64_t)pan * QM_NB * QM_NB + tid];
  } else {
    if (tid < QM_NB * QM_NB) {
      const int a = tid / QM_NB, b = tid % QM_NB;
      Tc s = qm_c<Tc>(0, 0);
      if (a < b && b < jb)
        for (int yy = 0; yy < nch; ++yy) {
          const Tc w = v.Wp[((int64_t)yy * QM_NB + a) * L + j0 + b];
          s.x += w.x;
          s.y += w.y;
        }
      Ss[a][b] = s;
    }
    __syncthreads();
    if (warp == 0 && lane < QM_NB) {
      // row a of T: T[a][a] = tau_a, T[a][i] = -tau_i sum_{b=a}^{i-1} T[a][b] S[b][i]
      const int a = lane;
      for (int i = 0; i < QM_NB; ++i) {
        Tc t = qm_c<Tc>(0, 0);
        if (i < jb) {
          const R ti = v.tau[j0 + i];
          if (a == i) {
            t = qm_c<Tc>(ti, 0);
          } else if (a < i) {
            Tc s = qm_c<Tc>(0, 0);
            for (int b = a; b < i; ++b) qm_fma_c(s, Ts[a][b], Ss[b][i]);
            t = qm_c<Tc>(-ti * s.x, -ti * s.y);
          }
        }
        Ts[a][i] = t;
      }
    }
    __syncthreads();
    if (store_t && tid < QM_NB * QM_NB) v.T[(int64_t)pan * QM_NB * QM_NB + tid] = Ts[tid / QM_NB][tid % QM_NB];
    if (c0 >= L) return;  // uniform over the block
  }
  __syncthreads();
  const int c = c0 + warp;
  const bool have = c < L;
  Tc w = qm_c<Tc>(0, 0);
  if (have && lane < jb)
    for (int yy = 0; yy < nch; ++yy) {
      const Tc x = v.Wp[((int64_t)yy * QM_NB + lane) * L + c];
      w.x += x.x;
      w.y += x.y;
    }
  if (lane < QM_NB) Wsh[lane][warp] = w;
  __syncwarp();
  Tc w2 = qm_c<Tc>(0, 0);
  if (lane < jb) {
    if (FORQ) {
      for (int b = lane; b < jb; ++b) qm_fma_c(w2, Ts[lane][b], Wsh[b][warp]);
    } else {
      for (int a = 0; a <= lane; ++a) qm_fmac(w2, Ts[a][lane], Wsh[a][warp]);
    }
  }
  __syncwarp();
  if (lane < QM_NB) Wsh[lane][warp] = w2;
  __syncwarp();
  if (!have) return;
  Tc w2r[QM_NB];
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) w2r[i] = Wsh[i][warp];
  const int rc = qm_rc(M, j0, nch);
  const int rlo = j0 + y * rc, rhi = min(M, rlo + rc);
  Tc* cc = (FORQ ? v.Q : v.A) + (int64_t)c * v.ld;
  const Tc* V = v.A + (int64_t)j0 * v.ld;
  for (int r = rlo + lane; r < rhi; r += 32) {
    Tc x = cc[r];
#pragma unroll
    for (int i = 0; i < QM_NB; ++i)
      if (i < jb && r >= j0 + i) qm_fms(x, V[(int64_t)i * v.ld + r], w2r[i]);
    cc[r] = x;
  }
}

template <typename Tc, class Src>
__global__ void qm_qinit(Src src) {
  QmView<Tc> v;
  if (!src.get(blockIdx.y, v)) return;
  const int64_t total = (int64_t)v.ld * v.Lq;  // [I; 0] over the stored layout
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / v.ld), r = (int)(e % v.ld);
    v.Q[e] = qm_c<Tc>(r == c && c < v.L ? 1 : 0, 0);
  }
}

// X = Rb^H into R (as k_qr): element (r, c) is conj(Rb[c][r]); Rb above the
// diagonal of the factored B^H, alpha on it.  After the Q formation (R held
// the partial products until then).
__global__ void qm_rextract(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  const Dims D = dims[blockIdx.y];
  if (!D.active) return;
  const ProbPtr P = ptrs[blockIdx.y];
  const int M = D.n, L = D.l;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * L; e += gridDim.x * blockDim.x) {
    const int c = e / L, r = e % L;
    cplx x = cmk(0.0, 0.0);
    if (c < r) x = cconj(P.Yt[(int64_t)r * M + c]);
    else if (c == r) x = cconj(P.J[c]);
    P.R[(int64_t)c * L + r] = x;
  }
}

template <typename Tc, class Src, bool F32>
static cudaError_t qm_run(const Src& src, int batch, int M, int L, cudaStream_t st) {
  const int npan = (L + QM_NB - 1) / QM_NB;
  const int nch = qm_nch(M, L);
  auto blocks = [](int cols) { return cols <= 0 ? 1 : (cols + QM_CW - 1) / QM_CW; };
  for (int pn = 0; pn < npan; ++pn) {
    const int j0 = pn * QM_NB, jb = (L - j0 < QM_NB) ? L - j0 : QM_NB;
    qm_panel_cl<Tc, Src, F32><<<batch * QM_PC, QM_PT, 0, st>>>(src, j0);
    qm_w<Tc, Src, false><<<dim3(blocks(L - j0), nch, batch), QM_AT, 0, st>>>(src, j0);
    qm_upd<Tc, Src, false><<<dim3(blocks(L - j0 - jb), nch, batch), QM_AT, 0, st>>>(src, j0);
  }
  const int64_t total = (int64_t)M * L;
  int bx = (int)((total + 255) / 256);
  bx = bx > 512 ? 512 : bx;
  qm_qinit<Tc, Src><<<dim3(bx, batch), 256, 0, st>>>(src);
  for (int pn = npan - 1; pn >= 0; --pn) {
    const int j0 = pn * QM_NB;
    qm_w<Tc, Src, true><<<dim3(blocks(L - j0), nch, batch), QM_AT, 0, st>>>(src, j0);
    qm_upd<Tc, Src, true><<<dim3(blocks(L - j0), nch, batch), QM_AT, 0, st>>>(src, j0);
  }
  return cudaGetLastError();
}

// Few tall instances: the one-CTA kernel would leave most SMs idle.  The
// scratch lives in each instance's R and J, sized by qr_multi_scratch_r/j of
// its own l (an l x l buffer holds it from l = 24 on).
static bool qr_multi_fits(int M, int L, int batch) {
  return M >= QM_MIN_M && L >= QM_MIN_L && batch <= QM_MAX_BATCH;
}

bool qr_multi_chosen(int stage, const Caps& cap, int batch, int force) {
  const int M = (stage == QR_Y) ? cap.m : cap.n;
  return force == 2 ? qr_multi_fits(M, cap.l, 1) : (force == 0 && qr_multi_fits(M, cap.l, batch));
}

cudaError_t launch_qr_sized(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                            cudaStream_t st, int force) {
  const int M = (stage == QR_Y) ? cap.m : cap.n;
  const bool multi = force == 2 ? qr_multi_fits(M, cap.l, 1) : (force == 0 && qr_multi_fits(M, cap.l, batch));
  if (!multi) return launch_qr(stage, dims, ptrs, batch, st);
  ProfScope ps("k_qr[multi]", st);
  cudaError_t e;
  switch (stage) {
    case QR_Y: e = qm_run<double2, QmSrc64<QR_Y>, false>(QmSrc64<QR_Y>{dims, ptrs}, batch, M, cap.l, st); break;
    case QR_YT: e = qm_run<double2, QmSrc64<QR_YT>, false>(QmSrc64<QR_YT>{dims, ptrs}, batch, M, cap.l, st); break;
    case QR_BH:
      e = qm_run<double2, QmSrc64<QR_BH>, false>(QmSrc64<QR_BH>{dims, ptrs}, batch, M, cap.l, st);
      if (e == cudaSuccess) {
        qm_rextract<<<dim3((cap.l * cap.l + 255) / 256, batch), 256, 0, st>>>(dims, ptrs);
        e = cudaGetLastError();
      }
      break;
    default: return cudaErrorInvalidValue;
  }
  return e;
}

// Scratch of an FP64 instance with l columns (complex words): the partial
// products of at most max(1, l / QM_NB) row chunks in R; alpha, tau and one
// QM_NB x QM_NB T per panel in J.
size_t qr_multi_scratch_r(int l) { return (size_t)(l / QM_NB > 1 ? l / QM_NB : 1) * QM_NB * l; }
size_t qr_multi_scratch_j(int l) {
  return (size_t)l + (l + 1) / 2 + (size_t)((l + QM_NB - 1) / QM_NB) * QM_NB * QM_NB;
}

bool qr_multi_f32_fits(int M, int L) { return M >= QM_MIN_M && L >= QM_MIN_L; }

size_t qr_multi_f32_scratch(int M, int L) {
  const size_t npan = (size_t)(L + QM_NB - 1) / QM_NB;
  return (size_t)(L + 1) / 2 + npan * QM_NB * QM_NB + (size_t)qm_nch(M, L) * QM_NB * L;
}

cudaError_t launch_qr_multi_f32(float2* A, float2* Q, float2* scr, size_t stride, int M, int L, int batch,
                                cudaStream_t st, const Dims* dims, int use_n) {
  if (stride < qr_multi_f32_scratch(M, L)) return cudaErrorInvalidValue;
  ProfScope ps("k_qr_f32[multi]", st);
  return qm_run<float2, QmSrc32, true>(QmSrc32{A, Q, scr, stride, M, L, dims, use_n}, batch, M, L, st);
}

}  // namespace tg
