// Householder QR of few, tall instances spread over many CTAs (FP64, sm_103a).
//
// The one-CTA-per-instance kernel (k_qr) keeps one SM busy per matrix: for a
// handful of large matrices (the long bonds of a chain with large local
// dimensions) the rest of the GPU idles.  Here the same reflectors as k_qr
// (alpha = -e^{i arg x0} ||x||, v = x - alpha e_1, tau = 1/(||x|| (||x|| + |x0|)))
// are grouped in panels of QM_NB columns (compact WY form, H_j0 ... H_j0+nb-1 =
// I - V T V^H; Golub & Van Loan 5.2.3) and every panel is one launch of each of:
//   qm_panel   one CTA per instance factors the panel and forms T;
//   qm_apply   one warp per trailing column, 16 columns per CTA, applies
//              I - V T^H V^H to the trailing columns (or, backwards,
//              I - V T V^H to Q when Q = H_0 ... H_{L-1} [I; 0] is formed).
// Kernel boundaries order the steps; no CTA waits on another.  The panel's
// tau, alpha and T live in the instance's J buffer (free until the SVD).
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "profiler.cuh"

namespace tg {

enum { QM_NB = 16, QM_THREADS = 512, QM_COLS = QM_THREADS / 32 };
enum { QM_MIN_M = 1024, QM_MIN_L = 32, QM_MAX_BATCH = 48 };

struct QmScratch {
  cplx* alph;   // L
  double* tau;  // L
  cplx* T;      // npan x QM_NB x QM_NB, T[a][b] at [a * QM_NB + b]
};

__device__ __forceinline__ QmScratch qm_scratch(const ProbPtr& P, int L) {
  QmScratch s;
  s.alph = P.J;
  s.tau = reinterpret_cast<double*>(P.J + L);
  s.T = P.J + L + (L + 1) / 2;
  return s;
}

template <int QS>
__device__ __forceinline__ void qm_operands(const Dims& D, const ProbPtr& P, int& M, cplx*& A, cplx*& Qo) {
  M = (QS == QR_Y) ? D.m : D.n;
  A = (QS == QR_Y) ? P.Y : P.Yt;
  Qo = (QS == QR_Y) ? P.Q : P.Qt;
}

// Panel [j0, j0 + jb): the column steps of k_qr restricted to the panel's
// columns, then T from S = V^H V.
template <int QS>
__global__ void __launch_bounds__(QM_THREADS) qm_panel(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                       int j0) {
  __shared__ double red[32];
  __shared__ double tau_s[QM_NB];
  __shared__ cplx S[QM_NB][QM_NB];
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  int M;
  cplx *A, *Qo;
  qm_operands<QS>(D, P, M, A, Qo);
  const int L = D.l;
  if (j0 >= L) return;
  const int jb = min((int)QM_NB, L - j0);
  const QmScratch sc = qm_scratch(P, L);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < jb; ++i) {
    const int j = j0 + i;
    cplx* aj = A + (int64_t)j * M;
    double s = 0.0;
    for (int r = j + tid; r < M; r += blockDim.x) s += cabs2(aj[r]);
    s = block_sum(s, red);
    if (tid == 0) {
      const cplx x0 = aj[j];
      const double ax0 = hypot(x0.x, x0.y);
      const double nx = sqrt(s);
      if (!(nx >= 1e-150)) {
        tau_s[i] = 0.0;
        sc.alph[j] = cmk(0.0, 0.0);
      } else {
        const cplx ph = (ax0 > 1e-15 * nx) ? cscale(x0, 1.0 / ax0) : cmk(1.0, 0.0);
        sc.alph[j] = cscale(ph, -nx);
        aj[j] = cscale(ph, ax0 + nx);
        tau_s[i] = 1.0 / (nx * (nx + ax0));
      }
      sc.tau[j] = tau_s[i];
    }
    __syncthreads();
    const double t = tau_s[i];
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < j0 + jb; c += nw) {
        cplx* ac = A + (int64_t)c * M;
        cplx sd = cmk(0.0, 0.0);
        for (int r = j + lane; r < M; r += 32) cfma_conj(sd, aj[r], ac[r]);
        sd = cscale(warp_sum(sd), t);
        for (int r = j + lane; r < M; r += 32) ac[r] = csub(ac[r], cmul(aj[r], sd));
      }
    }
    __syncthreads();
  }
  // S[a][b] = v_a^H v_b for a < b (v_b starts at row j0 + b, below v_a's start)
  for (int q = warp; q < jb * jb; q += nw) {
    const int a = q / jb, b = q % jb;
    if (a >= b) continue;
    const cplx* va = A + (int64_t)(j0 + a) * M;
    const cplx* vb = A + (int64_t)(j0 + b) * M;
    cplx sd = cmk(0.0, 0.0);
    for (int r = j0 + b + lane; r < M; r += 32) cfma_conj(sd, va[r], vb[r]);
    sd = warp_sum(sd);
    if (lane == 0) S[a][b] = sd;
  }
  __syncthreads();
  if (tid == 0) {
    cplx* T = sc.T + (int64_t)(j0 / QM_NB) * QM_NB * QM_NB;
    for (int e = 0; e < QM_NB * QM_NB; ++e) T[e] = cmk(0.0, 0.0);
    for (int i = 0; i < jb; ++i) {
      T[i * QM_NB + i] = cmk(tau_s[i], 0.0);
      for (int a = 0; a < i; ++a) {
        cplx s2 = cmk(0.0, 0.0);
        for (int b = a; b < i; ++b) cfma(s2, T[a * QM_NB + b], S[b][i]);
        T[a * QM_NB + i] = cscale(s2, -tau_s[i]);
      }
    }
  }
}

// C[j0:M, cols] <- C - V op(T) V^H C for 16 columns per CTA, one per warp:
// op(T) = T^H on the trailing columns of A (FORQ = false), T on the columns
// j0.. of Q (FORQ = true).
template <int QS, bool FORQ>
__global__ void __launch_bounds__(QM_THREADS) qm_apply(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                       int j0) {
  __shared__ cplx Ts[QM_NB][QM_NB];
  __shared__ cplx W[QM_NB][QM_COLS];
  __shared__ cplx W2[QM_NB][QM_COLS];
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  int M;
  cplx *A, *Qo;
  qm_operands<QS>(D, P, M, A, Qo);
  const int L = D.l;
  if (j0 >= L) return;
  const int jb = min((int)QM_NB, L - j0);
  const int c0 = (FORQ ? j0 : j0 + jb) + blockIdx.x * QM_COLS;
  if (c0 >= L) return;
  const QmScratch sc = qm_scratch(P, L);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < QM_NB * QM_NB) Ts[tid / QM_NB][tid % QM_NB] = sc.T[(int64_t)(j0 / QM_NB) * QM_NB * QM_NB + tid];
  cplx* C = FORQ ? Qo : A;
  const int c = c0 + warp;
  const bool have = c < L;
  cplx* cc = C + (int64_t)c * M;
  // W[:, warp] = V^H c
  cplx acc[QM_NB];
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) acc[i] = cmk(0.0, 0.0);
  if (have) {
    for (int r = j0 + lane; r < M; r += 32) {
      const cplx x = cc[r];
#pragma unroll
      for (int i = 0; i < QM_NB; ++i)
        if (i < jb && r >= j0 + i) cfma_conj(acc[i], A[(int64_t)(j0 + i) * M + r], x);
    }
  }
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) {
    const cplx s = warp_sum(acc[i]);
    if (lane == i) W[i][warp] = s;
  }
  __syncthreads();
  // W2 = op(T) W
  if (lane < jb) {
    const int i = lane;
    cplx s = cmk(0.0, 0.0);
    if (FORQ) {
      for (int b = i; b < jb; ++b) cfma(s, Ts[i][b], W[b][warp]);
    } else {
      for (int a = 0; a <= i; ++a) cfma_conj(s, Ts[a][i], W[a][warp]);
    }
    W2[i][warp] = s;
  }
  __syncthreads();
  if (!have) return;
  cplx w2[QM_NB];
#pragma unroll
  for (int i = 0; i < QM_NB; ++i) w2[i] = (i < jb) ? W2[i][warp] : cmk(0.0, 0.0);
  for (int r = j0 + lane; r < M; r += 32) {
    cplx x = cc[r];
#pragma unroll
    for (int i = 0; i < QM_NB; ++i)
      if (i < jb && r >= j0 + i) x = csub(x, cmul(A[(int64_t)(j0 + i) * M + r], w2[i]));
    cc[r] = x;
  }
}

template <int QS>
__global__ void qm_qinit(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  int M;
  cplx *A, *Qo;
  qm_operands<QS>(D, P, M, A, Qo);
  const int64_t total = (int64_t)M * D.l;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / M), r = (int)(e % M);
    Qo[e] = cmk(r == c ? 1.0 : 0.0, 0.0);
  }
}

// X = Rb^H into R (as k_qr): element (r, c) is conj(Rb[c][r]); Rb above the
// diagonal in A, alpha on it.
__global__ void qm_rextract(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs) {
  const int p = blockIdx.y;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr P = ptrs[p];
  const int M = D.n, L = D.l;
  const QmScratch sc = qm_scratch(P, L);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * L; e += gridDim.x * blockDim.x) {
    const int c = e / L, r = e % L;
    cplx v = cmk(0.0, 0.0);
    if (c < r) v = cconj(P.Yt[(int64_t)r * M + c]);
    else if (c == r) v = cconj(sc.alph[c]);
    P.R[(int64_t)c * L + r] = v;
  }
}

// Few tall instances: the one-CTA kernel would leave most SMs idle.  L >= 32
// also leaves room for the panel scratch (L + L/2 + 256 ceil(L/16) complex
// words) in the instance's L x L buffer J.
bool qr_multi_fits(int M, int L, int batch) { return M >= QM_MIN_M && L >= QM_MIN_L && batch <= QM_MAX_BATCH; }

template <int QS>
static cudaError_t qr_multi_stage(const Dims* dims, const ProbPtr* ptrs, int batch, int M, int L, cudaStream_t st) {
  const int npan = (L + QM_NB - 1) / QM_NB;
  const int cols_blocks = (L + QM_COLS - 1) / QM_COLS;
  for (int pn = 0; pn < npan; ++pn) {
    qm_panel<QS><<<batch, QM_THREADS, 0, st>>>(dims, ptrs, pn * QM_NB);
    qm_apply<QS, false><<<dim3(cols_blocks, batch), QM_THREADS, 0, st>>>(dims, ptrs, pn * QM_NB);
  }
  if (QS == QR_BH) qm_rextract<<<dim3((L * L + 255) / 256, batch), 256, 0, st>>>(dims, ptrs);
  int64_t total = (int64_t)M * L;
  int bx = (int)((total + 255) / 256);
  bx = bx > 256 ? 256 : bx;
  qm_qinit<QS><<<dim3(bx, batch), 256, 0, st>>>(dims, ptrs);
  for (int pn = npan - 1; pn >= 0; --pn)
    qm_apply<QS, true><<<dim3(cols_blocks, batch), QM_THREADS, 0, st>>>(dims, ptrs, pn * QM_NB);
  return cudaGetLastError();
}

static cudaError_t launch_qr_multi(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, int M, int L,
                                   cudaStream_t st) {
  ProfScope ps("k_qr[multi]", st);
  switch (stage) {
    case QR_Y: return qr_multi_stage<QR_Y>(dims, ptrs, batch, M, L, st);
    case QR_YT: return qr_multi_stage<QR_YT>(dims, ptrs, batch, M, L, st);
    case QR_BH: return qr_multi_stage<QR_BH>(dims, ptrs, batch, M, L, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_qr_sized(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                           cudaStream_t st) {
  const int M = (stage == QR_Y) ? cap.m : cap.n;
  if (qr_multi_fits(M, cap.l, batch)) return launch_qr_multi(stage, dims, ptrs, batch, M, cap.l, st);
  return launch_qr(stage, dims, ptrs, batch, st);
}

}  // namespace tg
