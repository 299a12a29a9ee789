// FP64-accurate projection on the tensor cores (sm_103a tcgen05, BF16 slices).
//
// The step B = Q^H A of Section IV (after Alg. 1), in the mixed form with the
// FP32 basis Q_f and its re-orthonormalisation Q = Q_f (I + D): C = Q_f^H A
// (l x n) is formed from error-free slices of both operands, then
// B^H = C^H (I + D) (the fold of qr_blocked.cu).
//
// Slices (Ozaki's error-free splitting; Ozaki, Ogita, Oishi, Rump, Numer.
// Algorithms 59, 2012): within each block of OZ_KB consecutive k, every row i
// of Q_f^H and every column j of A is scaled by a power of two s so that the
// block's entries x satisfy |x| < s 2^8, and x / s is cut into OZ_S = 6
// signed 8-bit digits d_1 .. d_6 (x = s (d_1 + d_2 2^-8 + ... ), truncated
// after 48 bits).  Digit t is stored as the BF16 number d_t 2^-8(t-1) (exact:
// 8 significant bits).  A product of digits t and u is then an integer times
// 2^-8(t+u-2) below 2^16 in that unit, and the tensor core sums them in FP32
// exactly as long as each sum stays below 2^24 units.  Per block of
// OZ_DRAIN = 32 k, with 2 real products per digit pair and k for C_r or C_i:
//   level 2 (t + u = 2): one digit pair, 64 products: exact;
//   level 3: two pairs, 128 products; level 4: three pairs, 192 products;
//   level 5: four pairs, 256 products (< 2^23.99 units): all exact;
//   levels 6 and 7: five and six pairs, rounded in FP32 (each rounding 2^-56
//   of the level-2 sum or less); digit pairs with t + u > 7 are dropped
//   (2^-48 relative).
// Each block therefore runs into twelve accumulators in tensor memory (C_r
// and C_i at levels 2 .. 7), which the epilogue warps read after every block,
// scale by the two block scales and add into double-float (FP32 pair) sums in
// registers.  Measured on 40-bit digits with levels 4 .. 6 in one
// inexact group: ~3e-10 relative (some 10^4 roundings of 2^-40 per output of
// a 2000-deep product add up like a random walk); with level 4 exact, 1.4e-11
// (the 40-bit truncation of the digits).  With 48-bit digits and levels 2 .. 5
// exact the roundings left are 2^-56 (levels 6+) and 2^-48 (combining the
// levels once per block): FP64-accurate, like the double-float path it
// replaces (~1e-14).
//
// Complex products: C_r = Ar Br - Ai Bi, C_i = Ar Bi + Ai Br with Ar, Ai the
// digits of Re and Im of Q_f^H (the conjugate folded in) and Br, Bi those of
// A; the minus sign is the MMA's negate-A bit.
//
// The same kernel serves the other FP64-accurate products of the mixed form
// (k_oz_gemm<stage>): the Cholesky QR of B^H (Gram matrices B B^H and
// Q1^H Q1, the triangular products B^H R1^-1 and Q1 R2^-1, and B Qb) and
// U = Q J_k, V = Qb W_k.  Their operands are FP64 (the stage table of
// stages.cuh gives the layout); k_oz_digits_op cuts them into the same
// digits, and a conjugated left operand flips the negate bits of the MMAs
// that take its imaginary digits instead of negating them.
//
// Kernel structure (one CTA = 128 rows of C (l) x OZ_BN = 32 columns (n), all
// k): warp 0 lane 0 streams the digit tiles of each 16-deep k step with 5-D
// TMA loads (k, row, digit, re/im, instance; 32-byte swizzle) into a ring of
// OZ_STAGES stages; warp 1 lane 0 issues 24 tcgen05.mma.kind::f16 per k step:
// the digit planes u = 1 .. 6 of a part of A's side lie one after another in
// shared memory and the accumulators of levels 2 .. 7 one after another in
// tensor memory, so digit t of the other operand times planes 1 .. 7 - t is
// one MMA of N = 32 (7 - t) into the accumulators of levels t + 1 .. 7 (six
// MMAs per real product instead of 21 small ones); warps 2 .. 17 read the
// accumulators after each k block (warp w reads TMEM lanes 32 (w % 4) .. +31
// and a quarter of the columns) and keep the double-float sums.  Every mbarrier wait is
// bounded; on expiry the kernel raises *err, waits for its own copies and
// MMAs, and frees its tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "../../include/tebd_gb300.h"
#include "dfsplit.cuh"
#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"
#include "stages.cuh"
#include "tc_sync.cuh"
#include "workspace.cuh"

namespace tg {

enum {
  OZ_S = 6,        // digits per operand
  OZ_KB = 64,      // k per block of the digit scales
  OZ_DRAIN = 32,   // k per exact accumulation (the accumulators are read and cleared after each)
  OZ_KS = 16,      // k per MMA / TMA stage
  OZ_BM = 128,     // rows of C per CTA (TMEM lanes)
  OZ_BN = 32,      // columns of C per CTA
  OZ_STAGES = 3,
  OZ_EPI_WARPS = 16,  // four per TMEM lane quadrant, 8 columns each
  OZ_THREADS = 64 + 32 * OZ_EPI_WARPS,
  OZ_NGRP = OZ_S,  // accumulators per part: levels 2 .. 7
  OZ_TMEM_COLS = 512  // twelve 32-column accumulators, rounded up to a power of two
};

static const uint32_t OZ_A_TILE = OZ_BM * OZ_KS * 2;  // one digit tile of Q_f^H: 4 KB
static const uint32_t OZ_B_TILE = OZ_BN * OZ_KS * 2;  // one digit tile of A: 1.5 KB
static const uint32_t OZ_A_STAGE = 2 * OZ_S * OZ_A_TILE;
static const uint32_t OZ_B_STAGE = 2 * OZ_S * OZ_B_TILE;


// ---------------------------------------------------------------------------
// Digits.  An FP64 or FP32 value and the block's largest biased exponent E
// give a 48-bit fixed-point magnitude N (x = +-N 2^(E - bias - mantissa - 5)
// for FP64), cut into six 8-bit digits, each stored as the BF16 number
// +-d_t 2^-8(t-1) (bit pattern built from FP32 arithmetic that is exact).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t oz_bf16_digit(unsigned d, int t, bool neg) {
  const float f = (float)d * __uint_as_float((unsigned)(127 - 8 * t) << 23);  // d 2^-8t, exact
  const unsigned u = __float_as_uint(f) >> 16;
  return (uint16_t)(u | (neg && d ? 0x8000u : 0u));
}

// 48-bit magnitude of an FP64 value relative to block exponent E (biased).
__device__ __forceinline__ uint64_t oz_n48_f64(double x, int E) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF) return 0;  // zero, subnormal (negligible), non-finite (flagged elsewhere)
  const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - e + 5;  // >= 5
  return sh >= 64 ? 0 : (m >> sh);
}

__device__ __forceinline__ uint64_t oz_n48_f32(float x, int E) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xFF);
  if (e == 0 || e == 0xFF) return 0;
  const uint64_t m = (uint64_t)((u & 0x7FFFFFu) | 0x800000u);
  const int sh = e - E + 24;  // <= 24
  return sh >= 0 ? (m << sh) : ((-sh) >= 64 ? 0 : (m >> (-sh)));
}

// Scale 2^(E - off) as an FP32 number, or 0 when it is below the normal range
// (the whole block is then negligible and its digits are zero).
__device__ __forceinline__ float oz_scale(int E, int off) {
  const int b = E - off + 127;
  return (b >= 1 && b <= 254) ? __uint_as_float((unsigned)b << 23) : 0.f;
}

// ---------------------------------------------------------------------------
// Digits of A (theta, m x n row-major FP64 per instance) into
// Bd[z][reim][t][j][k] (k contiguous, Kp per row, rows nc) and block scales
// Bs[z][kb][j].  A CTA takes 64 k x 16 j; rows past the instance's (m, n)
// become zero digits.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_oz_digits_theta(const Dims* __restrict__ dims,
                                                         const ProbPtr* __restrict__ ptrs, uint16_t* Bd, float* Bs,
                                                         int nc, int Kp) {
  __shared__ int emax[16][17];
  __shared__ uint16_t dig[2 * OZ_S][16][OZ_KB + 2];  // [reim t][j][k]
  const int z = blockIdx.z;
  const Dims D = dims[z];
  if (!D.active) return;
  const int m = D.m, n = D.n;
  const cplx* th = ptrs[z].theta;
  const int k0 = blockIdx.y * OZ_KB, j0 = blockIdx.x * 16;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int j = j0 + tx;
  cplx v[4];
  int e = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int k = k0 + ty + 16 * s;
    v[s] = (k < m && j < n) ? th[(int64_t)k * n + j] : cmk(0.0, 0.0);
    const uint64_t ur = (uint64_t)__double_as_longlong(v[s].x), ui = (uint64_t)__double_as_longlong(v[s].y);
    const int er = (int)((ur >> 52) & 0x7FF), ei = (int)((ui >> 52) & 0x7FF);
    e = max(e, max(er == 0x7FF ? 0 : er, ei == 0x7FF ? 0 : ei));
  }
  emax[ty][tx] = e;
  __syncthreads();
  int E = 0;
#pragma unroll
  for (int s = 0; s < 16; ++s) E = max(E, emax[s][tx]);
  const float sc = oz_scale(E, 1030);  // x = sum_t digit_t * 2^(E - 1030)
  const bool live = sc != 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int k = ty + 16 * s;
    const uint64_t nr = live ? oz_n48_f64(v[s].x, E) : 0, ni = live ? oz_n48_f64(v[s].y, E) : 0;
    const bool sr = v[s].x < 0.0, si = v[s].y < 0.0;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
      dig[t][tx][k] = oz_bf16_digit((unsigned)((nr >> (40 - 8 * t)) & 0xFF), t, sr);
      dig[OZ_S + t][tx][k] = oz_bf16_digit((unsigned)((ni >> (40 - 8 * t)) & 0xFF), t, si);
    }
  }
  if (ty == 0 && j < nc) Bs[((size_t)z * (Kp / OZ_KB) + blockIdx.y) * nc + j] = live ? sc : 0.f;
  __syncthreads();
  // rows (reim t, j) of 64 k = 128 bytes each: 8 threads per row, 16 bytes each
  uint16_t* base = Bd + (size_t)z * 2 * OZ_S * nc * Kp;
  for (int w = threadIdx.x; w < 2 * OZ_S * 16 * 8; w += 256) {
    const int q = w & 7, row = w >> 3, jj = row & 15, rt = row >> 4;
    if (j0 + jj >= nc) continue;
    const uint16_t* src = &dig[rt][jj][q * 8];
    uint4 pk;
    pk.x = (unsigned)src[0] | ((unsigned)src[1] << 16);
    pk.y = (unsigned)src[2] | ((unsigned)src[3] << 16);
    pk.z = (unsigned)src[4] | ((unsigned)src[5] << 16);
    pk.w = (unsigned)src[6] | ((unsigned)src[7] << 16);
    *reinterpret_cast<uint4*>(base + ((size_t)rt * nc + j0 + jj) * Kp + k0 + q * 8) = pk;
  }
}

// Digits of Q_f^H (Q_f m x l column-major FP32 complex per instance, capacity
// mc x lc) into Ad[z][reim][t][i][k] and scales As[z][kb][i]: one warp per
// (i, k block), two k per lane; Im negated (the conjugate).
__global__ void __launch_bounds__(256) k_oz_digits_q(const Dims* __restrict__ dims, const float2* __restrict__ Qf,
                                                     uint16_t* Ad, float* As, int mc, int lc, int Kp) {
  const int z = blockIdx.y;
  const Dims D = dims[z];
  if (!D.active) return;
  const int nkb = Kp / OZ_KB;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (wid >= lc * nkb) return;
  const int i = wid / nkb, kb = wid % nkb;
  const int k = kb * OZ_KB + 2 * lane;
  float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
  if (i < D.l) {
    const float2* q = Qf + (size_t)z * mc * lc + (size_t)i * mc;
    if (k < D.m) a = q[k];
    if (k + 1 < D.m) b = q[k + 1];
  }
  auto ex = [](float x) {
    const int e = (int)((__float_as_uint(x) >> 23) & 0xFF);
    return e == 0xFF ? 0 : e;
  };
  int E = max(max(ex(a.x), ex(a.y)), max(ex(b.x), ex(b.y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
  const float sc = oz_scale(E, 134);  // x = sum_t digit_t * 2^(E - 134)
  const bool live = sc != 0.f;
  uint16_t* base = Ad + (size_t)z * 2 * OZ_S * lc * Kp;
  const float re[2] = {a.x, b.x}, im[2] = {-a.y, -b.y};
#pragma unroll
  for (int t = 0; t < OZ_S; ++t) {
    uint16_t dr[2], di[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t nr = live ? oz_n48_f32(re[h], E) : 0, ni = live ? oz_n48_f32(im[h], E) : 0;
      dr[h] = oz_bf16_digit((unsigned)((nr >> (40 - 8 * t)) & 0xFF), t, re[h] < 0.f);
      di[h] = oz_bf16_digit((unsigned)((ni >> (40 - 8 * t)) & 0xFF), t, im[h] < 0.f);
    }
    *reinterpret_cast<unsigned*>(base + ((size_t)t * lc + i) * Kp + k) = (unsigned)dr[0] | ((unsigned)dr[1] << 16);
    *reinterpret_cast<unsigned*>(base + ((size_t)(OZ_S + t) * lc + i) * Kp + k) =
        (unsigned)di[0] | ((unsigned)di[1] << 16);
  }
  if (lane == 0) As[((size_t)z * nkb + kb) * lc + i] = live ? sc : 0.f;
}

// ---------------------------------------------------------------------------
// Stages.  OZ_PROJ is the projection C = Q_f^H A (l x n, K = m), written as
// B^H = C^H into Yt; the others are the GemmStage products of stages.cuh,
// C = op(A) op(B) with op(A) conjugated where StageFlags says so and C
// stored conjugated for G_V.
// ---------------------------------------------------------------------------
// OZ_THETA, OZ_GATE: the contraction and the gate of bonds whose gate is a
// GEMM (d_l d_r >= GATE_GEMM_MIN), the mixed forms' counterparts of
// k_cgemm_df<DgTheta> / <DgGate> (df_gemm.cu documents the operands).
enum { OZ_PROJ = 100, OZ_GRAM = 101, OZ_THETA = 102, OZ_GATE = 103 };
static_assert(OZ_THETA == OZ_THETA_STAGE && OZ_GATE == OZ_GATE_STAGE, "stage ids of mixed.cuh");

struct OzOp {
  int M, N, K;  // rows and columns of C, depth
  cplx* C;
  int64_t crs, ccs;
};

template <int ST>
__device__ __forceinline__ OzOp oz_op(const Dims& D, const ProbPtr& P) {
  OzOp o;
  if constexpr (ST == OZ_PROJ) {
    o.M = D.l; o.N = D.n; o.K = D.m;
    o.C = P.Yt; o.crs = D.n; o.ccs = 1;  // element (j, i) of the n x l column-major B^H
  } else if constexpr (ST == OZ_GRAM) {
    o.M = D.l; o.N = D.l; o.K = D.m;
    o.C = P.R; o.crs = 1; o.ccs = D.l;  // E = Q_f^H Q_f - I, l x l column-major
  } else if constexpr (ST == OZ_THETA) {
    o.M = D.dl * D.cl; o.N = D.dr * D.cr; o.K = D.cm;  // into the pre-gate buffer (oz_store)
    o.C = P.Cpre; o.crs = D.n; o.ccs = 1;
  } else if constexpr (ST == OZ_GATE) {
    o.M = D.dl * D.dr; o.N = D.cl * D.cr; o.K = D.dl * D.dr;  // into theta (oz_store)
    o.C = const_cast<cplx*>(P.theta); o.crs = 0; o.ccs = 0;
  } else {
    const GemmOp g = gemm_of<ST>(D, P);
    o.M = g.M; o.N = g.N; o.K = g.K;
    o.C = g.C; o.crs = g.crs; o.ccs = g.ccs;
  }
  return o;
}

template <int ST>
struct OzConj {
  // the projection and the Gram fold conj(Q_f) into Q_f's digits; the Gram
  // multiplies them by their own conjugate
  static constexpr bool own = ST < OZ_PROJ;  // a GemmStage of stages.cuh
  static constexpr bool A = own && StageFlags<ST>::conjA;
  static constexpr bool B = ST == OZ_GRAM;
  static constexpr bool C = ST == OZ_PROJ || (own && StageFlags<ST>::conjC);
};

// The stages that skip a bond: the contraction and gate GEMMs run only for
// bonds with a pre-gate buffer.
template <int ST>
__device__ __forceinline__ bool oz_skip(const ProbPtr& P) {
  return (ST == OZ_THETA || ST == OZ_GATE) && P.Cpre == nullptr;
}

// Element (i, j) of C into its destination.
template <int ST>
__device__ __forceinline__ void oz_store(const Dims& D, const ProbPtr& P, const OzOp& op, int i, int j, double re,
                                         double im) {
  if constexpr (ST == OZ_THETA) {
    // lam_l[alpha] lam_r[beta] scale the contraction (rows (i, alpha), columns (j, beta))
    op.C[(int64_t)i * D.n + j] = cscale(cmk(re, im), P.laml[i % D.cl] * P.lamr[j % D.cr]);
  } else if constexpr (ST == OZ_GATE) {
    const int a = i / D.dr, b = i - a * D.dr, al = j / D.cr, be = j - al * D.cr;  // rows (i, j), columns (alpha, beta)
    op.C[(int64_t)(a * D.cl + al) * D.n + b * D.cr + be] = cmk(re, im);
  } else {
    if (ST == OZ_GRAM && i == j) re -= 1.0;  // E = Q_f^H Q_f - I
    op.C[(int64_t)i * op.crs + (int64_t)j * op.ccs] = cmk(re, OzConj<ST>::C ? -im : im);
  }
}

// Operand sources of k_oz_digits_op in their K-major views: element (row, k)
// of side 0 (rows of op(A)) or side 1 (columns of op(B)), and whether
// consecutive rows are adjacent in memory (else consecutive k are).
template <int ST, int SIDE>
struct OzSrc {  // a GemmStage: strided operand of the stage table
  const cplx* X;
  int64_t rs, ks;
  int rows, K;
  __device__ OzSrc(const Dims& D, const ProbPtr& P) {
    const GemmOp g = gemm_of<ST>(D, P);
    rows = SIDE == 0 ? g.M : g.N;
    K = g.K;
    X = SIDE == 0 ? g.A : g.B;
    rs = SIDE == 0 ? g.ars : g.bcs;
    ks = SIDE == 0 ? g.acs : g.brs;
  }
  __device__ bool rows_contig() const { return rs == 1; }
  __device__ cplx at(int r, int k) const { return X[(int64_t)r * rs + (int64_t)k * ks]; }
};
template <int SIDE>
struct OzSrc<OZ_THETA, SIDE> {  // A = Gamma_l (rows (i, alpha)), B = lam_m Gamma_r (columns (j, beta))
  Dims D;
  const ProbPtr* P;
  int rows, K;
  __device__ OzSrc(const Dims& d, const ProbPtr& p) : D(d), P(&p) {
    rows = SIDE == 0 ? d.dl * d.cl : d.dr * d.cr;
    K = d.cm;
  }
  __device__ bool rows_contig() const { return SIDE == 1; }
  __device__ cplx at(int r, int g) const {
    if (SIDE == 0) {
      const int i = r / D.cl, al = r - i * D.cl;
      return P->gl[((int64_t)i * P->cap_l + al) * P->cap_m + g];
    }
    const int j = r / D.cr, be = r - j * D.cr;
    return cscale(P->gr[((int64_t)j * P->cap_m + g) * P->cap_r + be], P->lamm[g]);
  }
};
template <int SIDE>
struct OzSrc<OZ_GATE, SIDE> {  // A = the gate (rows (i, j)), B = the (i', j') x (alpha, beta) gather of C
  Dims D;
  const ProbPtr* P;
  int rows, K;
  __device__ OzSrc(const Dims& d, const ProbPtr& p) : D(d), P(&p) {
    rows = SIDE == 0 ? d.dl * d.dr : d.cl * d.cr;
    K = d.dl * d.dr;
  }
  __device__ bool rows_contig() const { return SIDE == 1; }
  __device__ cplx at(int r, int k) const {
    if (SIDE == 0) return P->gate[(int64_t)r * (D.dl * D.dr) + k];
    const int ip = k / D.dr, jp = k - ip * D.dr, al = r / D.cr, be = r - al * D.cr;
    return P->Cpre[(int64_t)(ip * D.cl + al) * D.n + jp * D.cr + be];
  }
};

// Digits of a stage operand in its K-major view: SIDE 0 the rows i of op(A)
// (element A[i ars + k acs], not conjugated: the MMAs conjugate), SIDE 1 the
// columns j of op(B) (element B[k brs + j bcs]); into Xd[z][reim][t][row][k]
// (rows rc, Kp per row) and scales Xs[z][kb][row].  A CTA takes 16 rows x 64
// k; rows and k past the instance's own extents become zero digits.
template <int ST, int SIDE>
__global__ void __launch_bounds__(256) k_oz_digits_op(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                      uint16_t* Xd, float* Xs, int rc, int Kp) {
  __shared__ cplx tile[16][OZ_KB + 1];
  __shared__ uint16_t dig[2 * OZ_S][16][OZ_KB + 2];  // [reim t][row][k]
  const int z = blockIdx.z;
  const Dims D = dims[z];
  if (!D.active || oz_skip<ST>(ptrs[z])) return;
  const OzSrc<ST, SIDE> src(D, ptrs[z]);
  const int rows = src.rows, K = src.K;
  const bool rowc = src.rows_contig();
  const int r0 = blockIdx.x * 16, k0 = blockIdx.y * OZ_KB;
  const int tid = threadIdx.x;
  for (int e = tid; e < 16 * OZ_KB; e += 256) {
    int r, k;  // consecutive threads along the unit-stride direction
    if (rowc) { r = e & 15; k = e >> 4; } else { k = e & (OZ_KB - 1); r = e >> 6; }
    const int gr = r0 + r, gk = k0 + k;
    tile[r][k] = (gr < rows && gk < K) ? src.at(gr, gk) : cmk(0.0, 0.0);
  }
  __syncthreads();
  const int r = tid >> 4, pq = tid & 15;  // 16 threads per row, 4 k each
  cplx v[4];
  int E = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = tile[r][pq * 4 + q];
    const uint64_t ur = (uint64_t)__double_as_longlong(v[q].x), ui = (uint64_t)__double_as_longlong(v[q].y);
    const int er = (int)((ur >> 52) & 0x7FF), ei = (int)((ui >> 52) & 0x7FF);
    E = max(E, max(er == 0x7FF ? 0 : er, ei == 0x7FF ? 0 : ei));
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));  // within the row's 16 lanes
  const float sc = oz_scale(E, 1030);
  const bool live = sc != 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = pq * 4 + q;
    const uint64_t nr = live ? oz_n48_f64(v[q].x, E) : 0, ni = live ? oz_n48_f64(v[q].y, E) : 0;
    const bool sr = v[q].x < 0.0, si = v[q].y < 0.0;
#pragma unroll
    for (int t = 0; t < OZ_S; ++t) {
      dig[t][r][k] = oz_bf16_digit((unsigned)((nr >> (40 - 8 * t)) & 0xFF), t, sr);
      dig[OZ_S + t][r][k] = oz_bf16_digit((unsigned)((ni >> (40 - 8 * t)) & 0xFF), t, si);
    }
  }
  if (pq == 0 && r0 + r < rc) Xs[((size_t)z * (Kp / OZ_KB) + blockIdx.y) * rc + r0 + r] = live ? sc : 0.f;
  __syncthreads();
  uint16_t* base = Xd + (size_t)z * 2 * OZ_S * rc * Kp;
  for (int w = tid; w < 2 * OZ_S * 16 * 8; w += 256) {
    const int q = w & 7, row = w >> 3, rr = row & 15, rt = row >> 4;
    if (r0 + rr >= rc) continue;
    const uint16_t* src = &dig[rt][rr][q * 8];
    uint4 pk;
    pk.x = (unsigned)src[0] | ((unsigned)src[1] << 16);
    pk.y = (unsigned)src[2] | ((unsigned)src[3] << 16);
    pk.z = (unsigned)src[4] | ((unsigned)src[5] << 16);
    pk.w = (unsigned)src[6] | ((unsigned)src[7] << 16);
    *reinterpret_cast<uint4*>(base + ((size_t)rt * rc + r0 + rr) * Kp + k0 + q * 8) = pk;
  }
}

// ---------------------------------------------------------------------------
// The digit-pair GEMM.
// ---------------------------------------------------------------------------
struct OzArgs {
  int lc, nc, Kp;      // capacities: rows of C, columns of C, padded k
  const float* As;     // [z][kb][i]
  const float* Bs;     // [z][kb][j]
  int* err;
  uint32_t poll_limit;
  int stall;
};

__device__ __forceinline__ void oz_tma_load_5d(void* dst, const CUtensorMap* tm, int c0, int c1, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(tc_smem_u32(dst)),
      "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(0), "r"(0), "r"(c4), "r"(tc_smem_u32(bar))
      : "memory");
}

// K-major, 32-byte swizzle: 8-row atoms of 256 bytes (stride byte offset 256).
__device__ __forceinline__ uint64_t oz_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused: one atom along k)
  d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)6 << 61;            // 32-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, K-major, M x N.
__host__ __device__ constexpr uint32_t oz_idesc(int M, int N, bool negA) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negA ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void oz_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void oz_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem_u32(bar)) : "memory");
}

// Warp-uniform bounded wait: lane 0 polls, the warp gets its answer.
__device__ __forceinline__ bool oz_warp_wait(uint64_t* bar, uint32_t parity, uint32_t limit, int* err,
                                             volatile int* abort_flag) {
  bool ok = false;
  if ((threadIdx.x & 31) == 0) ok = tc_mbar_wait(bar, parity, limit, err, abort_flag);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// four consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void oz_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}

// acc (h, l) += s (hs, ls), then renormalised
__device__ __forceinline__ void oz_df_add(float& h, float& l, float hs, float ls) {
  float t, e;
  two_sum(h, hs, t, e);
  e += l + ls;
  h = t + e;
  l = e - (h - t);
}

template <int ST>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs, OzArgs a) {
  extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
  const int z = blockIdx.z;
  const Dims D = dims[z];
  const int i0 = blockIdx.y * OZ_BM, j0 = blockIdx.x * OZ_BN;
  if (!D.active || oz_skip<ST>(ptrs[z])) return;
  const OzOp op = oz_op<ST>(D, ptrs[z]);
  if (i0 >= op.M || j0 >= op.N) return;  // uniform: before any barrier or allocation
  uint8_t* smem = (uint8_t*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + OZ_STAGES * OZ_A_STAGE;
  uint64_t* full = (uint64_t*)(sB + OZ_STAGES * OZ_B_STAGE);
  uint64_t* empty = full + OZ_STAGES;
  uint64_t* accf = empty + OZ_STAGES;
  uint64_t* accfree = accf + 1;
  uint64_t* drain = accfree + 1;
  uint32_t* tmem_holder = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nks = (min(op.K, a.Kp) + OZ_KS - 1) / OZ_KS;  // k steps of this instance
  const int nkb = (nks + (OZ_DRAIN / OZ_KS) - 1) / (OZ_DRAIN / OZ_KS);  // exact accumulation blocks
  const int iters = nkb * (OZ_DRAIN / OZ_KS);  // whole blocks (zero digits past m)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tmem_holder)),
                 "r"((uint32_t)OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      tc_mbar_init(&full[s], 1);
      tc_mbar_init(&empty[s], 1);
    }
    tc_mbar_init(accf, 1);
    tc_mbar_init(accfree, OZ_EPI_WARPS);
    tc_mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      int issued = 0;
      for (int it = 0; it < (a.stall ? 0 : iters); ++it) {
        const int s = it % OZ_STAGES;
        const uint32_t r = (uint32_t)(it / OZ_STAGES);
        if (it >= OZ_STAGES && !tc_mbar_wait(&empty[s], (r & 1u) ^ 1u, a.poll_limit, a.err, abort_flag)) break;
        tc_mbar_expect_tx(&full[s], OZ_A_STAGE + OZ_B_STAGE);
        oz_tma_load_5d(sA + s * OZ_A_STAGE, &tmA, it * OZ_KS, i0, z, &full[s]);
        oz_tma_load_5d(sB + s * OZ_B_STAGE, &tmB, it * OZ_KS, j0, z, &full[s]);
        issued = it + 1;
      }
      if (*abort_flag) {  // every copy issued lands before the teardown
        for (int it = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); it < issued; ++it)
          for (uint32_t i = 0; i < (1u << 22); ++i)
            if (tc_mbar_try_wait(&full[it % OZ_STAGES], (uint32_t)(it / OZ_STAGES) & 1u)) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: per k step the 21 digit pairs (t, u) with t + u <= 7,
      // as six MMAs per real product
      bool ok = true;
      int issued_mma = 0;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        if (kb > 0 && !tc_mbar_wait(accfree, (uint32_t)(kb - 1) & 1u, a.poll_limit, a.err, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int ks = 0; ks < OZ_DRAIN / OZ_KS; ++ks) {
          const int it = kb * (OZ_DRAIN / OZ_KS) + ks;
          const int s = it % OZ_STAGES;
          if (!tc_mbar_wait(&full[s], (uint32_t)(it / OZ_STAGES) & 1u, a.poll_limit, a.err, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = tc_smem_u32(sA + s * OZ_A_STAGE), bbase = tc_smem_u32(sB + s * OZ_B_STAGE);
          // digit t of A times planes u = 1 .. 7 - t of B (adjacent in shared
          // memory) into the accumulators of levels t + 1 .. 7 (adjacent in
          // tensor memory); the t = 1 MMAs of a block's first k step cover
          // every level and start the block's sums
          const uint64_t br = oz_desc_sw32(bbase), bi = oz_desc_sw32(bbase + OZ_S * OZ_B_TILE);
#pragma unroll 1
          for (int t = 1; t <= OZ_S; ++t) {
            const int N = OZ_BN * (OZ_S + 1 - t);
            const uint32_t ip = oz_idesc(OZ_BM, N, false), in = oz_idesc(OZ_BM, N, true);
            const uint32_t acc0 = (ks == 0 && t == 1) ? 0u : 1u;
            const uint32_t dr = tmem + (uint32_t)(OZ_BN * (t - 1)), di = tmem + (uint32_t)(OZ_BN * (OZ_NGRP + t - 1));
            const uint64_t ar = oz_desc_sw32(abase + (0 * OZ_S + t - 1) * OZ_A_TILE);
            const uint64_t ai = oz_desc_sw32(abase + (1 * OZ_S + t - 1) * OZ_A_TILE);
            // signs of a conjugated operand: C_r = Ar Br - sA sB Ai Bi,
            // C_i = sB Ar Bi + sA Ai Br with s = -1 for a conjugated side
            constexpr bool cA = OzConj<ST>::A, cB = OzConj<ST>::B;
            oz_mma(dr, ar, br, ip, acc0);                         // C_r += Ar Br
            oz_mma(dr, ai, bi, (cA != cB) ? ip : in, 1u);         // C_r -= Ai Bi
            oz_mma(di, ar, bi, cB ? in : ip, acc0);               // C_i += Ar Bi
            oz_mma(di, ai, br, cA ? in : ip, 1u);                 // C_i += Ai Br
          }
          oz_commit(&empty[s]);  // the stage is free once these MMAs have read it
          issued_mma = it + 1;
        }
        if (!ok) break;
        oz_commit(accf);  // block kb's sums are ready
      }
      if (!ok) {
        *abort_flag = 1;
        if (issued_mma > 0) {  // the MMAs issued read shared memory and write the tensor memory freed below
          oz_commit(drain);
          for (uint32_t i = 0; i < a.poll_limit; ++i)
            if (tc_mbar_try_wait(drain, 0)) break;
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads lanes 32 (w % 4) .. +31 and a quarter of the columns
    const int ew = warp - 2, quad = warp & 3, part = ew >> 2;
    const int i = i0 + 32 * quad + lane;  // row of C
    const int jq = j0 + 8 * part;         // first column of this warp
    const int nkbt = a.Kp / OZ_KB;        // k blocks of the scale arrays
    float hr[8], lr[8], hi[8], li[8];      // double-float sums (Re, Im) of 8 columns
#pragma unroll
    for (int c = 0; c < 8; ++c) hr[c] = lr[c] = hi[c] = li[c] = 0.f;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      // the block scales first: their loads overlap the wait for the MMAs
      const int sb = kb / (OZ_KB / OZ_DRAIN);  // the scale block holding this accumulation block
      const float sa = (i < a.lc) ? a.As[((size_t)z * nkbt + sb) * a.lc + i] : 0.f;
      const float* sbp = a.Bs + ((size_t)z * nkbt + sb) * a.nc;
      float sbv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) sbv[c] = (jq + c < a.nc) ? __ldg(sbp + jq + c) : 0.f;
      ok = oz_warp_wait(accf, (uint32_t)kb & 1u, a.poll_limit, a.err, abort_flag);
      if (!ok) break;
      tc_fence_after();
      const uint32_t lanes = (uint32_t)(32 * quad) << 16;
#pragma unroll
      for (int c4 = 0; c4 < 8; c4 += 4) {  // four columns of every accumulator per load
        float v[2 * OZ_NGRP][4];
#pragma unroll
        for (int g = 0; g < 2 * OZ_NGRP; ++g) oz_ld4(tmem + lanes + (uint32_t)(OZ_BN * g + 8 * part + c4), v[g]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float sc = sa * sbv[c4 + q];
          // levels 2, 3, 4 exactly into (s, e + e2), levels 5, 6, 7 into the low part
          float s, e, s2, e2;
          two_sum(v[0][q], v[1][q], s, e);
          two_sum(s, v[2][q], s2, e2);
          float lo = (e + e2) + (v[3][q] + (v[4][q] + v[5][q]));
          oz_df_add(hr[c4 + q], lr[c4 + q], s2 * sc, lo * sc);
          two_sum(v[6][q], v[7][q], s, e);
          two_sum(s, v[8][q], s2, e2);
          lo = (e + e2) + (v[9][q] + (v[10][q] + v[11][q]));
          oz_df_add(hi[c4 + q], li[c4 + q], s2 * sc, lo * sc);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) oz_arrive(accfree);  // the accumulators may be overwritten
    }
    if (ok && i < op.M) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = jq + c;
        if (j < op.N) oz_store<ST>(D, ptrs[z], op, i, j, (double)hr[c] + (double)lr[c], (double)hi[c] + (double)li[c]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)OZ_TMEM_COLS)
                 : "memory");
  }
}

static size_t oz_smem_bytes() { return 1024 + (size_t)OZ_STAGES * (OZ_A_STAGE + OZ_B_STAGE) + (2 * OZ_STAGES + 3) * 8 + 16; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*OzEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static OzEncodeFn oz_encode_fn() {
  static std::mutex mu;
  static OzEncodeFn fn = nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (OzEncodeFn)p;
  }
  return fn;
}

// 5-D map over digit arrays [z][reim][t][row][k] (BF16): box 16 k x box_rows
// rows x all digits x both parts x one instance, 32-byte swizzle.
static bool oz_make_map(CUtensorMap* m, const uint16_t* base, int Kp, int rows, int batch, int box_rows) {
  OzEncodeFn enc = oz_encode_fn();
  if (!enc) return false;
  cuuint64_t dims[5] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)OZ_S, 2, (cuuint64_t)batch};
  const cuuint64_t rb = (cuuint64_t)Kp * 2;
  cuuint64_t strides[4] = {rb, rb * rows, rb * rows * OZ_S, rb * rows * OZ_S * 2};
  cuuint32_t box[5] = {(cuuint32_t)OZ_KS, (cuuint32_t)box_rows, (cuuint32_t)OZ_S, 2, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)base, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int oz_kpad(int m) { return ((m + OZ_KB - 1) / OZ_KB) * OZ_KB; }

size_t oz_digits_bytes(int rows, int m) { return (size_t)2 * OZ_S * rows * oz_kpad(m) * sizeof(uint16_t); }
size_t oz_scales_bytes(int rows, int m) { return (size_t)(oz_kpad(m) / OZ_KB) * rows * sizeof(float); }

template <int ST>
static cudaError_t oz_attr() {
  return cudaFuncSetAttribute(k_oz_gemm<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
}

cudaError_t oz_prepare() {
  if (!oz_encode_fn()) return cudaErrorNotSupported;
  static int done = 0;
  if (!done) {
    const cudaError_t es[] = {oz_attr<OZ_PROJ>(), oz_attr<OZ_GRAM>(), oz_attr<G_G1>(), oz_attr<G_Q1>(), oz_attr<G_G2>(),
                              oz_attr<G_QB>(),    oz_attr<G_X>(),  oz_attr<G_U>(),  oz_attr<G_V>(),
                              oz_attr<OZ_THETA>(), oz_attr<OZ_GATE>()};
    for (cudaError_t e : es)
      if (e != cudaSuccess) return e;
    done = 1;
  }
  return cudaSuccess;
}

// Capacities (rows of C, columns of C, depth) of a stage's product.
static void oz_stage_caps(int stage, const Caps& c, int& Mc, int& Nc, int& Kc) {
  switch (stage) {
    case G_G1: case G_G2: case G_X: Mc = c.l; Nc = c.l; Kc = c.n; break;
    case G_Q1: case G_QB: Mc = c.n; Nc = c.l; Kc = c.l; break;
    case G_U: Mc = c.m; Nc = c.k; Kc = c.l; break;
    case OZ_THETA: Mc = c.m; Nc = c.n; Kc = c.cm; break;  // K = chi_m, at most its bond's capacity
    case OZ_GATE: Mc = c.dl * c.dr; Nc = c.cl * c.cr; Kc = c.dl * c.dr; break;
    default: Mc = c.n; Nc = c.k; Kc = c.l; break;  // G_V
  }
}

bool oz_stage_rule(const Caps& cap) { return cap.l >= 48 && (cap.m >= 256 || cap.n >= 256); }

static const int OZ_STAGE_LIST[] = {G_G1, G_Q1, G_G2, G_QB, G_X, G_U, G_V};

static void oz_grow(OzStageBytes& b, int stage, const Caps& c) {
  int Mc, Nc, Kc;
  oz_stage_caps(stage, c, Mc, Nc, Kc);
  b.ad = std::max(b.ad, oz_digits_bytes(Mc, Kc));
  b.as = std::max(b.as, oz_scales_bytes(Mc, Kc));
  b.bd = std::max(b.bd, oz_digits_bytes(Nc, Kc));
  b.bs = std::max(b.bs, oz_scales_bytes(Nc, Kc));
}

OzStageBytes oz_stage_bytes(int m, int n, int k, int l, const Caps* gate) {
  OzStageBytes b{0, 0, 0, 0};
  Caps c{};
  c.m = m; c.n = n; c.k = k; c.l = l;
  for (int stage : OZ_STAGE_LIST) oz_grow(b, stage, c);
  if (gate && gate->dl * gate->dr >= GATE_GEMM_MIN) {
    oz_grow(b, OZ_THETA, *gate);
    oz_grow(b, OZ_GATE, *gate);
  }
  return b;
}

bool oz_gate_rule(const Caps& cap) { return cap.dl * cap.dr >= GATE_GEMM_MIN; }

template <int ST>
static cudaError_t oz_stage_run(const Dims* dims, const ProbPtr* ptrs, int batch, int Mc, int Nc, int Kc,
                                const OzScratch& sc, int* err, cudaStream_t st) {
  const int Kp = oz_kpad(Kc);
  // G1 and G2 multiply an operand by its own adjoint: one set of digits
  const bool same = ST == G_G1 || ST == G_G2;
  {
    ProfScope ps("k_oz_digits[op]", st);
    k_oz_digits_op<ST, 0><<<dim3((Mc + 15) / 16, Kp / OZ_KB, batch), 256, 0, st>>>(dims, ptrs, sc.ad, sc.as, Mc, Kp);
    if (!same)
      k_oz_digits_op<ST, 1><<<dim3((Nc + 15) / 16, Kp / OZ_KB, batch), 256, 0, st>>>(dims, ptrs, sc.bd, sc.bs, Nc,
                                                                                      Kp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  CUtensorMap ta, tb;
  if (!oz_make_map(&ta, sc.ad, Kp, Mc, batch, OZ_BM) || !oz_make_map(&tb, same ? sc.ad : sc.bd, Kp, Nc, batch, OZ_BN))
    return cudaErrorInvalidValue;
  OzArgs oa;
  oa.lc = Mc;
  oa.nc = Nc;
  oa.Kp = Kp;
  oa.As = sc.as;
  oa.Bs = same ? sc.as : sc.bs;
  oa.err = err;
  oa.poll_limit = 1u << 24;
  oa.stall = 0;
  ProfScope ps(ST == G_U || ST == G_V ? "k_oz_gemm[uv]"
               : ST == OZ_THETA          ? "k_oz_gemm[theta]"
               : ST == OZ_GATE           ? "k_oz_gemm[gate]"
                                         : "k_oz_gemm[cholqr]",
               st);
  k_oz_gemm<ST><<<dim3((Nc + OZ_BN - 1) / OZ_BN, (Mc + OZ_BM - 1) / OZ_BM, batch), OZ_THREADS, oz_smem_bytes(), st>>>(
      ta, tb, dims, ptrs, oa);
  return cudaGetLastError();
}

cudaError_t launch_oz_stage(int stage, const Dims* dims, const ProbPtr* ptrs, int batch, const Caps& cap,
                            const OzScratch& sc, int* err, cudaStream_t st) {
  const cudaError_t e = oz_prepare();
  if (e != cudaSuccess) return e;
  int Mc, Nc, Kc;
  oz_stage_caps(stage, cap, Mc, Nc, Kc);
  switch (stage) {
    case OZ_THETA:
      if (!oz_gate_rule(cap)) return cudaSuccess;
      return oz_stage_run<OZ_THETA>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case OZ_GATE:
      if (!oz_gate_rule(cap)) return cudaSuccess;
      return oz_stage_run<OZ_GATE>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_G1: return oz_stage_run<G_G1>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_Q1: return oz_stage_run<G_Q1>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_G2: return oz_stage_run<G_G2>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_QB: return oz_stage_run<G_QB>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_X: return oz_stage_run<G_X>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_U: return oz_stage_run<G_U>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    case G_V: return oz_stage_run<G_V>(dims, ptrs, batch, Mc, Nc, Kc, sc, err, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_oz_digits_theta(const Dims* dims, const ProbPtr* ptrs, uint16_t* Bd, float* Bs, int m, int n,
                                   int batch, cudaStream_t st) {
  ProfScope ps("k_oz_digits[theta]", st);
  const int Kp = oz_kpad(m);
  k_oz_digits_theta<<<dim3((n + 15) / 16, Kp / OZ_KB, batch), 256, 0, st>>>(dims, ptrs, Bd, Bs, n, Kp);
  return cudaGetLastError();
}

cudaError_t launch_oz_digits_qf(const Dims* dims, const float2* Qf, uint16_t* Ad, float* As, int m, int l, int batch,
                                cudaStream_t st) {
  const int Kp = oz_kpad(m);
  ProfScope ps("k_oz_digits[q]", st);
  const int warps = l * (Kp / OZ_KB);
  k_oz_digits_q<<<dim3((warps + 7) / 8, batch), 256, 0, st>>>(dims, Qf, Ad, As, m, l, Kp);
  return cudaGetLastError();
}

cudaError_t launch_oz_gram(const Dims* dims, const ProbPtr* ptrs, const uint16_t* Ad, const float* As, int m, int l,
                           int batch, int* err, cudaStream_t st) {
  const cudaError_t e = oz_prepare();
  if (e != cudaSuccess) return e;
  const int Kp = oz_kpad(m);
  CUtensorMap ta, tb;
  if (!oz_make_map(&ta, Ad, Kp, l, batch, OZ_BM) || !oz_make_map(&tb, Ad, Kp, l, batch, OZ_BN))
    return cudaErrorInvalidValue;
  OzArgs oa;
  oa.lc = l;
  oa.nc = l;
  oa.Kp = Kp;
  oa.As = As;
  oa.Bs = As;
  oa.err = err;
  oa.poll_limit = 1u << 24;
  oa.stall = 0;
  ProfScope ps("k_oz_gemm[gram]", st);
  k_oz_gemm<OZ_GRAM><<<dim3((l + OZ_BN - 1) / OZ_BN, (l + OZ_BM - 1) / OZ_BM, batch), OZ_THREADS, oz_smem_bytes(),
                       st>>>(ta, tb, dims, ptrs, oa);
  return cudaGetLastError();
}

cudaError_t launch_proj_oz(const Dims* dims, const ProbPtr* ptrs, const float2* Qf, const float2* Dbuf,
                           uint16_t* Ad, float* As, const uint16_t* Bd, const float* Bs, int m, int n, int l, int batch,
                           int* err, cudaStream_t st, bool digits_done) {
  const int Kp = oz_kpad(m);
  if (!digits_done) {
    cudaError_t e = launch_oz_digits_qf(dims, Qf, Ad, As, m, l, batch, st);
    if (e != cudaSuccess) return e;
  }
  {
    cudaError_t e = oz_prepare();
    if (e != cudaSuccess) return e;
    CUtensorMap ta, tb;
    if (!oz_make_map(&ta, Ad, Kp, l, batch, OZ_BM) || !oz_make_map(&tb, Bd, Kp, n, batch, OZ_BN))
      return cudaErrorInvalidValue;
    OzArgs oa;
    oa.lc = l;
    oa.nc = n;
    oa.Kp = Kp;
    oa.As = As;
    oa.Bs = Bs;
    oa.err = err;
    // an injected pipeline stall (test hook), never inside a stream capture
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap_st) != cudaSuccess) cap_st = cudaStreamCaptureStatusActive;
    const bool stall = cap_st == cudaStreamCaptureStatusNone && fault_take(TEBD_FAULT_TC_STALL);
    oa.poll_limit = stall ? (1u << 12) : (1u << 24);
    oa.stall = stall ? 1 : 0;
    ProfScope ps("k_oz_proj[project]", st);
    k_oz_gemm<OZ_PROJ><<<dim3((n + OZ_BN - 1) / OZ_BN, (l + OZ_BM - 1) / OZ_BM, batch), OZ_THREADS, oz_smem_bytes(),
                         st>>>(ta, tb, dims, ptrs, oa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_fold_bh(Dbuf, dims, ptrs, n, l, batch, st);
}

}  // namespace tg
