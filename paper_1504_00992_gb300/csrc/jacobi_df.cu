// One-sided Jacobi SVD of X = Rb^H in double-float arithmetic (sm_103a), the
// small SVD of Section IV's step ii in the mixed form.
//
// The method of k_jacobi (round-robin pairs, one group of JD_G lanes per
// pair, the convergence test |g|^2 > tol^2 |x_a|^2 |x_b|^2, negligible
// columns skipped, X J = W S with J accumulating the rotations), with X and
// J held as FP32 pairs (hi + lo, 2^-48 relative) and every operation on
// their elements in FP32 arithmetic: products by FMA splitting (Dekker /
// Ogita-Rump-Oishi), sums by TwoSum.  GB300 runs FP64 at 1/64 of its FP32
// rate, and the element loops (inner products and rotations of X and J) are
// nearly all of the SVD's work, so they run several times faster this way.
//
// The rotation angle needs no more than FP32 accuracy: a rotation by a
// slightly wrong angle leaves an off-diagonal element ~1e-7 of the one it
// removes, which the next sweep removes (the convergence stays fast), but
// the rotation must be unitary to working accuracy, so c, s and the phase e
// (|e| = 1) are formed in double-float from the FP32 angle: c = 1 / sqrt(1 +
// t^2), s = c t with one Newton step each, e = g / |g| normalised likewise.
//
// X is scaled by a power of two to max |x| in [1, 2) first (exact), so that
// squares and products stay in FP32's range, and scaled back at the end;
// columns with |x|^2 below (L u)^2 ||X||_F^2 are left alone, as in k_jacobi.
// tol = 8 u sqrt(L) with u = 2^-48, above the rounding noise of a
// double-float inner product.  X and J are stored in place of the FP64
// matrices P.R and P.J (one complex element = 4 floats = 16 bytes) and
// converted back before jacobi_finish.
#include <cuda_runtime.h>
#include <math.h>

#include "dfsplit.cuh"
#include "internal.cuh"
#include "profiler.cuh"
#include "stages.cuh"

namespace tg {

enum { JD_G = 8, JD_THREADS = 512, JD_MAXSWEEPS = 60 };

// lazy accumulation of products into (h, lo), renormalised by the caller
__device__ __forceinline__ void acc_dd(float& h, float& lo, float xh, float xl, float yh, float yl) {
  dfx_dd(h, lo, xh, xl, yh, yl);
}

__device__ __forceinline__ dfl grp_dsum(dfl v, unsigned mask) {
#pragma unroll
  for (int o = JD_G / 2; o > 0; o >>= 1) {
    const dfl w{__shfl_xor_sync(mask, v.h, o), __shfl_xor_sync(mask, v.l, o)};
    v = dadd(v, w);
  }
  return v;
}

// u' = c u - conj(se) v, v' = se u + c v for one complex element of each
// column (float4 = Re hi, Re lo, Im hi, Im lo)
__device__ __forceinline__ void drot(float4& u, float4& v, dfl c, dfl sr, dfl si) {
  float h, lo;
  float4 nu, nv;
  // Re u' = c ur - sr vr - si vi
  h = 0.f; lo = 0.f;
  acc_dd(h, lo, c.h, c.l, u.x, u.y);
  acc_dd(h, lo, -sr.h, -sr.l, v.x, v.y);
  acc_dd(h, lo, -si.h, -si.l, v.z, v.w);
  fast2(h, lo); nu.x = h; nu.y = lo;
  // Im u' = c ui - sr vi + si vr
  h = 0.f; lo = 0.f;
  acc_dd(h, lo, c.h, c.l, u.z, u.w);
  acc_dd(h, lo, -sr.h, -sr.l, v.z, v.w);
  acc_dd(h, lo, si.h, si.l, v.x, v.y);
  fast2(h, lo); nu.z = h; nu.w = lo;
  // Re v' = sr ur - si ui + c vr
  h = 0.f; lo = 0.f;
  acc_dd(h, lo, sr.h, sr.l, u.x, u.y);
  acc_dd(h, lo, -si.h, -si.l, u.z, u.w);
  acc_dd(h, lo, c.h, c.l, v.x, v.y);
  fast2(h, lo); nv.x = h; nv.y = lo;
  // Im v' = sr ui + si ur + c vi
  h = 0.f; lo = 0.f;
  acc_dd(h, lo, sr.h, sr.l, u.z, u.w);
  acc_dd(h, lo, si.h, si.l, u.x, u.y);
  acc_dd(h, lo, c.h, c.l, v.z, v.w);
  fast2(h, lo); nv.z = h; nv.w = lo;
  u = nu;
  v = nv;
}

enum { JD_U = 4 };  // rows of a lane loaded before any is used (loads in flight together)

// g = x_a^H x_b over the rows gl, gl + JD_G, ... of this lane (lazy pair sums)
__device__ __forceinline__ void jd_dot(const float4* xa, const float4* xb, int L, int gl, float& gr, float& grl,
                                       float& gi, float& gil) {
  for (int r0 = gl; r0 < L; r0 += JD_G * JD_U) {
    float4 x[JD_U], y[JD_U];
#pragma unroll
    for (int u = 0; u < JD_U; ++u) {
      const int r = r0 + u * JD_G;
      x[u] = r < L ? xa[r] : make_float4(0.f, 0.f, 0.f, 0.f);
      y[u] = r < L ? xb[r] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < JD_U; ++u) {
      acc_dd(gr, grl, x[u].x, x[u].y, y[u].x, y[u].y);
      acc_dd(gr, grl, x[u].z, x[u].w, y[u].z, y[u].w);
      acc_dd(gi, gil, x[u].x, x[u].y, y[u].z, y[u].w);
      acc_dd(gi, gil, -x[u].z, -x[u].w, y[u].x, y[u].y);
    }
  }
}

// (x_a, x_b) <- (c x_a - conj(se) x_b, se x_a + c x_b) on this lane's rows
__device__ __forceinline__ void jd_rot(float4* xa, float4* xb, int L, int gl, dfl c, dfl sr, dfl si) {
  for (int r0 = gl; r0 < L; r0 += JD_G * JD_U) {
    float4 x[JD_U], y[JD_U];
#pragma unroll
    for (int u = 0; u < JD_U; ++u) {
      const int r = r0 + u * JD_G;
      if (r < L) {
        x[u] = xa[r];
        y[u] = xb[r];
      }
    }
#pragma unroll
    for (int u = 0; u < JD_U; ++u) {
      const int r = r0 + u * JD_G;
      if (r < L) {
        drot(x[u], y[u], c, sr, si);
        xa[r] = x[u];
        xb[r] = y[u];
      }
    }
  }
}

// Dynamic shared memory of an instance of L columns: X (XS: L^2 complex
// double-float), squared column norms, reduction scratch, and sigma / perm
// for jacobi_finish (in X's place once X is written back, XS).
// Every part starts on a 16-byte boundary.
__host__ __device__ inline size_t jd_up16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline size_t jd_head_bytes(int L, bool xs) {
  const size_t x = xs ? (size_t)L * L * sizeof(float4) : 0;
  const size_t fin = jd_up16((size_t)L * (sizeof(double) + sizeof(int)));
  return x > fin ? x : fin;
}
__host__ __device__ inline size_t jd_smem_bytes(int L, bool xs) {
  return jd_head_bytes(L, xs) + jd_up16((size_t)L * sizeof(float2)) + 32 * sizeof(double) + 33 * sizeof(int);
}

template <bool XS>
__global__ void __launch_bounds__(JD_THREADS) k_jacobi_df(const Dims* __restrict__ dims,
                                                          const ProbPtr* __restrict__ ptrs, int* status) {
  extern __shared__ __align__(16) unsigned char jd_smem[];
  const int p = blockIdx.x;
  const Dims D = dims[p];
  if (!D.active) return;
  const ProbPtr& P = ptrs[p];
  const int L = D.l;
  // shared layout (this instance's L): [X or sigma / perm][norms][red][emax][rotated]
  unsigned char* tail = jd_smem + jd_head_bytes(L, XS);
  float2* nrm = reinterpret_cast<float2*>(tail);  // squared column norms, double-float
  double* red = reinterpret_cast<double*>(tail + jd_up16((size_t)L * sizeof(float2)));
  int* emax = reinterpret_cast<int*>(red + 32);
  int& rotated = emax[32];
  double* sv = reinterpret_cast<double*>(jd_smem);
  int* perm = reinterpret_cast<int*>(jd_smem + (size_t)L * sizeof(double));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gl = lane & (JD_G - 1);
  const int grp = tid / JD_G, ngrp = blockDim.x / JD_G;
  const unsigned gmask = ((1u << JD_G) - 1u) << (lane & ~(JD_G - 1));
  cplx* X64 = P.R;
  cplx* J64 = P.J;
  float4* X = XS ? reinterpret_cast<float4*>(jd_smem) : reinterpret_cast<float4*>(P.R);
  float4* J = reinterpret_cast<float4*>(P.J);

  // the scale: largest biased exponent among the entries of X
  int e = 0;
  for (int i = tid; i < L * L; i += blockDim.x) {
    const cplx v = X64[i];
    const int er = (int)(((unsigned long long)__double_as_longlong(v.x) >> 52) & 0x7FF);
    const int ei = (int)(((unsigned long long)__double_as_longlong(v.y) >> 52) & 0x7FF);
    e = max(e, max(er == 0x7FF ? 0 : er, ei == 0x7FF ? 0 : ei));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) emax[warp] = e;
  __syncthreads();
  if (tid == 0) {
    int m = 0;
    for (int w = 0; w < nw; ++w) m = max(m, emax[w]);
    emax[0] = m;
  }
  __syncthreads();
  const int E = emax[0];
  __syncthreads();
  // scale to max |x| in [1, 2), split, identity J
  const double up = ldexp(1.0, 1023 - (E > 0 ? E : 1023));
  for (int i = tid; i < L * L; i += blockDim.x) {
    const cplx v = X64[i];
    float4 d;
    split_bits(v.x * up, d.x, d.y);
    split_bits(v.y * up, d.z, d.w);
    X[i] = d;
    J[i] = make_float4((i / L) == (i % L) ? 1.f : 0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  // ||X||_F^2 (FP32 is enough for the negligible-column threshold)
  float f2 = 0.f;
  for (int i = tid; i < L * L; i += blockDim.x) {
    const float4 d = X[i];
    f2 = fmaf(d.x, d.x, fmaf(d.z, d.z, f2));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  if (lane == 0) red[warp] = f2;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    red[0] = s;
  }
  __syncthreads();
  const float f2s = (float)red[0];
  const int Lp = (L + 1) & ~1;
  const float u = 3.5527136788005009e-15f;  // 2^-48
  const float tol = 8.0f * u * sqrtf((float)L);
  const float small = ((float)L * u) * ((float)L * u) * f2s;
  int sweep = 0;
  for (; sweep < JD_MAXSWEEPS && E > 0; ++sweep) {
    // squared column norms in double-float at the start of every sweep
    for (int c = warp; c < L; c += nw) {
      const float4* xc = X + (int64_t)c * L;
      float h = 0.f, lo = 0.f;
      for (int r = lane; r < L; r += 32) {
        const float4 d = xc[r];
        acc_dd(h, lo, d.x, d.y, d.x, d.y);
        acc_dd(h, lo, d.z, d.w, d.z, d.w);
      }
      fast2(h, lo);
      dfl s{h, lo};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = dadd(s, dfl{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)});
      if (lane == 0) nrm[c] = make_float2(s.h, s.l);
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
        float4* xa = X + (int64_t)a * L;
        float4* xb = X + (int64_t)b * L;
        const float2 na = nrm[a], nb = nrm[b];
        if (na.x <= small || nb.x <= small) continue;
        // g = x_a^H x_b
        float gr = 0.f, grl = 0.f, gi = 0.f, gil = 0.f;
        jd_dot(xa, xb, L, gl, gr, grl, gi, gil);
        fast2(gr, grl);
        fast2(gi, gil);
        const dfl g_r = grp_dsum(dfl{gr, grl}, gmask), g_i = grp_dsum(dfl{gi, gil}, gmask);
        // |g| against tol |x_a| |x_b|, as ratios (|g|^2 may lie below FP32's range)
        const float agf = hypotf(g_r.h, g_i.h);
        if (!(agf > 0.f) || !((agf / sqrtf(na.x)) / sqrtf(nb.x) > tol)) continue;
        // |g| and the phase e = g / |g| in double-float, from g scaled by a
        // power of two to its largest part in [1, 2)
        int kx;
        (void)frexpf(fmaxf(fabsf(g_r.h), fabsf(g_i.h)), &kx);
        const float gsc = ldexpf(1.0f, 1 - kx), gun = ldexpf(1.0f, kx - 1);
        const dfl gr_s{g_r.h * gsc, g_r.l * gsc}, gi_s{g_i.h * gsc, g_i.l * gsc};
        const dfl ags = dsqrt(dadd(dmul(gr_s, gr_s), dmul(gi_s, gi_s)));
        const dfl rinv = drecip(ags);
        const dfl ag{ags.h * gun, ags.l * gun};
        // the angle in FP32: zeta = (|x_b|^2 - |x_a|^2) / (2 |g|),
        // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), without overflow
        const dfl dba = dadd(dfl{nb.x, nb.y}, dfl{-na.x, -na.y});
        const float zeta = dba.h / (2.0f * ag.h);
        const float az = fabsf(zeta);
        const float den = az > 1e18f ? 2.0f * az : az + sqrtf(fmaf(zeta, zeta, 1.0f));
        const float t = (zeta >= 0.f ? 1.f : -1.f) / den;
        // c = 1 / sqrt(1 + t^2), s = c t: unitary to double-float accuracy
        const float t2 = t * t;
        const dfl c = drecip(dsqrt(dadd(dfl{1.0f, 0.0f}, dfl{t2, fmaf(t, t, -t2)})));
        const dfl s = dmulf(c, t);
        // se = s e with e = g / |g| of unit modulus to double-float accuracy
        const dfl er = dmul(gr_s, rinv), ei = dmul(gi_s, rinv);
        const dfl sr = dmul(s, er), si = dmul(s, ei);
        jd_rot(xa, xb, L, gl, c, sr, si);
        jd_rot(J + (int64_t)a * L, J + (int64_t)b * L, L, gl, c, sr, si);
        if (gl == 0) {
          // |x_a'|^2 = |x_a|^2 - t |g|, |x_b'|^2 = |x_b|^2 + t |g|
          const dfl tg = dmulf(ag, t);
          const dfl a2 = dadd(dfl{na.x, na.y}, dneg(tg)), b2 = dadd(dfl{nb.x, nb.y}, tg);
          nrm[a] = make_float2(a2.h, a2.l);
          nrm[b] = make_float2(b2.h, b2.l);
          rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  if (sweep == JD_MAXSWEEPS && tid == 0) atomicOr(status, 2);  // not converged (non-fatal)
  // back to FP64 in place, X unscaled
  const double down = ldexp(1.0, (E > 0 ? E : 1023) - 1023);
  for (int i = tid; i < L * L; i += blockDim.x) {
    const float4 x = X[i], j = J[i];
    X64[i] = cmk(((double)x.x + (double)x.y) * down, ((double)x.z + (double)x.w) * down);
    J64[i] = cmk((double)j.x + (double)j.y, (double)j.z + (double)j.w);
  }
  __syncthreads();
  jacobi_finish(D, P, sv, perm);
}

static int jd_smem_limit() {
  static int lim = -1;
  if (lim < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 48 * 1024;
    lim = v;
  }
  return lim;
}

cudaError_t jacobi_df_prepare() {
  static int done = 0;
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_jacobi_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, jd_smem_limit());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_jacobi_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)jd_smem_bytes(QR_MAXL, false));
    if (e != cudaSuccess) return e;
    done = 1;
  }
  return cudaSuccess;
}

cudaError_t launch_jacobi_df(const Dims* dims, const ProbPtr* ptrs, int batch, int lcap, int* status,
                             cudaStream_t st) {
  cudaError_t e = jacobi_df_prepare();
  if (e != cudaSuccess) return e;
  ProfScope ps("k_jacobi[df]", st);
  // X in shared memory wherever the widest instance's fits (l <= 120 on GB300)
  const size_t xs = jd_smem_bytes(lcap, true);
  if (xs <= (size_t)jd_smem_limit())
    k_jacobi_df<true><<<batch, JD_THREADS, xs, st>>>(dims, ptrs, status);
  else
    k_jacobi_df<false><<<batch, JD_THREADS, jd_smem_bytes(lcap, false), st>>>(dims, ptrs, status);
  return cudaGetLastError();
}

}  // namespace tg
