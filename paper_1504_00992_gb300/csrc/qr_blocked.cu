// Blocked Householder QR in FP32 and the FP64-accurate re-orthonormalisation
// of its Q (sm_103a), used by the mixed-precision RRSVD.
//
// k_qr_blk_f32: Householder reflectors H = I - tau v v^H with alpha =
// -e^{i arg x0} ||x||, normalised v = x / (x0 - alpha) (v_0 = 1) and
// tau = 1 + |x0| / ||x|| (Golub & Van Loan 5.1.2), grouped in panels of QB_NB columns (compact WY form,
// Schreiber & Van Loan 1989; Golub & Van Loan 5.2.3):
//   H_0 ... H_{nb-1} = I - V T V^H,  T upper triangular,
//   T[i][i] = tau_i,  T[0:i, i] = -tau_i T[0:i, 0:i] (V[:, 0:i]^H v_i).
// A panel is factored in shared memory; the trailing columns get
// A <- A - V T^H (V^H A) in two streaming passes instead of one pass per
// reflector, and Q = H_0 ... H_{L-1} [I; 0] is accumulated panel by panel
// backwards with Q <- Q - V T (V^H Q).  One CTA per instance.
//
// Re-orthonormalisation: the FP32 Q_f has ||Q_f^H Q_f - I|| ~ 1e-6.  With
// E = Q_f^H Q_f - I formed FP64-accurately (the digit-pair tensor-core Gram of
// oz_proj.cu, from exact BF16 digit splits of Q_f), the symmetric
// (Loewdin) orthonormalisation Q = Q_f (I + E)^{-1/2} is evaluated from the
// binomial series (I + E)^{-1/2} = I - E/2 + 3 E^2 / 8 - ..., whose first
// dropped term is of order ||E||^3 ~ 1e-18.  Q spans range(Q_f) and is
// orthonormal to ~1e-13: the "last QR in FP64" of the mixed form at FP32 cost.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "mixed.cuh"
#include "profiler.cuh"

namespace tg {

enum { QB_THREADS = 512, QB_WARPS = QB_THREADS / 32, QB_NB = 8, QB_CW = 4, QB_RED = 64 };

__device__ __forceinline__ float qb_wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout of k_qr_blk_f32 (bytes), shared with the host check.
__host__ __device__ inline size_t qb_smem_bytes(int M, int L, int nw = QB_WARPS) {
  const int npan = (L + QB_NB - 1) / QB_NB;
  return sizeof(float2) * ((size_t)QB_NB * M + 2 * (size_t)QB_NB * L + (size_t)npan * QB_NB * QB_NB) +
         sizeof(float) * ((size_t)L + (size_t)nw * QB_RED + QB_RED);
}

// C[j0:M, c0:L) <- C - V op(T) (V^H C), op(T) = T^H (trans) or T.  V holds jb
// reflectors in shared memory (local row r = global row j0 + r, zero above
// each reflector's first row).  When a column group's rows are split over
// several warps, their partial products go to the scratch `part`
// (warps x QB_NB x QB_CW real and imaginary parts) and are summed in a
// fixed order, so the result does not depend on scheduling.  All threads of
// the CTA call it.
template <int NT>
__device__ void qb_apply(float2* C, int ldc, int M, int j0, int jb, int c0, int L, const float2* Vs, int ldv,
                         const float2* Tp, bool trans, float2* W, float2* W2, float* part) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Mr = M - j0, ncol = L - c0;
  if (ncol <= 0) return;
  for (int e = tid; e < QB_NB * ncol; e += NT) W[(e / ncol) * L + c0 + e % ncol] = make_float2(0.f, 0.f);
  __syncthreads();
  const int ncg = (ncol + QB_CW - 1) / QB_CW;
  const int rs = ncg >= NW ? 1 : NW / ncg;
  const int ntask = ncg * rs;
  // pass 1: W = V^H C
  for (int t = warp; t < ntask; t += NW) {
    const int cg = t % ncg, h = t / ncg;
    const int cb = c0 + cg * QB_CW;
    const int nc = min(QB_CW, L - cb);
    float2 acc[QB_NB][QB_CW];
#pragma unroll
    for (int i = 0; i < QB_NB; ++i)
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) acc[i][w] = make_float2(0.f, 0.f);
    // the loads of the next row are issued before the products of this one
    const int rstep = 32 * rs;
    int r = h * 32 + lane;
    float2 an[QB_CW];
#pragma unroll
    for (int w = 0; w < QB_CW; ++w)
      an[w] = (w < nc && r < Mr) ? C[(size_t)(cb + w) * ldc + j0 + r] : make_float2(0.f, 0.f);
    for (; r < Mr; r += rstep) {
      float2 a[QB_CW];
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) a[w] = an[w];
      const int rn = r + rstep;
#pragma unroll
      for (int w = 0; w < QB_CW; ++w)
        if (w < nc && rn < Mr) an[w] = C[(size_t)(cb + w) * ldc + j0 + rn];
      float2 v[QB_NB];
#pragma unroll
      for (int i = 0; i < QB_NB; ++i) v[i] = (i < jb) ? Vs[i * ldv + r] : make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) {
#pragma unroll
        for (int i = 0; i < QB_NB; ++i) {
          acc[i][w].x = fmaf(v[i].x, a[w].x, fmaf(v[i].y, a[w].y, acc[i][w].x));
          acc[i][w].y = fmaf(v[i].x, a[w].y, fmaf(-v[i].y, a[w].x, acc[i][w].y));
        }
      }
    }
#pragma unroll
    for (int i = 0; i < QB_NB; ++i)
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) {
        const float sx = qb_wsum(acc[i][w].x), sy = qb_wsum(acc[i][w].y);
        if (lane == ((i * QB_CW + w) & 31)) {
          if (rs > 1) {  // one task per warp (ntask <= NW): a slot per warp
            part[(warp * QB_NB + i) * QB_CW + w] = sx;
            part[NW * QB_NB * QB_CW + (warp * QB_NB + i) * QB_CW + w] = sy;
          } else if (i < jb && w < nc) {  // the column group's only contributor
            W[i * L + cb + w] = make_float2(sx, sy);
          }
        }
      }
  }
  __syncthreads();
  if (rs > 1) {
    // task t = h ncg + cg ran on warp t: sum the row slices h in order
    for (int e = tid; e < jb * ncol; e += NT) {
      const int i = e / ncol, cl = e % ncol, cg = cl / QB_CW, w = cl % QB_CW;
      float sx = 0.f, sy = 0.f;
      for (int h = 0; h < rs; ++h) {
        const int slot = ((h * ncg + cg) * QB_NB + i) * QB_CW + w;
        sx += part[slot];
        sy += part[NW * QB_NB * QB_CW + slot];
      }
      W[i * L + c0 + cl] = make_float2(sx, sy);
    }
    __syncthreads();
  }
  // W2 = op(T) W
  for (int e = tid; e < jb * ncol; e += NT) {
    const int i = e / ncol, c = c0 + e % ncol;
    float2 s = make_float2(0.f, 0.f);
    if (trans) {
      for (int a = 0; a <= i; ++a) {  // conj(T[a][i]) W[a][c]
        const float2 t = Tp[a * QB_NB + i], w = W[a * L + c];
        s.x = fmaf(t.x, w.x, fmaf(t.y, w.y, s.x));
        s.y = fmaf(t.x, w.y, fmaf(-t.y, w.x, s.y));
      }
    } else {
      for (int b = i; b < jb; ++b) {  // T[i][b] W[b][c]
        const float2 t = Tp[i * QB_NB + b], w = W[b * L + c];
        s.x = fmaf(t.x, w.x, fmaf(-t.y, w.y, s.x));
        s.y = fmaf(t.x, w.y, fmaf(t.y, w.x, s.y));
      }
    }
    W2[i * L + c] = s;
  }
  __syncthreads();
  // pass 2: C -= V W2
  for (int t = warp; t < ntask; t += NW) {
    const int cg = t % ncg, h = t / ncg;
    const int cb = c0 + cg * QB_CW;
    const int nc = min(QB_CW, L - cb);
    float2 w2[QB_NB][QB_CW];
#pragma unroll
    for (int i = 0; i < QB_NB; ++i)
#pragma unroll
      for (int w = 0; w < QB_CW; ++w)
        w2[i][w] = (i < jb && w < nc) ? W2[i * L + cb + w] : make_float2(0.f, 0.f);
    const int rstep = 32 * rs;
    int r = h * 32 + lane;
    float2 an[QB_CW];
#pragma unroll
    for (int w = 0; w < QB_CW; ++w)
      an[w] = (w < nc && r < Mr) ? C[(size_t)(cb + w) * ldc + j0 + r] : make_float2(0.f, 0.f);
    for (; r < Mr; r += rstep) {
      float2 a[QB_CW];
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) a[w] = an[w];
      const int rn = r + rstep;
#pragma unroll
      for (int w = 0; w < QB_CW; ++w)
        if (w < nc && rn < Mr) an[w] = C[(size_t)(cb + w) * ldc + j0 + rn];
      float2 v[QB_NB];
#pragma unroll
      for (int i = 0; i < QB_NB; ++i) v[i] = (i < jb) ? Vs[i * ldv + r] : make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < QB_CW; ++w) {
        if (w < nc) {
#pragma unroll
          for (int i = 0; i < QB_NB; ++i) {
            a[w].x = fmaf(-v[i].x, w2[i][w].x, fmaf(v[i].y, w2[i][w].y, a[w].x));
            a[w].y = fmaf(-v[i].x, w2[i][w].y, fmaf(-v[i].y, w2[i][w].x, a[w].y));
          }
          C[(size_t)(cb + w) * ldc + j0 + r] = a[w];
        }
      }
    }
  }
  __syncthreads();
}

// A: Mc x Lc column-major per instance (overwritten by R and the reflectors);
// Q: Mc x Lc column-major output.  With dims, instance z factors only its own
// rows (D.n when use_n, else D.m) and D.l columns of the zero-padded capacity
// layout, and Q is [I; 0] outside them.  Requires Mc >= Lc and
// qb_smem_bytes(Mc, Lc) of dynamic shared memory.
template <int NT>
__global__ void __launch_bounds__(NT) k_qr_blk_f32(float2* Abase, float2* Qbase, int Mc, int Lc,
                                                  const Dims* __restrict__ dims, int use_n) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char qb_raw[];
  __shared__ float2 vscale;
  __shared__ float vnorm;
  const int ldv = Mc;  // shared memory is laid out for the capacity (Mc, Lc)
  const int npan_c = (Lc + QB_NB - 1) / QB_NB;
  float2* Vs = reinterpret_cast<float2*>(qb_raw);
  float2* W = Vs + (size_t)QB_NB * ldv;
  float2* W2 = W + QB_NB * Lc;
  float2* Tall = W2 + QB_NB * Lc;
  float* tau = reinterpret_cast<float*>(Tall + npan_c * QB_NB * QB_NB);
  float* red = tau + Lc;
  float* fin = red + NW * QB_RED;
  const int z = blockIdx.x;
  int M = Mc, L = Lc;  // this instance's rows and columns
  if (dims) {
    const Dims D = dims[z];
    if (!D.active) return;  // uniform over the block
    M = use_n ? D.n : D.m;
    L = D.l;
  }
  const int npan = (L + QB_NB - 1) / QB_NB;
  float2* A = Abase + (size_t)z * Mc * Lc;
  float2* Qo = Qbase + (size_t)z * Mc * Lc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int p = 0; p < npan; ++p) {
    const int j0 = p * QB_NB, jb = min(QB_NB, L - j0), Mr = M - j0;
    for (int e = tid; e < jb * Mr; e += NT) {
      const int i = e / Mr, r = e % Mr;
      Vs[i * ldv + r] = A[(size_t)(j0 + i) * Mc + j0 + r];
    }
    __syncthreads();
    // --- panel factorisation in shared memory
    for (int i = 0; i < jb; ++i) {
      const int j = j0 + i;
      float s = 0.f;
      for (int r = i + tid; r < Mr; r += NT) {
        const float2 v = Vs[i * ldv + r];
        s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
      }
      s = qb_wsum(s);
      if (lane == 0) red[warp] = s;
      __syncthreads();
      if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[w];
        vnorm = sqrtf(t);
      }
      __syncthreads();
      if (vnorm < 1e-12f) {
        // a column this small has squares in the FP32 subnormal range, whose
        // lost bits would make the reflector non-unitary: norm of x / max|x|
        float mx = 0.f;
        for (int r = i + tid; r < Mr; r += NT) {
          const float2 v = Vs[i * ldv + r];
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        float amax = 0.f;
        for (int w = 0; w < NW; ++w) amax = fmaxf(amax, red[w]);
        __syncthreads();
        float s2 = 0.f;
        if (amax > 0.f) {
          const float ia = 1.f / amax;
          for (int r = i + tid; r < Mr; r += NT) {
            const float2 v = Vs[i * ldv + r];
            const float a = v.x * ia, b = v.y * ia;
            s2 = fmaf(a, a, fmaf(b, b, s2));
          }
        }
        s2 = qb_wsum(s2);
        if (lane == 0) red[warp] = s2;
        __syncthreads();
        if (tid == 0) {
          float t = 0.f;
          for (int w = 0; w < NW; ++w) t += red[w];
          vnorm = amax * sqrtf(t);
        }
        __syncthreads();
      }
      if (tid == 0) {
        const float2 x0 = Vs[i * ldv + i];
        // |x0| without squaring (a square in the subnormal range would leave
        // the phase x0/|x0| off the unit circle and the reflector non-unitary)
        const float ax0 = hypotf(x0.x, x0.y);
        const float nx = vnorm;
        if (!(nx >= 1e-30f)) {  // zero column, or one below any meaningful scale: no reflection
          tau[j] = 0.f;
          vscale = make_float2(1.f, 0.f);
        } else {
          // normalised reflector: v = x / (x0 - alpha), v_0 = 1, tau = 1 + |x0| / ||x||
          // (in [1, 2], so columns of tiny norm neither overflow nor lose tau); the
          // phase of a leading entry negligible against ||x|| is not used
          const float2 ph = (ax0 > 1e-7f * nx) ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
          const float ri = 1.f / (ax0 + nx);
          vscale = make_float2(ph.x * ri, -ph.y * ri);  // 1 / (x0 - alpha)
          Vs[i * ldv + i] = make_float2(1.f, 0.f);
          tau[j] = 1.f + ax0 / nx;
        }
      }
      __syncthreads();
      const float tj = tau[j];
      if (tj != 0.f) {
        const float2 sc = vscale;
        for (int r = i + 1 + tid; r < Mr; r += NT) {
          const float2 v = Vs[i * ldv + r];
          Vs[i * ldv + r] = make_float2(v.x * sc.x - v.y * sc.y, v.x * sc.y + v.y * sc.x);
        }
        __syncthreads();
      }
      const int nc = jb - 1 - i;
      if (tj != 0.f && nc > 0) {
        float2 acc[QB_NB - 1];
#pragma unroll
        for (int c = 0; c < QB_NB - 1; ++c) acc[c] = make_float2(0.f, 0.f);
        for (int r = i + tid; r < Mr; r += NT) {
          const float2 v = Vs[i * ldv + r];
#pragma unroll
          for (int c = 0; c < QB_NB - 1; ++c)
            if (c < nc) {
              const float2 a = Vs[(i + 1 + c) * ldv + r];
              acc[c].x = fmaf(v.x, a.x, fmaf(v.y, a.y, acc[c].x));
              acc[c].y = fmaf(v.x, a.y, fmaf(-v.y, a.x, acc[c].y));
            }
        }
#pragma unroll
        for (int c = 0; c < QB_NB - 1; ++c) {
          const float sx = qb_wsum(acc[c].x), sy = qb_wsum(acc[c].y);
          if (lane == 0 && c < nc) {
            red[warp * QB_RED + 2 * c] = sx;
            red[warp * QB_RED + 2 * c + 1] = sy;
          }
        }
        __syncthreads();
        if (tid < 2 * nc) {
          float t = 0.f;
          for (int w = 0; w < NW; ++w) t += red[w * QB_RED + tid];
          fin[tid] = t * tj;
        }
        __syncthreads();
        for (int r = i + tid; r < Mr; r += NT) {
          const float2 v = Vs[i * ldv + r];
#pragma unroll
          for (int c = 0; c < QB_NB - 1; ++c)
            if (c < nc) {
              const float sx = fin[2 * c], sy = fin[2 * c + 1];
              float2* ap = &Vs[(i + 1 + c) * ldv + r];
              ap->x -= v.x * sx - v.y * sy;
              ap->y -= v.x * sy + v.y * sx;
            }
        }
        __syncthreads();
      }
    }
    // --- panel (R part and reflectors) back to global memory, then clear
    // the R part so that Vs holds V with its zeros
    for (int e = tid; e < jb * Mr; e += NT) {
      const int i = e / Mr, r = e % Mr;
      A[(size_t)(j0 + i) * Mc + j0 + r] = Vs[i * ldv + r];
    }
    __syncthreads();
    for (int e = tid; e < jb * jb; e += NT) {
      const int i = e / jb, r = e % jb;
      if (r < i) Vs[i * ldv + r] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    // --- T of this panel from S[a][b] = V_a^H V_b (a < b)
    {
      float2 sab[QB_NB * (QB_NB - 1) / 2];
#pragma unroll
      for (int q = 0; q < QB_NB * (QB_NB - 1) / 2; ++q) sab[q] = make_float2(0.f, 0.f);
      for (int r = 1 + tid; r < Mr; r += NT) {  // row 0 only meets V_0
        float2 v[QB_NB];
#pragma unroll
        for (int i = 0; i < QB_NB; ++i) v[i] = (i < jb) ? Vs[i * ldv + r] : make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 1; b < QB_NB; ++b)
#pragma unroll
          for (int a = 0; a < b; ++a) {
            float2& q = sab[b * (b - 1) / 2 + a];
            q.x = fmaf(v[a].x, v[b].x, fmaf(v[a].y, v[b].y, q.x));
            q.y = fmaf(v[a].x, v[b].y, fmaf(-v[a].y, v[b].x, q.y));
          }
      }
#pragma unroll
      for (int q = 0; q < QB_NB * (QB_NB - 1) / 2; ++q) {
        const float sx = qb_wsum(sab[q].x), sy = qb_wsum(sab[q].y);
        if (lane == 0) {
          red[warp * QB_RED + 2 * q] = sx;
          red[warp * QB_RED + 2 * q + 1] = sy;
        }
      }
      __syncthreads();
      if (tid < QB_NB * (QB_NB - 1)) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[w * QB_RED + tid];
        fin[tid] = t;
      }
      __syncthreads();
      if (tid == 0) {
        float2* Tp = Tall + p * QB_NB * QB_NB;
        for (int e = 0; e < QB_NB * QB_NB; ++e) Tp[e] = make_float2(0.f, 0.f);
        for (int i = 0; i < jb; ++i) {
          const float ti = tau[j0 + i];
          Tp[i * QB_NB + i] = make_float2(ti, 0.f);
          for (int a = 0; a < i; ++a) {
            float2 s = make_float2(0.f, 0.f);
            for (int b = a; b < i; ++b) {  // T[a][b] S[b][i]
              const float2 t = Tp[a * QB_NB + b];
              const int q = i * (i - 1) / 2 + b;
              const float2 sv = make_float2(fin[2 * q], fin[2 * q + 1]);
              s.x += t.x * sv.x - t.y * sv.y;
              s.y += t.x * sv.y + t.y * sv.x;
            }
            Tp[a * QB_NB + i] = make_float2(-ti * s.x, -ti * s.y);
          }
        }
      }
      __syncthreads();
    }
    // --- trailing columns: A <- A - V T^H V^H A
    qb_apply<NT>(A, Mc, M, j0, jb, j0 + jb, L, Vs, ldv, Tall + p * QB_NB * QB_NB, true, W, W2, red);
  }

  // --- Q = H_0 ... H_{L-1} [I; 0], panels backwards
  for (int64_t e = tid; e < (int64_t)Mc * Lc; e += NT) {  // [I; 0] over the whole capacity
    const int c = (int)(e / Mc), r = (int)(e % Mc);
    Qo[e] = make_float2(r == c && c < L ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * QB_NB, jb = min(QB_NB, L - j0), Mr = M - j0;
    for (int e = tid; e < jb * Mr; e += NT) {
      const int i = e / Mr, r = e % Mr;
      Vs[i * ldv + r] = (r < i) ? make_float2(0.f, 0.f) : A[(size_t)(j0 + i) * Mc + j0 + r];
    }
    __syncthreads();
    qb_apply<NT>(Qo, Mc, M, j0, jb, j0, L, Vs, ldv, Tall + p * QB_NB * QB_NB, false, W, W2, red);
  }
}

bool qr_blk_f32_fits(int M, int L) { return M >= L && L >= 1 && qb_smem_bytes(M, L) <= 227 * 1024 - 2048; }

// Raises a kernel's dynamic shared-memory limit to `bytes` (the first time a
// launch needs more than the last value set for it).
template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes, size_t* done) {
  if (bytes <= 48 * 1024 || bytes <= *done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *done = bytes;
  return e;
}

// Shared-memory limits set so far, per kernel (one record each, shared by the
// launchers and qr_blocked_prepare so that a limit is never lowered).
static size_t g_attr_qr = 0, g_attr_qr256 = 0, g_attr_ld = 0, g_attr_fold[2][2] = {{0, 0}, {0, 0}};

// Batches of many small matrices take smaller CTAs when several fit an SM
// (registers: 128 per thread; shared memory): the per-column barriers of one
// matrix then overlap with the others' work.  Four 128-thread CTAs per SM
// from four matrices per SM, two 256-thread CTAs from two.
static size_t g_attr_qr128 = 0;

cudaError_t launch_qr_blk_f32(float2* A, float2* Q, int M, int L, int batch, cudaStream_t st, const Dims* dims,
                              int use_n, int threads) {
  const bool t128 = threads == 128 || (threads == 0 && batch >= 4 * 152);
  const bool t256 = threads == 256 || (threads == 0 && batch >= 2 * 152);
  if (t128 && qb_smem_bytes(M, L, 4) <= 56 * 1024) {
    const size_t sm = qb_smem_bytes(M, L, 4);
    cudaError_t e = ensure_smem(k_qr_blk_f32<128>, sm, &g_attr_qr128);
    if (e != cudaSuccess) return e;
    k_qr_blk_f32<128><<<batch, 128, sm, st>>>(A, Q, M, L, dims, use_n);
    return cudaGetLastError();
  }
  if ((t128 || t256) && qb_smem_bytes(M, L, 8) <= 112 * 1024) {
    const size_t sm = qb_smem_bytes(M, L, 8);
    cudaError_t e = ensure_smem(k_qr_blk_f32<256>, sm, &g_attr_qr256);
    if (e != cudaSuccess) return e;
    k_qr_blk_f32<256><<<batch, 256, sm, st>>>(A, Q, M, L, dims, use_n);
    return cudaGetLastError();
  }
  const size_t sm = qb_smem_bytes(M, L);
  cudaError_t e = ensure_smem(k_qr_blk_f32<QB_THREADS>, sm, &g_attr_qr);
  if (e != cudaSuccess) return e;
  k_qr_blk_f32<QB_THREADS><<<batch, QB_THREADS, sm, st>>>(A, Q, M, L, dims, use_n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Re-orthonormalisation of an FP32 Q_f (M x L column-major per instance).
// ---------------------------------------------------------------------------
// D = -E/2 + 3 E^2 / 8 (E Hermitian, from its upper triangle), FP32, one CTA
// per instance; raises status bit 4 when E is not small or not finite.
__global__ void __launch_bounds__(512) k_lowdin(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                float2* Dbase, int Lc, int* status) {
  extern __shared__ __align__(16) unsigned char ld_raw[];
  float2* Ef = reinterpret_cast<float2*>(ld_raw);  // L x L, Ef[a * L + b] = E[a][b]
  __shared__ float red[32];
  const int z = blockIdx.x;
  if (!dims[z].active) return;
  const int L = dims[z].l;
  const cplx* E = ptrs[z].R;
  float2* D = Dbase + (size_t)z * Lc * Lc;
  const int tid = threadIdx.x;
  float mx = 0.f;
  for (int e = tid; e < L * L; e += blockDim.x) {
    const int a = e / L, b = e % L;
    cplx v = (a <= b) ? E[(size_t)b * L + a] : cconj(E[(size_t)a * L + b]);
    const float2 f = make_float2((float)v.x, (float)v.y);
    Ef[e] = f;
    const float m = fmaxf(fabsf(f.x), fabsf(f.y));
    mx = (m > mx || m != m) ? m : mx;  // NaN sticks
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (y > mx || y != y) ? y : mx;
  }
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = (red[w] > m || red[w] != red[w]) ? red[w] : m;
    if (!(m <= 1e-3f)) atomicOr(status, 4);
  }
  // D[a][b] = -E[a][b]/2 + 3/8 sum_k E[a][k] E[k][b]; stored column-major (D[b * L + a])
  for (int e = tid; e < L * L; e += blockDim.x) {
    const int b = e / L, a = e % L;
    float sx = 0.f, sy = 0.f;
    for (int k = 0; k < L; ++k) {
      const float2 x = Ef[a * L + k], y = Ef[k * L + b];
      sx = fmaf(x.x, y.x, fmaf(-x.y, y.y, sx));
      sy = fmaf(x.x, y.y, fmaf(x.y, y.x, sy));
    }
    const float2 ea = Ef[a * L + b];
    D[e] = make_float2(-0.5f * ea.x + 0.375f * sx, -0.5f * ea.y + 0.375f * sy);
  }
}

// Out = X + X D with the small correction X D in FP32 (|D| ~ 1e-6, so its
// relative FP32 error costs ~1e-13 absolute): Q = Q_f (I + D) from the FP32
// Q_f (capacity Mc x Lc per instance) into ptrs[z].Q (D.m x D.l, compact), or,
// in place, B^H = (A^H Q_f)(I + D) on ptrs[z].Yt (D.n x D.l, compact).  RPL
// rows per lane (32 RPL rows per CTA), staged column-major in shared memory
// as FP32; warp w owns the columns c = w (mod 8).
enum { QF_MAXL = 144, QF_MAXCPW = QF_MAXL / 8 };

template <bool FROM_F32, int RPL>
__global__ void __launch_bounds__(256) k_fold(const float2* __restrict__ Qf, const float2* __restrict__ Dbase,
                                              const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs, int Mc,
                                              int Lc) {
  constexpr int ROWS = 32 * RPL;
  extern __shared__ __align__(16) unsigned char qf_raw[];
  const int z = blockIdx.y;
  const Dims Dm = dims[z];
  if (!Dm.active) return;
  const int M = FROM_F32 ? Dm.m : Dm.n, L = Dm.l;
  const int r0 = blockIdx.x * ROWS;
  if (r0 >= M) return;
  float2* Ds = reinterpret_cast<float2*>(qf_raw);  // L x L column-major
  float2* Qs = Ds + ((L * L + 1) & ~1);            // ROWS x L column-major (16-byte aligned)
  const float2* q = FROM_F32 ? Qf + (size_t)z * Mc * Lc : nullptr;
  cplx* X = FROM_F32 ? ptrs[z].Q : ptrs[z].Yt;  // output (and FP64 source when !FROM_F32), ld M
  const float2* D = Dbase + (size_t)z * Lc * Lc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < L * L; e += 256) Ds[e] = D[e];
  for (int e = tid; e < ROWS * L; e += 256) {
    const int c = e / ROWS, r = e % ROWS;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + r < M) {
      if (FROM_F32) {
        v = q[(size_t)c * Mc + r0 + r];
      } else {
        const cplx x = X[(size_t)c * M + r0 + r];
        v = make_float2((float)x.x, (float)x.y);
      }
    }
    Qs[e] = v;
  }
  __syncthreads();
  float2 acc[RPL][QF_MAXCPW];
#pragma unroll
  for (int i = 0; i < RPL; ++i)
#pragma unroll
    for (int j = 0; j < QF_MAXCPW; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k = 0; k < L; ++k) {
    float2 x[RPL];
    if (RPL == 2) {
      const float4 x4 = *reinterpret_cast<const float4*>(&Qs[k * ROWS + 2 * lane]);  // rows 2 lane, 2 lane + 1
      x[0] = make_float2(x4.x, x4.y);
      x[RPL - 1] = make_float2(x4.z, x4.w);
    } else {
      x[0] = Qs[k * ROWS + lane];
    }
#pragma unroll
    for (int j = 0; j < QF_MAXCPW; ++j) {
      const int c = warp + 8 * j;
      if (c < L) {
        const float2 d = Ds[c * L + k];
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          acc[i][j].x = fmaf(x[i].x, d.x, fmaf(-x[i].y, d.y, acc[i][j].x));
          acc[i][j].y = fmaf(x[i].x, d.y, fmaf(x[i].y, d.x, acc[i][j].y));
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int r = RPL * lane + i;
    if (r0 + r >= M) continue;
#pragma unroll
    for (int j = 0; j < QF_MAXCPW; ++j) {
      const int c = warp + 8 * j;
      if (c < L) {
        cplx b;
        if (FROM_F32) {
          const float2 f = Qs[c * ROWS + r];
          b = cmk((double)f.x, (double)f.y);
        } else {
          b = X[(size_t)c * M + r0 + r];
        }
        X[(size_t)c * M + r0 + r] = cmk(b.x + (double)acc[i][j].x, b.y + (double)acc[i][j].y);
      }
    }
  }
}

// batch == 0 only raises the shared-memory limit.
template <bool FROM_F32>
static cudaError_t launch_fold(const float2* Qf, const float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int Mc,
                               int Lc, int batch, cudaStream_t st) {
  if (Lc <= 128) {
    const size_t sm = sizeof(float2) * ((size_t)((Lc * Lc + 1) & ~1) + 64 * (size_t)Lc);
    cudaError_t e = ensure_smem(k_fold<FROM_F32, 2>, sm, &g_attr_fold[FROM_F32][1]);
    if (e != cudaSuccess || batch == 0) return e;
    k_fold<FROM_F32, 2><<<dim3((Mc + 63) / 64, batch), 256, sm, st>>>(Qf, Dbuf, dims, ptrs, Mc, Lc);
  } else {
    const size_t sm = sizeof(float2) * ((size_t)((Lc * Lc + 1) & ~1) + 32 * (size_t)Lc);
    cudaError_t e = ensure_smem(k_fold<FROM_F32, 1>, sm, &g_attr_fold[FROM_F32][0]);
    if (e != cudaSuccess || batch == 0) return e;
    k_fold<FROM_F32, 1><<<dim3((Mc + 31) / 32, batch), 256, sm, st>>>(Qf, Dbuf, dims, ptrs, Mc, Lc);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The same steps for bases wider than QF_MAXL (D no longer fits in shared
// memory next to the rows), up to QF_MAXL_BIG columns.
// k_lowdin_big: D = -E/2 + 3 E^2 / 8 in 32 x 32 tiles over a grid (E read from
// its upper triangle in FP64 and staged as FP32, 32-deep K slices).
// k_fold_big: one CTA per 32 rows holding its rows of X (all L columns, FP32)
// in shared memory; each warp computes 16 output columns at a time with D
// read through L1 (every lane of a warp reads the same D element).  Out of
// place for Q; for B^H the rows are staged before any is overwritten, and a
// CTA owns whole rows, so the in-place update is safe.
// ---------------------------------------------------------------------------
enum { QF_MAXL_BIG = 512, QFB_ROWS = 32, QFB_CW = 16 };

__device__ __forceinline__ cplx herm_get(const cplx* E, int L, int a, int b) {
  return (a <= b) ? E[(size_t)b * L + a] : cconj(E[(size_t)a * L + b]);
}

__global__ void __launch_bounds__(256) k_lowdin_big(const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                    float2* Dbase, int Lc, int* status) {
  constexpr int T = 32;
  __shared__ float2 Ea[T][T + 1];  // E[a0 + i][k0 + kk] at [kk][i]
  __shared__ float2 Eb[T][T + 1];  // E[k0 + kk][b0 + j] at [kk][j]
  const int z = blockIdx.y;
  const Dims Dm = dims[z];
  if (!Dm.active) return;
  const int L = Dm.l;
  const int nt = (Lc + T - 1) / T;
  const int a0 = (blockIdx.x / nt) * T, b0 = (blockIdx.x % nt) * T;
  if (a0 >= L || b0 >= L) return;
  const cplx* E = ptrs[z].R;
  float2* D = Dbase + (size_t)z * Lc * Lc;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  int bad = 0;
  for (int k0 = 0; k0 < L; k0 += T) {
    for (int e = tid; e < T * T; e += 256) {
      const int kk = e % T, i = e / T;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (a0 + i < L && k0 + kk < L) {
        const cplx x = herm_get(E, L, a0 + i, k0 + kk);
        va = make_float2((float)x.x, (float)x.y);
        bad |= !(fmaxf(fabsf(va.x), fabsf(va.y)) <= 1e-3f);
      }
      if (k0 + kk < L && b0 + i < L) {
        const cplx x = herm_get(E, L, k0 + kk, b0 + i);
        vb = make_float2((float)x.x, (float)x.y);
      }
      Ea[kk][i] = va;
      Eb[kk][i] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < T; ++kk) {
      const float2 x0 = Ea[kk][ty], x1 = Ea[kk][ty + 16];
      const float2 y0 = Eb[kk][tx], y1 = Eb[kk][tx + 16];
      const float2 xs[2] = {x0, x1}, ys[2] = {y0, y1};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          acc[i][j].x = fmaf(xs[i].x, ys[j].x, fmaf(-xs[i].y, ys[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(xs[i].x, ys[j].y, fmaf(xs[i].y, ys[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(status, 4);  // E not small, or not finite
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < L && b < L) {
        const cplx ex = herm_get(E, L, a, b);
        D[(size_t)b * L + a] = make_float2(-0.5f * (float)ex.x + 0.375f * acc[i][j].x,
                                           -0.5f * (float)ex.y + 0.375f * acc[i][j].y);
      }
    }
}

template <bool FROM_F32>
__global__ void __launch_bounds__(256) k_fold_big(const float2* __restrict__ Qf, const float2* __restrict__ Dbase,
                                                  const Dims* __restrict__ dims, const ProbPtr* __restrict__ ptrs,
                                                  int Mc, int Lc) {
  extern __shared__ __align__(16) unsigned char qfb_raw[];
  const int z = blockIdx.y;
  const Dims Dm = dims[z];
  if (!Dm.active) return;
  const int M = FROM_F32 ? Dm.m : Dm.n, L = Dm.l;
  const int r0 = blockIdx.x * QFB_ROWS;
  if (r0 >= M) return;
  float2* Xs = reinterpret_cast<float2*>(qfb_raw);  // QFB_ROWS x L column-major
  const float2* q = FROM_F32 ? Qf + (size_t)z * Mc * Lc : nullptr;
  cplx* X = FROM_F32 ? ptrs[z].Q : ptrs[z].Yt;  // output (and FP64 source when !FROM_F32), ld M
  const float2* D = Dbase + (size_t)z * Lc * Lc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < QFB_ROWS * L; e += 256) {
    const int c = e / QFB_ROWS, r = e % QFB_ROWS;
    float2 v = make_float2(0.f, 0.f);
    if (r0 + r < M) {
      if (FROM_F32) {
        v = q[(size_t)c * Mc + r0 + r];
      } else {
        const cplx x = X[(size_t)c * M + r0 + r];
        v = make_float2((float)x.x, (float)x.y);
      }
    }
    Xs[e] = v;
  }
  __syncthreads();
  const int r = r0 + lane;
  for (int cb = warp * QFB_CW; cb < L; cb += 8 * QFB_CW) {
    float2 acc[QFB_CW];
#pragma unroll
    for (int j = 0; j < QFB_CW; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int k = 0; k < L; ++k) {
      const float2 x = Xs[k * QFB_ROWS + lane];
#pragma unroll
      for (int j = 0; j < QFB_CW; ++j) {
        if (cb + j < L) {
          const float2 d = __ldg(&D[(size_t)(cb + j) * L + k]);
          acc[j].x = fmaf(x.x, d.x, fmaf(-x.y, d.y, acc[j].x));
          acc[j].y = fmaf(x.x, d.y, fmaf(x.y, d.x, acc[j].y));
        }
      }
    }
    if (r < M) {
#pragma unroll
      for (int j = 0; j < QFB_CW; ++j) {
        const int c = cb + j;
        if (c < L) {
          cplx b;
          if (FROM_F32) {
            const float2 f = Xs[c * QFB_ROWS + lane];
            b = cmk((double)f.x, (double)f.y);
          } else {
            b = X[(size_t)c * M + r];
          }
          X[(size_t)c * M + r] = cmk(b.x + (double)acc[j].x, b.y + (double)acc[j].y);
        }
      }
    }
  }
}

static size_t g_attr_foldbig[2] = {0, 0};

// batch == 0 only raises the shared-memory limit.
template <bool FROM_F32>
static cudaError_t launch_fold_big(const float2* Qf, const float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int Mc,
                                   int Lc, int batch, cudaStream_t st) {
  const size_t sm = sizeof(float2) * (size_t)QFB_ROWS * Lc;
  cudaError_t e = ensure_smem(k_fold_big<FROM_F32>, sm, &g_attr_foldbig[FROM_F32]);
  if (e != cudaSuccess || batch == 0) return e;
  k_fold_big<FROM_F32><<<dim3((Mc + QFB_ROWS - 1) / QFB_ROWS, batch), 256, sm, st>>>(Qf, Dbuf, dims, ptrs, Mc, Lc);
  return cudaGetLastError();
}

// Raises the dynamic shared-memory limits the blocked QR, the Loewdin step
// and the folds need for capacities (M, N, L), outside any stream capture.
cudaError_t qr_blocked_prepare(int M, int N, int L) {
  cudaError_t e = cudaSuccess;
  const size_t qr = qb_smem_bytes(M > N ? M : N, L);
  if (qr <= 227 * 1024 - 1024) e = ensure_smem(k_qr_blk_f32<QB_THREADS>, qr, &g_attr_qr);
  const size_t qr256 = qb_smem_bytes(M > N ? M : N, L, 8), qr128 = qb_smem_bytes(M > N ? M : N, L, 4);
  if (e == cudaSuccess && qr256 <= 112 * 1024) e = ensure_smem(k_qr_blk_f32<256>, qr256, &g_attr_qr256);
  if (e == cudaSuccess && qr128 <= 56 * 1024) e = ensure_smem(k_qr_blk_f32<128>, qr128, &g_attr_qr128);
  if (e == cudaSuccess && L <= QF_MAXL) {
    e = ensure_smem(k_lowdin, sizeof(float2) * (size_t)L * L, &g_attr_ld);
    if (e == cudaSuccess) e = launch_fold<true>(nullptr, nullptr, nullptr, nullptr, M, L, 0, nullptr);
    if (e == cudaSuccess) e = launch_fold<false>(nullptr, nullptr, nullptr, nullptr, N, L, 0, nullptr);
  } else if (e == cudaSuccess && L <= QF_MAXL_BIG) {
    e = launch_fold_big<true>(nullptr, nullptr, nullptr, nullptr, M, L, 0, nullptr);
    if (e == cudaSuccess) e = launch_fold_big<false>(nullptr, nullptr, nullptr, nullptr, N, L, 0, nullptr);
  }
  return e;
}

bool reorth_fits(int M, int L) { return M >= L && L <= QF_MAXL_BIG; }

cudaError_t launch_reorth(const float2* Qf, float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int M, int L,
                          int batch, int* status, cudaStream_t st) {
  const int nt = (L + 31) / 32;
  if (L > QF_MAXL) {
    {
      ProfScope ps("k_lowdin", st);
      k_lowdin_big<<<dim3(nt * nt, batch), 256, 0, st>>>(dims, ptrs, Dbuf, L, status);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    ProfScope ps("k_fold[q]", st);
    return launch_fold_big<true>(Qf, Dbuf, dims, ptrs, M, L, batch, st);
  }
  const size_t sm_l = sizeof(float2) * (size_t)L * L;
  cudaError_t e0 = ensure_smem(k_lowdin, sm_l, &g_attr_ld);
  if (e0 != cudaSuccess) return e0;
  {
    ProfScope ps("k_lowdin", st);
    k_lowdin<<<batch, 512, sm_l, st>>>(dims, ptrs, Dbuf, L, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ProfScope ps("k_fold[q]", st);
  return launch_fold<true>(Qf, Dbuf, dims, ptrs, M, L, batch, st);
}

// B^H <- B^H (I + D) in place on ptrs[z].Yt (D.n x D.l column-major).
cudaError_t launch_fold_bh(const float2* Dbuf, const Dims* dims, const ProbPtr* ptrs, int n, int l, int batch,
                           cudaStream_t st) {
  ProfScope ps("k_fold[bh]", st);
  if (l > QF_MAXL) return launch_fold_big<false>(nullptr, Dbuf, dims, ptrs, n, l, batch, st);
  return launch_fold<false>(nullptr, Dbuf, dims, ptrs, n, l, batch, st);
}

}  // namespace tg
