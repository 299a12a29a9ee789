// Tensor-core GEMM for the low-precision sketch products (sm_103a tcgen05).
//
// Computes, per instance z of a batch, C = sum_pass A_pass * B_pass^T with
//   A: M x Kp real FP32 holding TF32-rounded values (KIND = TC_TF32) or BF16
//      values (KIND = TC_BF16), K-major (row-major),
//   B: Np x Kp of the same type, K-major,
// FP32 accumulation in tensor memory, and writes complex FP32 columns:
//   out[c * M + r] = (C[r][2c], C[r][2c+1])  for c < l, r < M
// (the real embedding of a complex product puts Re and Im of output column
// c in adjacent real columns 2c, 2c+1).
//
// npass = 1: A0 B0^T (one TF32 or BF16 product).  npass = 3 (TF32 only):
// A0 B0^T + A0 B1^T + A1 B0^T (the "3xTF32" split product, FP32-level
// accuracy).  A stage holds 128 bytes of every row: 32 TF32 or 64 BF16
// values, four MMAs of K = 8 (kind::tf32) or K = 16 (kind::f16) each.
//
// Structure (one CTA = 128 rows x up to 256 columns, 4 warps):
//   warp 0 / one lane : TMA producer (cp.async.bulk.tensor.3d into a ring of
//                       STAGES shared-memory slots, 128-byte swizzle),
//   warp 1 / one lane : MMA issuer (tcgen05.mma.cta_group::1.kind::tf32 or
//                       kind::f16, 4 per 128-byte slot), frees slots with
//                       tcgen05.commit -> mbarrier,
//   all 4 warps       : epilogue, tcgen05.ld 32x32b from the accumulator
//                       (warp w owns TMEM lanes 32w..32w+31 = tile rows).
// Every mbarrier wait is bounded (poll_limit polls); on expiry the kernel
// raises *err, skips the remaining work, waits (bounded) for its own copies
// and for the MMAs it already issued, and frees TMEM.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_sync.cuh"

namespace tg {

enum { TC_BM = 128, TC_BK = 32, TC_STAGES = 4, TC_MAXBN = 256, TC_TMEM_COLS = 256 };
enum { TC_TF32 = 0, TC_BF16 = 1 };
// k values per 128-byte stage row
__host__ __device__ constexpr int tc_bk(int kind) { return kind == TC_BF16 ? 64 : TC_BK; }

struct TcArgs {
  int M;          // rows of A and of the output
  int Kp;         // padded reduction length (multiple of TC_BK)
  int BN;         // columns per CTA (multiple of 16, <= 256)
  int l;          // complex output columns
  int npass;      // 1 or 3
  float2* out;    // complex output, column-major M x l, instance stride out_stride
  int64_t out_stride;
  int* err;       // error flag (timeouts)
  uint32_t poll_limit;  // polls of a pipeline wait before it gives up (1 << 24)
  int stall;      // test hook: the producer issues no copies, so the waits expire
};

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes stacked along M/N (stride byte offset 1024), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// kind::f16 with A = B = BF16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
              const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1, TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t bytesA = TC_BM * 128;     // 16 KB
  const uint32_t bytesB = (uint32_t)a.BN * 128;
  uint8_t* sA = smem;
  uint8_t* sB = smem + TC_STAGES * bytesA;
  uint64_t* full = (uint64_t*)(sB + TC_STAGES * bytesB);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accf = empty + TC_STAGES;
  uint64_t* drain = accf + 1;  // completion of the MMAs issued before an abort
  uint32_t* tmem_holder = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * a.BN, z = blockIdx.z;
  const int KB = a.Kp / tc_bk(KIND);
  const int iters = a.npass * KB;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(tmem_holder)),
                 "r"((uint32_t)TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < TC_STAGES; ++s) {
      tc_mbar_init(&full[s], 1);
      tc_mbar_init(&empty[s], 1);
    }
    tc_mbar_init(accf, 1);
    tc_mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---- producer
    int issued = 0;
    for (int it = 0; it < (a.stall ? 0 : iters); ++it) {
      const int s = it % TC_STAGES;
      const uint32_t r = (uint32_t)(it / TC_STAGES);
      if (it >= TC_STAGES && !tc_mbar_wait(&empty[s], (r & 1u) ^ 1u, a.poll_limit, a.err, abort_flag)) break;
      const int pass = it / KB, kb = it % KB;
      const CUtensorMap* ta = (pass == 2) ? &tmA1 : &tmA0;
      const CUtensorMap* tb = (pass == 1) ? &tmB1 : &tmB0;
      tc_mbar_expect_tx(&full[s], bytesA + bytesB);
      tc_tma_load_3d(sA + s * bytesA, ta, kb * tc_bk(KIND), m0, z, &full[s]);
      tc_tma_load_3d(sB + s * bytesB, tb, kb * tc_bk(KIND), n0, z, &full[s]);
      issued = it + 1;
    }
    // make sure every copy this thread issued has landed before teardown
    if (*abort_flag) {
      for (int it = (issued > TC_STAGES ? issued - TC_STAGES : 0); it < issued; ++it)
        for (uint32_t i = 0; i < (1u << 22); ++i)
          if (tc_mbar_try_wait(&full[it % TC_STAGES], (uint32_t)(it / TC_STAGES) & 1u)) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = KIND == TC_BF16 ? tc_idesc_bf16(TC_BM, a.BN) : tc_idesc_tf32(TC_BM, a.BN);
    bool ok = true;
    int issued_mma = 0;
    for (int it = 0; it < iters; ++it) {
      const int s = it % TC_STAGES;
      const uint32_t r = (uint32_t)(it / TC_STAGES);
      if (!tc_mbar_wait(&full[s], r & 1u, a.poll_limit, a.err, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const uint32_t aa = tc_smem_u32(sA + s * bytesA), bb = tc_smem_u32(sB + s * bytesB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of k per MMA
        const uint64_t ad = tc_desc_sw128(aa + kk * 32), bd = tc_desc_sw128(bb + kk * 32);
        const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
        if (KIND == TC_BF16)
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem_u32(&empty[s]))
                   : "memory");
      issued_mma = it + 1;
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem_u32(accf))
                   : "memory");
    } else {
      *abort_flag = 1;
      if (issued_mma > 0) {
        // the MMAs already issued read shared memory and write the tensor
        // memory freed below: wait (bounded) until they have completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         tc_smem_u32(drain))
                     : "memory");
        for (uint32_t i = 0; i < a.poll_limit; ++i)
          if (tc_mbar_try_wait(drain, 0)) break;
      }
    }
  }
  __syncwarp();
  // ---- epilogue: every thread owns one row of the tile
  const bool have = tc_mbar_wait(accf, 0, a.poll_limit, a.err, abort_flag);
  tc_fence_after();
  if (!have) {
    // aborted: defined (zero) output for the kernels that read it next; the
    // timeout flag already marks the result as invalid
    const int row = m0 + warp * 32 + lane;
    float2* out = a.out + a.out_stride * z;
    if (row < a.M)
      for (int cc = n0 / 2; cc < (n0 + a.BN) / 2 && cc < a.l; ++cc) out[(int64_t)cc * a.M + row] = make_float2(0.f, 0.f);
  } else {
    const int row = m0 + warp * 32 + lane;
    float2* out = a.out + a.out_stride * z;
    for (int c0 = 0; c0 < a.BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < a.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cc = (n0 + c0) / 2 + j;
          if (cc < a.l) out[(int64_t)cc * a.M + row] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_TMEM_COLS)
                 : "memory");
  }
}

inline size_t tc_smem_bytes(int BN) {
  return 1024 + (size_t)TC_STAGES * (TC_BM * 128 + (size_t)BN * 128) + (2 * TC_STAGES + 2) * 8 + 16;
}

}  // namespace tg
