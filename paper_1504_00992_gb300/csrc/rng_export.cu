// Exports of the sketch generator: the raw Philox4x64-10 words and the
// Gaussian test matrix Omega of Alg. 1 exactly as the sketch kernels draw
// them (the same device functions, common.cuh), so that a caller can check
// them against an independent implementation bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tebd_gb300.h"
#include "internal.cuh"
#include "profiler.cuh"

namespace tg {

__global__ void k_philox_words(const uint64_t* __restrict__ ctr, int64_t count, uint64_t k0, uint64_t k1,
                               uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const u64x4 w = philox4x64_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
#pragma unroll
    for (int j = 0; j < 4; ++j) out[4 * i + j] = w.v[j];
  }
}

// Row-major n x l: element (r, c) is sketch element r*l + c, the counter the
// sketch kernels give it.
__global__ void k_omega_export(int64_t total, uint64_t seed, uint64_t bond, uint64_t sweep, uint64_t chain,
                               cplx* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = gauss_c((uint64_t)e, bond, sweep, chain, seed, 0);
}

__global__ void k_omega_export_f32(int64_t total, uint64_t seed, uint64_t bond, uint64_t sweep, uint64_t chain,
                                   float2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = gauss_c_f32((uint64_t)e, bond, sweep, chain, seed);
}

static int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 1024) b = 1024;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace tg

using namespace tg;

extern "C" int tebd_philox4x64_10(const uint64_t* counters, int64_t count, uint64_t key0, uint64_t key1,
                                  uint64_t* words, void* stream) {
  if (count < 0 || (count > 0 && (!counters || !words))) return TEBD_EINVAL;
  if (count == 0) return TEBD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps("k_philox_words", st);
  k_philox_words<<<grid_for(count), 256, 0, st>>>(counters, count, key0, key1, words);
  return cudaGetLastError() == cudaSuccess ? TEBD_OK : TEBD_ECUDA;
}

extern "C" int rrsvd_sketch_omega(int n, int l, uint64_t seed, int64_t bond, int64_t sweep, int64_t chain,
                                  int precision, void* out, void* stream) {
  if (n < 0 || l < 0 || bond < 0 || sweep < 0 || chain < 0) return TEBD_EINVAL;
  if (precision != TEBD_PREC_FP64 && precision != TEBD_PREC_TF32 && precision != TEBD_PREC_BF16)
    return TEBD_ENOTIMPL;
  const int64_t total = (int64_t)n * l;
  if (total == 0) return TEBD_OK;
  if (!out) return TEBD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps("k_omega_export", st);
  if (precision == TEBD_PREC_FP64)
    k_omega_export<<<grid_for(total), 256, 0, st>>>(total, seed, (uint64_t)bond, (uint64_t)sweep, (uint64_t)chain,
                                                    (cplx*)out);
  else
    k_omega_export_f32<<<grid_for(total), 256, 0, st>>>(total, seed, (uint64_t)bond, (uint64_t)sweep,
                                                        (uint64_t)chain, (float2*)out);
  return cudaGetLastError() == cudaSuccess ? TEBD_OK : TEBD_ECUDA;
}
