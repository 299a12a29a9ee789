// rrsvd_execute_noalloc: the batched RRSVD truncation of rrsvd_execute for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- inside
// another library's scheduling loop or a host callback that must not block
// (cudaMalloc can synchronise the device), or in a process whose device
// memory has been reserved up front by a caching allocator or a fixed budget,
// so a fresh allocation may fail or evict.  Such a caller cannot create an
// rrsvd plan (which allocates descriptors) nor pass a workspace it cannot
// obtain.  This entry point needs neither: all of its scratch (descriptors,
// status word and the per-instance RRSVD workspace) lives in one file-scope
// device array that the library image carries, so every GPU that loads the
// library holds NOALLOC_SCRATCH_BYTES for the life of the process.
//
// Properties
//   * No cudaMalloc, cudaFree or allocating library call.
//   * Host code never hands the array's symbol to a kernel (in host code the
//     name is a host-side stand-in, not a device address): the device
//     address is looked up with cudaGetSymbolAddress once per device, on the
//     first call made while that device is current, and cached.  That first
//     call therefore does set-up work and should be made before any stream
//     capture begins.
//   * Every call reuses the same array, which keeps the previous call's
//     contents; the status word is cleared at the start of each call and
//     everything else is written before it is read.  Calls whose GPU work
//     overlaps (different streams, or several host threads) race on the
//     array and corrupt each other's results: the caller must order them.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/tebd_gb300.h"
#include "internal.cuh"
#include "profiler.cuh"
#include "workspace.cuh"

namespace tg {

static const size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

const size_t NA_ALIGN = 256;
inline size_t na_up(size_t x) { return (x + NA_ALIGN - 1) & ~(NA_ALIGN - 1); }

std::mutex na_mu;
const int NA_MAXDEV = 64;
void* na_addr[NA_MAXDEV] = {nullptr};

}  // namespace

}  // namespace tg

using namespace tg;

extern "C" int rrsvd_execute_noalloc(int m, int n, int k_max, int p, int q, int batch, uint64_t seed, int64_t chain0,
                                     const double* theta, double* sigma, double* U, double* Vh, double* w, int* rank,
                                     void* stream) {
  if (m < 1 || n < 1 || k_max < 1 || p < 0 || q < 0 || batch < 1 || chain0 < 0 || !theta || !sigma)
    return TEBD_EINVAL;
  const int k = k_max < (m < n ? m : n) ? k_max : (m < n ? m : n);
  const int mn = m < n ? m : n;
  const int l = (k + p < mn) ? k + p : mn;
  if (l > 512) return TEBD_EINVAL;
  // the workspace layout of an rrsvd plan of the same sizes (U and V^H have
  // room in it, for calls that pass NULL for them)
  const WsLayout lay = ws_layout(m, n, k, l, true, true, 0);
  const size_t head = na_up(sizeof(Dims) * (size_t)batch) + na_up(sizeof(ProbPtr) * (size_t)batch) + NA_ALIGN;
  const size_t need = head + lay.total * (size_t)batch;
  if (need > NOALLOC_SCRATCH_BYTES) return TEBD_EINVAL;  // beyond the fixed 16 MiB scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) return TEBD_ECUDA;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> g(na_mu);
    if (!na_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return TEBD_ECUDA;
      na_addr[dev] = ptr;
    }
    base = (char*)na_addr[dev];
  }
  Dims* dims = (Dims*)base;
  ProbPtr* ptrs = (ProbPtr*)(base + na_up(sizeof(Dims) * (size_t)batch));
  int* status = (int*)(base + na_up(sizeof(Dims) * (size_t)batch) + na_up(sizeof(ProbPtr) * (size_t)batch));
  char* ws = base + head;
  cudaStream_t st = (cudaStream_t)stream;
  {
    // descriptors of every instance, and the status word cleared (the one
    // value of the array that must start at zero)
    ProfScope ps("k_rrsvd_bind", st);
    k_rrsvd_bind<<<(batch + 127) / 128, 128, 0, st>>>(ptrs, batch, ws, lay.total, lay, (const cplx*)theta,
                                                       (size_t)m * n, (cplx*)U, (size_t)m * k, (cplx*)Vh,
                                                       (size_t)k * n, dims, m, n, k, l, status);
  }
  if (cudaGetLastError() != cudaSuccess) return TEBD_ECUDA;
  Caps cap;
  memset(&cap, 0, sizeof cap);
  cap.m = m; cap.n = n; cap.k = k; cap.l = l;
  if (run_rrsvd(dims, ptrs, batch, cap, q, seed, 0, chain0, 1, status, st) != cudaSuccess) return TEBD_ECUDA;
  if (launch_rrsvd_finalize(dims, ptrs, batch, cap, 1e-14, sigma, Vh, w, rank, status, st) != cudaSuccess)
    return TEBD_ECUDA;
  return TEBD_OK;
}
