// Per-kernel-class event timing (see profiler.cuh) and its C ABI.
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tebd_gb300.h"
#include "profiler.cuh"

namespace tg {
namespace {
struct Rec {
  std::string name;
  cudaEvent_t a, b;
  bool closed;
};
std::mutex mu;
bool on = false;
std::vector<Rec> recs;
std::vector<cudaEvent_t> pool;
struct Acc {
  double ms = 0.0;
  long long n = 0;
};
std::map<std::string, Acc> acc;

cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void drain_locked() {
  for (auto& r : recs) {
    if (!r.closed) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      Acc& x = acc[r.name];
      x.ms += ms;
      x.n += 1;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  std::vector<Rec> keep;
  for (auto& r : recs)
    if (!r.closed) keep.push_back(r);
  recs.swap(keep);
}
}  // namespace

bool prof_on() { return on; }

int prof_begin(const char* name, cudaStream_t st) {
  std::lock_guard<std::mutex> g(mu);
  if (recs.size() > 4096) drain_locked();
  Rec r;
  r.name = name;
  r.a = get_event();
  r.b = get_event();
  r.closed = false;
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void prof_end(int slot, cudaStream_t st) {
  std::lock_guard<std::mutex> g(mu);
  if (slot < 0 || slot >= (int)recs.size()) return;
  cudaEventRecord(recs[slot].b, st);
  recs[slot].closed = true;
}
}  // namespace tg

extern "C" int tebd_profiler_enable(int enable) {
  std::lock_guard<std::mutex> g(tg::mu);
  tg::on = enable != 0;
  return TEBD_OK;
}

extern "C" int tebd_profiler_reset(void) {
  std::lock_guard<std::mutex> g(tg::mu);
  tg::drain_locked();
  tg::acc.clear();
  return TEBD_OK;
}

extern "C" int tebd_profiler_read(int max_entries, char* names, double* total_ms, int64_t* launches, int* count) {
  if (max_entries < 0 || !count) return TEBD_EINVAL;
  std::lock_guard<std::mutex> g(tg::mu);
  tg::drain_locked();
  int i = 0;
  for (auto& kv : tg::acc) {
    if (i < max_entries) {
      if (names) {
        strncpy(names + 64 * i, kv.first.c_str(), 63);
        names[64 * i + 63] = 0;
      }
      if (total_ms) total_ms[i] = kv.second.ms;
      if (launches) launches[i] = kv.second.n;
    }
    ++i;
  }
  *count = i;
  return TEBD_OK;
}
