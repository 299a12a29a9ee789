// Optional per-kernel timing with CUDA events on the launching stream.
// Off by default; when on, every launch wrapper records a start/stop event
// pair under a kernel-class name, and tebd_profiler_read sums the elapsed
// times.  Not for use under stream capture.
#pragma once
#include <cuda_runtime.h>

namespace tg {
bool prof_on();
int prof_begin(const char* name, cudaStream_t st);  // returns a slot or -1
void prof_end(int slot, cudaStream_t st);

struct ProfScope {
  int slot;
  cudaStream_t st;
  ProfScope(const char* name, cudaStream_t s) : slot(prof_on() ? prof_begin(name, s) : -1), st(s) {}
  ~ProfScope() {
    if (slot >= 0) prof_end(slot, st);
  }
};
}  // namespace tg
