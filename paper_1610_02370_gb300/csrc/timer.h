// Per-kernel CUDA-event timing of every launch (off by default).  When
// enabled, each wrapped launch records an event before and after itself on the
// stream it is launched on; report() synchronises, sums the elapsed times per
// kernel name and returns launches and milliseconds.  One timer per process:
// contexts used from different threads at the same time share it.
#pragma once

#include <cuda_runtime.h>

#include <string>

namespace ddtm {

bool timer_on();
void timer_enable(bool on);
void timer_reset();
std::string timer_report_json();  // {"name": {"launches": n, "ms": t}, ...}

struct ScopedTimer {
  bool active;
  cudaStream_t st;
  ScopedTimer(const char* name, cudaStream_t s);
  ~ScopedTimer();
};

}  // namespace ddtm
