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
// {"name": {"launches": n, "ms": t, "units": u, "bytes": b}, ...}
std::string timer_report_json();

// units: work items of the launch (right-hand sides or vectors it processes);
// bytes: algorithmic memory traffic of the launch (every element it must read
// or write, once), 0 where the caller does not state it
struct ScopedTimer {
  bool active;
  cudaStream_t st;
  ScopedTimer(const char* name, cudaStream_t s, long units = 1, double bytes = 0);
  ~ScopedTimer();
};

}  // namespace ddtm
