#include <map>
#include <vector>

#include "ddtm_internal.h"
#include "timer.h"

namespace ddtm {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
  long units;
  double bytes;
};
struct Acc {
  long launches = 0, units = 0;
  double ms = 0, bytes = 0;
};
struct State {
  bool on = false;
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Acc> acc;
  const char* cur = nullptr;
  cudaEvent_t cur_a = nullptr;
  long cur_units = 0;
  double cur_bytes = 0;
  long launch_base = 0;
};
State& S() {
  static State s;
  return s;
}
cudaEvent_t get_event() {
  State& s = S();
  if (!s.pool.empty()) {
    cudaEvent_t e = s.pool.back();
    s.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}
void flush() {
  State& s = S();
  for (auto& r : s.pending) {
    CK(cudaEventSynchronize(r.b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    auto& v = s.acc[r.name];
    v.launches += 1;
    v.units += r.units;
    v.bytes += r.bytes;
    v.ms += ms;
    s.pool.push_back(r.a);
    s.pool.push_back(r.b);
  }
  s.pending.clear();
}
}  // namespace

bool timer_on() { return S().on; }
void timer_enable(bool on) {
  if (!on) flush();
  S().on = on;
}
void timer_reset() {
  flush();
  S().acc.clear();
  S().launch_base = kernel_launches();
}
std::string timer_report_json() {
  flush();
  // "_kernel_launches": every kernel launched by the library since the last reset
  std::string out = "{\"_kernel_launches\": " + std::to_string(kernel_launches() - S().launch_base);
  bool first = false;
  for (auto& kv : S().acc) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f, \"units\": %ld, \"bytes\": %.0f}",
             first ? "" : ", ", kv.first.c_str(), kv.second.launches, kv.second.ms, kv.second.units, kv.second.bytes);
    out += buf;
    first = false;
  }
  return out + "}";
}

ScopedTimer::ScopedTimer(const char* name, cudaStream_t s, long units, double bytes) : active(S().on), st(s) {
  if (!active) return;
  State& g = S();
  if (g.pending.size() > 20000) flush();
  g.cur = name;
  g.cur_units = units;
  g.cur_bytes = bytes;
  g.cur_a = get_event();
  CK(cudaEventRecord(g.cur_a, s));
}

ScopedTimer::~ScopedTimer() {
  if (!active) return;
  State& g = S();
  cudaEvent_t b = get_event();
  if (cudaEventRecord(b, st) == cudaSuccess) g.pending.push_back(Rec{g.cur, g.cur_a, b, g.cur_units, g.cur_bytes});
}

}  // namespace ddtm
