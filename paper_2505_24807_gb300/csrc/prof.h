// Per-kernel CUDA-event timing of libxs (enabled through xs_profile).  Each
// instrumented launch is bracketed by two events on the launching stream;
// elapsed times are summed when the profile is read.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <map>
#include <string>
#include <vector>

namespace xs {

struct ProfEntry {
  int launches = 0;
  double ms = 0.0;
  double bytes = 0.0;   // algorithmic bytes, summed over launches
  double flops = 0.0;   // algorithmic flops, summed over launches
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

struct Profiler {
  bool on = false;
  bool events = true;       // false: count launches, bytes and flops only
  bool timeline = false;    // also attribute the device idle time between launches
  struct Span {
    const ProfEntry* ent;
    cudaEvent_t a, b;
  };
  std::vector<Span> spans;  // launch order (timeline mode)
  long long launches = 0;   // every kernel launch of the library while on
  std::map<std::string, ProfEntry> e;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void flush();   // resolve pending event pairs (synchronises on them)
  void reset();
  ~Profiler();
};

// The profiler of the context whose API call is running on this thread.
extern thread_local Profiler* g_prof;

struct ProfScope {
  ProfEntry* ent = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s = nullptr;
  ProfScope(cudaStream_t stream, const char* name, double bytes, double flops);
  ~ProfScope();
};

// Host wall time of a region of an API call, recorded under its name (by
// convention "host:..."; launches counts the entries) while profiling is on.
struct HostScope {
  ProfEntry* ent = nullptr;
  std::chrono::steady_clock::time_point t0;
  explicit HostScope(const char* name);
  void stop();
  ~HostScope() { stop(); }
};

}  // namespace xs
