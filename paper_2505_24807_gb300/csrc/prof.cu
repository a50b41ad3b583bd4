// Per-kernel CUDA-event timing of libxs (see prof.h).
#include "prof.h"

namespace xs {

thread_local Profiler* g_prof = nullptr;

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t ev = nullptr;
  cudaEventCreate(&ev);
  return ev;
}

void Profiler::flush() {
  // timeline: the device idle time before each launch (end of the previous
  // launch to its start, same stream), charged to "gap:<kernel>"
  if (!spans.empty()) {
    std::map<const ProfEntry*, std::string> names;
    for (auto& kv : e) names[&kv.second] = kv.first;
    std::map<std::string, std::pair<int, double>> gaps;
    for (size_t i = 1; i < spans.size(); ++i) {
      cudaEventSynchronize(spans[i].a);
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, spans[i - 1].b, spans[i].a) == cudaSuccess && ms > 0.0f) {
        auto& g = gaps["gap:" + names[spans[i].ent]];
        g.first += 1;
        g.second += ms;
      }
    }
    spans.clear();
    for (auto& kv : gaps) {
      ProfEntry& ge = e[kv.first];
      ge.launches += kv.second.first;
      ge.ms += kv.second.second;
    }
  }
  for (auto& kv : e) {
    for (auto& pr : kv.second.pending) {
      cudaEventSynchronize(pr.second);
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) kv.second.ms += ms;
      pool.push_back(pr.first);
      pool.push_back(pr.second);
    }
    kv.second.pending.clear();
  }
}

void Profiler::reset() {
  flush();
  e.clear();
  launches = 0;
}

Profiler::~Profiler() {
  flush();
  for (auto ev : pool) cudaEventDestroy(ev);
}

ProfScope::ProfScope(cudaStream_t stream, const char* name, double bytes, double flops) {
  if (!g_prof || !g_prof->on) return;
  ent = &g_prof->e[name];
  ent->launches += 1;
  ent->bytes += bytes;
  ent->flops += flops;
  if (!g_prof->events) {
    ent = nullptr;
    return;
  }
  s = stream;
  a = g_prof->get();
  b = g_prof->get();
  cudaEventRecord(a, s);
  if (g_prof->timeline) g_prof->spans.push_back({ent, a, b});
}

ProfScope::~ProfScope() {
  if (!ent) return;
  cudaEventRecord(b, s);
  ent->pending.emplace_back(a, b);
}

HostScope::HostScope(const char* name) {
  if (!g_prof || !g_prof->on) return;
  ent = &g_prof->e[name];
  ent->launches += 1;
  t0 = std::chrono::steady_clock::now();
}

void HostScope::stop() {
  if (!ent) return;
  ent->ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ent = nullptr;
}

}  // namespace xs
