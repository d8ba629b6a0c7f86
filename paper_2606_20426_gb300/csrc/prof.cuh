// Opt-in per-kernel timing with CUDA events on the launching stream.
//
// When an env has profiling enabled, every kernel launch made on its behalf
// is bracketed by two events; completed pairs are folded into per-kernel
// totals (milliseconds and launch counts) at the env's next synchronisation.
// With profiling off a launch costs one thread-local pointer test.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

namespace tc {

struct ProfEntry {
  const char* name;
  double ms;
  long long launches;
};

struct Profiler {
  struct Pending {
    int idx;
    cudaEvent_t a, b;
  };
  std::vector<ProfEntry> entries;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;

  int index_of(const char* name) {
    for (size_t i = 0; i < entries.size(); ++i)
      if (std::strcmp(entries[i].name, name) == 0) return (int)i;
    entries.push_back({name, 0.0, 0});
    return (int)entries.size() - 1;
  }
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // fold completed pairs (call after the stream was synchronised)
  void collect() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        entries[p.idx].ms += ms;
        entries[p.idx].launches += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    collect();
    for (auto& e : entries) {
      e.ms = 0.0;
      e.launches = 0;
    }
  }
  ~Profiler() {
    for (auto& p : pending) {
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// The profiler of the env whose work is being launched (set by the API
// entry points for the duration of a call; null = profiling off).
extern thread_local Profiler* g_prof;

struct ProfScope {
  Profiler* p;
  cudaStream_t s;
  int idx;
  cudaEvent_t a;
  ProfScope(const char* name, cudaStream_t stream) : p(g_prof), s(stream), idx(-1), a(nullptr) {
    if (p) {
      idx = p->index_of(name);
      a = p->take();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (p) {
      cudaEvent_t b = p->take();
      cudaEventRecord(b, s);
      p->pending.push_back({idx, a, b});
    }
  }
};

}  // namespace tc

#define TC_LAUNCH(name, stream, ...)         \
  do {                                       \
    ::tc::ProfScope tc_prof_scope_(name, stream); \
    __VA_ARGS__;                             \
  } while (0)
