// Batch executor: device tables and pinned staging for batched launches.
#pragma once
#include <climits>
#include <cstdio>
#include <cstdint>
#include <initializer_list>
#include <vector>

#include "env.cuh"
#include "prof.cuh"
#include "solver.cuh"

namespace tc {

// CUDA-graph replay of phase launch sequences (TACAUCHY_GRAPHS=0 turns it off)
bool graphs_on();
bool trace_on();  // TACAUCHY_TRACE set (and not 0): per-iteration trace lines on stderr

template <class R> struct BatchExec {
  Arena* arena = nullptr;        // device memory comes from this arena
  cudaStream_t stream = nullptr;
  int cap_env = 0;
  int64_t cap_part = 0;
  EnvView<R>* d_views = nullptr;
  int* d_prefix = nullptr;
  double* d_part = nullptr;
  double* d_param = nullptr;
  Motion* d_motion = nullptr;
  Scalars* d_sc = nullptr;       // per-env scalars of the current phase
  EnvView<R>* h_views = nullptr; // pinned staging
  int* h_prefix = nullptr;
  double* h_param = nullptr;
  Motion* h_motion = nullptr;
  Scalars* h_sc = nullptr;
  BatchHost<R> host;
  std::vector<Env*> members;
  // Instantiated graphs of phase launch sequences.  A graph is keyed on the
  // phase, its launch parameters, the batch's unit tables (which fix every
  // grid) and `gen`, which moves whenever the device tables the kernels'
  // arguments point to are reallocated; the per-env contents of those
  // tables are uploaded by build() before every replay.
  struct Graph {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
    int seen = 0;
    uint64_t tick = 0;
  };
  static constexpr size_t kMaxGraphs = 24;
  std::vector<Graph> graphs;
  uint64_t gen = 0, tick = 0;
  cudaStream_t cap_stream = nullptr;  // captures run here (the legacy default stream cannot capture)

  ~BatchExec();
  void release();
  void drop_graphs();
  tc_status reserve(int nenv, int64_t part);
  // upload views / unit tables / params / motions of `set` and clear its scalars
  tc_status build(const std::vector<Env*>& set, const double* params, const Motion* motions);
  // copy the phase's scalars to h_sc and wait for the stream
  tc_status read();
  // Run the launch sequence f() of phase `phase` for the current batch: the
  // second time the same (phase, extra, batch tables) comes up it is captured
  // as a CUDA graph, and from then on replayed with one graph launch.  Off
  // while kernel profiling is on; a failed capture falls back to direct
  // launches for that key.
  template <class F> tc_status launch(int phase, std::initializer_list<int64_t> extra, F&& f);
};

template <class R>
template <class F>
tc_status BatchExec<R>::launch(int phase, std::initializer_list<int64_t> extra, F&& f) {
  if (g_prof != nullptr || !graphs_on()) return f();
  const int n = host.nenv;
  std::vector<int64_t> key;
  key.reserve(3 + extra.size() + (size_t)K_NKIND * (n + 1));
  key.push_back(phase);
  key.push_back((int64_t)gen);
  key.push_back(n);
  for (int64_t x : extra) key.push_back(x);
  for (int i = 0; i < K_NKIND * (n + 1); ++i) key.push_back(h_prefix[i]);
  ++tick;
  Graph* g = nullptr;
  for (auto& x : graphs)
    if (x.key == key) {
      g = &x;
      break;
    }
  if (!g) {
    if (graphs.size() >= kMaxGraphs) {  // evict the least recently used
      size_t lru = 0;
      for (size_t i = 1; i < graphs.size(); ++i)
        if (graphs[i].tick < graphs[lru].tick) lru = i;
      if (graphs[lru].exec) cudaGraphExecDestroy(graphs[lru].exec);
      graphs.erase(graphs.begin() + (long)lru);
    }
    graphs.push_back(Graph{key, nullptr, 0, tick});
    g = &graphs.back();
  }
  g->tick = tick;
  if (!g->exec) {
    if (g->seen < 0 || ++g->seen < 2) return f();  // capture on the second sighting
    cudaGraph_t cg = nullptr;
    if ((!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) ||
        cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g->seen = INT_MIN;
      if (trace_on()) std::fprintf(stderr, "[tc] graph of phase %d over %d envs: no capture, direct launches\n", phase, n);
      return f();
    }
    // f() launches on `stream`: point it at the capture stream meanwhile
    // (nothing runs during a capture; the graph is launched on the real one)
    const cudaStream_t real = stream;
    stream = cap_stream;
    const tc_status fs = f();
    const cudaError_t ce = cudaStreamEndCapture(cap_stream, &cg);
    stream = real;
    if (fs != TC_OK || ce != cudaSuccess || cg == nullptr || cudaGraphInstantiate(&g->exec, cg, 0) != cudaSuccess) {
      if (cg) cudaGraphDestroy(cg);
      g->exec = nullptr;
      g->seen = INT_MIN;  // this key runs directly from now on
      cudaGetLastError();
      if (trace_on()) std::fprintf(stderr, "[tc] graph of phase %d over %d envs: capture failed, direct launches\n", phase, n);
      return f();
    }
    cudaGraphDestroy(cg);
    if (trace_on()) std::fprintf(stderr, "[tc] graph of phase %d over %d envs captured\n", phase, n);
  }
  return cudaGraphLaunch(g->exec, stream) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

// State of one step request (Algorithm 2, physics line) in the scheduler.
struct StepCtl {
  Env* env = nullptr;
  uint64_t tag = 0;
  tc_pose pose0{}, target{};
  double s = 0.0, g0 = -1.0, E0 = 0.0, alpha = 1.0;
  double E1 = 0.0, ext = 0.0;  // energy after an accepted full step; continuation factor - 1
  int sub = 0, newton = 0, halvings = 0;
  bool tight = false;  // mixed mode: the substep's solves run to the verification tolerance
  double pmax = 0.0;   // max-norm of the current Newton direction
  enum Phase { START, ADVANCE, NEWTON, LINESEARCH, EXTEND, DONE, FAILED } phase = START;
  tc_status status = TC_OK;
};

struct StepDone {
  uint64_t tag;
  Env* env;
  tc_status status;
};

// Round-based scheduler over step requests: admit() adds a request at any
// time; round() advances every admitted request by one phase group (start,
// advance, Newton, PCG/CCD/trial, one halving, end) with one launch set per
// phase over all requests in it, and appends the requests that finished.
// One env may have at most one admitted request at a time.
template <class R> struct StepScheduler {
  BatchExec<R>* exec = nullptr;
  std::vector<StepCtl> tasks;
  void admit(Env* env, const tc_pose& target, uint64_t tag);
  tc_status round(std::vector<StepDone>& finished);
  bool empty() const { return tasks.empty(); }
};

void pose_interp(const tc_pose& a, const tc_pose& b, double s, tc_pose* out);
tc_status alloc_candidates(Env& env, int cap);
template <class R> tc_status ensure_candidates(BatchExec<R>& X, const std::vector<Env*>& envs);
template <class R>
tc_status step_batch(BatchExec<R>& X, const std::vector<Env*>& envs, const std::vector<tc_pose>& targets,
                     std::vector<tc_status>& result);
template <class R> tc_status energy_at_state(BatchExec<R>& X, Env& env, Scalars* out);
// Time the PCG of the envs' current Newton systems under every co-schedulable
// launch shape and keep the fastest per CG iteration of one env: mode 0 with
// each env's solve launched alone (latency), mode 1 with one launch over all
// envs (throughput).
struct PcgTune {
  int cs, threads, coresident;
  double us_per_env_iter;
  long long env_iters;
};
template <class R>
tc_status autotune_pcg(BatchExec<R>& X, const std::vector<Env*>& envs, int mode, std::vector<PcgTune>& out);
template <class R> tc_status contact_force_at_state(BatchExec<R>& X, Env& env, double* f);
template <class R> tc_status energy_gradient_at_state(BatchExec<R>& X, Env& env, double* E, double* grad);

}  // namespace tc
