// Batch executor: device tables and pinned staging for batched launches.
#pragma once
#include <vector>

#include "env.cuh"
#include "solver.cuh"

namespace tc {

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

  ~BatchExec();
  void release();
  tc_status reserve(int nenv, int64_t part);
  // upload views / unit tables / params / motions of `set` and clear its scalars
  tc_status build(const std::vector<Env*>& set, const double* params, const Motion* motions);
  // copy the phase's scalars to h_sc and wait for the stream
  tc_status read();
};

// State of one step request (Algorithm 2, physics line) in the scheduler.
struct StepCtl {
  Env* env = nullptr;
  uint64_t tag = 0;
  tc_pose pose0{}, target{};
  double s = 0.0, g0 = -1.0, E0 = 0.0, alpha = 1.0;
  double E1 = 0.0, ext = 0.0;  // energy after an accepted full step; continuation factor - 1
  int sub = 0, newton = 0, halvings = 0;
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

// TACAUCHY_TRACE set (and not 0): per-iteration trace lines on stderr
bool trace_on();
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
