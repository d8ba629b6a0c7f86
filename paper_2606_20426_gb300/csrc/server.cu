// Step server: continuous batching of tc_step requests from many envs.
//
// Callers submit (env, target pose, optional output buffers) from any thread
// and get a ticket back at once.  One worker thread per server owns a
// round-based step scheduler per precision: before every round it admits
// queued requests while a slot and HBM budget are free (an env's footprint is
// the device memory its arena holds), then runs one round -- every admitted
// request advances by one phase group, with one launch set per phase over all
// of them -- and finishes the requests that converged or failed: their
// stress and pressure map are written to the caller's buffers and their
// tickets complete.  A request that arrives while others are on the GPU joins
// at the next round boundary, so envs of different sizes and at different
// Newton iterations share every launch.  Env state (positions, velocities,
// candidate lists, PCG vectors) stays resident in the env between requests.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "env.cuh"

namespace tc {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  Env* env = nullptr;
  tc_pose target{};
  float* sigma = nullptr;
  float* map = nullptr;
  uint8_t* mask = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  int state = 0;  // 0 queued, 1 admitted, 2 done
  tc_status status = TC_OK;
  int rounds = 0;
  size_t bytes = 0;
};

struct Server {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int max_slots = 0;
  Arena arena;
  BatchExec<float> x32;
  BatchExec<double> x64;
  StepScheduler<float> s32;
  StepScheduler<double> s64;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;  // node-based: element addresses are stable
  int inflight = 0, peak_inflight = 0;
  size_t inflight_bytes = 0;
  int64_t submitted = 0, completed = 0;
  std::atomic<int64_t> rounds{0};
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;

  void run();
  void admit_locked(std::vector<Req*>& out);
  void complete_locked(Req& r, tc_status st);
};

void Server::complete_locked(Req& r, tc_status st) {
  r.status = st;
  r.state = 2;
  r.t_done = Clock::now();
  completed++;
}

// FIFO admission: a request waits while an earlier request of its env is in
// flight; the queue head waits for a free slot and for its footprint to fit
// the budget, except that a lone request always runs.
void Server::admit_locked(std::vector<Req*>& out) {
  for (auto it = queue.begin(); it != queue.end();) {
    Req& r = reqs.at(*it);
    if (r.env->in_flight.load()) {
      ++it;
      continue;
    }
    r.bytes = r.env->arena.bytes;
    if (r.bytes > budget) {  // can never fit
      complete_locked(r, TC_ERR_ADMISSION);
      r.env->busy.fetch_sub(1);
      it = queue.erase(it);
      continue;
    }
    const bool fits = inflight < max_slots && inflight_bytes + r.bytes <= budget;
    if (!fits && inflight > 0) break;
    r.state = 1;
    r.t_admit = Clock::now();
    r.env->in_flight.store(1);
    inflight++;
    inflight_bytes += r.bytes;
    peak_inflight = std::max(peak_inflight, inflight);
    out.push_back(&r);
    it = queue.erase(it);
  }
}

template <class R> static tc_status extract(Env& env, Req& r, cudaStream_t s) {
  EnvView<R> e = env.view<R>();
  if (r.sigma) launch_stress<R>(e, r.sigma, s);
  if (r.map && env.H * env.W > 0) {
    launch_traction<R>(e, env.cparent, nullptr, nullptr, nullptr, env.face_p, env.face_A, s);
    launch_vertex_avg(env.nvc, env.cv_face_off, env.cv_face_idx, env.face_p, env.face_A, env.vert_p, s);
    launch_splat(env.H * env.W, env.pix_face, env.pix_w, env.cface_slot, env.nfc, env.vert_p, r.map, r.mask, s);
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

void Server::run() {
  cudaSetDevice(device);
  std::vector<Req*> live;
  std::vector<StepDone> fin;
  for (;;) {
    std::vector<Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty() || inflight > 0; });
      if (stop && inflight == 0) break;
      if (!stop) admit_locked(admitted);
    }
    cv_done.notify_all();  // admission may have completed requests that can never fit
    // the env's earlier work (creation, extraction by the caller) is ordered
    // before its first launch on the server stream
    for (Req* r : admitted) {
      if (r->env->stream != stream) cudaStreamSynchronize(r->env->stream);
      if (r->env->precision == TC_FP64) s64.admit(r->env, r->target, r->ticket);
      else s32.admit(r->env, r->target, r->ticket);
      live.push_back(r);
    }
    fin.clear();
    tc_status st = TC_OK;
    const Clock::time_point t_round = Clock::now();
    if (!s32.empty()) st = s32.round(fin);
    if (st == TC_OK && !s64.empty()) st = s64.round(fin);
    if (trace_on())
      std::fprintf(stderr, "[tc] server round %lld: %zu in flight, %zu admitted, %zu finished, %.3f ms\n",
                   (long long)rounds.load(), live.size(), admitted.size(), fin.size(),
                   std::chrono::duration<double, std::milli>(Clock::now() - t_round).count());
    for (Req* r : live) r->rounds++;
    rounds++;
    std::vector<std::pair<Req*, tc_status>> done;
    if (st != TC_OK) {
      // a launch or copy failed: every request in flight ends with that status
      s32.tasks.clear();
      s64.tasks.clear();
      for (Req* r : live) done.push_back({r, st});
    } else {
      for (const StepDone& d : fin) {
        Req* r = nullptr;
        for (Req* q : live)
          if (q->ticket == d.tag) r = q;
        if (!r) continue;
        tc_status rs = d.status;
        if (rs == TC_OK && (r->sigma || r->map))
          rs = r->env->precision == TC_FP64 ? extract<double>(*r->env, *r, stream) : extract<float>(*r->env, *r, stream);
        done.push_back({r, rs});
      }
      if (!done.empty() && cudaStreamSynchronize(stream) != cudaSuccess)
        for (auto& d : done) d.second = TC_ERR_CUDA;
    }
    if (done.empty()) continue;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& d : done) {
        Req& r = *d.first;
        complete_locked(r, d.second);
        r.env->in_flight.store(0);
        r.env->busy.fetch_sub(1);
        inflight--;
        inflight_bytes -= r.bytes;
      }
    }
    std::vector<Req*> keep;
    for (Req* r : live) {
      bool fin_r = false;
      for (auto& d : done) fin_r = fin_r || d.first == r;
      if (!fin_r) keep.push_back(r);
    }
    live.swap(keep);
    cv_done.notify_all();
  }
}

}  // namespace tc

struct tc_server {
  tc::Server impl;
};

using tc::Clock;

static void fill_result(const tc::Req& r, tc_result* out) {
  if (!out) return;
  out->status = r.status;
  out->queue_us = r.state >= 1 && r.t_admit >= r.t_submit
                      ? std::chrono::duration<double, std::micro>(r.t_admit - r.t_submit).count()
                      : 0.0;
  out->latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
  out->rounds = r.rounds;
}

extern "C" {

tc_status tc_server_create(size_t hbm_budget_bytes, int32_t max_slots, tc_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots <= 0) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  tc_server* h = new (std::nothrow) tc_server;
  if (!h) return TC_ERR_OOM;
  tc::Server& s = h->impl;
  if (cudaGetDevice(&s.device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return TC_ERR_CUDA;
  }
  s.budget = hbm_budget_bytes;
  s.max_slots = max_slots;
  s.arena.stream = s.stream;
  s.x32.arena = &s.arena;
  s.x32.stream = s.stream;
  s.x64.arena = &s.arena;
  s.x64.stream = s.stream;
  s.s32.exec = &s.x32;
  s.s64.exec = &s.x64;
  try {
    s.worker = std::thread([&s] { s.run(); });
  } catch (...) {
    cudaStreamDestroy(s.stream);
    delete h;
    return TC_ERR_OOM;
  }
  *out = h;
  return TC_OK;
}

tc_status tc_submit(tc_server* h, tc_env* env, const tc_pose* target, float* sigma_out, float* map_out,
                    uint8_t* mask_out, uint64_t* ticket) {
  if (!h || !env || !target || !ticket) return TC_ERR_INVALID_ARG;
  for (double v : target->R)
    if (!std::isfinite(v)) return TC_ERR_NONFINITE;
  for (double v : target->t)
    if (!std::isfinite(v)) return TC_ERR_NONFINITE;
  tc::Server& s = h->impl;
  tc::Env& e = env->impl;
  if (e.device != s.device || (map_out && e.H * e.W == 0) || (mask_out && !map_out)) return TC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.stop) return TC_ERR_INVALID_ARG;
    const uint64_t t = s.next_ticket++;
    tc::Req& r = s.reqs[t];
    r.ticket = t;
    r.env = &e;
    r.target = *target;
    r.sigma = sigma_out;
    r.map = map_out;
    r.mask = mask_out;
    r.t_submit = Clock::now();
    s.queue.push_back(t);
    s.submitted++;
    e.busy.fetch_add(1);
    *ticket = t;
  }
  s.cv_work.notify_one();
  return TC_OK;
}

tc_status tc_poll(tc_server* h, uint64_t ticket, int32_t* done, tc_result* result) {
  if (!h || !done) return TC_ERR_INVALID_ARG;
  tc::Server& s = h->impl;
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.reqs.find(ticket);
  if (it == s.reqs.end()) return TC_ERR_INVALID_ARG;
  *done = it->second.state == 2;
  if (*done) {
    fill_result(it->second, result);
    s.reqs.erase(it);
  }
  return TC_OK;
}

tc_status tc_wait(tc_server* h, uint64_t ticket, int64_t timeout_us, tc_result* result) {
  if (!h || timeout_us < 0) return TC_ERR_INVALID_ARG;
  tc::Server& s = h->impl;
  std::unique_lock<std::mutex> lk(s.mu);
  auto it = s.reqs.find(ticket);
  if (it == s.reqs.end()) return TC_ERR_INVALID_ARG;
  tc::Req* r = &it->second;
  const bool ok = s.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->state == 2; });
  if (!ok) return TC_ERR_TIMEOUT;
  fill_result(*r, result);
  s.reqs.erase(ticket);
  return TC_OK;
}

tc_status tc_server_info(tc_server* h, tc_server_stats* out) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  tc::Server& s = h->impl;
  std::lock_guard<std::mutex> lk(s.mu);
  out->submitted = s.submitted;
  out->completed = s.completed;
  out->rounds = s.rounds.load();
  out->queued = (int32_t)s.queue.size();
  out->inflight = s.inflight;
  out->peak_inflight = s.peak_inflight;
  out->inflight_bytes = s.inflight_bytes;
  out->budget_bytes = s.budget;
  out->max_slots = s.max_slots;
  out->stream = (void*)s.stream;
  return TC_OK;
}

void tc_server_destroy(tc_server* h) {
  if (!h) return;
  tc::Server& s = h->impl;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.stop = true;
    // requests not yet admitted are cancelled; admitted ones run to the end
    for (uint64_t t : s.queue) {
      tc::Req& r = s.reqs.at(t);
      s.complete_locked(r, TC_ERR_ADMISSION);
      r.env->busy.fetch_sub(1);
    }
    s.queue.clear();
  }
  s.cv_work.notify_all();
  if (s.worker.joinable()) s.worker.join();
  s.cv_done.notify_all();
  cudaStreamSynchronize(s.stream);
  s.x32.release();
  s.x64.release();
  s.arena.release_all();
  cudaStreamSynchronize(s.stream);
  cudaStreamDestroy(s.stream);
  delete h;
}

}  // extern "C"
