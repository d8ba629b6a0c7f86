// Step server: continuous batching of tc_step requests from many envs.
//
// Callers submit (env, target pose, optional output buffers) from any thread
// and get a ticket back at once.  A pool of worker threads, each with its
// own CUDA stream and one round-based step scheduler per precision, drains a
// shared FIFO queue.  Before every round a worker admits queued requests
// while it has a free slot, the server has a free slot and the HBM budget
// allows (an env's footprint is the device memory its arena holds); then it
// runs one round -- every request it holds advances by one phase group, with
// one launch set per phase over all of them -- and finishes the requests that
// converged or failed: their stress and pressure map are written to the
// caller's buffers and their tickets complete.  A request that arrives while
// others are on the GPU joins at the next round boundary of a worker with
// room.  Workers run independently, so an env that needs many Newton or CG
// iterations delays only the requests batched with it, and the streams of
// different workers overlap on the device.  Env state (positions,
// velocities, candidate lists, PCG vectors) stays resident in the env
// between requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <memory>
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

struct Server;

struct Worker {
  Server* srv = nullptr;
  int id = 0;
  cudaStream_t stream = nullptr;
  Arena arena;
  BatchExec<float> x32;
  BatchExec<double> x64;
  StepScheduler<float> s32;
  StepScheduler<double> s64;
  int inflight = 0;  // guarded by the server mutex
  std::thread th;
  void run();
};

struct Server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  int slots_per_worker = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;  // node-based: element addresses are stable
  int inflight = 0, peak_inflight = 0;
  // working sets metered against the budget: every env ever submitted here
  // (until destroyed) and the bytes of those whose working set is resident
  std::vector<Env*> known;
  size_t inflight_bytes = 0;  // resident working-set bytes of the known envs
  uint64_t tick = 0;
  int64_t evictions = 0;
  int64_t submitted = 0, completed = 0;
  uint64_t gen = 0;  // bumped whenever a request arrives or capacity frees up
  std::atomic<int64_t> rounds{0};
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::unique_ptr<Worker>> workers;

  void admit_locked(Worker& w, std::vector<Req*>& out);
  void complete_locked(Req& r, tc_status st);
  void make_room_locked(size_t need, const Env* keep);
  void forget_locked(Env* e);
};

void Server::forget_locked(Env* e) {
  for (size_t i = 0; i < known.size(); ++i)
    if (known[i] == e) {
      if (e->work_resident) inflight_bytes -= std::min(inflight_bytes, e->work_bytes);
      known[i] = known.back();
      known.pop_back();
      break;
    }
  e->server = nullptr;
}

// Release the working sets of known envs with no request in flight, least
// recently used first, until `need` more bytes fit the budget.  An env whose
// API lock is held by a caller right now is skipped.
void Server::make_room_locked(size_t need, const Env* keep) {
  std::vector<Env*> cand;
  for (Env* e : known)
    if (e != keep && e->work_resident && !e->in_flight.load()) cand.push_back(e);
  std::sort(cand.begin(), cand.end(), [](const Env* a, const Env* b) { return a->server_tick < b->server_tick; });
  for (Env* e : cand) {
    if (inflight_bytes + need <= budget) break;
    if (!e->api_mu.try_lock()) continue;
    if (e->work_resident && !e->in_flight.load()) {
      cudaStreamSynchronize(e->stream);
      release_working(*e);
      inflight_bytes -= std::min(inflight_bytes, e->work_bytes);
      evictions++;
    }
    e->api_mu.unlock();
  }
}

void Server::complete_locked(Req& r, tc_status st) {
  r.status = st;
  r.state = 2;
  r.t_done = Clock::now();
  completed++;
}

// FIFO admission into worker w: a request waits while an earlier request of
// its env is in flight; the queue head waits for a free slot (the worker's
// and the server's) and for its footprint to fit the budget, except that a
// lone request always runs.
void Server::admit_locked(Worker& w, std::vector<Req*>& out) {
  for (auto it = queue.begin(); it != queue.end();) {
    Req& r = reqs.at(*it);
    if (r.env->in_flight.load()) {
      ++it;
      continue;
    }
    Env* e = r.env;
    if (e->server != this && e->server == nullptr) {  // first request of this env: meter its working set
      e->server = this;
      known.push_back(e);
      if (e->work_resident) inflight_bytes += e->work_bytes;
    }
    r.bytes = e->work_resident ? 0 : e->work_bytes;
    if (e->work_bytes > budget) {  // can never fit
      complete_locked(r, TC_ERR_ADMISSION);
      r.env->busy.fetch_sub(1);
      it = queue.erase(it);
      continue;
    }
    if (w.inflight >= slots_per_worker) break;
    if (inflight_bytes + r.bytes > budget) make_room_locked(r.bytes, e);
    const bool fits = inflight < max_slots && inflight_bytes + r.bytes <= budget;
    if (!fits && inflight > 0) break;
    e->server_tick = ++tick;
    r.state = 1;
    r.t_admit = Clock::now();
    r.env->in_flight.store(1);
    inflight++;
    w.inflight++;
    inflight_bytes += r.bytes;
    peak_inflight = std::max(peak_inflight, inflight);
    out.push_back(&r);
    it = queue.erase(it);
  }
}

// Stress and pressure maps of the requests a round finished, all of one
// precision, in one batched extraction launch on the worker's stream.
template <class R> static tc_status extract(const std::vector<Req*>& reqs, cudaStream_t s) {
  if (reqs.empty()) return TC_OK;
  std::vector<Env*> envs;
  std::vector<float*> sig, map;
  std::vector<uint8_t*> mask;
  for (Req* r : reqs) {
    envs.push_back(r->env);
    sig.push_back(r->sigma);
    map.push_back(r->map);
    mask.push_back(r->mask);
  }
  return extract_batch<R>(envs, sig, map, mask, s);
}

void Worker::run() {
  Server& S = *srv;
  cudaSetDevice(S.device);
  std::vector<Req*> live;
  std::vector<StepDone> fin;
  for (;;) {
    std::vector<Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(S.mu);
      for (;;) {
        if (!S.stop) S.admit_locked(*this, admitted);
        if (inflight > 0) break;
        if (S.stop) return;
        const uint64_t seen = S.gen;
        S.cv_work.wait(lk, [&] { return S.stop || S.gen != seen; });
      }
    }
    S.cv_done.notify_all();  // admission may have completed requests that can never fit
    // the env's earlier work (creation, extraction by the caller) is ordered
    // before its first launch on this worker's stream
    std::vector<std::pair<Req*, tc_status>> refused;
    for (Req* r : admitted) {
      // the working set of the env (released earlier to make room for others)
      tc_status ws;
      {
        std::lock_guard<std::mutex> g(r->env->api_mu);
        ws = acquire_working(*r->env);
      }
      if (ws != TC_OK) {
        refused.push_back({r, ws});
        continue;
      }
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
      std::fprintf(stderr, "[tc] worker %d round: %zu in flight, %zu admitted, %zu finished, %.3f ms\n", id,
                   live.size(), admitted.size(), fin.size(),
                   std::chrono::duration<double, std::milli>(Clock::now() - t_round).count());
    for (Req* r : live) r->rounds++;
    S.rounds++;
    std::vector<std::pair<Req*, tc_status>> done(refused);
    if (st != TC_OK) {
      // a launch or copy failed: every request this worker holds ends with that status
      s32.tasks.clear();
      s64.tasks.clear();
      for (Req* r : live) done.push_back({r, st});
    } else {
      std::vector<Req*> x32, x64;
      for (const StepDone& d : fin) {
        Req* r = nullptr;
        for (Req* q : live)
          if (q->ticket == d.tag) r = q;
        if (!r) continue;
        if (d.status == TC_OK && (r->sigma || r->map)) (r->env->precision == TC_FP64 ? x64 : x32).push_back(r);
        done.push_back({r, d.status});
      }
      // the requests finished in this round are extracted together
      const tc_status xs32 = extract<float>(x32, stream), xs64 = extract<double>(x64, stream);
      for (auto& d : done) {
        if (d.second != TC_OK || !(d.first->sigma || d.first->map)) continue;
        const tc_status xs = d.first->env->precision == TC_FP64 ? xs64 : xs32;
        if (xs != TC_OK) d.second = xs;
      }
      if (!done.empty() && cudaStreamSynchronize(stream) != cudaSuccess)
        for (auto& d : done) d.second = TC_ERR_CUDA;
    }
    if (done.empty()) continue;
    {
      std::lock_guard<std::mutex> lk(S.mu);
      for (auto& d : done) {
        Req& r = *d.first;
        S.complete_locked(r, d.second);
        r.env->in_flight.store(0);
        r.env->busy.fetch_sub(1);
        S.inflight--;
        inflight--;
        // the working set stays resident (metered) until the server needs
        // the room for another env; one that could not be acquired is not
        if (!r.env->work_resident) S.inflight_bytes -= std::min(S.inflight_bytes, r.bytes);
      }
      S.gen++;
    }
    if (!refused.empty()) S.cv_done.notify_all();
    std::vector<Req*> keep;
    for (Req* r : live) {
      bool fin_r = false;
      for (auto& d : done) fin_r = fin_r || d.first == r;
      if (!fin_r) keep.push_back(r);
    }
    live.swap(keep);
    S.cv_done.notify_all();
    S.cv_work.notify_all();  // freed capacity may let an idle worker admit
  }
}

void server_forget(Env& env) {
  Server* s = static_cast<Server*>(env.server);
  if (!s) return;
  std::lock_guard<std::mutex> lk(s->mu);
  s->forget_locked(&env);
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

static void stop_workers(tc::Server& s) {
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.stop = true;
  }
  s.cv_work.notify_all();
  for (auto& w : s.workers)
    if (w->th.joinable()) w->th.join();
  s.cv_done.notify_all();
  for (auto& w : s.workers) {
    if (!w->stream) continue;
    cudaStreamSynchronize(w->stream);
    w->x32.release();
    w->x64.release();
    w->arena.release_all();
    cudaStreamSynchronize(w->stream);
    cudaStreamDestroy(w->stream);
    w->stream = nullptr;
  }
}

extern "C" {

tc_status tc_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t workers, tc_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots <= 0) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  tc_server* h = new (std::nothrow) tc_server;
  if (!h) return TC_ERR_OOM;
  tc::Server& s = h->impl;
  if (cudaGetDevice(&s.device) != cudaSuccess) {
    delete h;
    return TC_ERR_CUDA;
  }
  const int nw = workers > 0 ? std::min(workers, max_slots) : max_slots;
  s.budget = hbm_budget_bytes;
  s.max_slots = max_slots;
  s.slots_per_worker = (max_slots + nw - 1) / nw;
  tc_status st = TC_OK;
  for (int i = 0; i < nw && st == TC_OK; ++i) {
    std::unique_ptr<tc::Worker> w(new (std::nothrow) tc::Worker());
    if (!w) {
      st = TC_ERR_OOM;
      break;
    }
    w->srv = &s;
    w->id = i;
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      st = TC_ERR_CUDA;
      break;
    }
    w->arena.stream = w->stream;
    w->x32.arena = &w->arena;
    w->x32.stream = w->stream;
    w->x64.arena = &w->arena;
    w->x64.stream = w->stream;
    w->s32.exec = &w->x32;
    w->s64.exec = &w->x64;
    s.workers.push_back(std::move(w));
  }
  if (st == TC_OK) {
    try {
      for (auto& w : s.workers) {
        tc::Worker* wp = w.get();
        w->th = std::thread([wp] { wp->run(); });
      }
    } catch (...) {
      st = TC_ERR_OOM;
    }
  }
  if (st != TC_OK) {
    stop_workers(s);
    delete h;
    return st;
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
    s.gen++;
    e.busy.fetch_add(1);
    *ticket = t;
  }
  s.cv_work.notify_all();
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
  out->max_slots = s.max_slots;
  out->workers = (int32_t)s.workers.size();
  out->inflight_bytes = s.inflight_bytes;
  out->budget_bytes = s.budget;
  out->evictions = s.evictions;
  out->known_envs = (int32_t)s.known.size();
  return TC_OK;
}

tc_status tc_server_stream(tc_server* h, int32_t worker, void** stream) {
  if (!h || !stream) return TC_ERR_INVALID_ARG;
  tc::Server& s = h->impl;
  if (worker < 0 || worker >= (int32_t)s.workers.size()) return TC_ERR_INVALID_ARG;
  *stream = (void*)s.workers[worker]->stream;
  return TC_OK;
}

void tc_server_destroy(tc_server* h) {
  if (!h) return;
  tc::Server& s = h->impl;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    // requests not yet admitted are cancelled; admitted ones run to the end
    for (uint64_t t : s.queue) {
      tc::Req& r = s.reqs.at(t);
      s.complete_locked(r, TC_ERR_ADMISSION);
      r.env->busy.fetch_sub(1);
    }
    s.queue.clear();
  }
  stop_workers(s);
  {
    std::lock_guard<std::mutex> lk(s.mu);
    for (tc::Env* e : s.known) e->server = nullptr;  // their working sets stay as they are
    s.known.clear();
  }
  delete h;
}

}  // extern "C"
