// Batched execution of the implicit step (Algorithm 2, physics line) over any
// number of envs.
//
// Each request (env, target pose) runs its own state machine -- step start,
// indenter advance (CCD-limited substep), Newton iteration (element + contact
// + assembly), PCG + CCD + first line-search trial, one halving per round,
// step end -- and every phase of a round is one set of launches over all
// requests currently in that phase, followed by one read of their scalars.
// Requests at different substeps or iterations share launches; a request that
// converges leaves at the end of its round and a new one can join at the start
// of the next (continuous batching).  A single-env call is a batch of one.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "prof.cuh"
#include "solver.cuh"

namespace tc {

// smallest and largest forcing term of the inexact Newton solve in the mixed mode
constexpr double kEtaFloor32 = 0.1;
constexpr double kEtaCap32 = 0.1;
// forcing term of the verification solves in the mixed mode: a step that
// passes a convergence test with the loose forcing term is taken, and the
// substep only ends when a step solved to this tolerance passes it too.  A
// loosely solved step can be small while the iterate is far from the
// minimiser along soft directions (tangential sliding under a flat
// frictionless face: block-Jacobi PCG stopped at a 10 % residual leaves those
// modes nearly untouched, so Newton crawls along them with tiny steps).
// 1e-2 gave the same positions as 1e-3 on graded-pad box cases at 12 % fewer
// CG iterations, but left a soft-barrier case (pairs at ~3e-3 dhat) 10x
// outside the position tolerance, which 1e-3 meets.
constexpr double kEtaTight32 = 1e-3;
// continuation of an accepted full step: taken when the energy fell by more
// than kExtendRatio times the model's predicted decrease, to at most
// kExtendMax times the step
constexpr double kExtendRatio = 1.2;
// start each dynamic substep's Newton solve from the CCD-bounded inertial
// prediction of the gel instead of the previous substep's solution
constexpr bool kPredict = true;
constexpr double kExtendMax = 8.0;

#define TC_CHECK(x)                                 \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return TC_ERR_CUDA;      \
  } while (0)

// TACAUCHY_TRACE=1 prints one line per env and Newton iteration to stderr.
bool trace_on() {
  static const bool on = [] {
    const char* v = std::getenv("TACAUCHY_TRACE");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

void pose_interp(const tc_pose& a, const tc_pose& b, double s, tc_pose* out) {
  for (int k = 0; k < 3; ++k) out->t[k] = (1.0 - s) * a.t[k] + s * b.t[k];
  bool same = true;
  for (int k = 0; k < 9; ++k) same = same && a.R[k] == b.R[k];
  if (same || s <= 0.0 || s >= 1.0) {
    std::memcpy(out->R, s >= 1.0 ? b.R : a.R, sizeof(out->R));
    return;
  }
  // geodesic interpolation R(s) = Ra exp(s log(Ra^T Rb)) via axis-angle
  double M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += a.R[3 * k + i] * b.R[3 * k + j];
      M[3 * i + j] = acc;
    }
  const double c = std::max(-1.0, std::min(1.0, 0.5 * (M[0] + M[4] + M[8] - 1.0)));
  const double th = std::acos(c);
  double ax[3] = {M[7] - M[5], M[2] - M[6], M[3] - M[1]};
  const double n = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
  if (n < 1e-15) {
    std::memcpy(out->R, a.R, sizeof(out->R));
    return;
  }
  for (double& v : ax) v /= n;
  const double ts = s * th, cs = std::cos(ts), sn = std::sin(ts), C = 1 - cs;
  const double x = ax[0], y = ax[1], z = ax[2];
  const double Rr[9] = {cs + x * x * C, x * y * C - z * sn, x * z * C + y * sn, y * x * C + z * sn, cs + y * y * C,
                        y * z * C - x * sn, z * x * C - y * sn, z * y * C + x * sn, cs + z * z * C};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += a.R[3 * i + k] * Rr[3 * k + j];
      out->R[3 * i + j] = acc;
    }
}

// ------------------------------------------------------------ executor

bool graphs_on() {
  static const bool on = [] {
    const char* v = std::getenv("TACAUCHY_GRAPHS");
    return !(v && v[0] == '0');
  }();
  return on;
}

template <class R> BatchExec<R>::~BatchExec() { release(); }

template <class R> void BatchExec<R>::drop_graphs() {
  for (auto& g : graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  graphs.clear();
  ++gen;
}

template <class R> void BatchExec<R>::release() {
  drop_graphs();
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
  if (arena) {
    arena->put(d_views);
    arena->put(d_prefix);
    arena->put(d_part);
    arena->put(d_param);
    arena->put(d_motion);
    arena->put(d_sc);
  }
  d_views = nullptr;
  d_prefix = nullptr;
  d_part = nullptr;
  d_param = nullptr;
  d_motion = nullptr;
  d_sc = nullptr;
  if (h_views) cudaFreeHost(h_views);
  if (h_prefix) cudaFreeHost(h_prefix);
  if (h_param) cudaFreeHost(h_param);
  if (h_motion) cudaFreeHost(h_motion);
  if (h_sc) cudaFreeHost(h_sc);
  h_views = nullptr;
  h_prefix = nullptr;
  h_param = nullptr;
  h_motion = nullptr;
  h_sc = nullptr;
  cap_env = 0;
  cap_part = 0;
}

template <class R> tc_status BatchExec<R>::reserve(int nenv, int64_t part) {
  if (nenv > cap_env || part > cap_part) drop_graphs();  // the tables move
  if (nenv > cap_env) {
    const int cap = std::max(nenv, 2 * cap_env);
    arena->put(d_views);
    arena->put(d_prefix);
    arena->put(d_param);
    arena->put(d_motion);
    arena->put(d_sc);
    if (h_views) cudaFreeHost(h_views);
    if (h_prefix) cudaFreeHost(h_prefix);
    if (h_param) cudaFreeHost(h_param);
    if (h_motion) cudaFreeHost(h_motion);
    if (h_sc) cudaFreeHost(h_sc);
    d_views = arena->alloc<EnvView<R>>(cap);
    d_prefix = arena->alloc<int>((int64_t)K_NKIND * (cap + 1));
    d_param = arena->alloc<double>(cap);
    d_motion = arena->alloc<Motion>(cap);
    d_sc = arena->alloc<Scalars>(cap);
    if (!d_views || !d_prefix || !d_param || !d_motion || !d_sc) return TC_ERR_OOM;
    if (cudaMallocHost(&h_views, sizeof(EnvView<R>) * cap) != cudaSuccess ||
        cudaMallocHost(&h_prefix, sizeof(int) * K_NKIND * (cap + 1)) != cudaSuccess ||
        cudaMallocHost(&h_param, sizeof(double) * cap) != cudaSuccess ||
        cudaMallocHost(&h_motion, sizeof(Motion) * cap) != cudaSuccess ||
        cudaMallocHost(&h_sc, sizeof(Scalars) * cap) != cudaSuccess)
      return TC_ERR_OOM;
    cap_env = cap;
  }
  if (part > cap_part) {
    const int64_t cap = std::max(part, 2 * cap_part);
    arena->put(d_part);
    d_part = arena->alloc<double>(cap);
    if (!d_part) return TC_ERR_OOM;
    cap_part = cap;
  }
  return TC_OK;
}

static int64_t units_of(const Env& e, int kind) {
  switch (kind) {
    case K_TET: return units_for(e.nt, K_TET);
    case K_VERT: return units_for(e.nv, K_VERT);
    case K_VGRP: return units_for(e.nv, K_VGRP);
    case K_CV: return units_for(e.nvc, K_CV);
    case K_CE: return units_for(e.nec, K_CE);
    default: return units_for(e.nfc, K_CF);
  }
}

template <class R>
tc_status BatchExec<R>::build(const std::vector<Env*>& set, const double* params, const Motion* motions) {
  const int n = (int)set.size();
  int64_t tot[K_NKIND];
  for (int k = 0; k < K_NKIND; ++k) tot[k] = 0;
  for (int k = 0; k < K_NKIND; ++k)
    for (int i = 0; i < n; ++i) tot[k] += units_of(*set[i], k);
  PartLayout L{};
  int64_t off = 0;
  auto take = [&](int64_t cnt) {
    const int64_t o = off;
    off += (cnt + 31) & ~int64_t(31);
    return o;
  };
  L.elem = take(tot[K_TET]);
  for (int k = 0; k < 3; ++k) L.cont[k] = take(2 * tot[K_CV + k]);
  L.asmb = take(2 * tot[K_VGRP]);
  L.inert = take(tot[K_VERT]);
  for (int k = 0; k < 3; ++k) L.ccd[k] = take(tot[K_CV + k]);
  L.rz = take(tot[K_VERT]);
  L.rr = take(tot[K_VERT]);
  L.env_s = take(8 * (int64_t)n);
  L.total = off;
  // the staging buffers below may still feed the previous phase's copies
  TC_CHECK(cudaStreamSynchronize(stream));
  tc_status st = reserve(n, L.total);
  if (st != TC_OK) return st;
  for (int k = 0; k < K_NKIND; ++k) {
    int acc = 0;
    for (int i = 0; i < n; ++i) {
      h_prefix[k * (n + 1) + i] = acc;
      acc += (int)units_of(*set[i], k);
    }
    h_prefix[k * (n + 1) + n] = acc;
  }
  for (int i = 0; i < n; ++i) {
    h_views[i] = set[i]->template view<R>();
    h_views[i].sc = d_sc + i;
    if (params) h_param[i] = params[i];
    if (motions) h_motion[i] = motions[i];
  }
  TC_CHECK(cudaMemcpyAsync(d_views, h_views, sizeof(EnvView<R>) * n, cudaMemcpyHostToDevice, stream));
  TC_CHECK(cudaMemcpyAsync(d_prefix, h_prefix, sizeof(int) * K_NKIND * (n + 1), cudaMemcpyHostToDevice, stream));
  if (params) TC_CHECK(cudaMemcpyAsync(d_param, h_param, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
  if (motions) TC_CHECK(cudaMemcpyAsync(d_motion, h_motion, sizeof(Motion) * n, cudaMemcpyHostToDevice, stream));
  TC_CHECK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * n, stream));
  host.nenv = n;
  for (int k = 0; k < K_NKIND; ++k) host.units[k] = (int)tot[k];
  host.bv.views = d_views;
  host.bv.nenv = n;
  host.bv.prefix = d_prefix;
  host.bv.part = d_part;
  host.bv.param = params ? d_param : nullptr;
  host.bv.motion = motions ? d_motion : nullptr;
  host.L = L;
  members = set;
  return TC_OK;
}

template <class R> tc_status BatchExec<R>::read() {
  const int n = host.nenv;
  TC_CHECK(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars) * n, cudaMemcpyDeviceToHost, stream));
  TC_CHECK(cudaStreamSynchronize(stream));
  TC_CHECK(cudaGetLastError());
  if (g_prof) g_prof->collect();
  return TC_OK;
}

// (Re)allocate an env's candidate lists for `cap` entries per gel primitive.
tc_status alloc_candidates(Env& env, int cap) {
  Arena& a = env.arena;
  const int n[3] = {env.nvc, env.nec, env.nfc};
  for (int k = 0; k < 3; ++k) {
    a.put(env.cand[k]);
    a.put(env.cand_n[k]);
    env.cand[k] = a.alloc<int32_t>((int64_t)cap * std::max(n[k], 1));
    env.cand_n[k] = a.alloc<int32_t>(std::max(n[k], 1));
    if (!env.cand[k] || !env.cand_n[k]) return TC_ERR_OOM;
    TC_CHECK(cudaMemsetAsync(env.cand_n[k], 0, sizeof(int32_t) * std::max(n[k], 1), env.stream));
  }
  env.cand_cap = cap;
  env.cand_valid = false;
  return TC_OK;
}

// Lagged-friction pair arrays sized for the current candidate capacity (the
// lagged pairs of a primitive are among its candidates).  Call with the
// batch stream idle.
template <class R> static tc_status ensure_friction(Env& env, cudaStream_t batch_stream) {
  if (!env.friction || (env.fr_cap == env.cand_cap && env.fr_n[0])) return TC_OK;
  Arena& a = env.arena;
  const int n[3] = {env.nvc, env.nec, env.nfc};
  const int cap = env.cand_cap;
  for (int k = 0; k < 3; ++k) {
    a.put(env.fr_n[k]);
    a.put(env.fr_ip[k]);
    a.put(env.fr_val[k]);
    env.fr_n[k] = a.alloc<int32_t>(std::max(n[k], 1));
    env.fr_ip[k] = a.alloc<int32_t>((int64_t)cap * std::max(n[k], 1));
    env.fr_val[k] = a.alloc<R>((int64_t)8 * cap * std::max(n[k], 1));
    if (!env.fr_n[k] || !env.fr_ip[k] || !env.fr_val[k]) return TC_ERR_OOM;
    TC_CHECK(cudaMemsetAsync(env.fr_n[k], 0, sizeof(int32_t) * std::max(n[k], 1), env.stream));
  }
  env.fr_cap = cap;
  if (env.stream != batch_stream) TC_CHECK(cudaStreamSynchronize(env.stream));
  return TC_OK;
}

static Motion make_motion(const tc_pose& a, const tc_pose& b, int use_dir) {
  Motion m;
  std::memcpy(m.Ra, a.R, sizeof(m.Ra));
  std::memcpy(m.ta, a.t, sizeof(m.ta));
  std::memcpy(m.Rb, b.R, sizeof(m.Rb));
  std::memcpy(m.tb, b.t, sizeof(m.tb));
  for (int k = 0; k < 9; ++k) {
    m.Raf[k] = (float)m.Ra[k];
    m.Rbf[k] = (float)m.Rb[k];
  }
  for (int k = 0; k < 3; ++k) {
    m.taf[k] = (float)m.ta[k];
    m.tbf[k] = (float)m.tb[k];
  }
  m.use_dir = use_dir;
  return m;
}

// CCD pass (rebuilding the candidate lists) for the envs in `set` with the
// given motions, optionally followed by the first line-search trial and its
// energy.  Envs whose lists overflowed get larger lists and are redone.
// On return X holds the scalars of all of `set`, in order.
template <class R>
static tc_status ccd_phase(BatchExec<R>& X, const std::vector<Env*>& set, const std::vector<Motion>& mot, bool trial,
                           std::vector<Scalars>& out) {
  out.assign(set.size(), Scalars{});
  std::vector<int> todo(set.size());
  for (size_t i = 0; i < set.size(); ++i) todo[i] = (int)i;
  for (int attempt = 0; attempt < 16 && !todo.empty(); ++attempt) {
    std::vector<Env*> sub;
    std::vector<Motion> m;
    for (int i : todo) {
      sub.push_back(set[i]);
      m.push_back(mot[i]);
    }
    tc_status st = X.build(sub, nullptr, m.data());
    if (st != TC_OK) return st;
    st = X.launch(3, {trial ? 1 : 0}, [&]() -> tc_status {
      b_ccd<R>(X.host, X.stream);
      if (trial) {
        b_trial<R>(X.host, X.stream);
        b_trial_energy<R>(X.host, X.stream);
      }
      return TC_OK;
    });
    if (st != TC_OK) return st;
    if ((st = X.read()) != TC_OK) return st;
    std::vector<int> again;
    for (size_t j = 0; j < todo.size(); ++j) {
      Env& e = *sub[j];
      const Scalars& sc = X.h_sc[j];
      if (sc.overflow > e.cand_cap) {
        int cap = e.cand_cap;
        while (cap < sc.overflow) cap *= 2;
        if ((st = alloc_candidates(e, cap)) != TC_OK) return st;
        // the new lists come from the env's own stream
        if (e.stream != X.stream) TC_CHECK(cudaStreamSynchronize(e.stream));
        again.push_back(todo[j]);
      } else {
        e.cand_valid = true;
        out[todo[j]] = sc;
      }
    }
    todo.swap(again);
  }
  return todo.empty() ? TC_OK : TC_ERR_CAPACITY;
}

// Candidate lists for the current state of every env that has none.
template <class R> tc_status ensure_candidates(BatchExec<R>& X, const std::vector<Env*>& envs) {
  std::vector<Env*> need;
  std::vector<Motion> mot;
  for (Env* e : envs)
    if (!e->cand_valid) {
      need.push_back(e);
      mot.push_back(make_motion(e->pose, e->pose, 0));
    }
  if (need.empty()) return TC_OK;
  std::vector<Scalars> out;
  return ccd_phase<R>(X, need, mot, false, out);
}

// ---------------------------------------------------------- step driver

template <class R> void StepScheduler<R>::admit(Env* env, const tc_pose& target, uint64_t tag) {
  StepCtl c;
  c.env = env;
  c.target = target;
  c.tag = tag;
  c.phase = StepCtl::START;
  tasks.push_back(c);
}

template <class R> tc_status StepScheduler<R>::round(std::vector<StepDone>& finished) {
  BatchExec<R>& X = *exec;
  tc_status st = TC_OK;
  auto pick = [&](StepCtl::Phase ph) {
    std::vector<int> ids;
    for (int i = 0; i < (int)tasks.size(); ++i)
      if (tasks[i].phase == ph) ids.push_back(i);
    return ids;
  };
  auto finish_substep = [&](StepCtl& c) {
    c.env->stats.substeps++;
    c.phase = c.s >= 1.0 ? StepCtl::DONE : StepCtl::ADVANCE;
  };
  auto fail = [&](StepCtl& c, tc_status code) {
    c.phase = StepCtl::FAILED;
    c.status = code;
  };
  // ---- step start: u0 = u, u_tilde = u + h v
  std::vector<int> S = pick(StepCtl::START);
  if (!S.empty()) {
    std::vector<Env*> set;
    for (int i : S) set.push_back(tasks[i].env);
    if ((st = X.build(set, nullptr, nullptr)) != TC_OK) return st;
    b_step_vectors<R>(X.host, 0, X.stream);
    for (int i : S) {
      tasks[i].pose0 = tasks[i].env->pose;
      tasks[i].env->pose_start = tasks[i].env->pose;
      tasks[i].phase = StepCtl::ADVANCE;
    }
  }
  // ---- indenter advance (CCD-limited substep)
  std::vector<int> A = pick(StepCtl::ADVANCE);
  if (!A.empty()) {
    std::vector<Env*> set;
    std::vector<Motion> mot;
    std::vector<int> live;
    for (int i : A) {
      StepCtl& c = tasks[i];
      if (c.sub >= 256) {
        fail(c, TC_ERR_NEWTON_MAXITER);
        continue;
      }
      tc_pose ps;
      pose_interp(c.pose0, c.target, c.s, &ps);
      c.env->pose = ps;
      set.push_back(c.env);
      mot.push_back(make_motion(ps, c.target, 0));
      live.push_back(i);
    }
    std::vector<Scalars> sc;
    if (!set.empty() && (st = ccd_phase<R>(X, set, mot, false, sc)) != TC_OK) return st;
    // lagged friction of the substep, at the converged state and the pose
    // before the advance (the candidate lists cover the advance's sweep)
    std::vector<Env*> fset;
    for (Env* e : set)
      if (e->friction) {
        if ((st = ensure_friction<R>(*e, X.stream)) != TC_OK) return st;
        fset.push_back(e);
      }
    if (!fset.empty()) {
      if ((st = X.build(fset, nullptr, nullptr)) != TC_OK) return st;
      b_friction_lag<R>(X.host, X.stream);
    }
    std::vector<Env*> pset;
    std::vector<double> pfac;
    std::vector<Motion> pmot;
    for (size_t j = 0; j < live.size(); ++j) {
      StepCtl& c = tasks[live[j]];
      const double frac = sc[j].ccd_t;
      const double s_old = c.s;
      c.s = frac >= 1.0 ? 1.0 : c.s + (1.0 - c.s) * frac;
      pose_interp(c.pose0, c.target, c.s, &c.env->pose);
      // inertial predictor (dynamic): the gel's start point for this
      // substep's solve moves by the substep's share of the inertial
      // increment dt v, as far as CCD against the advanced indenter allows
      if (kPredict && c.env->dynamic) {
        pset.push_back(c.env);
        pfac.push_back(c.s - s_old);
        pmot.push_back(make_motion(c.env->pose, c.env->pose, 1));
      }
      c.sub++;
      c.newton = 0;
      c.g0 = -1.0;
      c.tight = false;
      c.phase = StepCtl::NEWTON;
      if (trace_on())
        std::fprintf(stderr, "[tc] req %llu substep %d advance frac=%.6e s=%.9f\n", (unsigned long long)c.tag, c.sub,
                     frac, c.s);
    }
    if (!pset.empty()) {
      if ((st = X.build(pset, pfac.data(), nullptr)) != TC_OK) return st;
      b_step_vectors<R>(X.host, 2, X.stream);  // dx = f (utilde - u0)
      std::vector<Scalars> psc;
      if ((st = ccd_phase<R>(X, pset, pmot, true, psc)) != TC_OK) return st;
      for (size_t j = 0; j < pset.size(); ++j)
        if (!(psc[j].status & ST_NONFINITE) && psc[j].ccd_t > 0.0) {
          std::swap(pset[j]->u, pset[j]->utrial);  // the CCD pass's lists cover the moved state
        }
    }
  }
  // ---- Newton iteration: element + contact + assembly
  std::vector<int> N = pick(StepCtl::NEWTON);
  std::vector<int> P;
  std::vector<double> eta;
  if (!N.empty()) {
    std::vector<Env*> set;
    for (int i : N) set.push_back(tasks[i].env);
    if ((st = X.build(set, nullptr, nullptr)) != TC_OK) return st;
    st = X.launch(1, {}, [&]() -> tc_status {
      b_elem<R>(X.host, true, false, X.stream);
      b_contact<R>(X.host, true, false, X.stream);
      b_assemble<R>(X.host, X.stream);
      return TC_OK;
    });
    if (st != TC_OK) return st;
    if ((st = X.read()) != TC_OK) return st;
    for (size_t j = 0; j < N.size(); ++j) {
      StepCtl& c = tasks[N[j]];
      Env& e = *c.env;
      const Scalars& sc = X.h_sc[j];
      const double gn = std::sqrt(sc.gnorm2);
      if ((sc.status & ST_NONFINITE) || !std::isfinite(gn) || !std::isfinite(sc.energy)) {
        fail(c, TC_ERR_NONFINITE);
        continue;
      }
      c.E0 = sc.energy;
      if (c.g0 < 0) c.g0 = gn;
      e.stats.newton++;
      if (gn <= std::max(e.rtol * c.g0, e.gabs)) {
        finish_substep(c);
        continue;
      }
      if (c.newton >= e.newton_max) {
        fail(c, TC_ERR_NEWTON_MAXITER);
        continue;
      }
      // forcing term of the inexact Newton solve: min(0.5, sqrt(|g| / |g0|))
      // in FP64; 0.1 throughout in the mixed mode.  There the solve ends on
      // the step test (|dx|_inf <= ptol): near the solution each Newton step
      // then cuts the error at least tenfold, so the step that passes the
      // test leaves an error of ~0.1 ptol, while a tighter floor only
      // multiplies the CG iterations of the last Newton iterations, and a
      // looser start (0.5) spends extra Newton iterations on nearly
      // steepest-descent steps.
      double et = std::min(e.precision == TC_FP64 ? 0.5 : kEtaCap32, std::sqrt(gn / std::max(c.g0, 1e-300)));
      et = std::max(et, e.precision == TC_FP64 ? 1e-10 : kEtaFloor32);
      if (e.precision != TC_FP64 && c.tight) et = kEtaTight32;
      P.push_back(N[j]);
      eta.push_back(et * et * sc.gnorm2);  // squared PCG stopping tolerance (eta |g|)^2
    }
  }
  // ---- PCG, step bound, CCD along dx, first trial point and its energy
  if (!P.empty()) {
    std::vector<Env*> set;
    int pcg_max = 0;
    for (int i : P) {
      set.push_back(tasks[i].env);
      pcg_max = std::max(pcg_max, tasks[i].env->pcg_max);
    }
    // a substep's first solve warm-starts from the previous substep's first
    // solution (kept in dfirst, and replaced by this one); later solves from
    // the previous solve
    for (int i : P) tasks[i].env->warm_first = tasks[i].newton == 0;
    st = X.build(set, eta.data(), nullptr);
    for (int i : P) tasks[i].env->warm_first = false;
    if (st != TC_OK) return st;
    const PcgShape sh = pcg_shape<R>();
    st = X.launch(2, {pcg_max, sh.cs, sh.threads, sh.smem}, [&]() -> tc_status {
      const tc_status ps = b_pcg<R>(X.host, pcg_max, true, X.stream);
      b_pmax<R>(X.host, X.stream);
      return ps;
    });
    if (st != TC_OK) return st;
    for (int i : P)
      if (tasks[i].newton == 0) {
        Env& e = *tasks[i].env;
        TC_CHECK(cudaMemcpyAsync(e.dfirst, e.dx, sizeof(R) * 3 * (size_t)e.nv, cudaMemcpyDeviceToDevice, X.stream));
      }
    if ((st = X.read()) != TC_OK) return st;
    std::vector<Scalars> pre(X.h_sc, X.h_sc + set.size());
    std::vector<Motion> mot;
    for (int i : P) mot.push_back(make_motion(tasks[i].env->pose, tasks[i].env->pose, 1));
    std::vector<Scalars> sc;
    if ((st = ccd_phase<R>(X, set, mot, true, sc)) != TC_OK) return st;
    for (size_t j = 0; j < P.size(); ++j) {
      StepCtl& c = tasks[P[j]];
      Env& e = *c.env;
      e.stats.pcg += pre[j].pcg_iters;
      if (pre[j].pcg_capped) e.stats.pcg_capped++;
      if (pre[j].status & ST_NONFINITE) {
        fail(c, TC_ERR_NONFINITE);
        continue;
      }
      const double pmax = pre[j].pmax;
      c.pmax = pmax;
      const double decrement = -0.5 * pre[j].reduce_tmp[3];
      const double e_noise = (e.precision == TC_FP64 ? 1e-14 : 1e-7) * std::fabs(c.E0);
      const bool nonfinite = (sc[j].status & ST_NONFINITE) != 0;
      c.alpha = std::min(1.0, sc[j].ccd_t);
      const double Et = sc[j].energy;
      if (trace_on())
        std::fprintf(stderr, "[tc] req %llu newton %d E=%.17g pcg=%d pmax=%.3e dec=%.3e ccd=%.6f Etrial=%.17g\n",
                     (unsigned long long)c.tag, c.newton, c.E0, pre[j].pcg_iters, pmax, decrement, sc[j].ccd_t, Et);
      // converged: full step below ptol, or below 10 ptol with a predicted
      // decrease under the energy's rounding level -- take it without the
      // energy test
      // (every substep is verified: an unverified intermediate substep can
      // leave a close pair on the far side of the barrier's basin, from
      // which the next substep's minimiser differs)
      const bool loose = e.precision != TC_FP64 && !c.tight;
      if (pmax <= e.ptol || (pmax <= 10.0 * e.ptol && decrement <= e_noise)) {
        if (nonfinite) {
          fail(c, TC_ERR_NONFINITE);
          continue;
        }
        std::swap(e.u, e.utrial);
        if (loose) {  // take the step, then verify with a tightly solved one
          c.tight = true;
          c.newton++;
          c.phase = StepCtl::NEWTON;
          continue;
        }
        finish_substep(c);
        continue;
      }
      if (!nonfinite && std::isfinite(Et) && Et <= c.E0) {
        std::swap(e.u, e.utrial);
        c.newton++;
        c.phase = StepCtl::NEWTON;
        // rounding floor: the step is tiny and the energy did not move
        if (Et == c.E0 && pmax <= 10.0 * e.ptol) {
          if (loose) {
            c.tight = true;
            continue;
          }
          finish_substep(c);
          continue;
        }
        // continuation: a full step that lowered the energy clearly more than
        // the quadratic model predicted (model too stiff along dx -- the
        // Gauss-Newton contact blocks drop the barrier's negative curvature
        // term) goes on along dx to the minimiser of the parabola through
        // E0, the slope g.dx and E(1): alpha* = 1 / (2 - r), r = (E0 - E1) /
        // decrement, capped at kExtendMax
        const double dE = c.E0 - Et;
        if (c.alpha >= 1.0 && decrement > 0.0 && dE > 20.0 * e_noise) {
          const double r = dE / decrement;
          if (r > kExtendRatio) {
            const double astar = r >= 2.0 - 1.0 / kExtendMax ? kExtendMax : 1.0 / (2.0 - r);
            c.ext = astar - 1.0;
            c.E1 = Et;
            c.phase = StepCtl::EXTEND;
          }
        }
        continue;
      }
      c.alpha *= 0.5;
      c.halvings = 1;
      e.stats.halvings++;
      c.phase = StepCtl::LINESEARCH;
    }
  }
  // ---- one halving of every env in the line search
  // ---- continuation of accepted full steps along dx (CCD-bounded; kept
  // only if it lowers the energy further)
  std::vector<int> Ex = pick(StepCtl::EXTEND);
  if (!Ex.empty()) {
    std::vector<Env*> set;
    std::vector<double> fac;
    std::vector<Motion> mot;
    for (int i : Ex) {
      set.push_back(tasks[i].env);
      fac.push_back(tasks[i].ext);
      mot.push_back(make_motion(tasks[i].env->pose, tasks[i].env->pose, 1));
    }
    if ((st = X.build(set, fac.data(), nullptr)) != TC_OK) return st;
    b_scale_dx<R>(X.host, X.stream);
    std::vector<Scalars> sc;
    if ((st = ccd_phase<R>(X, set, mot, true, sc)) != TC_OK) return st;
    for (size_t j = 0; j < Ex.size(); ++j) {
      StepCtl& c = tasks[Ex[j]];
      Env& e = *c.env;
      const double Ee = sc[j].energy;
      const bool ok = !(sc[j].status & ST_NONFINITE) && std::isfinite(Ee) && Ee <= c.E1;
      if (ok) std::swap(e.u, e.utrial);
      if (trace_on())
        std::fprintf(stderr, "[tc] req %llu   continue x%.3f ccd=%.6f E=%.17g %s\n", (unsigned long long)c.tag,
                     1.0 + c.ext, sc[j].ccd_t, Ee, ok ? "kept" : "dropped");
      c.phase = StepCtl::NEWTON;
    }
  }
  std::vector<int> Ls = pick(StepCtl::LINESEARCH);
  if (!Ls.empty()) {
    std::vector<Env*> set;
    std::vector<double> al;
    for (int i : Ls) {
      set.push_back(tasks[i].env);
      al.push_back(tasks[i].alpha);
    }
    if ((st = X.build(set, al.data(), nullptr)) != TC_OK) return st;
    st = X.launch(4, {}, [&]() -> tc_status {
      b_trial<R>(X.host, X.stream);
      b_trial_energy<R>(X.host, X.stream);
      return TC_OK;
    });
    if (st != TC_OK) return st;
    if ((st = X.read()) != TC_OK) return st;
    for (size_t j = 0; j < Ls.size(); ++j) {
      StepCtl& c = tasks[Ls[j]];
      Env& e = *c.env;
      const Scalars& sc = X.h_sc[j];
      const double Et = sc.energy;
      if (!(sc.status & ST_NONFINITE) && std::isfinite(Et) && Et <= c.E0) {
        std::swap(e.u, e.utrial);
        c.newton++;
        c.phase = StepCtl::NEWTON;
        if (trace_on())
          std::fprintf(stderr, "[tc] req %llu   accepted alpha=%.6e\n", (unsigned long long)c.tag, c.alpha);
        // a short full step (within 10 ptol) that the energy could only
        // accept after halvings down to a move below ptol: the energy no
        // longer resolves the remaining decrease, so the substep ends here
        if (c.pmax <= 10.0 * e.ptol && c.alpha * c.pmax <= e.ptol) finish_substep(c);
        continue;
      }
      if (++c.halvings > 60) {
        fail(c, TC_ERR_LINESEARCH);
        continue;
      }
      c.alpha *= 0.5;
      e.stats.halvings++;
    }
  }
  // ---- step end: v = (u - u0) / h and the final pose for converged envs
  std::vector<int> D = pick(StepCtl::DONE);
  if (!D.empty()) {
    std::vector<Env*> set;
    for (int i : D) {
      StepCtl& c = tasks[i];
      c.env->pose = c.target;
      c.env->stats.steps++;
      set.push_back(c.env);
    }
    if ((st = X.build(set, nullptr, nullptr)) != TC_OK) return st;
    b_step_vectors<R>(X.host, 1, X.stream);
    TC_CHECK(cudaStreamSynchronize(X.stream));
  }
  // a failed step leaves its env as it was before the step: displacement of
  // the step start (kept in u0), indenter pose of the step start; the
  // velocity is only written by a completed step
  for (StepCtl& c : tasks)
    if (c.phase == StepCtl::FAILED) {
      Env& e = *c.env;
      TC_CHECK(cudaMemcpyAsync(e.u, e.ut, sizeof(R) * 3 * (size_t)e.nv, cudaMemcpyDeviceToDevice, X.stream));
      e.pose = c.pose0;
      e.cand_valid = false;
    }
  std::vector<StepCtl> keep;
  for (StepCtl& c : tasks) {
    if (c.phase == StepCtl::DONE) finished.push_back({c.tag, c.env, TC_OK});
    else if (c.phase == StepCtl::FAILED) finished.push_back({c.tag, c.env, c.status != TC_OK ? c.status : TC_ERR_NEWTON_MAXITER});
    else keep.push_back(c);
  }
  tasks.swap(keep);
  return TC_OK;
}

template <class R>
tc_status step_batch(BatchExec<R>& X, const std::vector<Env*>& envs, const std::vector<tc_pose>& targets,
                     std::vector<tc_status>& result) {
  const int n = (int)envs.size();
  result.assign(n, TC_ERR_NEWTON_MAXITER);
  StepScheduler<R> sched;
  sched.exec = &X;
  for (int i = 0; i < n; ++i) sched.admit(envs[i], targets[i], (uint64_t)i);
  std::vector<StepDone> fin;
  for (int guard = 0; guard < (1 << 22) && !sched.tasks.empty(); ++guard) {
    const tc_status st = sched.round(fin);
    if (st != TC_OK) return st;
  }
  for (const StepDone& d : fin) result[d.tag] = d.status;
  return TC_OK;
}

// Total energy and min pair distance at the current state (static candidate
// lists): used to reject a start pose that touches the gel.
template <class R> tc_status energy_at_state(BatchExec<R>& X, Env& env, Scalars* out) {
  std::vector<Env*> one{&env};
  tc_status st = ensure_candidates<R>(X, one);
  if (st != TC_OK) return st;
  const double zero = 0.0;
  if ((st = X.build(one, &zero, nullptr)) != TC_OK) return st;
  b_trial<R>(X.host, X.stream);  // ut = u + 0 dx
  b_trial_energy<R>(X.host, X.stream);
  if ((st = X.read()) != TC_OK) return st;
  *out = X.h_sc[0];
  return TC_OK;
}

template <class R> tc_status energy_gradient_at_state(BatchExec<R>& X, Env& env, double* E, double* grad) {
  std::vector<Env*> one{&env};
  tc_status st = ensure_candidates<R>(X, one);
  if (st != TC_OK) return st;
  if ((st = X.build(one, nullptr, nullptr)) != TC_OK) return st;
  b_elem<R>(X.host, true, false, X.stream);
  b_contact<R>(X.host, true, false, X.stream);
  b_assemble<R>(X.host, X.stream);
  if ((st = X.read()) != TC_OK) return st;
  if (X.h_sc[0].status & ST_NONFINITE) return TC_ERR_NONFINITE;
  if (E) *E = X.h_sc[0].energy;
  if (grad) {
    const int nv = env.nv;
    std::vector<R> g(3 * (size_t)nv);
    TC_CHECK(cudaMemcpyAsync(g.data(), env.g, sizeof(R) * 3 * nv, cudaMemcpyDeviceToHost, X.stream));
    TC_CHECK(cudaStreamSynchronize(X.stream));
    for (int v = 0; v < nv; ++v)
      for (int d = 0; d < 3; ++d) grad[3 * (size_t)v + d] = (double)g[(size_t)d * nv + v];
  }
  return TC_OK;
}

template <class R> tc_status contact_force_at_state(BatchExec<R>& X, Env& env, double* f) {
  std::vector<Env*> one{&env};
  tc_status st = ensure_candidates<R>(X, one);
  if (st != TC_OK) return st;
  if ((st = X.build(one, nullptr, nullptr)) != TC_OK) return st;
  b_contact<R>(X.host, true, false, X.stream);
  b_force<R>(X.host, X.stream);
  if ((st = X.read()) != TC_OK) return st;
  for (int d = 0; d < 3; ++d) f[d] = X.h_sc[0].force[d];
  return TC_OK;
}

template <class R>
tc_status autotune_pcg(BatchExec<R>& X, const std::vector<Env*>& envs, int mode, std::vector<PcgTune>& out) {
  out.clear();
  if (envs.empty()) return TC_OK;
  tc_status st = ensure_candidates<R>(X, envs);
  if (st != TC_OK) return st;
  // the current Newton systems: element + contact + assembly
  if ((st = X.build(envs, nullptr, nullptr)) != TC_OK) return st;
  b_elem<R>(X.host, true, false, X.stream);
  b_contact<R>(X.host, true, false, X.stream);
  b_assemble<R>(X.host, X.stream);
  if ((st = X.read()) != TC_OK) return st;
  std::vector<double> tol2(envs.size());
  int pcg_max = 0;
  for (size_t i = 0; i < envs.size(); ++i) {
    tol2[i] = 1e-6 * X.h_sc[i].gnorm2;  // a relative residual of 1e-3
    pcg_max = std::max(pcg_max, envs[i]->pcg_max);
  }
  const PcgShape keep = pcg_shape<R>();
  const int shapes[4][2] = {{16, 1024}, {8, 1024}, {16, 512}, {8, 512}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TC_ERR_CUDA;
  double best = 1e300;
  int best_k = -1;
  for (int k = 0; k < 4; ++k) {
    if (set_pcg_shape<R>(shapes[k][0], shapes[k][1]) != TC_OK) continue;
    const PcgShape sh = pcg_shape<R>();
    double us = 1e300;
    long long iters = 0;
    for (int rep = 0; rep < 3 && st == TC_OK; ++rep) {
      // mode 0: every env's solve alone, one after another (the latency of
      // one env's solve, as when requests run on their own workers);
      // mode 1: one launch over all envs (the throughput of a full batch)
      const size_t groups = mode == 0 ? envs.size() : 1;
      double ms_total = 0.0;
      long long it = 0;
      for (size_t gi = 0; gi < groups && st == TC_OK; ++gi) {
        std::vector<Env*> set = mode == 0 ? std::vector<Env*>{envs[gi]} : envs;
        std::vector<double> t2 = mode == 0 ? std::vector<double>{tol2[gi]} : tol2;
        if ((st = X.build(set, t2.data(), nullptr)) != TC_OK) break;
        cudaEventRecord(e0, X.stream);
        if ((st = b_pcg<R>(X.host, pcg_max, false, X.stream)) != TC_OK) break;
        cudaEventRecord(e1, X.stream);
        if ((st = X.read()) != TC_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_total += ms;
        for (size_t i = 0; i < set.size(); ++i) it += X.h_sc[i].pcg_iters;
      }
      if (it > 0 && rep > 0) us = std::min(us, 1e3 * ms_total / (double)it);
      iters = it;
    }
    if (st != TC_OK) break;
    out.push_back({sh.cs, sh.threads, sh.coresident, us, iters});
    if (us < best) {
      best = us;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TC_OK) {
    set_pcg_shape<R>(keep.cs, keep.threads);
    return st;
  }
  if (best_k >= 0) return set_pcg_shape<R>(shapes[best_k][0], shapes[best_k][1]);
  return set_pcg_shape<R>(keep.cs, keep.threads);
}

#define TC_INST(R)                                                                                              \
  template struct BatchExec<R>;                                                                                 \
  template tc_status ensure_candidates<R>(BatchExec<R>&, const std::vector<Env*>&);                             \
  template struct StepScheduler<R>;                                                                             \
  template tc_status step_batch<R>(BatchExec<R>&, const std::vector<Env*>&, const std::vector<tc_pose>&,        \
                                   std::vector<tc_status>&);                                                    \
  template tc_status energy_at_state<R>(BatchExec<R>&, Env&, Scalars*);                                         \
  template tc_status contact_force_at_state<R>(BatchExec<R>&, Env&, double*);                                \
  template tc_status energy_gradient_at_state<R>(BatchExec<R>&, Env&, double*, double*);                     \
  template tc_status autotune_pcg<R>(BatchExec<R>&, const std::vector<Env*>&, int, std::vector<PcgTune>&);
TC_INST(float)
TC_INST(double)
#undef TC_INST

}  // namespace tc
