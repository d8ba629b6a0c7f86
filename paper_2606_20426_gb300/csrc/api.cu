// C ABI (include/tacauchy.h): scene lifetime, steps, extraction, profiling.
//
// tc_step is a batch of one and tc_step_batch a batch of many; both run the
// implicit step of Algorithm 2 (physics line) through the batch executor,
// where every Newton phase is one launch over all envs taking part in it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "batch.cuh"
#include "env.cuh"
#include "solver.cuh"

namespace tc {

thread_local Profiler* g_prof = nullptr;

// Routes the launches of one API call to the env's profiler (if enabled).
struct ProfGuard {
  Profiler* saved;
  explicit ProfGuard(Env& env) : saved(g_prof) { g_prof = env.prof; }
  ~ProfGuard() { g_prof = saved; }
};

#define TC_CHECK(x)                                 \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return TC_ERR_CUDA;      \
  } while (0)

template <class R> static BatchExec<R>& exec_of(Env& env) { return *static_cast<BatchExec<R>*>(env.exec); }

static void destroy_exec(Env& env) {
  if (!env.exec) return;
  if (env.precision == TC_FP64) delete static_cast<BatchExec<double>*>(env.exec);
  else delete static_cast<BatchExec<float>*>(env.exec);
  env.exec = nullptr;
}

template <class R> static tc_status make_exec(Env& env) {
  auto* x = new (std::nothrow) BatchExec<R>();
  if (!x) return TC_ERR_OOM;
  x->arena = &env.arena;
  x->stream = env.stream;
  env.exec = x;
  return TC_OK;
}

template <class R> static tc_status do_step(Env& env, const tc_pose& target) {
  const tc_status ws = acquire_working(env);
  if (ws != TC_OK) return ws;
  std::vector<Env*> one{&env};
  std::vector<tc_pose> tg{target};
  std::vector<tc_status> res;
  tc_status st = step_batch<R>(exec_of<R>(env), one, tg, res);
  if (env.prof) env.prof->collect();
  return st != TC_OK ? st : res[0];
}

// Device state of an env in two parts.  The persistent part (positions,
// velocities, the step's start and inertial target, the PCG warm starts, the
// extraction scratch) lives as long as the env.  The working set -- the
// buffers a step fills and consumes (element stiffness blocks and gradient
// slots, the Newton matrix's values, gradient, block-Jacobi inverse, PCG
// vectors, line-search trial, contact slots and candidate lists) -- can be
// released between steps and acquired again; a step server does so to keep
// the working sets it holds within its HBM budget.
template <class R> static tc_status alloc_persistent(Env& env) {
  Arena& a = env.arena;
  const int64_t nv = env.nv;
  auto A = [&](void** p, int64_t n) {
    *p = a.alloc<R>(n);
    return *p != nullptr;
  };
  bool ok = A(&env.u, 3 * nv) && A(&env.ut, 3 * nv) && A(&env.dx, 3 * nv) && A(&env.dfirst, 3 * nv);
  if (ok && env.dynamic) ok = A(&env.vel, 3 * nv) && A(&env.utilde, 3 * nv);
  if (!ok) return TC_ERR_OOM;
  TC_CHECK(cudaMemsetAsync(env.u, 0, sizeof(R) * 3 * nv, env.stream));
  TC_CHECK(cudaMemsetAsync(env.dx, 0, sizeof(R) * 3 * nv, env.stream));
  TC_CHECK(cudaMemsetAsync(env.dfirst, 0, sizeof(R) * 3 * nv, env.stream));
  if (env.dynamic) {
    TC_CHECK(cudaMemsetAsync(env.vel, 0, sizeof(R) * 3 * nv, env.stream));
    TC_CHECK(cudaMemsetAsync(env.utilde, 0, sizeof(R) * 3 * nv, env.stream));
  }
  env.face_p = a.alloc<float>(std::max(env.nfc, 1));
  env.face_A = a.alloc<float>(std::max(env.nfc, 1));
  env.vert_p = a.alloc<float>(std::max(env.nvc, 1));
  if (!env.face_p || !env.face_A || !env.vert_p) return TC_ERR_OOM;
  return TC_OK;
}

template <class R> static tc_status alloc_working(Env& env) {
  if (env.work_resident) return TC_OK;
  Arena& a = env.arena;
  const int64_t nv = env.nv, nt = env.nt;
  const size_t before = a.bytes;
  auto A = [&](void** p, int64_t n) {
    *p = a.alloc<R>(n);
    return *p != nullptr;
  };
  bool ok = A(&env.utrial, 3 * nv) && A(&env.kblk, kblk_size(nt)) && A(&env.eslot, 12 * nt) &&
            A(&env.bsr_val, 9 * (int64_t)std::max(env.nsell, 1)) && A(&env.g, 3 * nv) && A(&env.Minv, 6 * nv) &&
            A(&env.r, 3 * nv) && A(&env.z, 3 * nv) && A(&env.p, 3 * nv) && A(&env.q, 3 * nv) && A(&env.p2, 3 * nv) &&
            A(&env.cv_slot, 9 * (int64_t)std::max(env.nvc, 1)) && A(&env.ce_slot, 27 * (int64_t)std::max(env.nec, 1)) &&
            A(&env.cf_slot, 54 * (int64_t)std::max(env.nfc, 1));
  tc_status st = ok ? alloc_candidates(env, std::max(env.cand_cap, 32)) : TC_ERR_OOM;
  if (st != TC_OK) {
    release_working(env);
    return st;
  }
  env.work_bytes = a.bytes - before;
  env.work_resident = true;
  return TC_OK;
}

// The API mutexes of several envs, taken in address order.
struct EnvLocks {
  std::vector<std::mutex*> m;
  explicit EnvLocks(const std::vector<Env*>& envs) {
    for (Env* e : envs) m.push_back(&e->api_mu);
    std::sort(m.begin(), m.end());
    for (std::mutex* x : m) x->lock();
  }
  ~EnvLocks() {
    for (auto it = m.rbegin(); it != m.rend(); ++it) (*it)->unlock();
  }
};

tc_status acquire_working(Env& env) {
  return env.precision == TC_FP64 ? alloc_working<double>(env) : alloc_working<float>(env);
}

void release_working(Env& env) {
  Arena& a = env.arena;
  void** bufs[] = {&env.utrial, &env.kblk, &env.eslot, &env.bsr_val, &env.g,  &env.Minv,    &env.r,
                   &env.z,      &env.p,    &env.q,     &env.p2,      &env.cv_slot, &env.ce_slot, &env.cf_slot};
  for (void** b : bufs) {
    a.put(*b);
    *b = nullptr;
  }
  for (int k = 0; k < 3; ++k) {
    a.put(env.cand[k]);
    a.put(env.cand_n[k]);
    env.cand[k] = nullptr;
    env.cand_n[k] = nullptr;
  }
  env.cand_valid = false;
  env.work_resident = false;
}

// Per-tet (mu, lam_hat) of a heterogeneous material (Eq. 1 per tet and the
// rest-stable lam_hat = lam + mu), uploaded as 2 x nt in the kernel type.
template <class R> static tc_status upload_material(Env& env, const double* E_nu) {
  const int64_t nt = env.nt;
  const bool lg = env.model == TC_MODEL_SNH_LOG;
  const int planes = lg ? 3 : 2;
  std::vector<R> h(planes * (size_t)nt);
  for (int64_t t = 0; t < nt; ++t) {
    const double E = E_nu[2 * t], nu = E_nu[2 * t + 1];
    const double mu = E / (2.0 * (1.0 + nu));
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    h[t] = (R)mu;
    h[nt + t] = (R)(lg ? lam + 5.0 / 6.0 * mu : lam + mu);
    if (lg) h[2 * nt + t] = (R)(mu / 3.0);
  }
  env.mat_tet = env.arena.alloc<R>(planes * nt);
  if (!env.mat_tet) return TC_ERR_OOM;
  TC_CHECK(cudaMemcpyAsync(env.mat_tet, h.data(), sizeof(R) * planes * nt, cudaMemcpyHostToDevice, env.stream));
  TC_CHECK(cudaStreamSynchronize(env.stream));
  return TC_OK;
}

template <class R> static tc_status initial_check(Env& env) {
  Scalars sc{};
  tc_status st = energy_at_state<R>(exec_of<R>(env), env, &sc);
  if (st != TC_OK) return st;
  if ((sc.status & ST_NONFINITE) || !(sc.reduce_tmp[1] > 0.0)) return TC_ERR_INITIAL_PENETRATION;
  int* flag = env.arena.alloc<int>(1);
  if (!flag) return TC_ERR_OOM;
  const int hit = intersect_test<R>(env.view<R>(), flag, env.stream);
  env.arena.put(flag);
  return hit ? TC_ERR_INITIAL_PENETRATION : TC_OK;
}

template <class R> static tc_status contact_force(Env& env, double* out) {
  const tc_status ws = acquire_working(env);
  if (ws != TC_OK) return ws;
  const tc_status st = contact_force_at_state<R>(exec_of<R>(env), env, out);
  if (env.prof) env.prof->collect();
  return st;
}

// Binning tables of `grid` (NULL: the grid given at create time), binned on
// first use and kept per env; the least recently used is dropped beyond
// Env::kGridCache grids.
static tc_status grid_table(Env& env, const tc_grid* grid, const int32_t** pf, const float** pw, int* npix) {
  if (!grid || (env.H * env.W > 0 && same_grid(*grid, env.grid0))) {
    if (env.H * env.W == 0) return TC_ERR_INVALID_ARG;
    *pf = env.pix_face;
    *pw = env.pix_w;
    *npix = env.H * env.W;
    return TC_OK;
  }
  if (!grid_valid(grid)) return TC_ERR_INVALID_ARG;
  const uint64_t now = ++env.grid_clock;
  for (auto& t : env.grid_tables)
    if (same_grid(t.key, *grid)) {
      t.last_use = now;
      *pf = t.pix_face;
      *pw = t.pix_w;
      *npix = grid->H * grid->W;
      return TC_OK;
    }
  if ((int)env.grid_tables.size() >= Env::kGridCache) {
    auto old = std::min_element(env.grid_tables.begin(), env.grid_tables.end(),
                                [](const Env::GridTable& a, const Env::GridTable& b) { return a.last_use < b.last_use; });
    if (cudaStreamSynchronize(env.stream) != cudaSuccess) return TC_ERR_CUDA;
    env.arena.put(old->pix_face);
    env.arena.put(old->pix_w);
    env.grid_tables.erase(old);
  }
  Env::GridTable t{*grid, nullptr, nullptr, now};
  const tc_status st = bin_pixel_grid(env, grid, &t.pix_face, &t.pix_w);
  if (st != TC_OK) return st;
  env.grid_tables.push_back(t);
  *pf = t.pix_face;
  *pw = t.pix_w;
  *npix = grid->H * grid->W;
  return TC_OK;
}

template <class R> static tc_status pressure_map(Env& env, const tc_grid* grid, float* out, uint8_t* mask) {
  const int32_t* pf = nullptr;
  const float* pw = nullptr;
  int npix = 0;
  const tc_status st = grid_table(env, grid, &pf, &pw, &npix);
  if (st != TC_OK) return st;
  EnvView<R> e = env.view<R>();
  launch_traction<R>(e, env.cparent, nullptr, nullptr, nullptr, env.face_p, env.face_A, env.stream);
  launch_vertex_avg(env.nvc, env.cv_face_off, env.cv_face_idx, env.face_p, env.face_A, env.vert_p, env.stream);
  launch_splat(npix, pf, pw, env.cface_slot, env.nfc, env.vert_p, out, mask, env.stream);
  TC_CHECK(cudaGetLastError());
  TC_CHECK(cudaStreamSynchronize(env.stream));
  if (env.prof) env.prof->collect();
  return TC_OK;
}

// Contact pass at the current state (fills the contact slots), then the
// per-vertex decomposition; with a grid, p goes to the env's vertex scratch
// and is splatted on that grid.
template <class R>
static tc_status vertex_forces(Env& env, float* f, float* fn, float* ft, float* p, const tc_grid* grid, bool map,
                               float* out, uint8_t* mask) {
  const int32_t* pf = nullptr;
  const float* pw = nullptr;
  int npix = 0;
  if (map) {
    const tc_status gs = grid_table(env, grid, &pf, &pw, &npix);
    if (gs != TC_OK) return gs;
  }
  double tot[3];
  tc_status st = acquire_working(env);
  if (st != TC_OK) return st;
  st = contact_force_at_state<R>(exec_of<R>(env), env, tot);
  if (st != TC_OK) return st;
  if (map) {
    launch_vertex_forces<R>(env.view<R>(), nullptr, nullptr, nullptr, env.vert_p, env.stream);
    launch_splat(npix, pf, pw, env.cface_slot, env.nfc, env.vert_p, out, mask, env.stream);
  } else {
    launch_vertex_forces<R>(env.view<R>(), f, fn, ft, p, env.stream);
  }
  TC_CHECK(cudaGetLastError());
  TC_CHECK(cudaStreamSynchronize(env.stream));
  if (env.prof) env.prof->collect();
  return TC_OK;
}

template <class R> static tc_status get_positions(Env& env, double* x) {
  const int nv = env.nv;
  std::vector<R> u(3 * (size_t)nv);
  std::vector<double> X(3 * (size_t)nv);
  TC_CHECK(cudaMemcpyAsync(u.data(), env.u, sizeof(R) * 3 * nv, cudaMemcpyDeviceToHost, env.stream));
  TC_CHECK(cudaMemcpyAsync(X.data(), env.X0, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost, env.stream));
  TC_CHECK(cudaStreamSynchronize(env.stream));
  for (int v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) x[3 * (size_t)v + d] = X[(size_t)d * nv + v] + (double)u[(size_t)d * nv + v];
  return TC_OK;
}

template <class R> static tc_status set_positions(Env& env, const double* x) {
  const int nv = env.nv;
  std::vector<R> u(3 * (size_t)nv);
  std::vector<double> X(3 * (size_t)nv);
  TC_CHECK(cudaMemcpyAsync(X.data(), env.X0, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost, env.stream));
  TC_CHECK(cudaStreamSynchronize(env.stream));
  for (int v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) u[(size_t)d * nv + v] = (R)(x[3 * (size_t)v + d] - X[(size_t)d * nv + v]);
  TC_CHECK(cudaMemcpyAsync(env.u, u.data(), sizeof(R) * 3 * nv, cudaMemcpyHostToDevice, env.stream));
  TC_CHECK(cudaStreamSynchronize(env.stream));
  env.cand_valid = false;
  return TC_OK;
}

}  // namespace tc

using tc::Env;

extern "C" {

const char* tc_status_str(tc_status s) {
  switch (s) {
    case TC_OK: return "ok";
    case TC_ERR_INVALID_ARG: return "invalid argument";
    case TC_ERR_INVALID_MESH: return "invalid mesh (non-positive tet or index out of range)";
    case TC_ERR_INITIAL_PENETRATION: return "indenter touches or intersects the gel";
    case TC_ERR_NEWTON_MAXITER: return "Newton iteration or substep cap reached";
    case TC_ERR_PCG_MAXITER: return "PCG iteration cap reached";
    case TC_ERR_LINESEARCH: return "line search found no decrease";
    case TC_ERR_NONFINITE: return "non-finite value";
    case TC_ERR_CUDA: return "CUDA runtime error";
    case TC_ERR_OOM: return "device allocation failed";
    case TC_ERR_ADMISSION: return "environment does not fit the memory budget";
    case TC_ERR_TIMEOUT: return "timed out";
    case TC_ERR_CAPACITY: return "capacity exceeded";
    default: return "unknown status";
  }
}

static bool pose_ok(const tc_pose* p) {
  if (!p) return false;
  for (double v : p->R)
    if (!std::isfinite(v)) return false;
  for (double v : p->t)
    if (!std::isfinite(v)) return false;
  return true;
}

tc_status tc_create_scene(const tc_mesh* mesh, const tc_material* material, const int32_t* fixed, int32_t nfixed,
                          const tc_trimesh* indenter, const tc_pose* start_pose, const tc_scene_opts* opts,
                          const tc_grid* grid, const tc_allocator* allocator, void* cuda_stream, tc_env** out) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !material || !indenter || !opts || !mesh->X || !mesh->tets || mesh->nv <= 0 || mesh->nt <= 0 ||
      nfixed < 0 || (nfixed > 0 && !fixed) || !indenter->V || !indenter->F || indenter->nv <= 0 ||
      indenter->nf <= 0)
    return TC_ERR_INVALID_ARG;
  if (!pose_ok(start_pose)) return TC_ERR_NONFINITE;
  if (mesh->nv >= (1 << 21)) return TC_ERR_INVALID_ARG;  // face keys pack three 21-bit ids
  if (!(material->E > 0) || !(material->nu > -1.0 && material->nu < 0.5) || !(opts->dhat > 0))
    return TC_ERR_INVALID_ARG;
  if (opts->precision != TC_FP64 && opts->precision != TC_FP32_MIXED) return TC_ERR_INVALID_ARG;
  if (material->model != TC_MODEL_SNH && material->model != TC_MODEL_SNH_LOG) return TC_ERR_INVALID_ARG;
  if (opts->dt > 0 && !(material->density > 0)) return TC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 4 * (int64_t)mesh->nt; ++i)
    if (mesh->tets[i] < 0 || mesh->tets[i] >= mesh->nv) return TC_ERR_INVALID_MESH;
  if (material->per_tet_E_nu)
    for (int64_t t = 0; t < mesh->nt; ++t) {
      const double E = material->per_tet_E_nu[2 * t], nu = material->per_tet_E_nu[2 * t + 1];
      if (!(E > 0) || !std::isfinite(E) || !(nu > -1.0 && nu < 0.5)) return TC_ERR_INVALID_ARG;
    }
  tc_env* h = new (std::nothrow) tc_env;
  if (!h) return TC_ERR_OOM;
  Env& env = h->impl;
  cudaGetDevice(&env.device);
  env.stream = (cudaStream_t)cuda_stream;
  env.arena.stream = env.stream;
  if (allocator && allocator->alloc && allocator->release) {
    env.arena.user = *allocator;
    env.arena.has_user = true;
  }
  env.precision = opts->precision;
  env.nv = mesh->nv;
  env.nt = mesh->nt;
  env.E = material->E;
  env.nu = material->nu;
  env.rho = material->density;
  env.mu = env.E / (2.0 * (1.0 + env.nu));                          // Eq. 1
  env.lam = env.E * env.nu / ((1.0 + env.nu) * (1.0 - 2.0 * env.nu));  // Eq. 1
  env.model = material->model;
  if (env.model == TC_MODEL_SNH_LOG) {
    // full stable Neo-Hookean as the rest-stable form with (mu, lam_hat) =
    // (3 mu_s / 4, lam_s) = (mu, lam + 5/6 mu) plus the log-term part with
    // coefficient mu_s / 4 = mu / 3
    env.lam_hat = env.lam + 5.0 / 6.0 * env.mu;
    env.kh = env.mu / 3.0;
  } else {
    env.lam_hat = env.lam + env.mu;
    env.kh = 0.0;
  }
  env.alpha = 1.0 + env.mu / env.lam_hat;
  env.dhat = opts->dhat;
  env.kappa = opts->kappa;
  env.dt = opts->dt;
  env.dynamic = opts->dt > 0;
  env.rtol = opts->newton_rtol > 0 ? opts->newton_rtol : 1e-6;
  env.newton_max = opts->newton_max > 0 ? opts->newton_max : 1024;
  env.pcg_max = opts->pcg_max > 0 ? opts->pcg_max : 1000;
  env.thick_axis = opts->contact_axis;
  if (!(opts->friction_mu >= 0.0) || !std::isfinite(opts->friction_mu)) {
    delete h;
    return TC_ERR_INVALID_ARG;
  }
  env.mu_f = opts->friction_mu;
  env.eps_v = opts->friction_eps_v > 0 && std::isfinite(opts->friction_eps_v) ? opts->friction_eps_v : 0.01;
  env.friction = env.dynamic && env.mu_f > 0.0;
  // Newton step tolerance: 1e-4 dhat in FP64; FP32 gradients carry rounding
  // noise of ~1e-5 of the contact force, whose Newton step is ~10 nm, so the
  // mixed mode stops at 1e-3 dhat.
  env.ptol = (env.precision == TC_FP64 ? 1e-4 : 1e-3) * env.dhat;
  env.pose = *start_pose;
  env.pose_start = *start_pose;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < mesh->nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], mesh->X[3 * (size_t)v + d]);
      hi[d] = std::max(hi[d], mesh->X[3 * (size_t)v + d]);
    }
  const double L2 = (hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) + (hi[2] - lo[2]) * (hi[2] - lo[2]);
  env.gabs = 1e-12 * env.E * L2;
  tc_status st = env.precision == TC_FP64 ? tc::make_exec<double>(env) : tc::make_exec<float>(env);
  if (st != TC_OK) {
    delete h;
    return st;
  }
  env.sc = env.arena.alloc<tc::Scalars>(1);
  if (!env.sc || cudaMallocHost(&env.sc_host, sizeof(tc::Scalars)) != cudaSuccess) st = TC_ERR_OOM;
  if (st == TC_OK && cudaMemsetAsync(env.sc, 0, sizeof(tc::Scalars), env.stream) != cudaSuccess) st = TC_ERR_CUDA;
  if (st == TC_OK) st = tc::setup_scene(env, mesh, fixed, nfixed, indenter, grid);
  if (st == TC_OK) st = tc::build_bsr(env, mesh->tets, fixed, nfixed);
  if (st == TC_OK)
    st = env.precision == TC_FP64 ? tc::alloc_persistent<double>(env) : tc::alloc_persistent<float>(env);
  if (st == TC_OK) st = tc::acquire_working(env);
  if (st == TC_OK && material->per_tet_E_nu)
    st = env.precision == TC_FP64 ? tc::upload_material<double>(env, material->per_tet_E_nu)
                                  : tc::upload_material<float>(env, material->per_tet_E_nu);
  if (st == TC_OK)
    st = env.precision == TC_FP64 ? tc::initial_check<double>(env) : tc::initial_check<float>(env);
  if (st == TC_OK && cudaStreamSynchronize(env.stream) != cudaSuccess) st = TC_ERR_CUDA;
  if (st != TC_OK) {
    tc_destroy(h);
    return st;
  }
  *out = h;
  return TC_OK;
}

tc_status tc_step(tc_env* h, const tc_pose* target) {
  if (!h || !target) return TC_ERR_INVALID_ARG;
  if (!pose_ok(target)) return TC_ERR_NONFINITE;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (env.busy.load()) return TC_ERR_INVALID_ARG;  // a server holds a request of this env
  tc::ProfGuard pg(env);
  tc_status st = env.precision == TC_FP64 ? tc::do_step<double>(env, *target) : tc::do_step<float>(env, *target);
  env.last_status = st;
  return st;
}

tc_status tc_step_batch(tc_env** envs, int32_t n, const tc_pose* targets, tc_status* statuses) {
  if (n < 0 || (n > 0 && (!envs || !targets || !statuses))) return TC_ERR_INVALID_ARG;
  if (n == 0) return TC_OK;
  for (int i = 0; i < n; ++i) {
    if (!envs[i] || envs[i]->impl.busy.load()) return TC_ERR_INVALID_ARG;
    if (envs[i]->impl.precision != envs[0]->impl.precision || envs[i]->impl.device != envs[0]->impl.device)
      return TC_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (envs[j] == envs[i]) return TC_ERR_INVALID_ARG;
  }
  std::vector<Env*> all;
  for (int i = 0; i < n; ++i) all.push_back(&envs[i]->impl);
  tc::EnvLocks locks(all);
  std::vector<Env*> set;
  std::vector<tc_pose> tg;
  std::vector<int> idx;
  for (int i = 0; i < n; ++i) {
    const tc_status ws = tc::acquire_working(envs[i]->impl);
    if (ws != TC_OK) return ws;
  }
  for (int i = 0; i < n; ++i) {
    if (!pose_ok(&targets[i])) {
      statuses[i] = TC_ERR_NONFINITE;
      continue;
    }
    set.push_back(&envs[i]->impl);
    tg.push_back(targets[i]);
    idx.push_back(i);
  }
  if (set.empty()) return TC_OK;
  Env& lead = *set[0];
  // every env's pending work must be complete before the lead stream runs
  for (Env* e : set)
    if (e->stream != lead.stream) cudaStreamSynchronize(e->stream);
  tc::ProfGuard pg(lead);
  std::vector<tc_status> res;
  tc_status st = lead.precision == TC_FP64 ? tc::step_batch<double>(tc::exec_of<double>(lead), set, tg, res)
                                           : tc::step_batch<float>(tc::exec_of<float>(lead), set, tg, res);
  if (st != TC_OK) return st;
  for (size_t k = 0; k < idx.size(); ++k) {
    statuses[idx[k]] = res[k];
    set[k]->last_status = res[k];
  }
  if (lead.prof) lead.prof->collect();
  return TC_OK;
}

tc_status tc_pcg_shape(int32_t precision, int32_t cluster_ctas, int32_t threads) {
  if (precision == TC_FP64) return tc::set_pcg_shape<double>(cluster_ctas, threads);
  if (precision == TC_FP32_MIXED) return tc::set_pcg_shape<float>(cluster_ctas, threads);
  return TC_ERR_INVALID_ARG;
}

tc_status tc_autotune_pcg(tc_env** envs, int32_t n, int32_t mode, tc_pcg_tune* results, int32_t max_results,
                          int32_t* n_results) {
  if (n <= 0 || !envs || (mode != 0 && mode != 1) || (max_results > 0 && !results)) return TC_ERR_INVALID_ARG;
  std::vector<Env*> set;
  for (int i = 0; i < n; ++i) {
    if (!envs[i] || envs[i]->impl.busy.load() || envs[i]->impl.precision != envs[0]->impl.precision ||
        envs[i]->impl.device != envs[0]->impl.device)
      return TC_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (envs[j] == envs[i]) return TC_ERR_INVALID_ARG;
    set.push_back(&envs[i]->impl);
  }
  tc::EnvLocks locks(set);
  for (Env* e : set) {
    const tc_status ws = tc::acquire_working(*e);
    if (ws != TC_OK) return ws;
  }
  Env& lead = *set[0];
  for (Env* e : set)
    if (e->stream != lead.stream) cudaStreamSynchronize(e->stream);
  tc::ProfGuard pg(lead);
  std::vector<tc::PcgTune> out;
  const tc_status st = lead.precision == TC_FP64
                           ? tc::autotune_pcg<double>(tc::exec_of<double>(lead), set, mode, out)
                           : tc::autotune_pcg<float>(tc::exec_of<float>(lead), set, mode, out);
  if (n_results) *n_results = (int32_t)out.size();
  for (int k = 0; k < (int)out.size() && k < max_results; ++k) {
    results[k].cluster_ctas = out[k].cs;
    results[k].threads = out[k].threads;
    results[k].coresident = out[k].coresident;
    results[k].us_per_env_iter = out[k].us_per_env_iter;
    results[k].env_iters = out[k].env_iters;
  }
  return st;
}

tc_status tc_stress(tc_env* h, float* sigma_out) {
  if (!h || !sigma_out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  tc::ProfGuard pg(env);
  if (env.precision == TC_FP64) tc::launch_stress<double>(env.view<double>(), sigma_out, env.stream);
  else tc::launch_stress<float>(env.view<float>(), sigma_out, env.stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(env.stream) != cudaSuccess) return TC_ERR_CUDA;
  if (env.prof) env.prof->collect();
  return TC_OK;
}

tc_status tc_traction(tc_env* h, float* t, float* p, float* t_tau) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  tc::ProfGuard pg(env);
  if (env.precision == TC_FP64)
    tc::launch_traction<double>(env.view<double>(), env.cparent, t, p, t_tau, nullptr, nullptr, env.stream);
  else
    tc::launch_traction<float>(env.view<float>(), env.cparent, t, p, t_tau, nullptr, nullptr, env.stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(env.stream) != cudaSuccess) return TC_ERR_CUDA;
  return TC_OK;
}

tc_status tc_pressure_map(tc_env* h, const tc_grid* grid, float* out, uint8_t* mask) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  tc::ProfGuard pg(env);
  return env.precision == TC_FP64 ? tc::pressure_map<double>(env, grid, out, mask)
                                  : tc::pressure_map<float>(env, grid, out, mask);
}

tc_status tc_extract_batch(tc_env** envs, int32_t n, float* const* sigma_out, float* const* map_out,
                           uint8_t* const* mask_out) {
  if (n < 0 || (n > 0 && !envs)) return TC_ERR_INVALID_ARG;
  if (n == 0) return TC_OK;
  std::vector<Env*> set;
  std::vector<float*> sig(n, nullptr), map(n, nullptr);
  std::vector<uint8_t*> mask(n, nullptr);
  for (int i = 0; i < n; ++i) {
    if (!envs[i] || envs[i]->impl.busy.load()) return TC_ERR_INVALID_ARG;
    Env& e = envs[i]->impl;
    if (e.precision != envs[0]->impl.precision || e.device != envs[0]->impl.device) return TC_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (envs[j] == envs[i]) return TC_ERR_INVALID_ARG;
    sig[i] = sigma_out ? sigma_out[i] : nullptr;
    map[i] = map_out ? map_out[i] : nullptr;
    mask[i] = mask_out ? mask_out[i] : nullptr;
    if (mask[i] && !map[i]) return TC_ERR_INVALID_ARG;
    if (map[i] && e.H * e.W == 0) return TC_ERR_INVALID_ARG;
    set.push_back(&e);
  }
  tc::EnvLocks locks(set);
  Env& lead = *set[0];
  for (Env* e : set)
    if (e->stream != lead.stream && cudaStreamSynchronize(e->stream) != cudaSuccess) return TC_ERR_CUDA;
  tc::ProfGuard pg(lead);
  const tc_status st = lead.precision == TC_FP64 ? tc::extract_batch<double>(set, sig, map, mask, lead.stream)
                                                 : tc::extract_batch<float>(set, sig, map, mask, lead.stream);
  if (lead.prof) lead.prof->collect();
  return st;
}

tc_status tc_contact_force(tc_env* h, double* out) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  tc::ProfGuard pg(env);
  return env.precision == TC_FP64 ? tc::contact_force<double>(env, out) : tc::contact_force<float>(env, out);
}

tc_status tc_depth_map(tc_env* h, const tc_grid* grid, float* height, uint8_t* mask) {
  if (!h || !height) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (grid && !tc::grid_valid(grid)) return TC_ERR_INVALID_ARG;
  if (!grid && env.H * env.W == 0) return TC_ERR_INVALID_ARG;
  const tc_grid& g = grid ? *grid : env.grid0;
  tc::ProfGuard pg(env);
  const tc_status st = env.precision == TC_FP64 ? tc::launch_depth_map<double>(env, g, height, mask, env.stream)
                                                : tc::launch_depth_map<float>(env, g, height, mask, env.stream);
  if (st != TC_OK) return st;
  if (cudaStreamSynchronize(env.stream) != cudaSuccess) return TC_ERR_CUDA;
  if (env.prof) env.prof->collect();
  return TC_OK;
}

tc_status tc_vertex_forces(tc_env* h, float* f, float* f_n, float* f_tau, float* p) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (env.busy.load()) return TC_ERR_INVALID_ARG;
  tc::ProfGuard pg(env);
  return env.precision == TC_FP64 ? tc::vertex_forces<double>(env, f, f_n, f_tau, p, nullptr, false, nullptr, nullptr)
                                  : tc::vertex_forces<float>(env, f, f_n, f_tau, p, nullptr, false, nullptr, nullptr);
}

tc_status tc_force_pressure_map(tc_env* h, const tc_grid* grid, float* out, uint8_t* mask) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (env.busy.load()) return TC_ERR_INVALID_ARG;
  tc::ProfGuard pg(env);
  return env.precision == TC_FP64 ? tc::vertex_forces<double>(env, nullptr, nullptr, nullptr, nullptr, grid, true, out, mask)
                                  : tc::vertex_forces<float>(env, nullptr, nullptr, nullptr, nullptr, grid, true, out, mask);
}

tc_status tc_energy_gradient(tc_env* h, double* energy, double* grad) {
  if (!h || (!energy && !grad)) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (env.busy.load()) return TC_ERR_INVALID_ARG;
  tc::ProfGuard pg(env);
  const tc_status ws = tc::acquire_working(env);
  if (ws != TC_OK) return ws;
  const tc_status st = env.precision == TC_FP64
                           ? tc::energy_gradient_at_state<double>(tc::exec_of<double>(env), env, energy, grad)
                           : tc::energy_gradient_at_state<float>(tc::exec_of<float>(env), env, energy, grad);
  if (env.prof) env.prof->collect();
  return st;
}

tc_status tc_surface_faces(tc_env* h, int32_t* faces, int32_t* parent) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  if (faces) std::memcpy(faces, env.h_cfaces.data(), sizeof(int32_t) * env.h_cfaces.size());
  if (parent) std::memcpy(parent, env.h_cparent.data(), sizeof(int32_t) * env.h_cparent.size());
  return TC_OK;
}

tc_status tc_boundary_faces(tc_env* h, int32_t* faces, int32_t* parent) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  if (faces) std::memcpy(faces, env.h_bfaces.data(), sizeof(int32_t) * env.h_bfaces.size());
  if (parent) std::memcpy(parent, env.h_bparent.data(), sizeof(int32_t) * env.h_bparent.size());
  return TC_OK;
}

tc_status tc_pixel_table(tc_env* h, int32_t* pix_face, float* pix_w) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  if (pix_face) std::memcpy(pix_face, env.h_pix_face.data(), sizeof(int32_t) * env.h_pix_face.size());
  if (pix_w) std::memcpy(pix_w, env.h_pix_w.data(), sizeof(float) * env.h_pix_w.size());
  return TC_OK;
}

tc_status tc_get_positions(tc_env* h, double* x) {
  if (!h || !x) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  return env.precision == TC_FP64 ? tc::get_positions<double>(env, x) : tc::get_positions<float>(env, x);
}

tc_status tc_set_positions(tc_env* h, const double* x) {
  if (!h || !x) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  if (env.busy.load()) return TC_ERR_INVALID_ARG;
  return env.precision == TC_FP64 ? tc::set_positions<double>(env, x) : tc::set_positions<float>(env, x);
}

tc_status tc_env_info(tc_env* h, tc_info* info) {
  if (!h || !info) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  info->nv = env.nv;
  info->nt = env.nt;
  info->nf = env.nf;
  info->nfc = env.nfc;
  info->nec = env.nec;
  info->nvc = env.nvc;
  info->ind_nv = env.ind_nv;
  info->ind_nf = env.ind_nf;
  info->ind_ne = env.ind_ne;
  info->H = env.H;
  info->W = env.W;
  info->newton_iters = env.stats.newton;
  info->pcg_iters = env.stats.pcg;
  info->substeps = env.stats.substeps;
  info->steps = env.stats.steps;
  info->line_search_halvings = env.stats.halvings;
  info->kappa = env.kappa;
  info->device_bytes = env.arena.bytes;
  info->nnzb = env.nnzb;
  info->pcg_capped = env.stats.pcg_capped;
  info->working_bytes = env.work_bytes;
  info->working_resident = env.work_resident ? 1 : 0;
  return TC_OK;
}

tc_status tc_profile_enable(tc_env* h, int32_t on) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  cudaStreamSynchronize(env.stream);
  if (on) {
    if (!env.prof) env.prof = new (std::nothrow) tc::Profiler();
    if (!env.prof) return TC_ERR_OOM;
    env.prof->reset();
  } else if (env.prof) {
    env.prof->collect();
    delete env.prof;
    env.prof = nullptr;
  }
  return TC_OK;
}

tc_status tc_profile_read(tc_env* h, tc_kernel_time* out, int32_t max, int32_t* n) {
  if (!h || !n || (max > 0 && !out)) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  std::lock_guard<std::mutex> api_lock(env.api_mu);
  *n = 0;
  if (!env.prof) return TC_OK;
  cudaStreamSynchronize(env.stream);
  env.prof->collect();
  const int cnt = (int)env.prof->entries.size();
  for (int i = 0; i < cnt && i < max; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, env.prof->entries[i].name, sizeof(out[i].name) - 1);
    out[i].ms = env.prof->entries[i].ms;
    out[i].launches = env.prof->entries[i].launches;
  }
  *n = cnt;
  return TC_OK;
}

void tc_destroy(tc_env* h) {
  if (!h) return;
  Env& env = h->impl;
  tc::server_forget(env);  // a server that meters this env's working set lets go of it first
  cudaStreamSynchronize(env.stream);
  delete env.prof;
  env.prof = nullptr;
  tc::destroy_exec(env);
  env.arena.release_all();
  cudaStreamSynchronize(env.stream);
  if (env.sc_host) cudaFreeHost(env.sc_host);
  if (env.x_host) cudaFreeHost(env.x_host);
  delete h;
}

tc_status tc_stress_from_F(const float* F, int64_t n, double E, double nu, float* sigma_out, void* stream) {
  if (n < 0 || (n > 0 && (!F || !sigma_out)) || !(E > 0) || !(nu > -1.0 && nu < 0.5)) return TC_ERR_INVALID_ARG;
  if (n == 0) return TC_OK;
  const double mu = E / (2.0 * (1.0 + nu));
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double lam_hat = lam + mu;
  tc::launch_stress_from_F(F, n, (float)mu, (float)lam_hat, (float)(1.0 + mu / lam_hat), sigma_out,
                           (cudaStream_t)stream);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TC_ERR_CUDA;
  return TC_OK;
}

}  // extern "C"
