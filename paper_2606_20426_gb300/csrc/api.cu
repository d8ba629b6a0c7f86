// C ABI (include/tacauchy.h) and the host side of one implicit step.
//
// tc_step (Algorithm 2, physics line) runs, on the env's stream:
//   indenter substeps s in [0, 1] (kinematic indenter, CCD-limited advance)
//     Newton iterations
//       K1 element pass + K3 barrier pass + K4 assembly   -> E, |g|
//       K5 PCG (chunks of iterations between flag reads)  -> dx
//       K6 CCD along dx                                    -> alpha_max
//       K7 backtracking line search on E(u + alpha dx)
// The host reads a handful of scalars per Newton iteration (energy, |g|,
// PCG flag, CCD bound, trial energies); everything else stays on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "env.cuh"

struct tc_env {
  tc::Env impl;
};

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

static void pose_interp(const tc_pose& a, const tc_pose& b, double s, tc_pose* out) {
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

// TACAUCHY_TRACE=1 prints one line per Newton iteration and substep to stderr.
static bool trace_on() {
  const char* v = std::getenv("TACAUCHY_TRACE");
  return v && v[0] && v[0] != '0';
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static tc_status read_scalars(Env& env) {
  TC_CHECK(cudaMemcpyAsync(env.sc_host, env.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, env.stream));
  TC_CHECK(cudaStreamSynchronize(env.stream));
  if (env.prof) env.prof->collect();
  if (env.sc_host->status & ST_NONFINITE) return TC_ERR_NONFINITE;
  return TC_OK;
}

// (Re)allocate the candidate lists for `cap` entries per gel primitive.
static tc_status alloc_candidates(Env& env, int cap) {
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

// One CCD pass (gel moving by dir from pose a to pose b), which also rebuilds
// the candidate lists; with `trial`, also the first line-search point
// u + min(1, TOI) dir and its energy.  Grows the lists and repeats when a
// primitive had more candidates than fit.
template <class R>
static tc_status ccd_pass(Env& env, const R* dir, const tc_pose& a, const tc_pose& b, bool trial) {
  for (int attempt = 0; attempt < 16; ++attempt) {
    EnvView<R> e = env.view<R>();
    launch_ccd<R>(e, dir, a.R, a.t, b.R, b.t, env.stream);
    if (trial) {
      launch_trial<R>(e, (R*)env.utrial, env.stream);
      launch_energy<R>(e, (R*)env.utrial, env.stream);
    }
    tc_status st = read_scalars(env);
    if (st != TC_OK && st != TC_ERR_NONFINITE) return st;
    const int need = env.sc_host->overflow;
    if (need > env.cand_cap) {
      int cap = env.cand_cap;
      while (cap < need) cap *= 2;
      TC_CHECK(cudaMemsetAsync(&env.sc->overflow, 0, sizeof(int), env.stream));
      const tc_status sa = alloc_candidates(env, cap);
      if (sa != TC_OK) return sa;
      continue;
    }
    env.cand_valid = true;
    return st;
  }
  return TC_ERR_CAPACITY;
}

// Candidate lists for the current state (static pass) if none are valid.
template <class R> static tc_status ensure_candidates(Env& env) {
  if (env.cand_valid) return TC_OK;
  const tc_status st = ccd_pass<R>(env, nullptr, env.pose, env.pose, false);
  return st == TC_ERR_NONFINITE ? TC_OK : st;
}

template <class R> static tc_status newton_solve(Env& env) {
  double g0 = -1.0;
  const int chunk = 8;
  for (int it = 0; it < env.newton_max; ++it) {
    const double t_iter0 = trace_on() ? now_ms() : 0.0;
    EnvView<R> e = env.view<R>();
    launch_elem<R>(e, true, e.u, env.stream);
    launch_contact<R>(e, true, e.u, env.stream);
    launch_assemble<R>(e, env.stream);
    tc_status st = read_scalars(env);
    if (st != TC_OK) return st;
    const double E0 = env.sc_host->energy;
    const double gn = std::sqrt(env.sc_host->gnorm2);
    if (!std::isfinite(gn) || !std::isfinite(E0)) return TC_ERR_NONFINITE;
    if (g0 < 0) g0 = gn;
    env.stats.newton++;
    if (gn <= std::max(env.rtol * g0, env.gabs)) return TC_OK;
    double eta = std::min(0.5, std::sqrt(gn / std::max(g0, 1e-300)));
    eta = std::max(eta, env.precision == TC_FP64 ? 1e-10 : 1e-5);
    launch_pcg_init<R>(e, eta, env.stream);
    if (!launch_pcg_persistent<R>(e, env.pcg_max, env.stream)) {
      int done_iters = 0;
      while (done_iters < env.pcg_max) {
        const int n = std::min(chunk, env.pcg_max - done_iters);
        for (int k = 0; k < n; ++k) launch_pcg_iter<R>(e, env.pcg_max, env.stream);
        done_iters += n;
        st = read_scalars(env);
        if (st != TC_OK) return st;
        if (env.sc_host->pcg_done) break;
      }
    }
    // direction bound, CCD along dx (rebuilding the candidate lists), and
    // the first trial point u + min(1, TOI) dx with its energy, all before
    // the next host read
    launch_pmax<R>(e, env.stream);
    st = ccd_pass<R>(env, e.dx, env.pose, env.pose, true);
    if (st != TC_OK && st != TC_ERR_NONFINITE) return st;
    e = env.view<R>();
    R* ut = (R*)env.utrial;
    env.stats.pcg += env.sc_host->pcg_iters;
    const int pcg_it = env.sc_host->pcg_iters;
    const double pcg_rr = env.sc_host->rr, pcg_tol2 = env.sc_host->pcg_tol2;
    const double t_pcg = trace_on() ? now_ms() : 0.0;
    double alpha = std::min(1.0, env.sc_host->ccd_t);
    if (trace_on())
      std::fprintf(stderr,
                   "[tc] newton %d E=%.17g |g|=%.6e g0=%.6e pcg=%d rr/tol=%.3e pq=%.3e rz=%.3e pmax=%.3e ccd=%.6f "
                   "Etrial=%.17g dmin=%.3e st=%d t=%.2fms\n",
                   it, E0, gn, g0, pcg_it, pcg_rr / std::max(pcg_tol2, 1e-300), env.sc_host->pq, env.sc_host->rz,
                   env.sc_host->pmax, env.sc_host->ccd_t, env.sc_host->energy, std::sqrt(env.sc_host->reduce_tmp[1]),
                   env.sc_host->status, t_pcg - t_iter0);
    // Converged when the full step is below ptol, or when it is below 10 ptol
    // and the predicted decrease -g.dx/2 is below the rounding level of the
    // energy (the line search could no longer measure progress): the step is
    // then taken without the energy test.
    const double decrement = -0.5 * env.sc_host->reduce_tmp[3];
    const double e_noise = (env.precision == TC_FP64 ? 1e-14 : 1e-7) * std::fabs(E0);
    if (env.sc_host->pmax <= env.ptol || (env.sc_host->pmax <= 10.0 * env.ptol && decrement <= e_noise)) {
      if (st == TC_ERR_NONFINITE) return st;
      std::swap(env.u, env.utrial);
      return TC_OK;
    }
    bool ok = false;
    for (int ls = 0; ls <= 60; ++ls) {
      if (ls > 0) {
        launch_axpy_u<R>(e, ut, e.u, (R)alpha, e.dx, env.stream);
        launch_energy<R>(e, ut, env.stream);
        st = read_scalars(env);
        if (st != TC_OK && st != TC_ERR_NONFINITE) return st;
      }
      const double Et = env.sc_host->energy;
      if (st == TC_OK && std::isfinite(Et) && Et <= E0) {
        ok = true;
        break;
      }
      if (st == TC_ERR_NONFINITE) {  // a trial point outside the barrier's domain: clear and keep halving
        int zero = 0;
        TC_CHECK(cudaMemcpyAsync(&env.sc->status, &zero, sizeof(int), cudaMemcpyHostToDevice, env.stream));
      }
      alpha *= 0.5;
      env.stats.halvings++;
    }
    if (trace_on())
      std::fprintf(stderr, "[tc]   line search alpha=%.6e ok=%d E_trial=%.17g dE=%.3e\n", alpha, (int)ok,
                   env.sc_host->energy, env.sc_host->energy - E0);
    if (!ok) return TC_ERR_LINESEARCH;
    std::swap(env.u, env.utrial);
    // Noise floor: the full Newton step is within 10 ptol and the energy can
    // no longer tell the trial point from the current one.
    if (env.sc_host->energy == E0 && env.sc_host->pmax <= 10.0 * env.ptol) return TC_OK;
  }
  return TC_ERR_NEWTON_MAXITER;
}

template <class R> static tc_status do_step(Env& env, const tc_pose& target) {
  const int64_t n3 = 3 * (int64_t)env.nv;
  TC_CHECK(cudaMemcpyAsync(env.ut, env.u, sizeof(R) * n3, cudaMemcpyDeviceToDevice, env.stream));
  if (env.dynamic) {  // u_tilde = u + h v
    EnvView<R> e = env.view<R>();
    launch_axpy_u<R>(e, (R*)env.utilde, (const R*)env.u, (R)env.dt, (const R*)env.vel, env.stream);
  }
  const tc_pose pose0 = env.pose;
  double s = 0.0;
  bool reached = false;
  for (int sub = 0; sub < 256; ++sub) {
    tc_pose ps;
    pose_interp(pose0, target, s, &ps);
    env.pose = ps;
    EnvView<R> e = env.view<R>();
    // indenter advance against the static gel (body frame: gel moves)
    tc_status st = ccd_pass<R>(env, (const R*)nullptr, ps, target, false);
    if (st != TC_OK) return st;
    const double frac = env.sc_host->ccd_t;
    s = frac >= 1.0 ? 1.0 : s + (1.0 - s) * frac;
    if (trace_on()) std::fprintf(stderr, "[tc] substep %d advance frac=%.6e s=%.9f\n", sub, frac, s);
    pose_interp(pose0, target, s, &env.pose);
    st = newton_solve<R>(env);
    env.stats.substeps++;
    if (st != TC_OK) return st;
    if (s >= 1.0) {
      reached = true;
      break;
    }
  }
  if (!reached) return TC_ERR_NEWTON_MAXITER;
  env.pose = target;
  if (env.dynamic) {  // v = (u - u_t) / h
    EnvView<R> e = env.view<R>();
    launch_axpy_u<R>(e, (R*)env.vel, (const R*)env.u, (R)-1.0, (const R*)env.ut, env.stream);
    launch_axpy_u<R>(e, (R*)env.vel, (R*)env.vel, (R)(1.0 / env.dt - 1.0), (const R*)env.vel, env.stream);
  }
  env.stats.steps++;
  TC_CHECK(cudaStreamSynchronize(env.stream));
  if (env.prof) env.prof->collect();
  return TC_OK;
}

template <class R> static tc_status alloc_state(Env& env) {
  Arena& a = env.arena;
  const int64_t nv = env.nv, nt = env.nt;
  auto A = [&](void** p, int64_t n) {
    *p = a.alloc<R>(n);
    return *p != nullptr;
  };
  bool ok = A(&env.u, 3 * nv) && A(&env.ut, 3 * nv) && A(&env.utrial, 3 * nv) && A(&env.H9, 45 * nt) &&
            A(&env.eslot, 36 * nt) && A(&env.yslot, 12 * nt) && A(&env.g, 3 * nv) && A(&env.Minv, 6 * nv) &&
            A(&env.dx, 3 * nv) && A(&env.r, 3 * nv) && A(&env.z, 3 * nv) && A(&env.p, 3 * nv) && A(&env.q, 3 * nv) &&
            A(&env.cv_slot, 9 * (int64_t)std::max(env.nvc, 1)) && A(&env.ce_slot, 27 * (int64_t)std::max(env.nec, 1)) &&
            A(&env.cf_slot, 54 * (int64_t)std::max(env.nfc, 1)) && A(&env.cv_y, 3 * (int64_t)std::max(env.nvc, 1)) &&
            A(&env.ce_y, 6 * (int64_t)std::max(env.nec, 1)) && A(&env.cf_y, 9 * (int64_t)std::max(env.nfc, 1));
  if (ok && env.dynamic) ok = A(&env.vel, 3 * nv) && A(&env.utilde, 3 * nv);
  if (!ok) return TC_ERR_OOM;
  TC_CHECK(cudaMemsetAsync(env.u, 0, sizeof(R) * 3 * nv, env.stream));
  TC_CHECK(cudaMemsetAsync(env.dx, 0, sizeof(R) * 3 * nv, env.stream));
  if (env.dynamic) {
    TC_CHECK(cudaMemsetAsync(env.vel, 0, sizeof(R) * 3 * nv, env.stream));
    TC_CHECK(cudaMemsetAsync(env.utilde, 0, sizeof(R) * 3 * nv, env.stream));
  }
  const int nc = (int)(std::max(1, (env.nvc + 127) / 128) + std::max(1, (env.nec + 127) / 128) +
                       std::max(1, (env.nfc + 127) / 128));
  // per-block partials: element + contact + assembly passes, or 3 per block
  // of the persistent PCG (at most grid_for(nt) + grid_for(nv) blocks)
  const int nbt = (int)grid_for(nt), nbv = (int)grid_for(nv), nbq = (int)grid_for(8 * (nv + 3));
  env.part_len = nbt + 2 * nc + 2 * nbq + 3 * (nbt + nbv) + nbq + 2 * nbv + 3 * nbv + 64;
  env.part = a.alloc<double>(env.part_len);
  const tc_status sc0 = alloc_candidates(env, 32);
  if (sc0 != TC_OK) return sc0;
  env.face_p = a.alloc<float>(std::max(env.nfc, 1));
  env.face_A = a.alloc<float>(std::max(env.nfc, 1));
  env.vert_p = a.alloc<float>(std::max(env.nvc, 1));
  if (!env.part || !env.face_p || !env.face_A || !env.vert_p) return TC_ERR_OOM;
  return TC_OK;
}

template <class R> static tc_status initial_check(Env& env) {
  tc_status sc0 = ensure_candidates<R>(env);
  if (sc0 != TC_OK) return sc0;
  EnvView<R> e = env.view<R>();
  launch_energy<R>(e, e.u, env.stream);
  tc_status st = read_scalars(env);
  if (st != TC_OK) return st == TC_ERR_NONFINITE ? TC_ERR_INITIAL_PENETRATION : st;
  if (!(env.sc_host->reduce_tmp[1] > 0.0)) return TC_ERR_INITIAL_PENETRATION;
  int* flag = env.arena.alloc<int>(1);
  if (!flag) return TC_ERR_OOM;
  const int hit = intersect_test<R>(e, flag, env.stream);
  env.arena.put(flag);
  return hit ? TC_ERR_INITIAL_PENETRATION : TC_OK;
}

template <class R> static tc_status contact_force(Env& env, double* out) {
  const tc_status sc0 = ensure_candidates<R>(env);
  if (sc0 != TC_OK) return sc0;
  EnvView<R> e = env.view<R>();
  launch_contact<R>(e, true, e.u, env.stream);
  launch_contact_force<R>(e, env.stream);
  tc_status st = read_scalars(env);
  if (st != TC_OK) return st;
  for (int d = 0; d < 3; ++d) out[d] = env.sc_host->force[d];
  return TC_OK;
}

template <class R> static tc_status pressure_map(Env& env, float* out, uint8_t* mask) {
  EnvView<R> e = env.view<R>();
  launch_traction<R>(e, env.cparent, nullptr, nullptr, nullptr, env.face_p, env.face_A, env.stream);
  launch_vertex_avg(env.nvc, env.cv_face_off, env.cv_face_idx, env.face_p, env.face_A, env.vert_p, env.stream);
  launch_splat(env.H * env.W, env.pix_face, env.pix_w, env.cface_slot, env.nfc, env.vert_p, out, mask, env.stream);
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
  if (opts->dt > 0 && !(material->density > 0)) return TC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 4 * (int64_t)mesh->nt; ++i)
    if (mesh->tets[i] < 0 || mesh->tets[i] >= mesh->nv) return TC_ERR_INVALID_MESH;
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
  env.lam_hat = env.lam + env.mu;
  env.alpha = 1.0 + env.mu / env.lam_hat;
  env.dhat = opts->dhat;
  env.kappa = opts->kappa;
  env.dt = opts->dt;
  env.dynamic = opts->dt > 0;
  env.rtol = opts->newton_rtol > 0 ? opts->newton_rtol : 1e-6;
  env.newton_max = opts->newton_max > 0 ? opts->newton_max : 1024;
  env.pcg_max = opts->pcg_max > 0 ? opts->pcg_max : 1000;
  env.thick_axis = opts->contact_axis;
  // Newton step tolerance: 1e-4 dhat in FP64; FP32 gradients carry rounding
  // noise of ~1e-5 of the contact force, whose Newton step is ~10 nm, so the
  // mixed mode stops at 1e-3 dhat.
  env.ptol = (env.precision == TC_FP64 ? 1e-4 : 1e-3) * env.dhat;
  env.pose = *start_pose;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < mesh->nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], mesh->X[3 * (size_t)v + d]);
      hi[d] = std::max(hi[d], mesh->X[3 * (size_t)v + d]);
    }
  const double L2 = (hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) + (hi[2] - lo[2]) * (hi[2] - lo[2]);
  env.gabs = 1e-12 * env.E * L2;
  tc_status st = TC_OK;
  env.sc = env.arena.alloc<tc::Scalars>(1);
  if (!env.sc || cudaMallocHost(&env.sc_host, sizeof(tc::Scalars)) != cudaSuccess) st = TC_ERR_OOM;
  if (st == TC_OK && cudaMemsetAsync(env.sc, 0, sizeof(tc::Scalars), env.stream) != cudaSuccess) st = TC_ERR_CUDA;
  if (st == TC_OK) st = tc::setup_scene(env, mesh, fixed, nfixed, indenter, grid);
  if (st == TC_OK)
    st = env.precision == TC_FP64 ? tc::alloc_state<double>(env) : tc::alloc_state<float>(env);
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
  tc::ProfGuard pg(env);
  tc_status st = env.precision == TC_FP64 ? tc::do_step<double>(env, *target) : tc::do_step<float>(env, *target);
  env.last_status = st;
  return st;
}

tc_status tc_stress(tc_env* h, float* sigma_out) {
  if (!h || !sigma_out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
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
  tc::ProfGuard pg(env);
  if (env.precision == TC_FP64)
    tc::launch_traction<double>(env.view<double>(), env.cparent, t, p, t_tau, nullptr, nullptr, env.stream);
  else
    tc::launch_traction<float>(env.view<float>(), env.cparent, t, p, t_tau, nullptr, nullptr, env.stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(env.stream) != cudaSuccess) return TC_ERR_CUDA;
  return TC_OK;
}

tc_status tc_pressure_map(tc_env* h, float* out, uint8_t* mask) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  tc::ProfGuard pg(env);
  if (env.H * env.W == 0) return TC_ERR_INVALID_ARG;
  return env.precision == TC_FP64 ? tc::pressure_map<double>(env, out, mask) : tc::pressure_map<float>(env, out, mask);
}

tc_status tc_contact_force(tc_env* h, double* out) {
  if (!h || !out) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  tc::ProfGuard pg(env);
  return env.precision == TC_FP64 ? tc::contact_force<double>(env, out) : tc::contact_force<float>(env, out);
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
  return env.precision == TC_FP64 ? tc::get_positions<double>(env, x) : tc::get_positions<float>(env, x);
}

tc_status tc_set_positions(tc_env* h, const double* x) {
  if (!h || !x) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
  return env.precision == TC_FP64 ? tc::set_positions<double>(env, x) : tc::set_positions<float>(env, x);
}

tc_status tc_env_info(tc_env* h, tc_info* info) {
  if (!h || !info) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
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
  return TC_OK;
}

tc_status tc_profile_enable(tc_env* h, int32_t on) {
  if (!h) return TC_ERR_INVALID_ARG;
  Env& env = h->impl;
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
  cudaStreamSynchronize(env.stream);
  delete env.prof;
  env.prof = nullptr;
  env.arena.release_all();
  cudaStreamSynchronize(env.stream);
  if (env.sc_host) cudaFreeHost(env.sc_host);
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
