// Host-side description of one batched launch and the launcher entry points.
#pragma once
#include "env.cuh"

namespace tc {

// Offsets (in doubles) of the per-unit partial regions of a batch.
struct PartLayout {
  int64_t elem;      // K_TET units: element energy
  int64_t cont[3];   // K_CV / K_CE / K_CF units: (energy, min d^2)
  int64_t asmb;      // K_VGRP units: (|g|^2, inertia energy)
  int64_t inert;     // K_VERT units: trial inertia energy
  int64_t ccd[3];    // contact units: min TOI
  int64_t rz, rr;    // K_VERT units: PCG start r.z, r.r
  int64_t env_s;     // 8 per env: PCG start values
  int64_t total;
};

// Launch shape of the per-env PCG cluster (process-wide per precision).
struct PcgShape {
  int cs = 16;          // CTAs per env (cluster size)
  int threads = 1024;   // threads per CTA
  int smem = 0;         // dynamic shared memory per CTA
  int coresident = 0;   // clusters of this shape the GPU holds at once
};
template <class R> PcgShape pcg_shape();
template <class R> tc_status set_pcg_shape(int cs, int threads);

template <class R> struct BatchHost {
  int nenv = 0;
  int units[K_NKIND] = {0, 0, 0, 0, 0, 0};
  BatchView<R> bv{};
  PartLayout L{};
};

template <class R> void b_elem(const BatchHost<R>& b, bool hess, bool trial, cudaStream_t s);
template <class R> void b_contact(const BatchHost<R>& b, bool hess, bool trial, cudaStream_t s);
template <class R> void b_ccd(const BatchHost<R>& b, cudaStream_t s);
template <class R> void b_force(const BatchHost<R>& b, cudaStream_t s);
// lagged friction pairs of every env (mu_f > 0) at its current state and pose
template <class R> void b_friction_lag(const BatchHost<R>& b, cudaStream_t s);
template <class R> void b_assemble(const BatchHost<R>& b, cudaStream_t s);
template <class R> void b_trial_energy(const BatchHost<R>& b, cudaStream_t s);
template <class R> tc_status b_pcg(const BatchHost<R>& b, int max_iter, bool warm, cudaStream_t s);
template <class R> void b_pmax(const BatchHost<R>& b, cudaStream_t s);
template <class R> void b_trial(const BatchHost<R>& b, cudaStream_t s);
template <class R> void b_scale_dx(const BatchHost<R>& b, cudaStream_t s);  // dx *= param per env
// mode 0: u0 = u and (dynamic) utilde = u + dt vel; mode 1: vel = (u - u0) / dt;
// mode 2: dx = param (utilde - u0)
template <class R> void b_step_vectors(const BatchHost<R>& b, int mode, cudaStream_t s);

}  // namespace tc
