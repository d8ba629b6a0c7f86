// Newton-step kernels over a batch of envs: per-vertex assembly (K4),
// matrix-free block-Jacobi PCG (K5), energies for the line search (K7) and
// step updates.
//
// Assembly is atomic-free: element and contact passes write their
// per-element / per-primitive contributions to slots, and one lane group per
// vertex sums its incident slots through fixed incidence lists into the
// gradient and into its row of the block-sparse (3x3 BSR) Newton matrix,
// which the PCG then multiplies row by row.  Every block
// reduction writes one partial per work unit; per-env finalize blocks fold an
// env's partials in unit order.  Dot products and energies accumulate in
// double.  Results do not depend on the batch composition or the schedule.
#include <cooperative_groups.h>

#include "env.cuh"
#include "prof.cuh"
#include "solver.cuh"

namespace cg = cooperative_groups;

namespace tc {

// Per-vertex gathers use a group of kLanes consecutive lanes: each lane sums
// every kLanes-th incidence and the group combines the partial sums with a
// fixed shuffle tree (deterministic), giving kLanes times more independent
// loads in flight than one thread per vertex.
constexpr int kLanes = 8;
static_assert(kBlock / kLanes == 32, "K_VGRP units hold 32 vertices");

template <class T> TC_D T group_sum(T v) {
#pragma unroll
  for (int o = kLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kLanes);
  return v;
}

// An env's per-unit partials part[u * stride + offset], u over its units of
// `kind`, folded in unit order by one block.
template <class R>
TC_D double env_unit_sum(const BatchView<R>& bv, int kind, int env, const double* part, int stride = 1,
                         int offset = 0) {
  const int* p = bv.prefix + kind * (bv.nenv + 1);
  double s = 0.0;
  for (int u = p[env] + threadIdx.x; u < p[env + 1]; u += blockDim.x) s += part[(int64_t)u * stride + offset];
  return block_sum<kBlock>(s);
}
template <class R>
TC_D double env_unit_min(const BatchView<R>& bv, int kind, int env, const double* part, int stride = 1,
                         int offset = 0) {
  const int* p = bv.prefix + kind * (bv.nenv + 1);
  double s = 1e300;
  for (int u = p[env] + threadIdx.x; u < p[env + 1]; u += blockDim.x) s = fmin(s, part[(int64_t)u * stride + offset]);
  return block_min<kBlock>(s);
}

// ---------------------------------------------------------------- assembly
// One lane group per vertex (row) gathers, through fixed-order lists:
//   g_v     = element gradient slots + contact gradient slots (+ inertia)
//   row v   = every 3x3 block (v, j) of the Newton matrix: element stiffness
//             blocks + contact Hessian blocks (+ M/h^2 on the diagonal)
//   M^-1_v  = inverse of the diagonal block (block-Jacobi preconditioner).
// Partials per K_VGRP unit: |g|^2 and the inertia energy 1/(2h^2)|u - u~|_M^2.
TC_D int pair_index(int a, int b) { return a * 4 - (a * (a - 1)) / 2 + (b - a); }  // corners a <= b

template <class R> TC_D void add_contact_block(const EnvView<R>& e, uint32_t code, R B[9]) {
  const int kind = (int)(code >> 30), a = (int)((code >> 28) & 3u), b = (int)((code >> 26) & 3u);
  const int prim = (int)(code & ((1u << 26) - 1u));
  const R* slot;
  int n, N;
  if (kind == 0) {
    slot = e.cv_slot;
    n = e.nvc;
    N = 3;
  } else if (kind == 1) {
    slot = e.ce_slot;
    n = e.nec;
    N = 6;
  } else {
    slot = e.cf_slot;
    n = e.nfc;
    N = 9;
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) B[3 * r + c] += slot[(int64_t)(N + sym_index(3 * a + r, 3 * b + c, N)) * n + prim];
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_assemble(const BatchView<R> bv, PartLayout L) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VGRP, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int lane = threadIdx.x & (kLanes - 1);
  const int v = l.chunk * 32 + threadIdx.x / kLanes;
  const int nt = e.nt, nv = e.nv;
  const bool valid = v < nv;
  double gn2 = 0.0, ein = 0.0;
  R g[3] = {0, 0, 0};
  bool finite = true;
  if (valid) {
    for (int k = e.vt_off[v] + lane; k < e.vt_off[v + 1]; k += kLanes) {
      const int code = e.vt_idx[k];
      const int el = code >> 2, c = code & 3;
      for (int i = 0; i < 3; ++i) g[i] += e.eslot[(int64_t)(3 * c + i) * nt + el];
    }
    const int s = e.vslot[v];
    if (s >= 0) {
      if (lane == 0)
        for (int i = 0; i < 3; ++i) g[i] += e.cv_slot[(int64_t)i * e.nvc + s];
      for (int k = e.cv_edge_off[s] + lane; k < e.cv_edge_off[s + 1]; k += kLanes) {
        const int code = e.cv_edge_idx[k], p = code >> 2, q = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.ce_slot[(int64_t)(3 * q + i) * e.nec + p];
      }
      for (int k = e.cv_face_off[s] + lane; k < e.cv_face_off[s + 1]; k += kLanes) {
        const int code = e.cv_face_idx[k], p = code >> 2, q = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.cf_slot[(int64_t)(3 * q + i) * e.nfc + p];
      }
    }
    // the matrix row (empty for a fixed vertex)
    const R mh = e.mass ? e.mass[v] * e.inv_h2 : R(0);
    for (int k = e.bsr_rp[v] + lane; k < e.bsr_rp[v + 1]; k += kLanes) {
      R B[9];
      for (int q = 0; q < 9; ++q) B[q] = R(0);
      for (int c = e.be_off[k]; c < e.be_off[k + 1]; ++c) {
        const int code = e.be_idx[c];
        const int t = code >> 4, a = (code >> 2) & 3, b = code & 3;
        const R* K = e.kblk + (int64_t)t * 90;
        if (a <= b) {
          const R* Kb = K + 9 * pair_index(a, b);
          for (int q = 0; q < 9; ++q) B[q] += Kb[q];
        } else {
          const R* Kb = K + 9 * pair_index(b, a);
          for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) B[3 * r + cc] += Kb[3 * cc + r];
        }
      }
      for (int c = e.bc_off[k]; c < e.bc_off[k + 1]; ++c) add_contact_block<R>(e, (uint32_t)e.bc_idx[c], B);
      if (k == e.bsr_diag[v]) {
        B[0] += mh;
        B[4] += mh;
        B[8] += mh;
        // inverse of the (symmetric) diagonal block: adjugate / det
        const R xx = B[0], yy = B[4], zz = B[8], xy = B[1], yz = B[5], zx = B[2];
        const R c00 = yy * zz - yz * yz, c01 = yz * zx - xy * zz, c02 = xy * yz - yy * zx;
        const R det = xx * c00 + xy * c01 + zx * c02;
        R M[6];
        if (det > R(0) && isfinite((double)det)) {
          const R id = R(1) / det;
          M[0] = c00 * id;
          M[1] = (xx * zz - zx * zx) * id;
          M[2] = (xx * yy - xy * xy) * id;
          M[3] = c01 * id;
          M[4] = (xy * zx - xx * yz) * id;
          M[5] = c02 * id;
        } else {
          const R tr = xx + yy + zz;
          const R d = tr > R(0) ? R(3) / tr : R(1);
          M[0] = M[1] = M[2] = d;
          M[3] = M[4] = M[5] = R(0);
        }
        for (int i = 0; i < 6; ++i) {
          e.Minv[(int64_t)i * nv + v] = M[i];
          finite = finite && isfinite((double)M[i]);
        }
      }
      for (int q = 0; q < 9; ++q) {
        e.bsr_val[(int64_t)q * e.nnzb + k] = B[q];
        finite = finite && isfinite((double)B[q]);
      }
    }
  }
  for (int i = 0; i < 3; ++i) g[i] = group_sum(g[i]);
  if (valid && lane == 0) {
    if (e.mass) {
      const R mh = e.mass[v] * e.inv_h2;
      for (int i = 0; i < 3; ++i) {
        const R du = e.u[i * nv + v] - e.utilde[i * nv + v];
        g[i] += mh * du;
        ein += 0.5 * (double)mh * (double)du * (double)du;
      }
    }
    if (e.fixed[v]) {
      g[0] = g[1] = g[2] = R(0);
      for (int i = 0; i < 6; ++i) e.Minv[(int64_t)i * nv + v] = R(0);
    }
    for (int i = 0; i < 3; ++i) {
      e.g[i * nv + v] = g[i];
      gn2 += (double)g[i] * (double)g[i];
      finite = finite && isfinite((double)g[i]);
    }
  }
  if (!finite) atomicOr(&e.sc->status, ST_NONFINITE);
  gn2 = block_sum<kBlock>(gn2);
  ein = block_sum<kBlock>(ein);
  if (threadIdx.x == 0) {
    bv.part[L.asmb + 2 * (int64_t)blockIdx.x] = gn2;
    bv.part[L.asmb + 2 * (int64_t)blockIdx.x + 1] = ein;
  }
}

// inertia energy at the trial point (K_VERT units)
template <class R>
__global__ void __launch_bounds__(kBlock) k_inertia(const BatchView<R> bv, PartLayout L) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  double ein = 0.0;
  if (v < e.nv && e.mass) {
    const R mh = e.mass[v] * e.inv_h2;
    for (int i = 0; i < 3; ++i) {
      const double du = (double)e.ut[i * e.nv + v] - (double)e.utilde[i * e.nv + v];
      ein += 0.5 * (double)mh * du * du;
    }
  }
  ein = block_sum<kBlock>(ein);
  if (threadIdx.x == 0) bv.part[L.inert + blockIdx.x] = ein;
}

// per env: total energy (elastic + contact + inertia), min pair distance and
// (after assembly) |g|^2 -> the env's Scalars
template <class R>
__global__ void __launch_bounds__(kBlock) k_finalize_energy(const BatchView<R> bv, PartLayout L, int assembly) {
  const int env = blockIdx.x;
  const EnvView<R>& e = bv.views[env];
  double E = env_unit_sum(bv, K_TET, env, bv.part + L.elem);
  double dm = 1e300;
  for (int k = 0; k < 3; ++k) {
    E += env_unit_sum(bv, K_CV + k, env, bv.part + L.cont[k], 2, 0);
    dm = fmin(dm, env_unit_min(bv, K_CV + k, env, bv.part + L.cont[k], 2, 1));
  }
  double gn2 = 0.0;
  if (assembly) {
    E += env_unit_sum(bv, K_VGRP, env, bv.part + L.asmb, 2, 1);
    gn2 = env_unit_sum(bv, K_VGRP, env, bv.part + L.asmb, 2, 0);
  } else {
    E += env_unit_sum(bv, K_VERT, env, bv.part + L.inert);
  }
  if (threadIdx.x == 0) {
    e.sc->energy = E;
    if (assembly) e.sc->gnorm2 = gn2;
    e.sc->reduce_tmp[1] = dm;  // min squared pair distance seen by the contact pass
    if (!isfinite(E)) e.sc->status |= ST_NONFINITE;
  }
}

template <class R> void b_assemble(const BatchHost<R>& b, cudaStream_t s) {
  if (b.units[K_VGRP] > 0) TC_LAUNCH("k_assemble", s, k_assemble<R><<<b.units[K_VGRP], kBlock, 0, s>>>(b.bv, b.L));
  TC_LAUNCH("k_finalize_energy", s, k_finalize_energy<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L, 1));
}

// energy at the trial displacement ut (elastic + contact + inertia)
template <class R> void b_trial_energy(const BatchHost<R>& b, cudaStream_t s) {
  b_elem<R>(b, false, true, s);
  b_contact<R>(b, false, true, s);
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_inertia", s, k_inertia<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, b.L));
  TC_LAUNCH("k_finalize_energy", s, k_finalize_energy<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L, 0));
}

// ------------------------------------------------------------------ PCG

template <class R> TC_D void apply_minv(const EnvView<R>& e, int v, const R r[3], R z[3]) {
  const int nv = e.nv;
  const R m0 = e.Minv[v], m1 = e.Minv[nv + v], m2 = e.Minv[2 * nv + v];
  const R m3 = e.Minv[3 * nv + v], m4 = e.Minv[4 * nv + v], m5 = e.Minv[5 * nv + v];
  z[0] = m0 * r[0] + m3 * r[1] + m5 * r[2];
  z[1] = m3 * r[0] + m1 * r[1] + m4 * r[2];
  z[2] = m5 * r[0] + m4 * r[1] + m2 * r[2];
}

// r = -g, z = M^-1 r, p = z, dx = 0; partials r.z, r.r per K_VERT unit
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_init(const BatchView<R> bv, PartLayout L) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  const int nv = e.nv;
  double rz = 0.0, rr = 0.0;
  if (v < nv) {
    R r[3], z[3];
    for (int i = 0; i < 3; ++i) r[i] = e.fixed[v] ? R(0) : -e.g[i * nv + v];
    apply_minv<R>(e, v, r, z);
    for (int i = 0; i < 3; ++i) {
      e.r[i * nv + v] = r[i];
      e.z[i * nv + v] = z[i];
      e.p[i * nv + v] = z[i];
      e.dx[i * nv + v] = R(0);
      rz += (double)r[i] * (double)z[i];
      rr += (double)r[i] * (double)r[i];
    }
  }
  rz = block_sum<kBlock>(rz);
  rr = block_sum<kBlock>(rr);
  if (threadIdx.x == 0) {
    bv.part[L.rz + blockIdx.x] = rz;
    bv.part[L.rr + blockIdx.x] = rr;
  }
}

// Per-env PCG scalars, double-buffered by iteration parity: iteration `it`
// reads buffer it & 1 and the env's designated block writes buffer
// (it + 1) & 1, so no block reads a value while it is being replaced.
// Fields: 0 r.z, 1 r.r, 2 done (0 running, 1 stopped), 3 iterations,
// 4 squared tolerance, 5 p.q of the last iteration.
constexpr int kEnvScalars = 8;

// per env: r.z, r.r and the squared stopping tolerance (param[env]) -> buffer 0
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_init_env(const BatchView<R> bv, PartLayout L) {
  const int env = blockIdx.x;
  const EnvView<R>& e = bv.views[env];
  const double rz = env_unit_sum(bv, K_VERT, env, bv.part + L.rz);
  const double rr = env_unit_sum(bv, K_VERT, env, bv.part + L.rr);
  if (threadIdx.x == 0) {
    Scalars* sc = e.sc;
    if (!isfinite(rz) || !isfinite(rr)) sc->status |= ST_NONFINITE;
    const double tol2 = bv.param[env];
    double* es = bv.part + L.env_s + kEnvScalars * env;
    es[0] = rz;
    es[1] = rr;
    es[2] = (rr <= tol2) ? 1.0 : 0.0;
    es[3] = 0.0;
    es[4] = tol2;
    es[5] = 0.0;
  }
}

// q = A p for row v (BSR, one lane group per row); returns p.q on the
// group's lane 0 (0 elsewhere).  Every lane of the warp calls it.
template <class R> TC_D double bsr_q_group(const EnvView<R>& e, int v, bool valid) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int nv = e.nv;
  R q0 = 0, q1 = 0, q2 = 0;
  if (valid) {
    const int64_t nb = e.nnzb;
    for (int k = e.bsr_rp[v] + lane; k < e.bsr_rp[v + 1]; k += kLanes) {
      const int j = e.bsr_ci[k];
      const R p0 = e.p[j], p1 = e.p[nv + j], p2 = e.p[2 * nv + j];
      const R* B = e.bsr_val + k;
      q0 += B[0] * p0 + B[nb] * p1 + B[2 * nb] * p2;
      q1 += B[3 * nb] * p0 + B[4 * nb] * p1 + B[5 * nb] * p2;
      q2 += B[6 * nb] * p0 + B[7 * nb] * p1 + B[8 * nb] * p2;
    }
  }
  q0 = group_sum(q0);
  q1 = group_sum(q1);
  q2 = group_sum(q2);
  double pq = 0.0;
  if (valid && lane == 0) {
    e.q[v] = q0;
    e.q[nv + v] = q1;
    e.q[2 * nv + v] = q2;
    pq = (double)e.p[v] * (double)q0 + (double)e.p[nv + v] * (double)q1 + (double)e.p[2 * nv + v] * (double)q2;
  }
  return pq;
}

// block-wide sum broadcast to every thread
TC_D double block_sum_all(double v) {
  __shared__ double s_tot;
  const double t = block_sum<kBlock>(v);
  if (threadIdx.x == 0) s_tot = t;
  __syncthreads();
  const double r = s_tot;
  __syncthreads();
  return r;
}

template <class R> TC_D double env_sum_all(const BatchView<R>& bv, int kind, int env, const double* part) {
  const int* p = bv.prefix + kind * (bv.nenv + 1);
  double s = 0.0;
  for (int u = p[env] + threadIdx.x; u < p[env + 1]; u += blockDim.x) s += part[u];
  return block_sum_all(s);
}

// ------------------------------------------------------ persistent PCG
// All CG iterations of all envs of the batch in one cooperative launch, over
// contiguous ranges of work units per block.  Per iteration:
//   A  q = A p (BSR rows), p.q partials                           | sync
//   B  alpha = r.z / p.q per env, dx += alpha p, r -= alpha q,
//      z = M^-1 r; r.z, r.r partials                              | sync
//   C  beta = r.z_new / r.z per env, stop test, p = z + beta p;
//      each env's designated block publishes its new scalars      | sync
// Every block folds the partials of the envs it touches itself, in unit
// order with the same reduction tree, so all blocks hold bit-identical
// per-env scalars without waiting for one writer; converged envs skip their
// work while the others continue.  Results do not depend on the grid size or
// on which other envs are in the batch.
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_batched(const BatchView<R> bv, PartLayout L, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x;
  const int nenv = bv.nenv;
  const int* pre = bv.prefix;
  const int nG = pre[K_VGRP * (nenv + 1) + nenv];
  const int nV = pre[K_VERT * (nenv + 1) + nenv];
  const int g0 = (int)((int64_t)nG * blockIdx.x / G), g1 = (int)((int64_t)nG * (blockIdx.x + 1) / G);
  const int w0 = (int)((int64_t)nV * blockIdx.x / G), w1 = (int)((int64_t)nV * (blockIdx.x + 1) / G);
  double* es0 = bv.part + L.env_s;
  int it = 0;
  for (; it < max_iter; ++it) {
    const double* cur = es0 + (int64_t)(it & 1) * kEnvScalars * nenv;
    double* nxt = es0 + (int64_t)((it + 1) & 1) * kEnvScalars * nenv;
    int all_done = 1;
    for (int env = 0; env < nenv; ++env) all_done &= cur[kEnvScalars * env + 2] != 0.0;
    if (all_done) break;
    // A. q = A p
    for (int u = g0; u < g1; ++u) {
      const Loc l = locate(pre, nenv, K_VGRP, u);
      double pq = 0.0;
      if (cur[kEnvScalars * l.env + 2] == 0.0) {
        const EnvView<R>& e = bv.views[l.env];
        const int v = l.chunk * 32 + threadIdx.x / kLanes;
        pq = bsr_q_group<R>(e, v, v < e.nv && !e.fixed[v]);
      }
      pq = block_sum<kBlock>(pq);
      if (threadIdx.x == 0) bv.part[L.pq + u] = pq;
    }
    grid.sync();
    // B. vector update
    {
      int cenv = -1;
      R alpha = 0;
      for (int u = w0; u < w1; ++u) {
        const Loc l = locate(pre, nenv, K_VERT, u);
        double rz = 0.0, rr = 0.0;
        if (cur[kEnvScalars * l.env + 2] == 0.0) {
          if (l.env != cenv) {
            cenv = l.env;
            const double pq = env_sum_all(bv, K_VGRP, cenv, bv.part + L.pq);
            alpha = (R)(pq > 0.0 ? cur[kEnvScalars * cenv + 0] / pq : 0.0);
          }
          const EnvView<R>& e = bv.views[l.env];
          const int nv = e.nv;
          const int v = l.chunk * kBlock + threadIdx.x;
          if (v < nv) {
            R r[3], z[3];
            for (int i = 0; i < 3; ++i) {
              e.dx[i * nv + v] += alpha * e.p[i * nv + v];
              r[i] = e.r[i * nv + v] - alpha * e.q[i * nv + v];
              e.r[i * nv + v] = r[i];
            }
            apply_minv<R>(e, v, r, z);
            for (int i = 0; i < 3; ++i) {
              e.z[i * nv + v] = z[i];
              rz += (double)r[i] * (double)z[i];
              rr += (double)r[i] * (double)r[i];
            }
          }
        }
        rz = block_sum<kBlock>(rz);
        rr = block_sum<kBlock>(rr);
        if (threadIdx.x == 0) {
          bv.part[L.rz + u] = rz;
          bv.part[L.rr + u] = rr;
        }
      }
    }
    grid.sync();
    // C. direction update and the published scalars
    {
      int cenv = -1;
      R beta = 0;
      for (int u = w0; u < w1; ++u) {
        const Loc l = locate(pre, nenv, K_VERT, u);
        if (cur[kEnvScalars * l.env + 2] != 0.0) continue;
        if (l.env != cenv) {
          cenv = l.env;
          const double rz_new = env_sum_all(bv, K_VERT, cenv, bv.part + L.rz);
          const double rz_old = cur[kEnvScalars * cenv + 0];
          beta = (R)(rz_old > 0.0 ? rz_new / rz_old : 0.0);
        }
        const EnvView<R>& e = bv.views[l.env];
        const int nv = e.nv;
        const int v = l.chunk * kBlock + threadIdx.x;
        if (v < nv)
          for (int i = 0; i < 3; ++i) e.p[i * nv + v] = e.z[i * nv + v] + beta * e.p[i * nv + v];
      }
      for (int env = blockIdx.x; env < nenv; env += G) {
        const double* c = cur + kEnvScalars * env;
        double* n = nxt + kEnvScalars * env;
        if (c[2] != 0.0) {
          if (threadIdx.x == 0)
            for (int f = 0; f < kEnvScalars; ++f) n[f] = c[f];
          continue;
        }
        const double rz_new = env_sum_all(bv, K_VERT, env, bv.part + L.rz);
        const double rr = env_sum_all(bv, K_VERT, env, bv.part + L.rr);
        const double pq = env_sum_all(bv, K_VGRP, env, bv.part + L.pq);
        if (threadIdx.x == 0) {
          const double iters = c[3] + 1.0;
          const bool done = rr <= c[4] || !(pq > 0.0) || !isfinite(rr) || iters >= max_iter;
          n[0] = rz_new;
          n[1] = rr;
          n[2] = done ? 1.0 : 0.0;
          n[3] = iters;
          n[4] = c[4];
          n[5] = pq;
        }
      }
    }
    grid.sync();
  }
  // publish per-env results (the buffer the last iteration wrote)
  const double* fin = es0 + (int64_t)(it & 1) * kEnvScalars * nenv;
  for (int env = blockIdx.x; env < nenv; env += G)
    if (threadIdx.x == 0) {
      const double* c = fin + kEnvScalars * env;
      Scalars* sc = bv.views[env].sc;
      sc->pcg_iters = (int)c[3];
      sc->rz = c[0];
      sc->rr = c[1];
      sc->pq = c[5];
      sc->pcg_tol2 = c[4];
      sc->pcg_done = 1;
      if (!isfinite(sc->rr) || !isfinite(sc->pq)) sc->status |= ST_NONFINITE;
    }
}

template <class R> struct CoopInfo {
  static int max_blocks() {
    static int cached = -1;
    if (cached < 0) {
      int dev = 0, sms = 0, per_sm = 0, coop = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batched<R>, kBlock, 0);
      cached = coop ? sms * per_sm : 0;
    }
    return cached;
  }
};

template <class R> tc_status b_pcg(const BatchHost<R>& b, int max_iter, cudaStream_t s) {
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_pcg_init", s, k_pcg_init<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, b.L));
  TC_LAUNCH("k_pcg_init_env", s, k_pcg_init_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
  const int cap = CoopInfo<R>::max_blocks();
  if (cap <= 0) return TC_ERR_CUDA;
  const int work = std::max(b.nenv, std::max(b.units[K_VGRP], b.units[K_VERT]));
  const int G = std::max(1, std::min(work, cap));
  BatchView<R> bv = b.bv;
  PartLayout L = b.L;
  int mi = max_iter;
  void* args[] = {(void*)&bv, (void*)&L, (void*)&mi};
  cudaError_t err = cudaSuccess;
  TC_LAUNCH("k_pcg_batched", s,
            err = cudaLaunchCooperativeKernel((void*)k_pcg_batched<R>, dim3(G), dim3(kBlock), args, 0, s));
  return err == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

// ------------------------------------------------------ per-env reductions

// max-norm of dx -> pmax, and g.dx (minus twice the Newton decrement)
template <class R>
__global__ void __launch_bounds__(kBlock) k_pmax(const BatchView<R> bv) {
  const EnvView<R>& e = bv.views[blockIdx.x];
  double m = 0.0, gd = 0.0;
  for (int v = threadIdx.x; v < e.nv; v += blockDim.x)
    for (int i = 0; i < 3; ++i) {
      const double d = (double)e.dx[i * e.nv + v];
      m = fmax(m, fabs(d));
      gd += (double)e.g[i * e.nv + v] * d;
    }
  m = block_max<kBlock>(m);
  gd = block_sum<kBlock>(gd);
  if (threadIdx.x == 0) {
    e.sc->pmax = m;
    e.sc->reduce_tmp[3] = gd;
    if (!isfinite(m)) e.sc->status |= ST_NONFINITE;
  }
}

template <class R> void b_pmax(const BatchHost<R>& b, cudaStream_t s) {
  TC_LAUNCH("k_pmax", s, k_pmax<R><<<b.nenv, kBlock, 0, s>>>(b.bv));
}

// trial point ut = u + alpha dx; alpha = min(1, TOI) when param < 0 (or no
// param), else param
template <class R>
__global__ void __launch_bounds__(kBlock) k_trial(const BatchView<R> bv) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const double a = bv.param ? bv.param[l.env] : -1.0;
  const R alpha = (R)(a < 0.0 ? fmin(1.0, e.sc->ccd_t) : a);
  const int v = l.chunk * kBlock + threadIdx.x;
  if (v < e.nv)
    for (int i = 0; i < 3; ++i) e.ut[i * e.nv + v] = e.u[i * e.nv + v] + alpha * e.dx[i * e.nv + v];
}

template <class R> void b_trial(const BatchHost<R>& b, cudaStream_t s) {
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_trial", s, k_trial<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv));
}

// mode 0 (step start): u0 = u and, when dynamic, utilde = u + dt vel;
// mode 1 (step end, dynamic): vel = (u - u0) / dt
template <class R>
__global__ void __launch_bounds__(kBlock) k_step_vectors(const BatchView<R> bv, int mode) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  if (v >= e.nv) return;
  for (int i = 0; i < 3; ++i) {
    const int k = i * e.nv + v;
    if (mode == 0) {
      e.u0[k] = e.u[k];
      if (e.dt > 0.0) e.utilde[k] = e.u[k] + (R)e.dt * e.vel[k];
    } else if (e.dt > 0.0) {
      e.vel[k] = (R)((double)(e.u[k] - e.u0[k]) / e.dt);
    }
  }
}

template <class R> void b_step_vectors(const BatchHost<R>& b, int mode, cudaStream_t s) {
  if (b.units[K_VERT] > 0)
    TC_LAUNCH("k_step_vectors", s, k_step_vectors<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, mode));
}

#define TC_INST(R)                                                            \
  template void b_assemble<R>(const BatchHost<R>&, cudaStream_t);             \
  template void b_trial_energy<R>(const BatchHost<R>&, cudaStream_t);         \
  template tc_status b_pcg<R>(const BatchHost<R>&, int, cudaStream_t);        \
  template void b_pmax<R>(const BatchHost<R>&, cudaStream_t);                 \
  template void b_trial<R>(const BatchHost<R>&, cudaStream_t);                \
  template void b_step_vectors<R>(const BatchHost<R>&, int, cudaStream_t);
TC_INST(float)
TC_INST(double)
#undef TC_INST

}  // namespace tc
