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

#include <cstdio>
#include <cstdlib>

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

// Per-env PCG start values written by k_pcg_init_env: 0 r.z, 1 r.r,
// 2 done (1 when the start residual already meets the tolerance),
// 3 iterations, 4 squared tolerance, 5 p.q.
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

// ------------------------------------------------- PCG, one cluster per env
// Every env of the batch runs all of its CG iterations in one thread-block
// cluster (16 CTAs where the GPU can co-schedule them, else 8; 1024 threads
// each) over a contiguous share of the env's rows, so envs iterate
// independently: an env that converges frees its SMs at once, and no grid-wide
// barrier ties envs together.  Per iteration:
//   A  q = A p (BSR rows, one 8-lane group per row), p.q          | cluster barrier
//   B  alpha = r.z / p.q, dx += alpha p, r -= alpha q, z = M^-1 r;
//      r.z, r.r                                                    | cluster barrier
//   C  beta = r.z_new / r.z, stop test, p = z + beta p             | cluster barrier
// Each CTA reduces its rows in a fixed tree and posts the result in its
// shared memory; after the barrier every CTA adds the CS posts in rank order
// through distributed shared memory, so all CTAs hold bit-identical scalars
// and take the same branch.  Results do not depend on the other envs.
constexpr int kPcgThreads = 1024;

// Sum of `nval` posted values over the CS ranks of the cluster, in a fixed
// shuffle tree on warp 0 (the same tree in every CTA), broadcast to the block.
template <int NVAL>
TC_D void cluster_gather(cg::cluster_group& cluster, int CS, double* s_post, double* s_bcast, double out[NVAL]) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double* remote = lane < CS ? cluster.map_shared_rank(s_post, lane) : nullptr;
#pragma unroll
    for (int k = 0; k < NVAL; ++k) {
      double v = lane < CS ? remote[k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_bcast[k] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NVAL; ++k) out[k] = s_bcast[k];
}

// q = A p for two rows per lane group at once (independent loads in flight)
template <class R>
TC_D void bsr_rows2(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const R* __restrict__ val,
                    int64_t nb, const R* p, R* q, int nv, int v0, int v1, int r1, double& pq) {
  const int lane = threadIdx.x & (kLanes - 1);
  const bool ok0 = v0 < r1, ok1 = v1 < r1;
  R a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
  const int k0s = ok0 ? __ldg(rp + v0) : 0, k0e = ok0 ? __ldg(rp + v0 + 1) : 0;
  const int k1s = ok1 ? __ldg(rp + v1) : 0, k1e = ok1 ? __ldg(rp + v1 + 1) : 0;
  int k0 = k0s + lane, k1 = k1s + lane;
  while (k0 < k0e || k1 < k1e) {
    if (k0 < k0e) {
      const int j = __ldg(ci + k0);
      const R p0 = p[j], p1 = p[nv + j], p2 = p[2 * nv + j];
      const R* B = val + k0;
      a0 += __ldg(B) * p0 + __ldg(B + nb) * p1 + __ldg(B + 2 * nb) * p2;
      a1 += __ldg(B + 3 * nb) * p0 + __ldg(B + 4 * nb) * p1 + __ldg(B + 5 * nb) * p2;
      a2 += __ldg(B + 6 * nb) * p0 + __ldg(B + 7 * nb) * p1 + __ldg(B + 8 * nb) * p2;
      k0 += kLanes;
    }
    if (k1 < k1e) {
      const int j = __ldg(ci + k1);
      const R p0 = p[j], p1 = p[nv + j], p2 = p[2 * nv + j];
      const R* B = val + k1;
      b0 += __ldg(B) * p0 + __ldg(B + nb) * p1 + __ldg(B + 2 * nb) * p2;
      b1 += __ldg(B + 3 * nb) * p0 + __ldg(B + 4 * nb) * p1 + __ldg(B + 5 * nb) * p2;
      b2 += __ldg(B + 6 * nb) * p0 + __ldg(B + 7 * nb) * p1 + __ldg(B + 8 * nb) * p2;
      k1 += kLanes;
    }
  }
  a0 = group_sum(a0);
  a1 = group_sum(a1);
  a2 = group_sum(a2);
  b0 = group_sum(b0);
  b1 = group_sum(b1);
  b2 = group_sum(b2);
  if (lane == 0) {
    if (ok0) {
      q[v0] = a0;
      q[nv + v0] = a1;
      q[2 * nv + v0] = a2;
      pq += (double)p[v0] * (double)a0 + (double)p[nv + v0] * (double)a1 + (double)p[2 * nv + v0] * (double)a2;
    }
    if (ok1) {
      q[v1] = b0;
      q[nv + v1] = b1;
      q[2 * nv + v1] = b2;
      pq += (double)p[v1] * (double)b0 + (double)p[nv + v1] * (double)b1 + (double)p[2 * nv + v1] * (double)b2;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_cluster(const BatchView<R> bv, PartLayout L, int max_iter) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int env = blockIdx.x / CS;
  __shared__ double s_post[3];
  __shared__ double s_bcast[3];
  const EnvView<R>& ev = bv.views[env];
  const int nv = ev.nv;
  const int64_t nb = ev.nnzb;
  const int32_t* __restrict__ rp = ev.bsr_rp;
  const int32_t* __restrict__ ci = ev.bsr_ci;
  const R* __restrict__ val = ev.bsr_val;
  const R* __restrict__ Minv = ev.Minv;
  R* p = ev.p;
  R* q = ev.q;
  R* r = ev.r;
  R* z = ev.z;
  R* dx = ev.dx;
  const int r0 = (int)((int64_t)nv * rank / CS), r1 = (int)((int64_t)nv * (rank + 1) / CS);
  const double* es = bv.part + L.env_s + kEnvScalars * env;
  double rz = es[0], rr = es[1], pq = 0.0;
  const double tol2 = es[4];
  bool done = es[2] != 0.0;
  int it = 0;
  constexpr int kGroups = kPcgThreads / kLanes;
  while (!done && it < max_iter) {
    // A. q = A p
    double loc = 0.0;
    const int g = (int)threadIdx.x / kLanes;
    for (int base = r0; base < r1; base += 2 * kGroups)  // block-uniform trip count
      bsr_rows2<R>(rp, ci, val, nb, p, q, nv, base + g, base + g + kGroups, r1, loc);
    loc = block_sum<kPcgThreads>(loc);
    if (threadIdx.x == 0) s_post[0] = loc;
    cluster.sync();
    double g1[1];
    cluster_gather<1>(cluster, CS, s_post, s_bcast, g1);
    pq = g1[0];
    const R alpha = (R)(pq > 0.0 ? rz / pq : 0.0);
    // B. vector update
    double lrz = 0.0, lrr = 0.0;
    for (int v = r0 + (int)threadIdx.x; v < r1; v += kPcgThreads) {
      R rv[3], zv[3];
      for (int i = 0; i < 3; ++i) {
        dx[i * nv + v] += alpha * p[i * nv + v];
        rv[i] = r[i * nv + v] - alpha * q[i * nv + v];
        r[i * nv + v] = rv[i];
      }
      const R m0 = __ldg(Minv + v), m1 = __ldg(Minv + nv + v), m2 = __ldg(Minv + 2 * nv + v);
      const R m3 = __ldg(Minv + 3 * nv + v), m4 = __ldg(Minv + 4 * nv + v), m5 = __ldg(Minv + 5 * nv + v);
      zv[0] = m0 * rv[0] + m3 * rv[1] + m5 * rv[2];
      zv[1] = m3 * rv[0] + m1 * rv[1] + m4 * rv[2];
      zv[2] = m5 * rv[0] + m4 * rv[1] + m2 * rv[2];
      for (int i = 0; i < 3; ++i) {
        z[i * nv + v] = zv[i];
        lrz += (double)rv[i] * (double)zv[i];
        lrr += (double)rv[i] * (double)rv[i];
      }
    }
    lrz = block_sum<kPcgThreads>(lrz);
    lrr = block_sum<kPcgThreads>(lrr);
    if (threadIdx.x == 0) {
      s_post[1] = lrz;
      s_post[2] = lrr;
    }
    cluster.sync();
    double g3[3];
    cluster_gather<3>(cluster, CS, s_post, s_bcast, g3);
    const double rz_new = g3[1];
    rr = g3[2];
    ++it;
    done = rr <= tol2 || !(pq > 0.0) || !isfinite(rr) || it >= max_iter;
    const R beta = (R)(rz > 0.0 ? rz_new / rz : 0.0);
    rz = rz_new;
    if (done) break;
    // C. direction update
    for (int v = r0 + (int)threadIdx.x; v < r1; v += kPcgThreads)
      for (int i = 0; i < 3; ++i) p[i * nv + v] = z[i * nv + v] + beta * p[i * nv + v];
    cluster.sync();
  }
  if (rank == 0 && threadIdx.x == 0) {
    Scalars* sc = ev.sc;
    sc->pcg_iters = it;
    sc->rz = rz;
    sc->rr = rr;
    sc->pq = pq;
    sc->pcg_tol2 = tol2;
    sc->pcg_done = 1;
    if (!isfinite(rr) || !isfinite(pq)) sc->status |= ST_NONFINITE;
  }
  // no CTA may leave while another can still read its shared memory
  cluster.sync();
}

// Largest cluster the GPU co-schedules for the PCG kernel: 16 (non-portable)
// if possible, else the portable 8.
template <class R> static int pcg_cluster_size() {
  static int cached = -1;
  if (cached < 0) {
    cached = 8;
    if (cudaFuncSetAttribute(k_pcg_cluster<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kPcgThreads);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster<R>, &cfg) == cudaSuccess && n > 0) cached = 16;
      const char* tr = std::getenv("TACAUCHY_TRACE");
      if (tr && tr[0] && tr[0] != '0') {
        int n8 = 0;
        attr[0].val.clusterDim.x = 8;
        cfg.gridDim = dim3(8);
        cudaOccupancyMaxActiveClusters(&n8, k_pcg_cluster<R>, &cfg);
        std::fprintf(stderr, "[tc] pcg cluster size %d (co-resident clusters: %d of 16 CTAs, %d of 8)\n", cached, n, n8);
      }
    }
    cudaGetLastError();
  }
  return cached;
}

template <class R> tc_status b_pcg(const BatchHost<R>& b, int max_iter, cudaStream_t s) {
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_pcg_init", s, k_pcg_init<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, b.L));
  TC_LAUNCH("k_pcg_init_env", s, k_pcg_init_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
  const int CS = pcg_cluster_size<R>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b.nenv * CS));
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err = cudaSuccess;
  TC_LAUNCH("k_pcg_cluster", s, err = cudaLaunchKernelEx(&cfg, k_pcg_cluster<R>, b.bv, b.L, max_iter));
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
