// Newton-step kernels over a batch of envs: per-vertex assembly (K4),
// block-Jacobi PCG on the assembled block-sparse matrix (K5), energies for the line search (K7) and
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
#include <mutex>
#include <cstdlib>

#include "env.cuh"
#include "prof.cuh"
#include "batch.cuh"
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

// slot of block kk of the row with free index f (sliced layout, EnvView::bsr_val)
template <class R> TC_D int64_t sell_slot(const EnvView<R>& e, int f, int kk) {
  return (int64_t)e.sell_off[f >> 5] + 32 * kk + (f & 31);
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
    const int k0 = e.bsr_rp[v], fr = e.free_of[v];
    for (int k = k0 + lane; k < e.bsr_rp[v + 1]; k += kLanes) {
      R B[9];
      for (int q = 0; q < 9; ++q) B[q] = R(0);
      for (int c = e.be_off[k]; c < e.be_off[k + 1]; ++c) {
        const int code = e.be_idx[c];
        const int t = code >> 4, a = (code >> 2) & 3, b = code & 3;
        const R* K = e.kblk;
        if (a <= b) {
          const int q0 = 9 * pair_index(a, b);
          for (int q = 0; q < 9; ++q) B[q] += K[kblk_index(t, q0 + q)];
        } else {
          const int q0 = 9 * pair_index(b, a);
          for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) B[3 * r + cc] += K[kblk_index(t, q0 + 3 * cc + r)];
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
      const int64_t t = sell_slot(e, fr, k - k0);
      for (int q = 0; q < 9; ++q) {
        e.bsr_val[(int64_t)q * e.nsell + t] = B[q];
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

// Per-env PCG start values written by k_pcg_init_env: 0 r.z, 1 r.r,
// 2 done (1 when the start residual already meets the tolerance),
// 3 iterations, 4 squared tolerance, 5 p.q; 6 the warm-start scale s.
constexpr int kEnvScalars = 8;

// Warm start from a previous solve: its solution d scaled by the minimiser
// s = -g.d / d.A d of the quadratic model along d, so the start point s d is
// never worse for the model than 0.  d (EnvView::wd) is the previous solve's
// solution (still in dx), or for the first Newton solve of a substep the
// first solve of the previous substep (the response to the previous
// indenter advance).  This pass forms q = A d
// (one lane group per row, blocks in row order) and the per-unit partials
// -g.d and d.q (K_VGRP units, in the assembly's partial region, which is
// free once the assembly has been folded).
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_warm(const BatchView<R> bv, PartLayout L) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VGRP, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int lane = threadIdx.x & (kLanes - 1);
  const int v = l.chunk * 32 + threadIdx.x / kLanes;
  const int nv = e.nv;
  const int64_t nb = e.nsell;
  double gd = 0.0, dq = 0.0;
  R a[3] = {0, 0, 0};
  if (v < nv) {
    const int k0 = e.bsr_rp[v], fr = e.free_of[v];
    for (int k = k0 + lane; k < e.bsr_rp[v + 1]; k += kLanes) {
      const int j = e.bsr_ci[k];
      const R d0 = e.wd[j], d1 = e.wd[nv + j], d2 = e.wd[2 * nv + j];
      const R* B = e.bsr_val + sell_slot(e, fr, k - k0);
      a[0] += B[0] * d0 + B[nb] * d1 + B[2 * nb] * d2;
      a[1] += B[3 * nb] * d0 + B[4 * nb] * d1 + B[5 * nb] * d2;
      a[2] += B[6 * nb] * d0 + B[7 * nb] * d1 + B[8 * nb] * d2;
    }
  }
  for (int i = 0; i < 3; ++i) a[i] = group_sum(a[i]);
  if (v < nv && lane == 0)
    for (int i = 0; i < 3; ++i) {
      const R d = e.wd[i * nv + v];
      e.q[i * nv + v] = a[i];
      gd -= (double)e.g[i * nv + v] * (double)d;
      dq += (double)d * (double)a[i];
    }
  gd = block_sum<kBlock>(gd);
  dq = block_sum<kBlock>(dq);
  if (threadIdx.x == 0) {
    bv.part[L.asmb + 2 * (int64_t)blockIdx.x] = gd;
    bv.part[L.asmb + 2 * (int64_t)blockIdx.x + 1] = dq;
  }
}

// per env: the warm-start scale s (0 when d.A d is not positive or the
// quotient is not finite: then the solve starts from 0)
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_warm_env(const BatchView<R> bv, PartLayout L) {
  const int env = blockIdx.x;
  const double gd = env_unit_sum(bv, K_VGRP, env, bv.part + L.asmb, 2, 0);
  const double dq = env_unit_sum(bv, K_VGRP, env, bv.part + L.asmb, 2, 1);
  if (threadIdx.x == 0) {
    double sc = dq > 0.0 ? gd / dq : 0.0;
    if (!isfinite(sc)) sc = 0.0;
    bv.part[L.env_s + kEnvScalars * env + 6] = sc;
  }
}

// dx = s d, r = -g - s A d (cold start: s = 0, dx = 0, r = -g), z = M^-1 r,
// p = z; partials r.z, r.r per K_VERT unit
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_init(const BatchView<R> bv, PartLayout L, int warm) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  const int nv = e.nv;
  const R sw = warm ? (R)bv.part[L.env_s + kEnvScalars * l.env + 6] : R(0);
  double rz = 0.0, rr = 0.0;
  if (v < nv) {
    R r[3], z[3];
    for (int i = 0; i < 3; ++i) {
      r[i] = e.fixed[v] ? R(0) : -e.g[i * nv + v];
      if (sw != R(0) && !e.fixed[v]) r[i] -= sw * e.q[i * nv + v];
    }
    apply_minv<R>(e, v, r, z);
    for (int i = 0; i < 3; ++i) {
      e.r[i * nv + v] = r[i];
      e.z[i * nv + v] = z[i];
      e.p[i * nv + v] = z[i];
      e.dx[i * nv + v] = sw != R(0) ? sw * e.wd[i * nv + v] : R(0);
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

// ------------------------------------------------- PCG, one cluster per env
// Every env of the batch runs all of its CG iterations in one thread-block
// cluster (16 CTAs where the GPU co-schedules them, else 8; 1024 threads
// each) over a contiguous share of the env's matrix slices (32 free rows
// each, split so that every CTA holds about the same number of block
// slots), so envs iterate independently: an env that converges frees its
// SMs at once, and no grid-wide barrier ties envs together.  Per
// iteration, two cluster barriers:
//   S  p = z + beta p over the CTA's halo (the columns its rows touch),
//      staged in shared memory; the CTA's own rows also go to the next p
//      buffer in HBM (two buffers alternate, so no CTA overwrites values
//      another may still read)
//   A  q = A p, one lane per row of a slice, summing the row's blocks in
//      column order in registers; p.q                             | barrier
//   B  alpha = r.z / p.q, dx += alpha p, r -= alpha q, z = M^-1 r;
//      r.z, r.r                                                     | barrier
// Resident mode (the usual case): when the halo, a staging copy of it and
// the CTA's rows' r, z, dx, q and M^-1 all fit in shared memory, those
// vectors stay there for the whole solve and only z and p are published to
// HBM for the neighbours' halos.  Otherwise every vector lives in HBM (and
// when even the halo does not fit, the SpMV forms p = z + beta p of each
// column from HBM).  Dot products accumulate in double-float pairs (FP64
// issues at a small fraction of the FP32 rate on this part) with fixed
// reduction trees; each CTA pushes its partials into a slot of every CTA's
// shared memory before the cluster barrier, and every CTA adds the slots of
// all ranks in the same order, so all derive bit-identical alpha, beta and
// stop decisions (the quotients are taken in float from the double-float
// sums with one residual correction, so no FP64 division sits on the
// critical path).  Results do not depend on the other envs.
constexpr int kPcgMaxCluster = 16;
// blocks per lane and round of the SpMV: all their loads are issued before
// the first product, so a round waits on L2 once
template <class R> constexpr int kPcgUnroll = sizeof(R) == 4 ? 3 : 2;

// Items [r0, r1) of cluster rank `rank` out of nv items with offsets rp
// (rp[nv] in total): rank k starts at the first item r whose offset rp[r]
// reaches k rp[nv] / CS, so every rank holds about the same share.  Rank 0
// starts at item 0 and the last rank ends at item nv.  (The PCG splits the
// matrix slices by their slot offsets.)  Two rounds of
// parallel search over the row pointers; s_w holds 4 ints of scratch.
template <int NT>
TC_D void pcg_rows(const int32_t* __restrict__ rp, int nv, int CS, int rank, int* s_w, int& r0, int& r1) {
  const int64_t wtot = rp[nv];
  const int64_t tgt[2] = {wtot * rank / CS, wtot * (rank + 1) / CS};
  const int s1 = (nv + NT) / NT;  // NT * s1 >= nv + 1
  if (threadIdx.x < 2) {
    s_w[threadIdx.x] = 0;
    s_w[2 + threadIdx.x] = nv;
  }
  __syncthreads();
  {
    // coarse: the last sample row c s1 whose offset is below the target
    const int rc = min(nv, (int)threadIdx.x * s1);
    const int64_t wc = rp[rc];
    for (int b = 0; b < 2; ++b)
      if (wc < tgt[b]) atomicMax(&s_w[b], (int)threadIdx.x);
  }
  __syncthreads();
  // fine: the first row reaching the target among c s1 .. (c + 1) s1
  for (int b = 0; b < 2; ++b) {
    const int lo = s_w[b] * s1;
    for (int j = (int)threadIdx.x; j <= s1; j += NT) {
      const int r = min(nv, lo + j);
      if ((int64_t)rp[r] >= tgt[b]) atomicMin(&s_w[2 + b], r);
    }
  }
  __syncthreads();
  r0 = rank == 0 ? 0 : s_w[2];
  r1 = rank == CS - 1 ? nv : s_w[3];
}

// Block sums of NV accumulators (fixed tree) pushed into slot
// s_all[rank][slot + k] of every CTA of the cluster; the cluster barrier that
// follows makes them visible.  Ends without a block barrier: s_red is next
// written after that cluster barrier.
template <class R, int NV>
TC_D void cluster_push(typename Acc<R>::T* v, typename Acc<R>::T (*s_red)[32], typename Acc<R>::T (*s_all)[3],
                       int slot, cg::cluster_group& cluster, int rank, int CS) {
  using A = Acc<R>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    typename A::T x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl_xor(x, o));
    if (lane == 0) s_red[k][w] = x;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      typename A::T x = lane < (int)(blockDim.x >> 5) ? s_red[k][lane] : A::zero();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl_xor(x, o));
      if (lane < CS) cluster.map_shared_rank(&s_all[rank][slot + k], lane)[0] = x;
    }
  }
}

// Sum over ranks of slot `slot` (warp 0; fixed tree, the same in every CTA).
template <class R> TC_D typename Acc<R>::T cluster_total(typename Acc<R>::T (*s_all)[3], int slot, int CS) {
  using A = Acc<R>;
  const int lane = threadIdx.x & 31;
  typename A::T x = lane < CS ? s_all[lane][slot] : A::zero();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = A::add(x, A::shfl_xor(x, o));
  return x;
}

TC_D size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <class R, int kPcgThreads>
__global__ void __launch_bounds__(kPcgThreads, 1024 / kPcgThreads)
    k_pcg_cluster(const BatchView<R> bv, PartLayout L, int max_iter, int smem_bytes) {
  using A = Acc<R>;
  using AT = typename A::T;
  constexpr int NW = kPcgThreads / 32;
  constexpr int U = kPcgUnroll<R>;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ AT s_red[3][32];
  __shared__ AT s_all[kPcgMaxCluster][3];  // [rank][0 p.q, 1 r.z, 2 r.r]
  __shared__ R s_coef;
  __shared__ int s_flag;
  __shared__ int s_lohi[2];
  __shared__ int s_rows[4];
  __shared__ AT s_at[2];      // r.z, p.q (thread 0)
  __shared__ double s_sc[2];  // r.r, squared tolerance (thread 0)
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int env = blockIdx.x / CS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const EnvView<R>& ev = bv.views[env];
  const int nv = ev.nv, nfree = ev.nfree, nsl = (nfree + 31) >> 5;
  const int64_t ns = ev.nsell;
  const int32_t* __restrict__ rp = ev.bsr_rp;
  const int32_t* __restrict__ ci = ev.bsr_ci;
  const int32_t* __restrict__ soff = ev.sell_off;
  const int32_t* __restrict__ sci = ev.sell_ci;
  const int32_t* __restrict__ fv = ev.free_v;
  const R* __restrict__ val = ev.bsr_val;
  const R* __restrict__ Minv = ev.Minv;
  R* q = ev.q;
  R* r = ev.r;
  R* z = ev.z;
  R* dx = ev.dx;
  R* pbuf[2] = {ev.p, ev.p2};
  // the rank's slices [s0, s1), its free rows [f0, f1) and their vertex
  // range [r0, r1) (the free rows between r0 and r1 are exactly its rows)
  int s0, s1;
  pcg_rows<kPcgThreads>(soff, nsl, CS, rank, s_rows, s0, s1);
  const int f0 = min(32 * s0, nfree), f1 = min(32 * s1, nfree), nf = f1 - f0;
  const int r0 = nf > 0 ? fv[f0] : 0, r1 = nf > 0 ? fv[f1 - 1] + 1 : 0;
  // halo of the rows (columns within a row ascend, so its first and last
  // blocks bound it)
  if (threadIdx.x == 0) {
    s_lohi[0] = r0;
    s_lohi[1] = r1 - 1;
  }
  __syncthreads();
  if (nf > 0) {
    int lo = r0, hi = r1 - 1;
    for (int f = f0 + (int)threadIdx.x; f < f1; f += kPcgThreads) {
      const int v = fv[f];
      lo = min(lo, ci[rp[v]]);
      hi = max(hi, ci[rp[v + 1] - 1]);
    }
    atomicMin(&s_lohi[0], lo);
    atomicMax(&s_lohi[1], hi);
  }
  __syncthreads();
  const int cmin = s_lohi[0];
  const int H = nf > 0 ? s_lohi[1] - cmin + 1 : 0;
  // shared memory: p over the halo | (resident) the neighbours' old p, the
  // rows' r, z, dx, q, M^-1 and their vertex ids
  const size_t stage_bytes = align16((size_t)3 * H * sizeof(R));
  const size_t vec_bytes = align16((size_t)18 * nf * sizeof(R));
  const size_t lst_bytes = align16((size_t)nf * sizeof(int));
  const bool res = nf > 0 && 2 * stage_bytes + vec_bytes + lst_bytes <= (size_t)smem_bytes;
  const bool staged = res || stage_bytes <= (size_t)smem_bytes;
  R* sp = reinterpret_cast<R*>(s_dyn);
  R* sy = reinterpret_cast<R*>(s_dyn + stage_bytes);
  R* rs = reinterpret_cast<R*>(s_dyn + 2 * stage_bytes);  // resident: r, z, dx, q (3 nf each), M^-1 (6 nf)
  R* zs = rs + 3 * nf;
  R* dxs = zs + 3 * nf;
  R* qs = dxs + 3 * nf;
  R* ms = qs + 3 * nf;
  int* lst = reinterpret_cast<int*>(s_dyn + 2 * stage_bytes + vec_bytes);  // vertex of each row
  if (res)
    for (int idx = (int)threadIdx.x; idx < nf; idx += kPcgThreads) {
      const int v = fv[f0 + idx];
      lst[idx] = v;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rs[i * nf + idx] = r[i * nv + v];
        zs[i * nf + idx] = z[i * nv + v];
        dxs[i * nf + idx] = dx[i * nv + v];
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) ms[i * nf + idx] = Minv[i * nv + v];
    }
  // every CTA of the cluster runs (and has set up its shared memory) before
  // the first partials are pushed into it
  cluster.sync();
  const double* es = bv.part + L.env_s + kEnvScalars * env;
  if (threadIdx.x == 0) {
    s_at[0] = A::from_double(es[0]);
    s_at[1] = A::zero();
    s_sc[0] = es[1];
    s_sc[1] = es[4];
  }
  bool done = es[2] != 0.0;
  // each env stops at its own cap (max_iter bounds the launch as a whole), so
  // its iterations do not depend on the caps of the other envs in the batch
  const int cap = ev.pcg_max > 0 ? min(max_iter, ev.pcg_max) : max_iter;
  R beta = R(0);
  int it = 0;
  while (!done) {
    const R* pc = pbuf[it & 1];
    R* pn = pbuf[(it + 1) & 1];
    // S. direction update over the halo (or the own rows)
    if (res) {
      // the neighbours' halo rows from HBM: z into the halo buffer and the
      // old p into the staging buffer by asynchronous copies, so every load
      // of the thread is in flight at once; each thread then combines the
      // words it copied
      const int nlo = r0 - cmin, nother = H - (r1 - r0);
      for (int j = (int)threadIdx.x; j < nother; j += kPcgThreads) {
        const int v = j < nlo ? cmin + j : r1 + (j - nlo), l = v - cmin;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          cp_async_word(&sp[i * H + l], &z[i * nv + v]);
          cp_async_word(&sy[i * H + l], &pc[i * nv + v]);
        }
      }
      cp_async_wait_all();
      for (int j = (int)threadIdx.x; j < nother; j += kPcgThreads) {
        const int v = j < nlo ? cmin + j : r1 + (j - nlo), l = v - cmin;
#pragma unroll
        for (int i = 0; i < 3; ++i) sp[i * H + l] = sp[i * H + l] + beta * sy[i * H + l];
      }
      // the own rows from shared memory
      for (int idx = (int)threadIdx.x; idx < nf; idx += kPcgThreads) {
        const int v = lst[idx], l = v - cmin;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const R x = it == 0 ? zs[i * nf + idx] : zs[i * nf + idx] + beta * sp[i * H + l];
          sp[i * H + l] = x;
          pn[i * nv + v] = x;
        }
      }
    } else {
      if (staged)
        for (int v = cmin + (int)threadIdx.x; v < cmin + H; v += kPcgThreads)
#pragma unroll
          for (int i = 0; i < 3; ++i) sp[i * H + (v - cmin)] = z[i * nv + v] + beta * pc[i * nv + v];
      for (int f = f0 + (int)threadIdx.x; f < f1; f += kPcgThreads) {
        const int v = fv[f];
#pragma unroll
        for (int i = 0; i < 3; ++i) pn[i * nv + v] = z[i * nv + v] + beta * pc[i * nv + v];
      }
    }
    __syncthreads();
    // A. q = A p: one lane per row of a slice, its blocks in column order
    // (block kk of the slice's 32 rows is one coalesced load per entry)
    AT pq_loc = A::zero();
    for (int s = s0 + wid; s < s1; s += NW) {
      const int f = 32 * s + lane;
      const bool row = f < nfree;
      int v = 0, len = 0;
      if (row) {
        v = res ? lst[f - f0] : fv[f];
        len = rp[v + 1] - rp[v];
      }
      const int64_t base = soff[s] + lane;
      const int W = (soff[s + 1] - soff[s]) >> 5;
      R a0 = 0, a1 = 0, a2 = 0;
      for (int k0 = 0; k0 < W; k0 += U) {
        int jj[U];
        R Bv[U][9];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u < len) {
            const int64_t t = base + 32 * (k0 + u);
            jj[u] = sci[t];
#pragma unroll
            for (int e9 = 0; e9 < 9; ++e9) Bv[u][e9] = val[t + e9 * ns];
          }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (k0 + u < len) {
            const int j = jj[u];
            R p0, p1, p2;
            if (staged) {
              const int l = j - cmin;
              p0 = sp[l];
              p1 = sp[H + l];
              p2 = sp[2 * H + l];
            } else {
              p0 = z[j] + beta * pc[j];
              p1 = z[nv + j] + beta * pc[nv + j];
              p2 = z[2 * nv + j] + beta * pc[2 * nv + j];
            }
            const R* B = Bv[u];
            a0 += B[0] * p0 + B[1] * p1 + B[2] * p2;
            a1 += B[3] * p0 + B[4] * p1 + B[5] * p2;
            a2 += B[6] * p0 + B[7] * p1 + B[8] * p2;
          }
      }
      if (row) {
        R pv0, pv1, pv2;
        if (res) {
          const int idx = f - f0;
          qs[idx] = a0;
          qs[nf + idx] = a1;
          qs[2 * nf + idx] = a2;
        } else {
          q[v] = a0;
          q[nv + v] = a1;
          q[2 * nv + v] = a2;
        }
        if (staged) {
          const int l = v - cmin;
          pv0 = sp[l];
          pv1 = sp[H + l];
          pv2 = sp[2 * H + l];
        } else {
          pv0 = pn[v];
          pv1 = pn[nv + v];
          pv2 = pn[2 * nv + v];
        }
        pq_loc = A::add(pq_loc, A::add(A::add(A::prod(pv0, a0), A::prod(pv1, a1)), A::prod(pv2, a2)));
      }
    }
    cluster_push<R, 1>(&pq_loc, s_red, s_all, 0, cluster, rank, CS);
    cluster.sync();
    if (wid == 0) {
      const AT x = cluster_total<R>(s_all, 0, CS);
      if (threadIdx.x == 0) {
        s_at[1] = x;
        s_coef = A::positive(x) ? (R)A::ratio(s_at[0], x) : R(0);
      }
    }
    __syncthreads();
    const R alpha = s_coef;
    // B. vector update
    AT acc[2] = {A::zero(), A::zero()};
    if (res) {
      for (int idx = (int)threadIdx.x; idx < nf; idx += kPcgThreads) {
        const int v = lst[idx], l = v - cmin;
        R rv[3], zv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dxs[i * nf + idx] += alpha * sp[i * H + l];
          rv[i] = rs[i * nf + idx] - alpha * qs[i * nf + idx];
          rs[i * nf + idx] = rv[i];
        }
        const R m0 = ms[idx], m1 = ms[nf + idx], m2 = ms[2 * nf + idx];
        const R m3 = ms[3 * nf + idx], m4 = ms[4 * nf + idx], m5 = ms[5 * nf + idx];
        zv[0] = m0 * rv[0] + m3 * rv[1] + m5 * rv[2];
        zv[1] = m3 * rv[0] + m1 * rv[1] + m4 * rv[2];
        zv[2] = m5 * rv[0] + m4 * rv[1] + m2 * rv[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          zs[i * nf + idx] = zv[i];
          z[i * nv + v] = zv[i];
          acc[0] = A::add(acc[0], A::prod(rv[i], zv[i]));
          acc[1] = A::add(acc[1], A::prod(rv[i], rv[i]));
        }
      }
    } else {
      for (int f = f0 + (int)threadIdx.x; f < f1; f += kPcgThreads) {
        const int v = fv[f];
        R rv[3], zv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const R pv = staged ? sp[i * H + (v - cmin)] : pn[i * nv + v];
          dx[i * nv + v] += alpha * pv;
          rv[i] = r[i * nv + v] - alpha * q[i * nv + v];
          r[i * nv + v] = rv[i];
        }
        const R m0 = Minv[v], m1 = Minv[nv + v], m2 = Minv[2 * nv + v];
        const R m3 = Minv[3 * nv + v], m4 = Minv[4 * nv + v], m5 = Minv[5 * nv + v];
        zv[0] = m0 * rv[0] + m3 * rv[1] + m5 * rv[2];
        zv[1] = m3 * rv[0] + m1 * rv[1] + m4 * rv[2];
        zv[2] = m5 * rv[0] + m4 * rv[1] + m2 * rv[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          z[i * nv + v] = zv[i];
          acc[0] = A::add(acc[0], A::prod(rv[i], zv[i]));
          acc[1] = A::add(acc[1], A::prod(rv[i], rv[i]));
        }
      }
    }
    cluster_push<R, 2>(acc, s_red, s_all, 1, cluster, rank, CS);
    cluster.sync();
    if (wid == 0) {
      const AT x = cluster_total<R>(s_all, 1, CS);
      const AT y = cluster_total<R>(s_all, 2, CS);
      if (threadIdx.x == 0) {
        const double rr = A::to_double(y);
        s_coef = A::positive(s_at[0]) ? (R)A::ratio(x, s_at[0]) : R(0);
        s_at[0] = x;
        s_sc[0] = rr;
        s_flag = (rr <= s_sc[1] || !A::positive(s_at[1]) || !isfinite(rr) || it + 1 >= cap) ? 1 : 0;
      }
    }
    __syncthreads();
    beta = s_coef;
    done = s_flag != 0;
    ++it;
    __syncthreads();  // s_coef / s_flag are rewritten in the next iteration
  }
  if (res)
    for (int idx = (int)threadIdx.x; idx < nf; idx += kPcgThreads) {
      const int v = lst[idx];
#pragma unroll
      for (int i = 0; i < 3; ++i) dx[i * nv + v] = dxs[i * nf + idx];
    }
  if (rank == 0 && threadIdx.x == 0) {
    Scalars* sc = ev.sc;
    const double rr = s_sc[0], pq = A::to_double(s_at[1]);
    sc->pcg_iters = it;
    sc->pcg_capped = (it >= cap && !(rr <= s_sc[1])) ? 1 : 0;
    sc->rz = A::to_double(s_at[0]);
    sc->rr = rr;
    sc->pq = pq;
    sc->pcg_tol2 = s_sc[1];
    sc->pcg_done = 1;
    if (!isfinite(rr) || !isfinite(pq)) sc->status |= ST_NONFINITE;
  }
  // no CTA may leave while another can still write into its shared memory
  cluster.sync();
}

// Launch shape of the PCG kernel: cluster size (CTAs per env) and threads
// per CTA.  The dynamic shared memory of a CTA is the SM's share for the
// CTAs it holds (one of 1024 threads or two of 512) less the static part.
// The shape in use is process-wide per precision (so an env's result does
// not depend on when or with whom it is stepped): the largest co-schedulable
// cluster of 1024-thread CTAs unless tc_pcg_shape / tc_autotune_pcg chose
// another.
template <class R, int NT> static PcgShape pcg_probe(int cs) {
  PcgShape sh;
  sh.cs = cs;
  sh.threads = NT;
  int dev = 0, optin = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k_pcg_cluster<R, NT>);
  const int ctas = 1024 / NT;
  sh.smem = std::max(0, std::min(optin, per_sm / ctas - 1024) - (int)fa.sharedSizeBytes - 1024);
  cudaFuncSetAttribute(k_pcg_cluster<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem);
  if (cs > 8) cudaFuncSetAttribute(k_pcg_cluster<R, NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sh.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster<R, NT>, &cfg) != cudaSuccess) n = 0;
  sh.coresident = n;
  cudaGetLastError();
  return sh;
}

template <class R> static PcgShape pcg_probe_any(int cs, int threads) {
  return threads == 512 ? pcg_probe<R, 512>(cs) : pcg_probe<R, 1024>(cs);
}

template <class R> struct PcgSel {
  std::mutex mu;
  bool set = false;
  PcgShape cur;
};
template <class R> static PcgSel<R>& pcg_sel() {
  static PcgSel<R> sel;
  return sel;
}

template <class R> PcgShape pcg_shape() {
  PcgSel<R>& sel = pcg_sel<R>();
  std::lock_guard<std::mutex> lk(sel.mu);
  if (!sel.set) {
    sel.cur = pcg_probe_any<R>(16, 1024);
    if (sel.cur.coresident <= 0) sel.cur = pcg_probe_any<R>(8, 1024);
    sel.set = true;
    if (trace_on())
      std::fprintf(stderr, "[tc] pcg shape: %d CTAs x %d threads, %d co-resident clusters, %d B shared per CTA\n",
                   sel.cur.cs, sel.cur.threads, sel.cur.coresident, sel.cur.smem);
  }
  return sel.cur;
}

template <class R> tc_status set_pcg_shape(int cs, int threads) {
  if (cs < 1 || cs > kPcgMaxCluster || (threads != 512 && threads != 1024)) return TC_ERR_INVALID_ARG;
  const PcgShape sh = pcg_probe_any<R>(cs, threads);
  if (sh.coresident <= 0) return TC_ERR_CAPACITY;
  PcgSel<R>& sel = pcg_sel<R>();
  std::lock_guard<std::mutex> lk(sel.mu);
  sel.cur = sh;
  sel.set = true;
  return TC_OK;
}

template <class R> tc_status b_pcg(const BatchHost<R>& b, int max_iter, bool warm, cudaStream_t s) {
  if (warm && b.units[K_VGRP] > 0) {
    TC_LAUNCH("k_pcg_warm", s, k_pcg_warm<R><<<b.units[K_VGRP], kBlock, 0, s>>>(b.bv, b.L));
    TC_LAUNCH("k_pcg_warm_env", s, k_pcg_warm_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
  }
  if (b.units[K_VERT] > 0)
    TC_LAUNCH("k_pcg_init", s, k_pcg_init<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, b.L, warm ? 1 : 0));
  TC_LAUNCH("k_pcg_init_env", s, k_pcg_init_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
  const PcgShape sh = pcg_shape<R>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b.nenv * sh.cs));
  cfg.blockDim = dim3((unsigned)sh.threads);
  cfg.dynamicSmemBytes = (size_t)sh.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)sh.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err = cudaSuccess;
  if (sh.threads == 512)
    TC_LAUNCH("k_pcg_cluster", s, err = cudaLaunchKernelEx(&cfg, k_pcg_cluster<R, 512>, b.bv, b.L, max_iter, sh.smem));
  else
    TC_LAUNCH("k_pcg_cluster", s, err = cudaLaunchKernelEx(&cfg, k_pcg_cluster<R, 1024>, b.bv, b.L, max_iter, sh.smem));
  return err == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

// ------------------------------------------------------ per-env reductions

// max-norm of dx -> pmax, and g.dx (minus twice the Newton decrement):
// partials per K_VERT unit (the PCG's r.z / r.r regions, free again once the
// PCG has run), folded per env in unit order
template <class R>
__global__ void __launch_bounds__(kBlock) k_pmax(const BatchView<R> bv, PartLayout L) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  double m = 0.0, gd = 0.0;
  if (v < e.nv)
    for (int i = 0; i < 3; ++i) {
      const double d = (double)e.dx[i * e.nv + v];
      m = fmax(m, fabs(d));
      gd += (double)e.g[i * e.nv + v] * d;
    }
  m = block_max<kBlock>(m);
  gd = block_sum<kBlock>(gd);
  if (threadIdx.x == 0) {
    bv.part[L.rz + blockIdx.x] = m;
    bv.part[L.rr + blockIdx.x] = gd;
  }
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_pmax_env(const BatchView<R> bv, PartLayout L) {
  const int env = blockIdx.x;
  const EnvView<R>& e = bv.views[env];
  const int* p = bv.prefix + K_VERT * (bv.nenv + 1);
  double m = 0.0;
  for (int u = p[env] + threadIdx.x; u < p[env + 1]; u += blockDim.x) m = fmax(m, bv.part[L.rz + u]);
  m = block_max<kBlock>(m);
  const double gd = env_unit_sum(bv, K_VERT, env, bv.part + L.rr);
  if (threadIdx.x == 0) {
    e.sc->pmax = m;
    e.sc->reduce_tmp[3] = gd;
    if (!isfinite(m)) e.sc->status |= ST_NONFINITE;
  }
}

template <class R> void b_pmax(const BatchHost<R>& b, cudaStream_t s) {
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_pmax", s, k_pmax<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv, b.L));
  TC_LAUNCH("k_pmax_env", s, k_pmax_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
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

// dx *= param (per env): the continuation of an accepted step along its
// direction, whose length the CCD pass that follows then bounds
template <class R>
__global__ void __launch_bounds__(kBlock) k_scale_dx(const BatchView<R> bv) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const R f = (R)bv.param[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  if (v < e.nv)
    for (int i = 0; i < 3; ++i) e.dx[i * e.nv + v] *= f;
}

template <class R> void b_scale_dx(const BatchHost<R>& b, cudaStream_t s) {
  if (b.units[K_VERT] > 0) TC_LAUNCH("k_scale_dx", s, k_scale_dx<R><<<b.units[K_VERT], kBlock, 0, s>>>(b.bv));
}

// mode 0 (step start): u0 = u and, when dynamic, utilde = u + dt vel;
// mode 1 (step end, dynamic): vel = (u - u0) / dt;
// mode 2 (substep start, dynamic): dx = param (utilde - u0), the substep's
// share of the inertial increment (the predictor direction)
template <class R>
__global__ void __launch_bounds__(kBlock) k_step_vectors(const BatchView<R> bv, int mode) {
  const Loc l = locate(bv.prefix, bv.nenv, K_VERT, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const int v = l.chunk * kBlock + threadIdx.x;
  if (v >= e.nv) return;
  for (int i = 0; i < 3; ++i) {
    const int k = i * e.nv + v;
    if (mode == 2) {
      e.dx[k] = (R)bv.param[l.env] * (e.utilde[k] - e.u0[k]);
    } else if (mode == 0) {
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
  template tc_status b_pcg<R>(const BatchHost<R>&, int, bool, cudaStream_t);        \
  template void b_pmax<R>(const BatchHost<R>&, cudaStream_t);                 \
  template void b_trial<R>(const BatchHost<R>&, cudaStream_t);                \
  template void b_scale_dx<R>(const BatchHost<R>&, cudaStream_t);             \
  template void b_step_vectors<R>(const BatchHost<R>&, int, cudaStream_t);    \
  template PcgShape pcg_shape<R>();                                           \
  template tc_status set_pcg_shape<R>(int, int);
TC_INST(float)
TC_INST(double)
#undef TC_INST

}  // namespace tc
