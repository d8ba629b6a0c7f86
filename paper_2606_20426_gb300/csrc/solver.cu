// Newton-step kernels over a batch of envs: per-vertex assembly (K4),
// matrix-free block-Jacobi PCG (K5), energies for the line search (K7) and
// step updates.
//
// Assembly and SpMV are atomic-free: element and contact passes write their
// per-element / per-primitive contributions to slots, and one lane group per
// vertex sums its incident slots through fixed incidence lists.  Every block
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

template <class R> struct Sym3 {
  R xx, yy, zz, xy, yz, zx;
};

template <class R> TC_D void add_packed_block(Sym3<R>& D, const R* slot, int64_t stride, int64_t prim, int l, int N) {
  const int b = 3 * l;
  D.xx += slot[(int64_t)sym_index(b + 0, b + 0, N) * stride + prim];
  D.yy += slot[(int64_t)sym_index(b + 1, b + 1, N) * stride + prim];
  D.zz += slot[(int64_t)sym_index(b + 2, b + 2, N) * stride + prim];
  D.xy += slot[(int64_t)sym_index(b + 0, b + 1, N) * stride + prim];
  D.yz += slot[(int64_t)sym_index(b + 1, b + 2, N) * stride + prim];
  D.zx += slot[(int64_t)sym_index(b + 2, b + 0, N) * stride + prim];
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
// g_v = sum of element and contact gradient slots (+ inertia), 3x3 diagonal
// block -> inverse for block-Jacobi.  Partials per K_VGRP unit: |g|^2 and the
// inertia energy 1/(2h^2)|u - u_tilde|_M^2.
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
  Sym3<R> D{0, 0, 0, 0, 0, 0};
  if (valid) {
    for (int k = e.vt_off[v] + lane; k < e.vt_off[v + 1]; k += kLanes) {
      const int code = e.vt_idx[k];
      const int el = code >> 2, c = code & 3;
      for (int i = 0; i < 3; ++i) g[i] += e.eslot[(int64_t)(3 * c + i) * nt + el];
      const R* ds = e.eslot + (int64_t)(12 + 6 * c) * nt + el;
      D.xx += ds[0];
      D.yy += ds[(int64_t)nt];
      D.zz += ds[2 * (int64_t)nt];
      D.xy += ds[3 * (int64_t)nt];
      D.yz += ds[4 * (int64_t)nt];
      D.zx += ds[5 * (int64_t)nt];
    }
    const int s = e.vslot[v];
    if (s >= 0) {
      if (lane == 0) {
        for (int i = 0; i < 3; ++i) g[i] += e.cv_slot[(int64_t)i * e.nvc + s];
        add_packed_block<R>(D, e.cv_slot + 3 * (int64_t)e.nvc, e.nvc, s, 0, 3);
      }
      for (int k = e.cv_edge_off[s] + lane; k < e.cv_edge_off[s + 1]; k += kLanes) {
        const int code = e.cv_edge_idx[k], p = code >> 2, q = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.ce_slot[(int64_t)(3 * q + i) * e.nec + p];
        add_packed_block<R>(D, e.ce_slot + 6 * (int64_t)e.nec, e.nec, p, q, 6);
      }
      for (int k = e.cv_face_off[s] + lane; k < e.cv_face_off[s + 1]; k += kLanes) {
        const int code = e.cv_face_idx[k], p = code >> 2, q = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.cf_slot[(int64_t)(3 * q + i) * e.nfc + p];
        add_packed_block<R>(D, e.cf_slot + 9 * (int64_t)e.nfc, e.nfc, p, q, 9);
      }
    }
  }
  for (int i = 0; i < 3; ++i) g[i] = group_sum(g[i]);
  D.xx = group_sum(D.xx);
  D.yy = group_sum(D.yy);
  D.zz = group_sum(D.zz);
  D.xy = group_sum(D.xy);
  D.yz = group_sum(D.yz);
  D.zx = group_sum(D.zx);
  if (valid && lane == 0) {
    if (e.mass) {
      const R mh = e.mass[v] * e.inv_h2;
      for (int i = 0; i < 3; ++i) {
        const R du = e.u[i * nv + v] - e.utilde[i * nv + v];
        g[i] += mh * du;
        ein += 0.5 * (double)mh * (double)du * (double)du;
      }
      D.xx += mh;
      D.yy += mh;
      D.zz += mh;
    }
    R M[6] = {0, 0, 0, 0, 0, 0};
    if (e.fixed[v]) {
      g[0] = g[1] = g[2] = R(0);
    } else {
      // inverse of the symmetric 3x3 block (adjugate / det)
      const R c00 = D.yy * D.zz - D.yz * D.yz, c01 = D.yz * D.zx - D.xy * D.zz, c02 = D.xy * D.yz - D.yy * D.zx;
      const R det = D.xx * c00 + D.xy * c01 + D.zx * c02;
      if (det > R(0) && isfinite((double)det)) {
        const R id = R(1) / det;
        M[0] = c00 * id;
        M[1] = (D.xx * D.zz - D.zx * D.zx) * id;
        M[2] = (D.xx * D.yy - D.xy * D.xy) * id;
        M[3] = c01 * id;
        M[4] = (D.xy * D.zx - D.xx * D.yz) * id;
        M[5] = c02 * id;
      } else {
        const R tr = D.xx + D.yy + D.zz;
        const R d = tr > R(0) ? R(3) / tr : R(1);
        M[0] = M[1] = M[2] = d;
      }
    }
    bool finite = true;
    for (int i = 0; i < 3; ++i) {
      e.g[i * nv + v] = g[i];
      gn2 += (double)g[i] * (double)g[i];
      finite = finite && isfinite((double)g[i]);
    }
    for (int i = 0; i < 6; ++i) {
      e.Minv[(int64_t)i * nv + v] = M[i];
      finite = finite && isfinite((double)M[i]);
    }
    if (!finite) atomicOr(&e.sc->status, ST_NONFINITE);
  }
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

// per env: r.z, r.r and the squared stopping tolerance (param[env]) ->
// published scalars
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
    double* es = bv.part + L.env_s + 8 * env;
    es[0] = 0.0;
    es[1] = 0.0;
    es[2] = rz;
    es[3] = rr;
    es[4] = 0.0;
    es[5] = (rr <= tol2) ? 1.0 : 0.0;
    es[6] = 0.0;
    es[7] = tol2;
  }
}

// element share of A p: y_e = V D^T H9 D p_e  (12 per tet)
template <class R> TC_D void spmv_elem_one(const EnvView<R>& e, int el) {
  const int nt = e.nt, nv = e.nv;
  const int4 t = e.tets[el];
  const int v[4] = {t.x, t.y, t.z, t.w};
  R Bm[3][3];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 3; ++j) Bm[a][j] = e.Dminv[(int64_t)(a * 3 + j) * nt + el];
  R Dp[3][3];
  for (int i = 0; i < 3; ++i) {
    const R p0 = e.p[i * nv + v[0]];
    for (int a = 0; a < 3; ++a) Dp[i][a] = e.p[i * nv + v[a + 1]] - p0;
  }
  R f[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) f[3 * i + j] = Dp[i][0] * Bm[0][j] + Dp[i][1] * Bm[1][j] + Dp[i][2] * Bm[2][j];
  R y[9];
  for (int a = 0; a < 9; ++a) y[a] = R(0);
  int idx = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
#pragma unroll
    for (int b = a; b < 9; ++b) {
      const R h = e.H9[(int64_t)(idx++) * nt + el];
      y[a] += h * f[b];
      if (b != a) y[b] += h * f[a];
    }
  }
  const R V = e.vol[el];
  for (int i = 0; i < 3; ++i) {
    R s0 = 0;
    for (int a = 0; a < 3; ++a) {
      const R ya = V * (y[3 * i + 0] * Bm[a][0] + y[3 * i + 1] * Bm[a][1] + y[3 * i + 2] * Bm[a][2]);
      e.yslot[(int64_t)(3 * (a + 1) + i) * nt + el] = ya;
      s0 += ya;
    }
    e.yslot[(int64_t)i * nt + el] = -s0;
  }
}

// contact share of A p per primitive: y = H_prim p_prim
template <class R, int NGP>
TC_D void contact_spmv_prim(const EnvView<R>& e, const R* slot, int n, int prim, const int* verts, R* yout) {
  constexpr int NG = 3 * NGP;
  R x[NG];
  for (int l = 0; l < NGP; ++l)
    for (int i = 0; i < 3; ++i) x[3 * l + i] = e.p[i * e.nv + verts[l]];
  R y[NG];
  for (int a = 0; a < NG; ++a) y[a] = R(0);
  int idx = NG;
  for (int a = 0; a < NG; ++a)
    for (int b = a; b < NG; ++b) {
      const R h = slot[(int64_t)(idx++) * n + prim];
      y[a] += h * x[b];
      if (b != a) y[b] += h * x[a];
    }
  for (int a = 0; a < NG; ++a) yout[(int64_t)a * n + prim] = y[a];
}

template <class R> TC_D void spmv_contact_one(const EnvView<R>& e, int kind, int i) {
  if (kind == K_CV) {
    if (i >= e.nvc) return;
    const int v[1] = {e.cverts[i]};
    contact_spmv_prim<R, 1>(e, e.cv_slot, e.nvc, i, v, e.cv_y);
  } else if (kind == K_CE) {
    if (i >= e.nec) return;
    const int v[2] = {e.cedges[i], e.cedges[e.nec + i]};
    contact_spmv_prim<R, 2>(e, e.ce_slot, e.nec, i, v, e.ce_y);
  } else {
    if (i >= e.nfc) return;
    const int v[3] = {e.cfaces[i], e.cfaces[e.nfc + i], e.cfaces[2 * e.nfc + i]};
    contact_spmv_prim<R, 3>(e, e.cf_slot, e.nfc, i, v, e.cf_y);
  }
}

// q = A p at vertex v gathered by a lane group; returns p.q on the group's
// lane 0 (0 elsewhere).  Every lane of the warp calls it.
template <class R> TC_D double pcg_q_group(const EnvView<R>& e, int v, bool valid) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int nv = e.nv, nt = e.nt;
  R q[3] = {0, 0, 0};
  const bool act = valid && !e.fixed[v];
  if (act) {
    for (int k = e.vt_off[v] + lane; k < e.vt_off[v + 1]; k += kLanes) {
      const int code = e.vt_idx[k];
      const int el = code >> 2, c = code & 3;
      for (int i = 0; i < 3; ++i) q[i] += e.yslot[(int64_t)(3 * c + i) * nt + el];
    }
    const int s = e.vslot[v];
    if (s >= 0) {
      if (lane == 0)
        for (int i = 0; i < 3; ++i) q[i] += e.cv_y[(int64_t)i * e.nvc + s];
      for (int k = e.cv_edge_off[s] + lane; k < e.cv_edge_off[s + 1]; k += kLanes) {
        const int code = e.cv_edge_idx[k], p = code >> 2, l = code & 3;
        for (int i = 0; i < 3; ++i) q[i] += e.ce_y[(int64_t)(3 * l + i) * e.nec + p];
      }
      for (int k = e.cv_face_off[s] + lane; k < e.cv_face_off[s + 1]; k += kLanes) {
        const int code = e.cv_face_idx[k], p = code >> 2, l = code & 3;
        for (int i = 0; i < 3; ++i) q[i] += e.cf_y[(int64_t)(3 * l + i) * e.nfc + p];
      }
    }
  }
  for (int i = 0; i < 3; ++i) q[i] = group_sum(q[i]);
  double pq = 0.0;
  if (valid && lane == 0) {
    if (act && e.mass) {
      const R mh = e.mass[v] * e.inv_h2;
      for (int i = 0; i < 3; ++i) q[i] += mh * e.p[i * nv + v];
    }
    for (int i = 0; i < 3; ++i) {
      e.q[i * nv + v] = q[i];
      pq += (double)e.p[i * nv + v] * (double)q[i];
    }
  }
  return pq;
}

// ------------------------------------------------------ persistent PCG
// All CG iterations of all envs of the batch in one cooperative launch.  Per
// iteration: element + contact SpMV | gather q = A p (p.q partials) | per-env
// alpha | vector update (r.z, r.r partials) | per-env beta and stop test |
// direction update, with grid-wide syncs between the phases.  Per-env scalars
// are folded by one block per env and published through global memory before
// the next sync, so every block reads the same values; converged envs skip
// their work while the others continue.  Published scalars, 8 per env at
// part + env_s: alpha, beta, r.z, r.r, p.q, done (0 running, 1 stopped before
// the iteration, 2 stopped in it), iterations, tolerance^2.

template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_batched(const BatchView<R> bv, PartLayout L, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x;
  const int nenv = bv.nenv;
  double* es = bv.part + L.env_s;
  const int* pre = bv.prefix;
  const int nT = pre[K_TET * (nenv + 1) + nenv];
  const int nC[3] = {pre[K_CV * (nenv + 1) + nenv], pre[K_CE * (nenv + 1) + nenv], pre[K_CF * (nenv + 1) + nenv]};
  const int nG = pre[K_VGRP * (nenv + 1) + nenv];
  const int nV = pre[K_VERT * (nenv + 1) + nenv];
  for (int it = 0; it < max_iter; ++it) {
    int all_done = 1;
    for (int env = 0; env < nenv; ++env) all_done &= es[8 * env + 5] != 0.0;
    if (all_done) break;
    // 1. SpMV
    for (int u = blockIdx.x; u < nT; u += G) {
      const Loc l = locate(pre, nenv, K_TET, u);
      if (es[8 * l.env + 5] != 0.0) continue;
      const EnvView<R>& e = bv.views[l.env];
      const int el = l.chunk * kBlock + threadIdx.x;
      if (el < e.nt) spmv_elem_one<R>(e, el);
    }
    for (int k = 0; k < 3; ++k)
      for (int u = blockIdx.x; u < nC[k]; u += G) {
        const Loc l = locate(pre, nenv, K_CV + k, u);
        if (es[8 * l.env + 5] != 0.0) continue;
        if (threadIdx.x < unit_items(K_CV + k))
          spmv_contact_one<R>(bv.views[l.env], K_CV + k, l.chunk * unit_items(K_CV + k) + threadIdx.x);
      }
    grid.sync();
    // 2. gather q = A p; partial p.q per unit
    for (int u = blockIdx.x; u < nG; u += G) {
      const Loc l = locate(pre, nenv, K_VGRP, u);
      double pq = 0.0;
      if (es[8 * l.env + 5] == 0.0) {
        const EnvView<R>& e = bv.views[l.env];
        const int v = l.chunk * 32 + threadIdx.x / kLanes;
        pq = pcg_q_group<R>(e, v, v < e.nv);
      }
      pq = block_sum<kBlock>(pq);
      if (threadIdx.x == 0) bv.part[L.pq + u] = pq;
    }
    grid.sync();
    // 3. per-env alpha = r.z / p.q
    for (int env = blockIdx.x; env < nenv; env += G) {
      const double pq = env_unit_sum(bv, K_VGRP, env, bv.part + L.pq);
      if (threadIdx.x == 0 && es[8 * env + 5] == 0.0) {
        es[8 * env + 4] = pq;
        es[8 * env + 0] = pq > 0.0 ? es[8 * env + 2] / pq : 0.0;
      }
    }
    grid.sync();
    // 4. dx += alpha p, r -= alpha q, z = M^-1 r; partials r.z, r.r
    for (int u = blockIdx.x; u < nV; u += G) {
      const Loc l = locate(pre, nenv, K_VERT, u);
      double rz = 0.0, rr = 0.0;
      if (es[8 * l.env + 5] == 0.0) {
        const EnvView<R>& e = bv.views[l.env];
        const int nv = e.nv;
        const int v = l.chunk * kBlock + threadIdx.x;
        const R alpha = (R)es[8 * l.env + 0];
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
    grid.sync();
    // 5. per-env beta and stop test
    for (int env = blockIdx.x; env < nenv; env += G) {
      const double rz_new = env_unit_sum(bv, K_VERT, env, bv.part + L.rz);
      const double rr = env_unit_sum(bv, K_VERT, env, bv.part + L.rr);
      if (threadIdx.x == 0 && es[8 * env + 5] == 0.0) {
        const double rz_old = es[8 * env + 2];
        es[8 * env + 1] = rz_old > 0.0 ? rz_new / rz_old : 0.0;
        es[8 * env + 2] = rz_new;
        es[8 * env + 3] = rr;
        es[8 * env + 6] += 1.0;
        const double pq = es[8 * env + 4];
        const bool done = rr <= es[8 * env + 7] || !(pq > 0.0) || !isfinite(rr) || es[8 * env + 6] >= max_iter;
        es[8 * env + 5] = done ? 2.0 : 0.0;
      }
    }
    grid.sync();
    // 6. p = z + beta p for envs still running
    for (int u = blockIdx.x; u < nV; u += G) {
      const Loc l = locate(pre, nenv, K_VERT, u);
      if (es[8 * l.env + 5] != 0.0) continue;
      const EnvView<R>& e = bv.views[l.env];
      const int nv = e.nv;
      const int v = l.chunk * kBlock + threadIdx.x;
      const R beta = (R)es[8 * l.env + 1];
      if (v < nv)
        for (int i = 0; i < 3; ++i) e.p[i * nv + v] = e.z[i * nv + v] + beta * e.p[i * nv + v];
    }
    grid.sync();
  }
  // publish per-env results
  for (int env = blockIdx.x; env < nenv; env += G)
    if (threadIdx.x == 0) {
      Scalars* sc = bv.views[env].sc;
      sc->pcg_iters = (int)es[8 * env + 6];
      sc->rz = es[8 * env + 2];
      sc->rr = es[8 * env + 3];
      sc->pq = es[8 * env + 4];
      sc->pcg_tol2 = es[8 * env + 7];
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
  int work = std::max(b.units[K_TET], std::max(b.units[K_VGRP], b.units[K_VERT]));
  work = std::max(work, std::max(b.nenv, b.units[K_CV] + b.units[K_CE] + b.units[K_CF]));
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
