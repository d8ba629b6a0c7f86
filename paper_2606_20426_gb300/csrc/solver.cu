// Newton-step kernels: per-vertex assembly (K4), matrix-free block-Jacobi
// PCG (K5), energy reductions for the line search (K7), step updates.
//
// Assembly and SpMV are atomic-free: element and contact passes write their
// per-element / per-primitive contributions to slots, and one thread per
// vertex sums its incident slots through fixed incidence lists, so results
// do not depend on scheduling.  All dot products accumulate in double;
// block partials are combined in a fixed order by every block that needs the
// scalar (no separate finalize launch).
#include <cooperative_groups.h>

#include "env.cuh"
#include "prof.cuh"

namespace cg = cooperative_groups;

namespace tc {

// ------------------------------------------------------------------ helpers

// Sum of partials[0..n) in a fixed order, computed by every block that needs
// it (n is a few hundred at most per env phase).
TC_D double sum_partials(const double* part, int n, int stride = 1, int offset = 0) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[(int64_t)i * stride + offset];
  return block_sum<kBlock>(s);
}

__shared__ double s_bcast;

TC_D double bcast(double v) {
  if (threadIdx.x == 0) s_bcast = v;
  __syncthreads();
  const double r = s_bcast;
  __syncthreads();
  return r;
}

// Per-vertex gathers are done by a group of kLanes consecutive lanes: each
// lane sums every kLanes-th incidence and the group combines the partial sums
// with a fixed shuffle tree (deterministic), which gives the gathers kLanes
// times more independent loads in flight than one thread per vertex.
constexpr int kLanes = 8;

template <class T> TC_D T group_sum(T v) {
#pragma unroll
  for (int o = kLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kLanes);
  return v;
}

TC_HD int round_up(int n, int m) { return (n + m - 1) / m * m; }

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

// ---------------------------------------------------------------- assembly
// g_v = sum of element and contact gradient slots (+ inertia), 3x3 diagonal
// block -> inverse for block-Jacobi.  part layout: [0..nb) gnorm2, [nb..2nb)
// inertia energy.
template <class R>
__global__ void __launch_bounds__(kBlock) k_assemble(const EnvView<R> e, double* part) {
  const int lane = threadIdx.x & (kLanes - 1);
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) / kLanes;
  const bool valid = v < e.nv;
  double gn2 = 0.0, ein = 0.0;
  const int nt = e.nt, nv = e.nv;
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
        const int code = e.cv_edge_idx[k], p = code >> 2, l = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.ce_slot[(int64_t)(3 * l + i) * e.nec + p];
        add_packed_block<R>(D, e.ce_slot + 6 * (int64_t)e.nec, e.nec, p, l, 6);
      }
      for (int k = e.cv_face_off[s] + lane; k < e.cv_face_off[s + 1]; k += kLanes) {
        const int code = e.cv_face_idx[k], p = code >> 2, l = code & 3;
        for (int i = 0; i < 3; ++i) g[i] += e.cf_slot[(int64_t)(3 * l + i) * e.nfc + p];
        add_packed_block<R>(D, e.cf_slot + 9 * (int64_t)e.nfc, e.nfc, p, l, 9);
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
    if (e.mass) {  // inertia 1/(2h^2) |u - u_tilde|_M^2
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
    part[blockIdx.x] = gn2;
    part[gridDim.x + blockIdx.x] = ein;
  }
}

// total energy = elastic partials + contact partials + inertia partials
__global__ void k_energy_total(const double* part_elem, int ne, const double* part_contact, int nc,
                               const double* part_in, int ni, int in_stride_off, Scalars* sc, int write_gn2,
                               const double* part_gn2) {
  double s = 0.0;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) s += part_elem[i];
  for (int i = threadIdx.x; i < nc; i += blockDim.x) s += part_contact[2 * i];
  for (int i = threadIdx.x; i < ni; i += blockDim.x) s += part_in[in_stride_off + i];
  s = block_sum<kBlock>(s);
  double g = 0.0;
  if (write_gn2)
    for (int i = threadIdx.x; i < ni; i += blockDim.x) g += part_gn2[i];
  g = block_sum<kBlock>(g);
  double dm = 1e300;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) dm = fmin(dm, part_contact[2 * i + 1]);
  dm = block_min<kBlock>(dm);
  if (threadIdx.x == 0) {
    sc->energy = s;
    if (write_gn2) sc->gnorm2 = g;
    sc->reduce_tmp[1] = dm;  // min squared pair distance seen by the contact pass
    if (!isfinite(s)) sc->status |= ST_NONFINITE;
  }
}

static unsigned contact_blocks(int n) { return (unsigned)std::max(1, (n + 127) / 128); }

template <class R> static int n_contact_blocks(const EnvView<R>& e) {
  return (int)(contact_blocks(e.nvc) + contact_blocks(e.nec) + contact_blocks(e.nfc));
}

// part layout during assembly: [elem nb_t][contact 2*nc][assemble gn2 nb_v][assemble inertia nb_v]
template <class R> void launch_assemble(const EnvView<R>& e, cudaStream_t s) {
  const int nbt = (int)grid_for(e.nt), nc = n_contact_blocks(e);
  const int nba = (int)grid_for((int64_t)round_up(e.nv, kWarp / kLanes) * kLanes);
  double* pa = e.part + nbt + 2 * nc;
  TC_LAUNCH("k_assemble", s, k_assemble<R><<<nba, kBlock, 0, s>>>(e, pa));
  TC_LAUNCH("k_energy_total", s, k_energy_total<<<1, kBlock, 0, s>>>(e.part, nbt, e.part + nbt, nc, pa, nba, nba, e.sc, 1, pa));
}

// inertia energy only (line-search trial)
template <class R>
__global__ void __launch_bounds__(kBlock) k_inertia(const EnvView<R> e, const R* __restrict__ u, double* part) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double ein = 0.0;
  if (v < e.nv && e.mass) {
    const R mh = e.mass[v] * e.inv_h2;
    for (int i = 0; i < 3; ++i) {
      const double du = (double)u[i * e.nv + v] - (double)e.utilde[i * e.nv + v];
      ein += 0.5 * (double)mh * du * du;
    }
  }
  ein = block_sum<kBlock>(ein);
  if (threadIdx.x == 0) part[blockIdx.x] = ein;
}

template <class R> void launch_energy(const EnvView<R>& e, const R* u_eval, cudaStream_t s) {
  const int nbt = (int)grid_for(e.nt), nbv = (int)grid_for(e.nv), nc = n_contact_blocks(e);
  launch_elem<R>(e, false, u_eval, s);
  launch_contact<R>(e, false, u_eval, s);
  double* pa = e.part + nbt + 2 * nc;
  TC_LAUNCH("k_inertia", s, k_inertia<R><<<nbv, kBlock, 0, s>>>(e, u_eval, pa));
  TC_LAUNCH("k_energy_total", s, k_energy_total<<<1, kBlock, 0, s>>>(e.part, nbt, e.part + nbt, nc, pa, nbv, 0, e.sc, 0, nullptr));
}

// --------------------------------------------------------------------- PCG
// Layout of e.part during PCG: [0, nbv) p.q; [nbv, 2 nbv) r.z; [2 nbv, 3 nbv) r.r

template <class R> TC_D void apply_minv(const EnvView<R>& e, int v, const R r[3], R z[3]) {
  const int nv = e.nv;
  const R m0 = e.Minv[v], m1 = e.Minv[nv + v], m2 = e.Minv[2 * nv + v];
  const R m3 = e.Minv[3 * nv + v], m4 = e.Minv[4 * nv + v], m5 = e.Minv[5 * nv + v];
  z[0] = m0 * r[0] + m3 * r[1] + m5 * r[2];
  z[1] = m3 * r[0] + m1 * r[1] + m4 * r[2];
  z[2] = m5 * r[0] + m4 * r[1] + m2 * r[2];
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_init(const EnvView<R> e) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
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
  const int nbv = gridDim.x;
  if (threadIdx.x == 0) {
    e.part[nbv + blockIdx.x] = rz;
    e.part[2 * nbv + blockIdx.x] = rr;
  }
}

__global__ void k_pcg_init_scalars(const double* part, int nbv, Scalars* sc, double eta, int max_iter) {
  const double rz = sum_partials(part + nbv, nbv);
  const double rr = sum_partials(part + 2 * nbv, nbv);
  if (threadIdx.x == 0) {
    if (!isfinite(rz) || !isfinite(rr)) sc->status |= ST_NONFINITE;
    sc->rz = rz;
    sc->rz_next = rz;
    sc->rr = rr;
    sc->pcg_tol2 = eta * eta * sc->gnorm2;
    sc->pcg_done = (rr <= sc->pcg_tol2 || max_iter <= 0) ? 1 : 0;
    sc->pcg_iters = 0;
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

template <class R>
__global__ void __launch_bounds__(kBlock) k_spmv_elem(const EnvView<R> e) {
  if (e.sc->pcg_done) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) e.sc->rz = e.sc->rz_next;
  const int el = blockIdx.x * blockDim.x + threadIdx.x;
  if (el < e.nt) spmv_elem_one<R>(e, el);
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

template <class R> TC_D void spmv_contact_one(const EnvView<R>& e, int i) {
  if (i < e.nvc) {
    const int v[1] = {e.cverts[i]};
    contact_spmv_prim<R, 1>(e, e.cv_slot, e.nvc, i, v, e.cv_y);
  } else if (i < e.nvc + e.nec) {
    const int p = i - e.nvc;
    const int v[2] = {e.cedges[p], e.cedges[e.nec + p]};
    contact_spmv_prim<R, 2>(e, e.ce_slot, e.nec, p, v, e.ce_y);
  } else if (i < e.nvc + e.nec + e.nfc) {
    const int p = i - e.nvc - e.nec;
    const int v[3] = {e.cfaces[p], e.cfaces[e.nfc + p], e.cfaces[2 * e.nfc + p]};
    contact_spmv_prim<R, 3>(e, e.cf_slot, e.nfc, p, v, e.cf_y);
  }
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_spmv_contact(const EnvView<R> e) {
  if (e.sc->pcg_done) return;
  spmv_contact_one<R>(e, blockIdx.x * blockDim.x + threadIdx.x);
}

// q = A p at vertex v gathered by a lane group; returns p.q on the group's
// lane 0 (0 elsewhere).  Every lane of the warp calls it (valid may differ
// per group).
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

// Per-iteration kernels (used when a cooperative launch is unavailable).
// Partials: part[0, nbq) p.q, part[nbq, nbq + nbv) r.z, then r.r.
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_q(const EnvView<R> e) {
  if (e.sc->pcg_done) return;
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) / kLanes;
  double pq = pcg_q_group<R>(e, v, v < e.nv);
  pq = block_sum<kBlock>(pq);
  if (threadIdx.x == 0) e.part[blockIdx.x] = pq;
}

// dx += alpha p, r -= alpha q, z = M^-1 r; partials r.z, r.r
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_update(const EnvView<R> e, int nbq) {
  if (e.sc->pcg_done) return;
  const int nbv = gridDim.x;
  const double pq = bcast(sum_partials(e.part, nbq));
  const double alpha = pq > 0.0 ? e.sc->rz / pq : 0.0;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int nv = e.nv;
  double rz = 0.0, rr = 0.0;
  if (v < nv) {
    R r[3], z[3];
    for (int i = 0; i < 3; ++i) {
      e.dx[i * nv + v] += (R)alpha * e.p[i * nv + v];
      r[i] = e.r[i * nv + v] - (R)alpha * e.q[i * nv + v];
      e.r[i * nv + v] = r[i];
    }
    apply_minv<R>(e, v, r, z);
    for (int i = 0; i < 3; ++i) {
      e.z[i * nv + v] = z[i];
      rz += (double)r[i] * (double)z[i];
      rr += (double)r[i] * (double)r[i];
    }
  }
  rz = block_sum<kBlock>(rz);
  rr = block_sum<kBlock>(rr);
  if (threadIdx.x == 0) {
    e.part[nbq + blockIdx.x] = rz;
    e.part[nbq + nbv + blockIdx.x] = rr;
    if (blockIdx.x == 0) e.sc->pq = pq;
  }
}

// beta = rz_new / rz; p = z + beta p; convergence flag (block 0 writes)
template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_p(const EnvView<R> e, int max_iter, int nbq) {
  if (e.sc->pcg_done) return;
  const int nbv = gridDim.x;
  const double rz_new = bcast(sum_partials(e.part + nbq, nbv));
  const double rr = bcast(sum_partials(e.part + nbq + nbv, nbv));
  const double rz_old = e.sc->rz;
  const double beta = rz_old > 0.0 ? rz_new / rz_old : 0.0;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int nv = e.nv;
  if (v < nv)
    for (int i = 0; i < 3; ++i) e.p[i * nv + v] = e.z[i * nv + v] + (R)beta * e.p[i * nv + v];
  // sc->rz is read by every block above, so the new value goes to rz_next;
  // k_spmv_elem (next iteration, where nobody reads rz) moves it into rz.
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scalars* sc = e.sc;
    sc->rz_next = rz_new;
    sc->rr = rr;
    sc->pcg_iters += 1;
    if (rr <= sc->pcg_tol2 || sc->pcg_iters >= max_iter || !(sc->pq > 0.0) || !isfinite(rr)) sc->pcg_done = 1;
  }
}

// ------------------------------------------------------ persistent PCG
// All iterations in one cooperative launch: grid-stride element / contact
// SpMV, per-vertex gather, then the vector updates, separated by grid-wide
// barriers (four per iteration).  Each block sums the per-block partials in
// the same fixed order, so alpha, beta and the stopping test are identical in
// every block and no scalar is shared through global memory mid-iteration.
// Partials: part[0, G) p.q, part[G, 2G) r.z, part[2G, 3G) r.r (G = gridDim.x).

TC_D double sum_part_all(const double* part, int n) {
  // every thread of the block gets the same value
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = block_sum<kBlock>(s);
  return bcast(s);
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_pcg_persistent(const EnvView<R> e, int max_iter) {
  cg::grid_group grid = cg::this_grid();
  const int G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = G * blockDim.x;
  const int nv = e.nv, nc = e.nvc + e.nec + e.nfc;
  const int nv_pad = round_up(nv, kWarp / kLanes);
  double rz = e.sc->rz;
  const double tol2 = e.sc->pcg_tol2;
  int it = 0;
  bool done = e.sc->pcg_done != 0;
  double rr = e.sc->rr, pq = 0.0;
  while (!done && it < max_iter) {
    for (int el = tid; el < e.nt; el += nth) spmv_elem_one<R>(e, el);
    for (int i = tid; i < nc; i += nth) spmv_contact_one<R>(e, i);
    grid.sync();
    double lpq = 0.0;
    for (int v = tid / kLanes; v < nv_pad; v += nth / kLanes) lpq += pcg_q_group<R>(e, v, v < nv);
    lpq = block_sum<kBlock>(lpq);
    if (threadIdx.x == 0) e.part[blockIdx.x] = lpq;
    grid.sync();
    pq = sum_part_all(e.part, G);
    const double alpha = pq > 0.0 ? rz / pq : 0.0;
    double lrz = 0.0, lrr = 0.0;
    for (int v = tid; v < nv; v += nth) {
      R r[3], z[3];
      for (int i = 0; i < 3; ++i) {
        e.dx[i * nv + v] += (R)alpha * e.p[i * nv + v];
        r[i] = e.r[i * nv + v] - (R)alpha * e.q[i * nv + v];
        e.r[i * nv + v] = r[i];
      }
      apply_minv<R>(e, v, r, z);
      for (int i = 0; i < 3; ++i) {
        e.z[i * nv + v] = z[i];
        lrz += (double)r[i] * (double)z[i];
        lrr += (double)r[i] * (double)r[i];
      }
    }
    lrz = block_sum<kBlock>(lrz);
    lrr = block_sum<kBlock>(lrr);
    if (threadIdx.x == 0) {
      e.part[G + blockIdx.x] = lrz;
      e.part[2 * G + blockIdx.x] = lrr;
    }
    grid.sync();
    const double rz_new = sum_part_all(e.part + G, G);
    rr = sum_part_all(e.part + 2 * G, G);
    const double beta = rz > 0.0 ? rz_new / rz : 0.0;
    rz = rz_new;
    ++it;
    done = rr <= tol2 || !(pq > 0.0) || !isfinite(rr);
    if (!done && it < max_iter) {
      for (int v = tid; v < nv; v += nth)
        for (int i = 0; i < 3; ++i) e.p[i * nv + v] = e.z[i * nv + v] + (R)beta * e.p[i * nv + v];
      grid.sync();
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!isfinite(rr) || !isfinite(pq)) e.sc->status |= ST_NONFINITE;
    e.sc->pcg_iters = it;
    e.sc->rz = rz;
    e.sc->rr = rr;
    e.sc->pq = pq;
    e.sc->pcg_done = 1;
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
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<R>, kBlock, 0);
      cached = coop ? sms * per_sm : 0;
    }
    return cached;
  }
};

// Runs the whole PCG solve; returns false if a cooperative launch is not
// available (the caller then uses the per-iteration kernels).
template <class R> bool launch_pcg_persistent(const EnvView<R>& e, int max_iter, cudaStream_t s) {
  const int cap = CoopInfo<R>::max_blocks();
  if (cap <= 0) return false;
  const int64_t work = std::max<int64_t>(e.nt, std::max<int64_t>(e.nv, e.nvc + e.nec + e.nfc));
  int G = (int)std::min<int64_t>((work + kBlock - 1) / kBlock, cap);
  G = std::max(G, 1);
  // 3 G partials must fit: part holds at least 3 * grid_for(nv) + the element blocks
  G = std::min(G, (int)(grid_for(e.nt) + grid_for(e.nv)));
  EnvView<R> ev = e;
  int mi = max_iter;
  void* args[] = {(void*)&ev, (void*)&mi};
  cudaError_t err;
  TC_LAUNCH("k_pcg_persistent", s,
            err = cudaLaunchCooperativeKernel((void*)k_pcg_persistent<R>, dim3(G), dim3(kBlock), args, 0, s));
  return err == cudaSuccess;
}

template <class R> void launch_pcg_init(const EnvView<R>& e, double eta, cudaStream_t s) {
  const int nbv = (int)grid_for(e.nv);
  TC_LAUNCH("k_pcg_init", s, k_pcg_init<R><<<nbv, kBlock, 0, s>>>(e));
  TC_LAUNCH("k_pcg_init_scalars", s, k_pcg_init_scalars<<<1, kBlock, 0, s>>>(e.part, nbv, e.sc, eta, 1 << 30));
}

template <class R> void launch_pcg_iter(const EnvView<R>& e, int max_iter, cudaStream_t s) {
  const int nbv = (int)grid_for(e.nv);
  TC_LAUNCH("k_spmv_elem", s, k_spmv_elem<R><<<grid_for(e.nt), kBlock, 0, s>>>(e));
  const int nc = e.nvc + e.nec + e.nfc;
  if (nc > 0) TC_LAUNCH("k_spmv_contact", s, k_spmv_contact<R><<<grid_for(nc), kBlock, 0, s>>>(e));
  const int nbq = (int)grid_for((int64_t)round_up(e.nv, kWarp / kLanes) * kLanes);
  TC_LAUNCH("k_pcg_q", s, k_pcg_q<R><<<nbq, kBlock, 0, s>>>(e));
  TC_LAUNCH("k_pcg_update", s, k_pcg_update<R><<<nbv, kBlock, 0, s>>>(e, nbq));
  TC_LAUNCH("k_pcg_p", s, k_pcg_p<R><<<nbv, kBlock, 0, s>>>(e, max_iter, nbq));
}

// max-norm of dx -> sc->pmax, and g.dx (minus the Newton decrement)
// -> sc->reduce_tmp[3]
template <class R>
__global__ void k_pmax(const EnvView<R> e) {
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

template <class R> void launch_pmax(const EnvView<R>& e, cudaStream_t s) { k_pmax<R><<<1, kBlock, 0, s>>>(e); }

template <class R>
__global__ void k_axpy(int n3, R* out, const R* u, R alpha, const R* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) out[i] = u[i] + alpha * d[i];
}

template <class R> void launch_axpy_u(const EnvView<R>& e, R* out, const R* u, R alpha, const R* d, cudaStream_t s) {
  TC_LAUNCH("k_axpy", s, k_axpy<R><<<grid_for(3 * (int64_t)e.nv), kBlock, 0, s>>>(3 * e.nv, out, u, alpha, d));
}

// first line-search trial: alpha = min(1, TOI) read on the device
template <class R>
__global__ void k_trial(int n3, R* out, const R* u, const R* d, const Scalars* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const R alpha = (R)fmin(1.0, sc->ccd_t);
  if (i < n3) out[i] = u[i] + alpha * d[i];
}

template <class R> void launch_trial(const EnvView<R>& e, R* out, cudaStream_t s) {
  TC_LAUNCH("k_trial", s, k_trial<R><<<grid_for(3 * (int64_t)e.nv), kBlock, 0, s>>>(3 * e.nv, out, e.u, e.dx, e.sc));
}

#define TC_INST(R)                                                                              \
  template void launch_assemble<R>(const EnvView<R>&, cudaStream_t);                            \
  template void launch_energy<R>(const EnvView<R>&, const R*, cudaStream_t);                    \
  template void launch_pcg_init<R>(const EnvView<R>&, double, cudaStream_t);                    \
  template void launch_pcg_iter<R>(const EnvView<R>&, int, cudaStream_t);                       \
  template bool launch_pcg_persistent<R>(const EnvView<R>&, int, cudaStream_t);                 \
  template void launch_trial<R>(const EnvView<R>&, R*, cudaStream_t);                           \
  template void launch_pmax<R>(const EnvView<R>&, cudaStream_t);                                \
  template void launch_axpy_u<R>(const EnvView<R>&, R*, const R*, R, const R*, cudaStream_t);
TC_INST(float)
TC_INST(double)
#undef TC_INST

}  // namespace tc
