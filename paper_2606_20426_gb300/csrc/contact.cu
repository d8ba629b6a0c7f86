// Contact (K2 query, K3 barrier, K6 CCD, K11 force).
//
// The indenter is rigid, so its primitives are binned once, in its body
// frame, into a uniform grid (built at scene setup).  Every Newton iteration
// each gel contact primitive (vertex, edge, face) maps its points into the
// body frame, walks the grid cells its padded box overlaps, and visits each
// indenter primitive once (in the cell holding the low corner of the
// intersection of the two boxes).  The pairs are
//   gel vertex  - indenter triangle   (point-triangle, gel slot 0)
//   gel face    - indenter vertex     (point-triangle, gel slots 1, 2, 3)
//   gel edge    - indenter edge       (edge-edge, gel slots 0, 1, mollified)
// and every pair with d < dhat contributes kappa * b(d) (Li et al. 2020).
//
// Precision: the body-frame coordinates of a pair are formed in FP64
// relative to the primitive's first gel point and rounded once, so the pair
// arithmetic runs in the kernel type R on small numbers; pairs closer than
// 1e-2 dhat are redone in FP64.
//
// Hessian: each pair adds kappa J^T [d2f]_+ J, where f is the barrier as a
// function of the distance d (and, for edge-edge pairs, of the mollifier
// argument c), J stacks the gradients of d and c on the gel points, and
// [.]_+ clamps the 1x1 or 2x2 Hessian of f to PSD in closed form.  This is
// PSD by construction and needs no eigensolver; it drops the curvature of
// d itself, which only changes the Newton path, not the minimiser.
//
// One thread owns one gel primitive and sums its pairs in registers, so the
// result per primitive is deterministic and the per-vertex assembly needs no
// atomics.
#include "env.cuh"
#include "geom.cuh"
#include "prof.cuh"
#include "solver.cuh"

namespace tc {

TC_D void to_body(const double* Rm, const double* tr, const double* x, double* b) {
  const double dx = x[0] - tr[0], dy = x[1] - tr[1], dz = x[2] - tr[2];
  b[0] = Rm[0] * dx + Rm[3] * dy + Rm[6] * dz;
  b[1] = Rm[1] * dx + Rm[4] * dy + Rm[7] * dz;
  b[2] = Rm[2] * dx + Rm[5] * dy + Rm[8] * dz;
}

// gel primitive kinds
enum { GV = 0, GE = 1, GF = 2 };
// indenter primitive kind queried by each gel kind: vertex->faces, edge->edges, face->vertices
TC_HD int ind_kind_for(int gk) { return gk == GV ? 2 : (gk == GE ? 1 : 0); }

template <class R> TC_D int prim_count(const EnvView<R>& e, int gk) { return gk == GV ? e.nvc : (gk == GE ? e.nec : e.nfc); }

template <class R> TC_D int gel_vertex(const EnvView<R>& e, int gk, int prim, int l) {
  if (gk == GV) return e.cverts[prim];
  if (gk == GE) return e.cedges[l * e.nec + prim];
  return e.cfaces[l * e.nfc + prim];
}

template <class R> TC_D void gel_world(const EnvView<R>& e, const R* u, int v, double* x) {
  for (int d = 0; d < 3; ++d) x[d] = e.X0[d * e.nv + v] + (double)u[d * e.nv + v];
}

template <class R> TC_D int ind_vertex(const EnvView<R>& e, int ik, int prim, int l) {
  if (ik == 0) return prim;
  if (ik == 1) return e.IE[l * e.ind_ne + prim];
  return e.IF[l * e.ind_nf + prim];
}

// Origin of a primitive's local frame (its first gel point, body frame) in
// FP64 and as an FP32 hi/lo pair.
struct Origin {
  double d[3];
  float hi[3], lo[3];
};

TC_D Origin make_origin(const double* o) {
  Origin r;
  for (int k = 0; k < 3; ++k) {
    r.d[k] = o[k];
    r.hi[k] = __double2float_rn(o[k]);
    r.lo[k] = __double2float_rn(o[k] - (double)r.hi[k]);
  }
  return r;
}

// indenter vertex v in the body frame relative to the origin: FP64
// difference rounded once (double path), or the same difference formed from
// FP32 hi/lo pairs without FP64 instructions (float path; both hi parts are
// close to each other, so hi - hi is exact)
template <class T, class R> TC_D Vec3<T> ind_rel(const EnvView<R>& e, int v, const Origin& o) {
  const int n = e.ind_nv;
  if constexpr (sizeof(T) == 4) {
    return v3<T>((e.IVhi[v] - o.hi[0]) + (e.IVlo[v] - o.lo[0]), (e.IVhi[n + v] - o.hi[1]) + (e.IVlo[n + v] - o.lo[1]),
                 (e.IVhi[2 * n + v] - o.hi[2]) + (e.IVlo[2 * n + v] - o.lo[2]));
  } else {
    return v3<T>((T)(e.IV[v] - o.d[0]), (T)(e.IV[n + v] - o.d[1]), (T)(e.IV[2 * n + v] - o.d[2]));
  }
}

template <class T> TC_D Vec3<T> rel(const double* b, const double* o) {
  return v3<T>((T)(b[0] - o[0]), (T)(b[1] - o[1]), (T)(b[2] - o[2]));
}

// Visit the indenter primitives of kind ik whose boxes overlap the FP32
// body-frame query box [lo, hi]; f(prim) is called once per primitive.
template <class R, class F> TC_D void grid_visit(const EnvView<R>& e, int ik, const float* lo, const float* hi, F f) {
  const GridView& g = e.grid;
  const float cell = 1.0f / g.inv_cell;
  for (int d = 0; d < 3; ++d)
    if (hi[d] < g.org[d] || lo[d] > g.org[d] + g.dims[d] * cell) return;
  int c0[3], c1[3];
  for (int d = 0; d < 3; ++d) {
    c0[d] = grid_cell(lo[d], g.org[d], g.inv_cell, g.dims[d]);
    c1[d] = grid_cell(hi[d], g.org[d], g.inv_cell, g.dims[d]);
  }
  const int32_t* start = g.start[ik];
  const int32_t* items = g.items[ik];
  const float* box = g.box[ik];
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const int cell_id = x + g.dims[0] * (y + g.dims[1] * z);
        const int k1 = start[cell_id + 1];
        for (int k = start[cell_id]; k < k1; ++k) {
          const int p = items[k];
          const float* b = box + 6 * (int64_t)p;
          if (b[0] > hi[0] || b[1] > hi[1] || b[2] > hi[2] || b[3] < lo[0] || b[4] < lo[1] || b[5] < lo[2]) continue;
          // visit in the cell of the low corner of the intersection box
          if (grid_cell(fmaxf(lo[0], b[0]), g.org[0], g.inv_cell, g.dims[0]) != x ||
              grid_cell(fmaxf(lo[1], b[1]), g.org[1], g.inv_cell, g.dims[1]) != y ||
              grid_cell(fmaxf(lo[2], b[2]), g.org[2], g.inv_cell, g.dims[2]) != z)
            continue;
          f(p);
        }
      }
}

// The same visit by a group of NL consecutive lanes that share one query box:
// the lanes take a cell's items NL at a time and a ballot over the group
// compacts the hits, so write(pos, prim) receives the primitives in exactly
// the order of grid_visit.  Every lane of the group must call it.  Returns the
// number of primitives found.
template <int NL, class R, class W>
TC_D int grid_collect(const EnvView<R>& e, int ik, const float* lo, const float* hi, W write) {
  const GridView& g = e.grid;
  const float cell = 1.0f / g.inv_cell;
  for (int d = 0; d < 3; ++d)
    if (hi[d] < g.org[d] || lo[d] > g.org[d] + g.dims[d] * cell) return 0;
  const int lane = (int)(threadIdx.x & 31) % NL;
  const int base = (int)(threadIdx.x & 31) - lane;
  const unsigned gmask = ((NL == 32) ? 0xffffffffu : ((1u << NL) - 1u)) << base;
  int c0[3], c1[3];
  for (int d = 0; d < 3; ++d) {
    c0[d] = grid_cell(lo[d], g.org[d], g.inv_cell, g.dims[d]);
    c1[d] = grid_cell(hi[d], g.org[d], g.inv_cell, g.dims[d]);
  }
  const int32_t* start = g.start[ik];
  const int32_t* items = g.items[ik];
  const float* box = g.box[ik];
  int cnt = 0;
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const int cell_id = x + g.dims[0] * (y + g.dims[1] * z);
        const int k0 = start[cell_id], k1 = start[cell_id + 1];
        for (int kb = k0; kb < k1; kb += NL) {
          const int k = kb + lane;
          bool hit = false;
          int p = -1;
          if (k < k1) {
            p = items[k];
            const float* b = box + 6 * (int64_t)p;
            hit = !(b[0] > hi[0] || b[1] > hi[1] || b[2] > hi[2] || b[3] < lo[0] || b[4] < lo[1] || b[5] < lo[2]) &&
                  grid_cell(fmaxf(lo[0], b[0]), g.org[0], g.inv_cell, g.dims[0]) == x &&
                  grid_cell(fmaxf(lo[1], b[1]), g.org[1], g.inv_cell, g.dims[1]) == y &&
                  grid_cell(fmaxf(lo[2], b[2]), g.org[2], g.inv_cell, g.dims[2]) == z;
          }
          const unsigned gm = (__ballot_sync(gmask, hit) & gmask) >> base;
          if (hit) write(cnt + __popc(gm & ((1u << lane) - 1u)), p);
          cnt += __popc(gm);
        }
      }
  return cnt;
}

// Mollifier of an edge-edge pair in its dimensionless argument
// t = c / eps_x, c = |(x1-x0) x (x3-x2)|^2: m(t) = (2 - t) t for t < 1, its
// first two derivatives in t, and grad t on the gel edge (points 0, 1).
// Working in t keeps every factor in range (1/eps_x^2 overflows FP32).
template <class T> TC_D void mollifier_t(const Vec3<T>* x, T eps_x, T* m, T* mt, T* mtt, T* gt) {
  const Vec3<T> u = x[1] - x[0], v = x[3] - x[2];
  const T uu = dot(u, u), vv = dot(v, v), uv = dot(u, v);
  const T c = uu * vv - uv * uv;
  const T t = c / eps_x;
  if (!(t < T(1))) {
    *m = T(1);
    *mt = *mtt = T(0);
    for (int i = 0; i < 6; ++i) gt[i] = T(0);
    return;
  }
  *m = (T(2) - t) * t;
  *mt = T(2) - T(2) * t;
  *mtt = T(-2);
  const T s = T(2) / eps_x;
  const T gu[3] = {s * (vv * u.x - uv * v.x), s * (vv * u.y - uv * v.y), s * (vv * u.z - uv * v.z)};
  for (int j = 0; j < 3; ++j) {
    gt[j] = -gu[j];
    gt[3 + j] = gu[j];
  }
}

// Barrier of one pair in arithmetic T.  Adds kappa * grad to g[NG] and the
// PSD Gauss-Newton block to the packed upper triangle Hp[NG(NG+1)/2].
template <class T, int NG>
TC_D T pair_gn(int kind, const Vec3<T>* x, const int* gs, T dhat, T kappa, bool ee, T eps_x, bool hess, T* g,
               T* Hp) {
  int which;
  const T d2 = pair_dist2<T>(kind, x, &which);
  const T d = sqrt(d2);
  if (!(d < dhat) || !(d > T(0)) || which < 0) return T(0);
  T b, b1, b2;
  barrier3<T>(d, dhat, &b, &b1, &b2);
  T m = T(1), mt = T(0), mtt = T(0);
  T gt[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  if (NG == 6 && ee) mollifier_t<T>(x, eps_x, &m, &mt, &mtt, gt);
  if (!hess) return kappa * m * b;
  const CandEval<T> ev = eval_cand<T>(kind == 0 ? c_pt_cand[which] : c_ee_cand[which], x);
  const T id = T(1) / d;
  T gd[NG];
#pragma unroll
  for (int s = 0; s < NG / 3; ++s) {
    const T w = ev.w[gs[s]] * id;
    gd[3 * s + 0] = w * ev.r.x;
    gd[3 * s + 1] = w * ev.r.y;
    gd[3 * s + 2] = w * ev.r.z;
  }
  if (NG == 6 && ee && mt != T(0)) {
    // f(d, t) = m(t) b(d): 2x2 Hessian in (d, t), clamped to PSD
    const T a = m * b2, bb = mt * b1, c = mtt * b;
    const T tr = T(0.5) * (a + c), df = T(0.5) * (a - c);
    const T disc = sqrt(df * df + bb * bb);
    const T l1 = tr + disc, l2 = tr - disc;
    T P00 = T(0), P01 = T(0), P11 = T(0);
    if (disc > T(0)) {
      // unit eigenvector of l1: (l1 - c, bb), or (bb, l1 - a) when that vanishes
      T v1x = df + disc, v1y = bb;
      if (fabs(v1x) + fabs(v1y) == T(0)) { v1x = bb; v1y = disc - df; }
      const T nv = sqrt(v1x * v1x + v1y * v1y);
      v1x /= nv;
      v1y /= nv;
      const T v2x = -v1y, v2y = v1x;
      const T L1 = l1 > T(0) ? l1 : T(0), L2 = l2 > T(0) ? l2 : T(0);
      P00 = L1 * v1x * v1x + L2 * v2x * v2x;
      P01 = L1 * v1x * v1y + L2 * v2x * v2y;
      P11 = L1 * v1y * v1y + L2 * v2y * v2y;
    } else {
      P00 = a > T(0) ? a : T(0);
      P11 = c > T(0) ? c : T(0);
    }
    int idx = 0;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      g[i] += kappa * (m * b1 * gd[i] + mt * b * gt[i]);
#pragma unroll
      for (int j = i; j < NG; ++j)
        Hp[idx++] += kappa * (P00 * gd[i] * gd[j] + P01 * (gd[i] * gt[j] + gt[i] * gd[j]) + P11 * gt[i] * gt[j]);
    }
  } else {
    const T s1 = kappa * m * b1, s2 = kappa * m * (b2 > T(0) ? b2 : T(0));
    int idx = 0;
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      g[i] += s1 * gd[i];
#pragma unroll
      for (int j = i; j < NG; ++j) Hp[idx++] += s2 * gd[i] * gd[j];
    }
  }
  return kappa * m * b;
}

// Pair points of gel primitive gk with indenter primitive ip, relative to o.
template <class T, class R, int GK>
TC_D void pair_points(const EnvView<R>& e, const Vec3<T>* xg, int ip, const Origin& o, Vec3<T>* x) {
  constexpr int ik = GK == GV ? 2 : (GK == GE ? 1 : 0);
  if (GK == GV) {
    x[0] = xg[0];
    for (int l = 0; l < 3; ++l) x[1 + l] = ind_rel<T>(e, ind_vertex(e, ik, ip, l), o);
  } else if (GK == GF) {
    x[0] = ind_rel<T>(e, ip, o);
    for (int l = 0; l < 3; ++l) x[1 + l] = xg[l];
  } else {
    x[0] = xg[0];
    x[1] = xg[1];
    for (int l = 0; l < 2; ++l) x[2 + l] = ind_rel<T>(e, ind_vertex(e, ik, ip, l), o);
  }
}

// Body-frame points of gel primitive `prim` at displacement u, relative to the
// origin o of its first point.
template <class R, int GK>
TC_D void contact_prim_points(const EnvView<R>& e, const R* u, int prim, double bw[3][3], Origin* o) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  for (int l = 0; l < NGP; ++l) {
    double w[3];
    gel_world(e, u, gel_vertex(e, GK, prim, l), w);
    to_body(e.Rm, e.tr, w, bw[l]);
  }
  *o = make_origin(bw[0]);
}

// Pairs per chunk of the pass with slots, and its dynamic shared memory.
template <class R> constexpr int contact_chunk() { return sizeof(R) == 4 ? 512 : 256; }
template <class R, int GK> constexpr size_t contact_smem() {
  constexpr int NG = 3 * (GK == GV ? 1 : (GK == GE ? 2 : 3));
  return (size_t)contact_chunk<R>() * (NG + NG * (NG + 1) / 2) * sizeof(R);
}

// One contact primitive pass over the candidate lists built by the last CCD
// pass.  MODE 0: energy only; 1: energy + slots.  One unit = 128 gel
// primitives; the unit's (primitive, candidate) pairs are flattened and
// spread over all threads of the block, in chunks.  With MODE 1 each pair
// writes its gradient and Hessian to shared memory, and the thread owning a
// primitive then adds its pairs in candidate order (fixed-order sums, no
// atomics) before rotating the sums to the world frame into the slots.
// In place: s_off[1..128] holds 128 counts on entry (stored before a block
// barrier) and their inclusive prefix sums on exit (s_off[0] stays 0).
// Warps 0-3 scan one count per lane (integer sums: the same as a serial
// pass).  Needs at least 128 threads; ends with a block barrier.
TC_D void prefix128(int* s_off) {
  __shared__ int s_w4[4];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int incl = 0;
  if (t < 128) {
    incl = s_off[t + 1];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) s_w4[w] = incl;
  }
  __syncthreads();
  if (t < 128) {
    int off = 0;
    for (int k = 0; k < w; ++k) off += s_w4[k];
    s_off[t + 1] = off + incl;
  }
  __syncthreads();
}

// ------------------------------------------------------------ friction
// Lagged IPC friction (Li et al. 2020) with the friction ratio and velocity
// threshold of Sec. III-B.  At the start of each indenter substep every
// candidate pair within dhat (at the converged gel state and the pre-advance
// pose) fixes its normal force lambda = kappa m(c) |b'(d)|, the world-frame
// unit normal n of its closest-point vector r = sum_i w_i x_i, and the
// weights w (all in FP64, rounded once).  During the substep's Newton solve
// the pair adds mu lambda f0(y), y = |P rel|, P = I - n n^T, rel = sum_i w_i
// (x_i - x_i^t) the closest points' relative displacement since the step
// start (gel points: u - u0; indenter points: (R - R0) V + (t - t0)), with
// f0 the C1 smoothing of |.| below eps_x = eps_v dt.  Gradient w.r.t. rel:
// mu lambda (f1 / y) P rel; Hessian mu lambda [(f1 / y) P + (f1' y - f1) / y^3
// u u^T], PSD (eigenvalues f1' >= 0 along u, f1 / y across it, 0 along n).

// slot of gel point l in the pair's 4 points, and the indenter slots
template <int GK> TC_HD int gel_pair_slot(int l) { return GK == GF ? 1 + l : l; }

template <class R, int GK>
TC_D void friction_lag_prim(const EnvView<R>& e, int prim) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  const int n = prim_count(e, GK);
  const int kind = GK == GE ? 1 : 0;
  const int kept = min(e.cand_n[GK][prim], e.cand_cap);
  int cnt = 0;
  if (kept > 0) {
    double bw[3][3];
    Origin o;
    contact_prim_points<R, GK>(e, e.u, prim, bw, &o);
    Vec3<double> xg[NGP];
    for (int l = 0; l < NGP; ++l) xg[l] = rel<double>(bw[l], o.d);
    for (int j = 0; j < kept; ++j) {
      const int ip = e.cand[GK][(int64_t)j * n + prim];
      Vec3<double> x[4];
      pair_points<double, R, GK>(e, xg, ip, o, x);
      int which;
      const double d = sqrt(pair_dist2<double>(kind, x, &which));
      if (!(d < e.dhat) || !(d > 0.0) || which < 0) continue;
      double b, b1, b2;
      barrier3<double>(d, e.dhat, &b, &b1, &b2);
      double m = 1.0;
      if (GK == GE) {
        double mt, mtt, gt[6];
        mollifier_t<double>(x, 1e-3 * e.gel_elen2[prim] * e.ind_elen2[ip], &m, &mt, &mtt, gt);
      }
      const CandEval<double> ev = eval_cand<double>(kind == 0 ? c_pt_cand[which] : c_ee_cand[which], x);
      const double rn = sqrt(ev.r.x * ev.r.x + ev.r.y * ev.r.y + ev.r.z * ev.r.z);
      if (!(rn > 0.0)) continue;
      const double nb[3] = {ev.r.x / rn, ev.r.y / rn, ev.r.z / rn};
      double vals[8];
      vals[0] = e.kappa * m * (-b1);
      for (int i = 0; i < 3; ++i)  // body -> world
        vals[1 + i] = e.Rm[3 * i + 0] * nb[0] + e.Rm[3 * i + 1] * nb[1] + e.Rm[3 * i + 2] * nb[2];
      for (int q = 0; q < 4; ++q) vals[4 + q] = ev.w[q];
      e.fr_ip[GK][(int64_t)cnt * n + prim] = ip;
      for (int q = 0; q < 8; ++q) e.fr_val[GK][((int64_t)8 * cnt + q) * n + prim] = (R)vals[q];
      ++cnt;
    }
  }
  e.fr_n[GK][prim] = cnt;
}

// one unit = 128 gel primitives of one kind; edges, faces, vertices in one launch
template <class R> __global__ void __launch_bounds__(128) k_friction_lag(const BatchView<R> bv, int ne, int nf) {
  int unit = blockIdx.x, gk;
  if (unit < ne) gk = GE;
  else if (unit < ne + nf) { gk = GF; unit -= ne; }
  else { gk = GV; unit -= ne + nf; }
  const Loc lc = locate(bv.prefix, bv.nenv, K_CV + gk, unit);
  const EnvView<R>& e = bv.views[lc.env];
  const int prim = lc.chunk * 128 + (int)threadIdx.x;
  if (e.mu_f <= R(0) || e.fr_n[gk] == nullptr) return;
  if (gk == GE) { if (prim < e.nec) friction_lag_prim<R, GE>(e, prim); }
  else if (gk == GF) { if (prim < e.nfc) friction_lag_prim<R, GF>(e, prim); }
  else if (prim < e.nvc) friction_lag_prim<R, GV>(e, prim);
}

template <class R> void b_friction_lag(const BatchHost<R>& b, cudaStream_t s) {
  const int nv = b.units[K_CV], ne = b.units[K_CE], nf = b.units[K_CF];
  if (nv + ne + nf == 0) return;
  TC_LAUNCH("k_friction_lag", s, k_friction_lag<R><<<nv + ne + nf, 128, 0, s>>>(b.bv, ne, nf));
}

// Friction of gel primitive `prim` at displacement u: returns its energy and,
// with MODE 1, adds its gradient and Hessian, rotated into the indenter's
// body frame, to the primitive's accumulators (which the caller rotates back).
template <class R, int GK, int MODE>
TC_D double friction_prim(const EnvView<R>& e, const R* __restrict__ u, int prim, R* gacc, R* hacc) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  constexpr int NG = 3 * NGP;
  const int n = prim_count(e, GK);
  const int nv = e.nv;
  const int cnt = e.fr_n[GK][prim];
  R dg[NGP][3];
  for (int l = 0; l < NGP; ++l) {
    const int v = gel_vertex(e, GK, prim, l);
    for (int d = 0; d < 3; ++d) dg[l][d] = u[d * nv + v] - e.u0[d * nv + v];
  }
  double dR[9];
  for (int k = 0; k < 9; ++k) dR[k] = e.Rm[k] - e.Rm0[k];
  const double dt3[3] = {e.tr[0] - e.tr0[0], e.tr[1] - e.tr0[1], e.tr[2] - e.tr0[2]};
  const R mu = e.mu_f, ex = e.eps_x;
  const int ik = GK == GV ? 2 : (GK == GE ? 1 : 0);
  const int nind = GK == GV ? 3 : (GK == GE ? 2 : 1);
  const int ind_slot0 = GK == GV ? 1 : (GK == GE ? 2 : 0);
  double energy = 0.0;
  for (int j = 0; j < cnt; ++j) {
    const int ip = e.fr_ip[GK][(int64_t)j * n + prim];
    R val[8];
    for (int q = 0; q < 8; ++q) val[q] = e.fr_val[GK][((int64_t)8 * j + q) * n + prim];
    const R lam = val[0];
    const R nw[3] = {val[1], val[2], val[3]};
    R relv[3] = {R(0), R(0), R(0)};
    for (int l = 0; l < NGP; ++l) {
      const R w = val[4 + gel_pair_slot<GK>(l)];
      for (int d = 0; d < 3; ++d) relv[d] += w * dg[l][d];
    }
    for (int l = 0; l < nind; ++l) {
      const int iv = ind_vertex(e, ik, ip, l);
      const double V[3] = {e.IV[iv], e.IV[e.ind_nv + iv], e.IV[2 * e.ind_nv + iv]};
      const R w = val[4 + ind_slot0 + l];
      for (int d = 0; d < 3; ++d)
        relv[d] += w * (R)(dR[3 * d] * V[0] + dR[3 * d + 1] * V[1] + dR[3 * d + 2] * V[2] + dt3[d]);
    }
    const R un = relv[0] * nw[0] + relv[1] * nw[1] + relv[2] * nw[2];
    R ut[3];
    for (int d = 0; d < 3; ++d) ut[d] = relv[d] - un * nw[d];
    const R y = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    const R ml = mu * lam;
    const R f0 = y < ex ? (-y * y * y / (R(3) * ex * ex) + y * y / ex + ex / R(3)) : y;
    energy += (double)(ml * f0);
    if (MODE != 1) continue;
    const R a = ml * (y < ex ? (R(2) / ex - y / (ex * ex)) : R(1) / y);  // mu lambda f1 / y
    const R c = y > R(0) ? ml * (y < ex ? -R(1) / (y * ex * ex) : -R(1) / (y * y * y)) : R(0);
    // world gradient w.r.t. rel and Hessian M = a P + c ut ut^T, rotated to the body frame
    R gw[3], M[3][3];
    for (int i = 0; i < 3; ++i) {
      gw[i] = a * ut[i];
      for (int k = 0; k < 3; ++k) M[i][k] = a * ((i == k ? R(1) : R(0)) - nw[i] * nw[k]) + c * ut[i] * ut[k];
    }
    R Rm[9];
    for (int k = 0; k < 9; ++k) Rm[k] = (R)e.Rm[k];
    R gb[3], T1[3][3], Mb[3][3];
    for (int i = 0; i < 3; ++i) gb[i] = Rm[i] * gw[0] + Rm[3 + i] * gw[1] + Rm[6 + i] * gw[2];  // R^T g
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) T1[i][k] = Rm[i] * M[0][k] + Rm[3 + i] * M[1][k] + Rm[6 + i] * M[2][k];  // R^T M
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) Mb[i][k] = T1[i][0] * Rm[k] + T1[i][1] * Rm[3 + k] + T1[i][2] * Rm[6 + k];  // (R^T M) R
    R wl[NGP];
    for (int l = 0; l < NGP; ++l) wl[l] = val[4 + gel_pair_slot<GK>(l)];
    for (int la = 0; la < NGP; ++la) {
      for (int i = 0; i < 3; ++i) gacc[3 * la + i] += wl[la] * gb[i];
      for (int lb = la; lb < NGP; ++lb) {
        const R s = wl[la] * wl[lb];
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) {
            const int ra = 3 * la + i, cb = 3 * lb + k;
            if (ra > cb) continue;
            hacc[sym_index(ra, cb, NG)] += s * Mb[i][k];
          }
      }
    }
  }
  return energy;
}

template <class R, int GK, int MODE>
TC_D void contact_unit(const BatchView<R>& bv, const PartLayout& L, int trial, int unit) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  constexpr int NG = 3 * NGP;
  constexpr int NH = NG * (NG + 1) / 2;
  // a unit's pairs are spread over 512 threads; with slots, each pair's
  // gradient and Hessian go through dynamic shared memory in chunks of CH
  constexpr int NT = 512;
  constexpr int CH = MODE == 1 ? contact_chunk<R>() : NT;  // pairs per chunk
  __shared__ int s_off[129];
  extern __shared__ __align__(16) unsigned char s_dyn_contact[];
  R(*s_gh)[NG + NH] = reinterpret_cast<R(*)[NG + NH]>(s_dyn_contact);
  __shared__ Origin s_o[128];
  __shared__ Vec3<R> s_xg[128][NGP];
  const Loc lc = locate(bv.prefix, bv.nenv, K_CV + GK, unit);
  const EnvView<R>& e = bv.views[lc.env];
  const R* __restrict__ u = trial ? e.ut : e.u;
  double* part_out = bv.part + L.cont[GK];
  const int base = lc.chunk * 128;
  const int n = prim_count(e, GK);
  const int32_t* cl = e.cand[GK];
  const int mine = base + (int)threadIdx.x;
  const int kept = (threadIdx.x < 128 && mine < n) ? min(e.cand_n[GK][mine], e.cand_cap) : 0;
  if (kept > 0) {  // the primitive's FP64 geometry, once, for all its pairs
    double bw[3][3];
    Origin o;
    contact_prim_points<R, GK>(e, u, mine, bw, &o);
    s_o[threadIdx.x] = o;
    for (int l = 0; l < NGP; ++l) s_xg[threadIdx.x][l] = rel<R>(bw[l], o.d);
  }
  if (threadIdx.x == 0) s_off[0] = 0;
  if (threadIdx.x < 128) s_off[threadIdx.x + 1] = kept;
  __syncthreads();
  prefix128(s_off);
  const int total = s_off[128];
  double energy = 0.0;
  double dmin2 = 1e300;
  R gacc[MODE == 1 ? NG : 1];
  R hacc[MODE == 1 ? NH : 1];
  if (MODE == 1) {
#pragma unroll
    for (int a = 0; a < NG; ++a) gacc[a] = R(0);
#pragma unroll
    for (int a = 0; a < NH; ++a) hacc[a] = R(0);
  }
  const int kind = GK == GE ? 1 : 0;
  int gs[3];
  if (GK == GV) { gs[0] = 0; gs[1] = 0; gs[2] = 0; }
  else if (GK == GE) { gs[0] = 0; gs[1] = 1; gs[2] = 0; }
  else { gs[0] = 1; gs[1] = 2; gs[2] = 3; }
  const R dhat2 = (R)(e.dhat * e.dhat);
  for (int c0 = 0; c0 < total; c0 += CH) {
    for (int q = c0 + (int)threadIdx.x; q < total && q < c0 + CH; q += NT) {
      int lo_i = 0, hi_i = 127;  // last i with s_off[i] <= q
      while (lo_i < hi_i) {
        const int mid = (lo_i + hi_i + 1) >> 1;
        if (s_off[mid] <= q) lo_i = mid;
        else hi_i = mid - 1;
      }
      const int prim = base + lo_i, j = q - s_off[lo_i];
      R* gp = MODE == 1 ? &s_gh[q - c0][0] : nullptr;
      R* hp = MODE == 1 ? &s_gh[q - c0][NG] : nullptr;
      if (MODE == 1)
        for (int a = 0; a < NG + NH; ++a) s_gh[q - c0][a] = R(0);
      const Origin o = s_o[lo_i];
      Vec3<R> xg[NGP];
      for (int l = 0; l < NGP; ++l) xg[l] = s_xg[lo_i][l];
      const int ip = cl[(int64_t)j * n + prim];
      Vec3<R> x[4];
      pair_points<R, R, GK>(e, xg, ip, o, x);
      const R d2 = pair_dist2<R>(kind, x, nullptr);
      dmin2 = fmin(dmin2, (double)d2);
      if (!(d2 < dhat2)) continue;
      const double eps_x = GK == GE ? 1e-3 * e.gel_elen2[prim] * e.ind_elen2[ip] : 0.0;
      if (sizeof(R) == 4 && d2 < (R)(1e-4 * e.dhat * e.dhat)) {  // FP64 island for very close pairs
        double bw[3][3];
        Origin od;
        contact_prim_points<R, GK>(e, u, prim, bw, &od);
        Vec3<double> xgd[NGP];
        for (int l = 0; l < NGP; ++l) xgd[l] = rel<double>(bw[l], o.d);
        Vec3<double> xd[4];
        pair_points<double, R, GK>(e, xgd, ip, o, xd);
        double gd[MODE == 1 ? NG : 1], hd[MODE == 1 ? NH : 1];
        if (MODE == 1) {
          for (int a = 0; a < NG; ++a) gd[a] = 0.0;
          for (int a = 0; a < NH; ++a) hd[a] = 0.0;
        }
        energy += pair_gn<double, NG>(kind, xd, gs, e.dhat, e.kappa, GK == GE, eps_x, MODE == 1, gd, hd);
        if (MODE == 1) {
          for (int a = 0; a < NG; ++a) gp[a] = (R)gd[a];
          for (int a = 0; a < NH; ++a) hp[a] = (R)hd[a];
        }
      } else {
        energy += (double)pair_gn<R, NG>(kind, x, gs, (R)e.dhat, (R)e.kappa, GK == GE, (R)eps_x, MODE == 1, gp, hp);
      }
    }
    if (MODE == 1) {
      __syncthreads();
      if (kept > 0) {
        const int a0 = max(s_off[threadIdx.x], c0), a1 = min(s_off[threadIdx.x + 1], c0 + CH);
        for (int q = a0; q < a1; ++q) {
#pragma unroll
          for (int a = 0; a < NG; ++a) gacc[a] += s_gh[q - c0][a];
#pragma unroll
          for (int a = 0; a < NH; ++a) hacc[a] += s_gh[q - c0][NG + a];
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < 128 && mine < n && e.mu_f > R(0) && e.fr_n[GK] != nullptr && e.fr_n[GK][mine] > 0)
    energy += friction_prim<R, GK, MODE>(e, u, mine, gacc, hacc);
  if (MODE == 1 && threadIdx.x < 128 && mine < n) {
    const int prim = mine;
    // body -> world: g_w = R g_b per point, H_w = R H_b R^T per 3x3 block
    R Rm[9];
    for (int k = 0; k < 9; ++k) Rm[k] = (R)e.Rm[k];
    R* slot = GK == GV ? e.cv_slot : (GK == GE ? e.ce_slot : e.cf_slot);
    for (int l = 0; l < NGP; ++l)
      for (int i = 0; i < 3; ++i) {
        R s = 0;
        for (int k = 0; k < 3; ++k) s += Rm[3 * i + k] * gacc[3 * l + k];
        slot[(int64_t)(3 * l + i) * n + prim] = s;
      }
    for (int la = 0; la < NGP; ++la)
      for (int lb = la; lb < NGP; ++lb) {
        R B[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) B[i][j] = hacc[sym_index(3 * la + i, 3 * lb + j, NG)];
        R T1[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) T1[i][j] = Rm[3 * i + 0] * B[0][j] + Rm[3 * i + 1] * B[1][j] + Rm[3 * i + 2] * B[2][j];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const int ra = 3 * la + i, cb = 3 * lb + j;
            if (ra > cb) continue;  // packed upper triangle
            const R v = T1[i][0] * Rm[3 * j + 0] + T1[i][1] * Rm[3 * j + 1] + T1[i][2] * Rm[3 * j + 2];
            slot[(int64_t)(NG + sym_index(ra, cb, NG)) * n + prim] = v;
          }
      }
  }
  energy = block_sum<NT>(energy);
  dmin2 = block_min<NT>(dmin2);
  if (threadIdx.x == 0) {
    part_out[2 * unit] = energy;
    part_out[2 * unit + 1] = dmin2;
  }
}

// All three gel primitive kinds in one launch, the slowest kind (edges)
// first: blocks [0, ne) edges, then faces, then vertices.
template <class R, int MODE>
__global__ void __launch_bounds__(512) k_contact(const BatchView<R> bv, PartLayout L, int trial, int ne, int nf) {
  const int b = blockIdx.x;
  if (b < ne) contact_unit<R, GE, MODE>(bv, L, trial, b);
  else if (b < ne + nf) contact_unit<R, GF, MODE>(bv, L, trial, b - ne);
  else contact_unit<R, GV, MODE>(bv, L, trial, b - ne - nf);
}

template <class R> struct ContactGrid {
  static unsigned blocks(int n) { return (unsigned)std::max(1, (n + 127) / 128); }
};

// (energy, min d^2) per unit into the contact partial regions
template <class R> void b_contact(const BatchHost<R>& b, bool hess, bool trial, cudaStream_t s) {
  const int t = trial ? 1 : 0;
  const int nv = b.units[K_CV], ne = b.units[K_CE], nf = b.units[K_CF];
  const unsigned n = (unsigned)(nv + ne + nf);
  if (n == 0) return;
  constexpr size_t smem = std::max(contact_smem<R, GV>(), std::max(contact_smem<R, GE>(), contact_smem<R, GF>()));
  if (hess) {
    static const bool smem_set = [] {
      cudaFuncSetAttribute(k_contact<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      return true;
    }();
    (void)smem_set;
    TC_LAUNCH("k_contact", s, k_contact<R, 1><<<n, 512, smem, s>>>(b.bv, b.L, t, ne, nf));
  } else {
    TC_LAUNCH("k_contact_energy", s, k_contact<R, 0><<<n, 512, 0, s>>>(b.bv, b.L, t, ne, nf));
  }
}

// ------------------------------------------------------------------- CCD
// Gel points move linearly in the indenter's body frame from b0 to b1 (the
// indenter is static there); additive CCD per candidate pair in type R on
// coordinates relative to the primitive's first gel point.

// Swept geometry of one gel primitive in the indenter's body frame: start
// points b0, end points b1 and the FP32 box (outward-rounded, grown by dhat).
template <class R, int GK>
TC_D void ccd_prim_geom(const EnvView<R>& e, const Motion& mo, const R* dir, int prim, double b0[3][3],
                        double b1[3][3], float lo[3], float hi[3]) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  for (int d = 0; d < 3; ++d) {
    lo[d] = 3e38f;
    hi[d] = -3e38f;
  }
  for (int l = 0; l < NGP; ++l) {
    const int v = gel_vertex(e, GK, prim, l);
    double w[3];
    gel_world(e, e.u, v, w);
    to_body(mo.Ra, mo.ta, w, b0[l]);
    if (dir)
      for (int d = 0; d < 3; ++d) w[d] += (double)dir[d * e.nv + v];
    to_body(mo.Rb, mo.tb, w, b1[l]);
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __double2float_rd(fmin(b0[l][d], b1[l][d]) - e.dhat));
      hi[d] = fmaxf(hi[d], __double2float_ru(fmax(b0[l][d], b1[l][d]) + e.dhat));
    }
  }
}

// FP32 swept box of one gel primitive in the body frame for the broad phase:
// the FP64 geometry rounds to within ~1e-8 m of these coordinates, and the
// box is grown by dhat plus a margin of 1e-6 of the coordinate magnitude
// (>= 1e-7 m), so it contains the FP64 box.
template <class R, int GK>
TC_D void ccd_prim_box32(const EnvView<R>& e, const Motion& mo, const R* dir, int prim, float lo[3], float hi[3]) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  for (int d = 0; d < 3; ++d) {
    lo[d] = 3e38f;
    hi[d] = -3e38f;
  }
  float mag = 0.f;
  for (int l = 0; l < NGP; ++l) {
    const int v = gel_vertex(e, GK, prim, l);
    float w[3], wb[3];
    for (int d = 0; d < 3; ++d) {
      w[d] = e.X0f[d * e.nv + v] + (float)e.u[d * e.nv + v];
      wb[d] = w[d] + (dir ? (float)dir[d * e.nv + v] : 0.f);
    }
    float b0[3], b1[3];
    const float dx0 = w[0] - mo.taf[0], dy0 = w[1] - mo.taf[1], dz0 = w[2] - mo.taf[2];
    const float dx1 = wb[0] - mo.tbf[0], dy1 = wb[1] - mo.tbf[1], dz1 = wb[2] - mo.tbf[2];
    for (int d = 0; d < 3; ++d) {
      b0[d] = mo.Raf[d] * dx0 + mo.Raf[3 + d] * dy0 + mo.Raf[6 + d] * dz0;
      b1[d] = mo.Rbf[d] * dx1 + mo.Rbf[3 + d] * dy1 + mo.Rbf[6 + d] * dz1;
      lo[d] = fminf(lo[d], fminf(b0[d], b1[d]));
      hi[d] = fmaxf(hi[d], fmaxf(b0[d], b1[d]));
      mag = fmaxf(mag, fmaxf(fabsf(w[d]) + fabsf(mo.taf[d]), fabsf(wb[d]) + fabsf(mo.tbf[d])));
    }
  }
  const float grow = (float)e.dhat + fmaxf(1e-7f, 1e-6f * mag);
  for (int d = 0; d < 3; ++d) {
    lo[d] -= grow;
    hi[d] += grow;
  }
}

// One unit = 128 gel primitives.  Broad phase, one thread per primitive, in
// FP32: visit the grid cells of the swept box and write every indenter
// primitive found to the candidate list (these lists feed the contact and
// energy passes until the next CCD pass).  The FP64 swept geometry is then
// formed once per primitive that has candidates and kept in shared memory,
// and the narrow phase runs all threads of the block over the unit's
// flattened (primitive, candidate) pairs: additive CCD per pair, so the few
// primitives near the indenter do not serialise the block.
// A unit's 128 primitives run the broad phase on kCcdLanes lanes each; all
// kCcdThreads share its narrow phase.
constexpr int kCcdThreads = 512;
constexpr int kCcdLanes = kCcdThreads / 128;
// registers per thread of the fused CCD kernel (one 512-thread block per SM)
constexpr int kCcdRegs = 96;

template <class R, int GK>
TC_D void ccd_unit(const BatchView<R>& bv, const PartLayout& L, int unit) {
  constexpr int NGP = GK == GV ? 1 : (GK == GE ? 2 : 3);
  constexpr int ik = GK == GV ? 2 : (GK == GE ? 1 : 0);
  __shared__ int s_off[129];
  __shared__ Origin s_o[128];
  __shared__ Vec3<R> s_xg[128][NGP], s_pg[128][NGP];
  const Loc lc = locate(bv.prefix, bv.nenv, K_CV + GK, unit);
  const EnvView<R>& e = bv.views[lc.env];
  const Motion& mo = bv.motion[lc.env];
  const R* __restrict__ dir = mo.use_dir ? e.dx : nullptr;
  double* part_out = bv.part + L.ccd[GK];
  const int base = lc.chunk * 128;
  const int n = prim_count(e, GK);
  int32_t* cl = e.cand[GK];
  // broad phase: kCcdLanes consecutive lanes per primitive share its grid
  // visit (same candidate order as one thread alone)
  const int pl = (int)threadIdx.x / kCcdLanes;  // primitive of the unit
  const int prim = base + pl;
  int kept = 0;
  if (prim < n) {
    float lo[3], hi[3];
    ccd_prim_box32<R, GK>(e, mo, dir, prim, lo, hi);
    const int cap = e.cand_cap;
    const int cnt = grid_collect<kCcdLanes, R>(e, ik, lo, hi, [&](int pos, int ip) {
      if (pos < cap) cl[(int64_t)pos * n + prim] = ip;
    });
    kept = cnt < cap ? cnt : cap;
    if ((int)threadIdx.x % kCcdLanes == 0) {
      e.cand_n[GK][prim] = cnt;
      if (cnt > cap) atomicMax(&e.sc->overflow, cnt);
      if (kept > 0) {
        double b0[3][3], b1[3][3];
        float blo[3], bhi[3];
        ccd_prim_geom<R, GK>(e, mo, dir, prim, b0, b1, blo, bhi);
        const Origin o = make_origin(b0[0]);
        s_o[pl] = o;
        for (int l = 0; l < NGP; ++l) {
          s_xg[pl][l] = rel<R>(b0[l], o.d);
          s_pg[pl][l] = rel<R>(b1[l], b0[l]);
        }
      }
    }
  }
  // exclusive prefix of the kept counts (128 primitives, fixed order)
  if (threadIdx.x == 0) s_off[0] = 0;
  if ((int)threadIdx.x % kCcdLanes == 0) s_off[pl + 1] = kept;
  __syncthreads();
  prefix128(s_off);
  const int total = s_off[128];
  double tmin = 1.0;
  const int kind = GK == GE ? 1 : 0;
  for (int q = threadIdx.x; q < total; q += kCcdThreads) {
    int lo_i = 0, hi_i = 127;  // last i with s_off[i] <= q
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (s_off[mid] <= q) lo_i = mid;
      else hi_i = mid - 1;
    }
    const int prim = base + lo_i, j = q - s_off[lo_i];
    const Origin o = s_o[lo_i];
    Vec3<R> xg[NGP], pg[NGP];
    for (int l = 0; l < NGP; ++l) {
      xg[l] = s_xg[lo_i][l];
      pg[l] = s_pg[lo_i][l];
    }
    const int ip = cl[(int64_t)j * n + prim];
    Vec3<R> x0[4], p[4];
    pair_points<R, R, GK>(e, xg, ip, o, x0);
    const Vec3<R> zero = v3<R>(0, 0, 0);
    if (GK == GV) {
      p[0] = pg[0];
      p[1] = p[2] = p[3] = zero;
    } else if (GK == GF) {
      p[0] = zero;
      for (int l = 0; l < 3; ++l) p[1 + l] = pg[l];
    } else {
      p[0] = pg[0];
      p[1] = pg[1];
      p[2] = p[3] = zero;
    }
    const R t = accd<R>(kind, x0, p, (R)1.0, 4096);
    tmin = fmin(tmin, (double)t);
  }
  tmin = block_min<kCcdThreads>(tmin);
  if (threadIdx.x == 0) part_out[unit] = tmin;
}

// All three gel primitive kinds in one launch, edges first (the slowest
// kind), then faces, then vertices.
template <class R>
__global__ void __maxnreg__(kCcdRegs) k_ccd(const BatchView<R> bv, PartLayout L, int ne, int nf) {
  const int b = blockIdx.x;
  if (b < ne) ccd_unit<R, GE>(bv, L, b);
  else if (b < ne + nf) ccd_unit<R, GF>(bv, L, b - ne);
  else ccd_unit<R, GV>(bv, L, b - ne - nf);
}

// per env: min TOI over its contact units -> ccd_t
template <class R>
__global__ void __launch_bounds__(kBlock) k_ccd_env(const BatchView<R> bv, PartLayout L) {
  const int env = blockIdx.x;
  double m = 1.0;
  for (int k = 0; k < 3; ++k) {
    const int* p = bv.prefix + (K_CV + k) * (bv.nenv + 1);
    for (int u = p[env] + threadIdx.x; u < p[env + 1]; u += blockDim.x) m = fmin(m, bv.part[L.ccd[k] + u]);
  }
  m = block_min<kBlock>(m);
  if (threadIdx.x == 0) bv.views[env].sc->ccd_t = m;
}

template <class R> void b_ccd(const BatchHost<R>& b, cudaStream_t s) {
  const int nv = b.units[K_CV], ne = b.units[K_CE], nf = b.units[K_CF];
  if (nv + ne + nf > 0)
    TC_LAUNCH("k_ccd", s, k_ccd<R><<<(unsigned)(nv + ne + nf), kCcdThreads, 0, s>>>(b.bv, b.L, ne, nf));
  TC_LAUNCH("k_ccd_env", s, k_ccd_env<R><<<b.nenv, kBlock, 0, s>>>(b.bv, b.L));
}

// ------------------------------------------------------------ contact force
// f = -sum over all gel points of the barrier gradient (Algorithm 2:
// f_k = -g_k / dt^2 with the potential scaled by dt^2).
template <class R>
__global__ void k_force(const BatchView<R> bv) {
  const EnvView<R>& e = bv.views[blockIdx.x];
  double* out = e.sc->force;
  double f[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < e.nvc + e.nec + e.nfc; i += blockDim.x) {
    if (i < e.nvc) {
      for (int d = 0; d < 3; ++d) f[d] -= (double)e.cv_slot[(int64_t)d * e.nvc + i];
    } else if (i < e.nvc + e.nec) {
      const int p = i - e.nvc;
      for (int l = 0; l < 2; ++l)
        for (int d = 0; d < 3; ++d) f[d] -= (double)e.ce_slot[(int64_t)(3 * l + d) * e.nec + p];
    } else {
      const int p = i - e.nvc - e.nec;
      for (int l = 0; l < 3; ++l)
        for (int d = 0; d < 3; ++d) f[d] -= (double)e.cf_slot[(int64_t)(3 * l + d) * e.nfc + p];
    }
  }
  for (int d = 0; d < 3; ++d) {
    const double s = block_sum<kBlock>(f[d]);
    if (threadIdx.x == 0) out[d] = s;
  }
}

// Algorithm 2's contact decomposition per contact vertex s, from the contact
// slots of the last contact pass: f = -(vertex slot + its shares of the
// incident edges' and faces' slots), the unit normal n of sum_f A_f n_f over
// the incident deformed contact faces, the area A = sum_f A_f / 3,
// f_n = (f.n) n, f_tau = f - f_n, p = |f| / A (any output may be null).
template <class R>
__global__ void __launch_bounds__(kBlock)
    k_vertex_forces(const EnvView<R> e, float* __restrict__ f_out, float* __restrict__ fn_out,
                    float* __restrict__ ft_out, float* __restrict__ p_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int nvc = e.nvc, nec = e.nec, nfc = e.nfc, nv = e.nv;
  if (s >= nvc) return;
  double f[3];
  for (int d = 0; d < 3; ++d) f[d] = -(double)e.cv_slot[(int64_t)d * nvc + s];
  for (int k = e.cv_edge_off[s]; k < e.cv_edge_off[s + 1]; ++k) {
    const int ed = e.cv_edge_idx[k] >> 2, l = e.cv_edge_idx[k] & 3;
    for (int d = 0; d < 3; ++d) f[d] -= (double)e.ce_slot[(int64_t)(3 * l + d) * nec + ed];
  }
  double cs[3] = {0, 0, 0}, area2 = 0;
  for (int k = e.cv_face_off[s]; k < e.cv_face_off[s + 1]; ++k) {
    const int fc = e.cv_face_idx[k] >> 2, l = e.cv_face_idx[k] & 3;
    for (int d = 0; d < 3; ++d) f[d] -= (double)e.cf_slot[(int64_t)(3 * l + d) * nfc + fc];
    const int a = e.cfaces[fc], b = e.cfaces[nfc + fc], c = e.cfaces[2 * nfc + fc];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = (e.X0[d * nv + b] - e.X0[d * nv + a]) + (double)(e.u[d * nv + b] - e.u[d * nv + a]);
      e2[d] = (e.X0[d * nv + c] - e.X0[d * nv + a]) + (double)(e.u[d * nv + c] - e.u[d * nv + a]);
    }
    const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                 cz = e1[0] * e2[1] - e1[1] * e2[0];
    cs[0] += cx;
    cs[1] += cy;
    cs[2] += cz;
    area2 += sqrt(cx * cx + cy * cy + cz * cz);
  }
  const double cn = sqrt(cs[0] * cs[0] + cs[1] * cs[1] + cs[2] * cs[2]);
  double n[3] = {0, 0, 0};
  if (cn > 0)
    for (int d = 0; d < 3; ++d) n[d] = cs[d] / cn;
  const double fdn = f[0] * n[0] + f[1] * n[1] + f[2] * n[2];
  for (int d = 0; d < 3; ++d) {
    if (f_out) f_out[(int64_t)d * nvc + s] = (float)f[d];
    if (fn_out) fn_out[(int64_t)d * nvc + s] = (float)(fdn * n[d]);
    if (ft_out) ft_out[(int64_t)d * nvc + s] = (float)(f[d] - fdn * n[d]);
  }
  const double A = area2 / 6.0;
  if (p_out) p_out[s] = (float)(A > 0 ? sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]) / A : 0.0);
}

template <class R>
void launch_vertex_forces(const EnvView<R>& e, float* f, float* fn, float* ft, float* p, cudaStream_t s) {
  if (e.nvc > 0) TC_LAUNCH("k_vertex_forces", s, k_vertex_forces<R><<<grid_for(e.nvc), kBlock, 0, s>>>(e, f, fn, ft, p));
}
template void launch_vertex_forces<float>(const EnvView<float>&, float*, float*, float*, float*, cudaStream_t);
template void launch_vertex_forces<double>(const EnvView<double>&, float*, float*, float*, float*, cudaStream_t);

template <class R> void b_force(const BatchHost<R>& b, cudaStream_t s) {
  TC_LAUNCH("k_force", s, k_force<R><<<b.nenv, kBlock, 0, s>>>(b.bv));
}

// ------------------------------------------------------ intersection test
// Closed segment vs triangle with orientation signs in FP64 (used once, to
// reject a start pose where the indenter already crosses the gel surface).

TC_D double orient3(const double* a, const double* b, const double* c, const double* d) {
  const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double w[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
  return u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
}

TC_D bool seg_tri(const double* a, const double* b, const double* p0, const double* p1, const double* p2) {
  const double sa = orient3(p0, p1, p2, a), sb = orient3(p0, p1, p2, b);
  const bool straddle = (sa <= 0 && sb >= 0) || (sa >= 0 && sb <= 0);
  if (!straddle || (sa == 0 && sb == 0)) return false;
  const double s0 = orient3(a, b, p0, p1), s1 = orient3(a, b, p1, p2), s2 = orient3(a, b, p2, p0);
  return (s0 >= 0 && s1 >= 0 && s2 >= 0) || (s0 <= 0 && s1 <= 0 && s2 <= 0);
}

template <class R, int GK>
__global__ void k_intersect(const EnvView<R> e, int* flag) {
  // GK == GE: gel edges vs indenter faces; GK == GF: gel faces vs indenter edges
  constexpr int NGP = GK == GE ? 2 : 3;
  const int prim = blockIdx.x * blockDim.x + threadIdx.x;
  if (prim >= prim_count(e, GK)) return;
  double gw[3][3];
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  for (int l = 0; l < NGP; ++l) {
    gel_world(e, e.u, gel_vertex(e, GK, prim, l), gw[l]);
    double b[3];
    to_body(e.Rm, e.tr, gw[l], b);
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __double2float_rd(b[d]));
      hi[d] = fmaxf(hi[d], __double2float_ru(b[d]));
    }
  }
  const int ik = GK == GE ? 2 : 1;
  grid_visit<R>(e, ik, lo, hi, [&](int ip) {
    double w[3][3];
    const int nI = GK == GE ? 3 : 2;
    for (int l = 0; l < nI; ++l) {
      const int v = ind_vertex(e, ik, ip, l);
      const double yb[3] = {e.IV[v], e.IV[e.ind_nv + v], e.IV[2 * e.ind_nv + v]};
      for (int i = 0; i < 3; ++i)
        w[l][i] = e.Rm[3 * i] * yb[0] + e.Rm[3 * i + 1] * yb[1] + e.Rm[3 * i + 2] * yb[2] + e.tr[i];
    }
    const bool hit = GK == GE ? seg_tri(gw[0], gw[1], w[0], w[1], w[2]) : seg_tri(w[0], w[1], gw[0], gw[1], gw[2]);
    if (hit) atomicOr(flag, 1);
  });
}

template <class R> int intersect_test(const EnvView<R>& e, int* dflag, cudaStream_t s) {
  cudaMemsetAsync(dflag, 0, sizeof(int), s);
  TC_LAUNCH("k_intersect", s, k_intersect<R, GE><<<ContactGrid<R>::blocks(e.nec), 128, 0, s>>>(e, dflag));
  TC_LAUNCH("k_intersect", s, k_intersect<R, GF><<<ContactGrid<R>::blocks(e.nfc), 128, 0, s>>>(e, dflag));
  int h = 0;
  cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return h;
}

template void b_contact<float>(const BatchHost<float>&, bool, bool, cudaStream_t);
template void b_contact<double>(const BatchHost<double>&, bool, bool, cudaStream_t);
template void b_ccd<float>(const BatchHost<float>&, cudaStream_t);
template void b_ccd<double>(const BatchHost<double>&, cudaStream_t);
template void b_friction_lag<float>(const BatchHost<float>&, cudaStream_t);
template void b_friction_lag<double>(const BatchHost<double>&, cudaStream_t);
template void b_force<float>(const BatchHost<float>&, cudaStream_t);
template void b_force<double>(const BatchHost<double>&, cudaStream_t);
template int intersect_test<float>(const EnvView<float>&, int*, cudaStream_t);
template int intersect_test<double>(const EnvView<double>&, int*, cudaStream_t);

}  // namespace tc
