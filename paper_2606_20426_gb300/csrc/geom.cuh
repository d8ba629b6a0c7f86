// Contact geometry on the device: unsigned point-triangle and edge-edge
// distances, their gradient / Hessian restricted to the gel's points, the
// IPC log barrier b(d) = -(d - dhat)^2 ln(d / dhat) (Li et al. 2020) with the
// edge-edge mollifier, and additive CCD (Li, Kaufman & Jiang 2021).
//
// A pair is four points x0..x3 (point-triangle: point, t0, t1, t2; edge-edge:
// a0, a1, b0, b1).  The distance is the smallest distance between a face of
// one primitive and a face of the other whose closest points lie strictly
// inside both faces.  For the active pair of faces the difference vector is
// r = sum_i w_i x_i with weights affine in k <= 2 face parameters beta, and
//   d(d^2)/dx_i = 2 w_i r,
//   d2(d^2)/dx2 = 2 (w w^T (x) I) - Fxb (2 D^T D)^-1 Fxb^T,
//   Fxb[(i,j), c] = 2 (B_ic r_j + w_i D_cj),  D_c = sum_i B_ic x_i.
#pragma once
#include "common.cuh"

namespace tc {

// Candidate face pairs: slots of face A (nA, A[]) and face B (nB, B[]).
struct Cand {
  int nA, A[3], nB, B[3];
};

__constant__ Cand c_pt_cand[7] = {
    {1, {0, 0, 0}, 1, {1, 0, 0}}, {1, {0, 0, 0}, 1, {2, 0, 0}}, {1, {0, 0, 0}, 1, {3, 0, 0}},
    {1, {0, 0, 0}, 2, {1, 2, 0}}, {1, {0, 0, 0}, 2, {1, 3, 0}}, {1, {0, 0, 0}, 2, {2, 3, 0}},
    {1, {0, 0, 0}, 3, {1, 2, 3}}};
__constant__ Cand c_ee_cand[9] = {
    {1, {0, 0, 0}, 1, {2, 0, 0}}, {1, {0, 0, 0}, 1, {3, 0, 0}}, {1, {0, 0, 0}, 2, {2, 3, 0}},
    {1, {1, 0, 0}, 1, {2, 0, 0}}, {1, {1, 0, 0}, 1, {3, 0, 0}}, {1, {1, 0, 0}, 2, {2, 3, 0}},
    {2, {0, 1, 0}, 1, {2, 0, 0}}, {2, {0, 1, 0}, 1, {3, 0, 0}}, {2, {0, 1, 0}, 2, {2, 3, 0}}};

template <class T> struct CandEval {
  T d2;
  int k;          // number of face parameters
  T w[4];         // weights at the optimum
  T B[4][2];      // parameter columns
  Vec3<T> r;      // difference vector
  Vec3<T> D[2];   // parameter directions
  bool feasible;
};

template <class T> TC_D CandEval<T> eval_cand(const Cand& c, const Vec3<T>* x) {
  CandEval<T> ev;
  for (int i = 0; i < 4; ++i) {
    ev.w[i] = T(0);
    ev.B[i][0] = ev.B[i][1] = T(0);
  }
  ev.w[c.A[0]] += T(1);
  ev.w[c.B[0]] -= T(1);
  int k = 0;
  for (int m = 1; m < c.nA; ++m, ++k) {
    ev.B[c.A[m]][k] += T(1);
    ev.B[c.A[0]][k] -= T(1);
  }
  const int ka = k;
  for (int m = 1; m < c.nB; ++m, ++k) {
    ev.B[c.B[m]][k] -= T(1);
    ev.B[c.B[0]][k] += T(1);
  }
  ev.k = k;
  Vec3<T> r0 = x[c.A[0]] - x[c.B[0]];
  for (int q = 0; q < k; ++q) {
    Vec3<T> d = v3<T>(0, 0, 0);
    for (int i = 0; i < 4; ++i)
      if (ev.B[i][q] != T(0)) d = d + ev.B[i][q] * x[i];
    ev.D[q] = d;
  }
  T beta[2] = {T(0), T(0)};
  ev.feasible = true;
  if (k == 1) {
    const T dd = dot(ev.D[0], ev.D[0]);
    if (!(dd > T(0))) {
      ev.feasible = false;
    } else {
      beta[0] = -dot(ev.D[0], r0) / dd;
      ev.feasible = beta[0] > T(0) && beta[0] < T(1);
    }
  } else if (k == 2) {
    const T a = dot(ev.D[0], ev.D[0]), b = dot(ev.D[0], ev.D[1]), d = dot(ev.D[1], ev.D[1]);
    const T det = a * d - b * b;
    // near-parallel directions: the lower-dimensional candidates cover them
    const T tiny = sizeof(T) == 4 ? T(1e-6) : T(1e-20);
    if (!(det > tiny * a * d) || !(det > T(0))) {
      ev.feasible = false;
    } else {
      const T r1 = -dot(ev.D[0], r0), r2 = -dot(ev.D[1], r0);
      beta[0] = (d * r1 - b * r2) / det;
      beta[1] = (a * r2 - b * r1) / det;
      if (ka == 2) {  // both parameters on face A (triangle side never happens here)
        ev.feasible = beta[0] > T(0) && beta[1] > T(0) && beta[0] + beta[1] < T(1);
      } else if (ka == 0) {  // both on face B (point-triangle interior)
        ev.feasible = beta[0] > T(0) && beta[1] > T(0) && beta[0] + beta[1] < T(1);
      } else {  // one on each face (edge-edge interior)
        ev.feasible = beta[0] > T(0) && beta[0] < T(1) && beta[1] > T(0) && beta[1] < T(1);
      }
    }
  }
  if (!ev.feasible) {
    ev.d2 = T(0);
    return ev;
  }
  Vec3<T> r = r0;
  for (int q = 0; q < k; ++q) r = r + beta[q] * ev.D[q];
  for (int i = 0; i < 4; ++i) ev.w[i] += ev.B[i][0] * beta[0] + ev.B[i][1] * beta[1];
  ev.r = r;
  ev.d2 = dot(r, r);
  return ev;
}

// Squared distance and index of the active candidate (kind 0: PT, 1: EE).
template <class T> TC_D T pair_dist2(int kind, const Vec3<T>* x, int* which) {
  const int nc = kind == 0 ? 7 : 9;
  T best = T(sizeof(T) == 4 ? 3e38 : 1e300);
  int arg = -1;
  for (int c = 0; c < nc; ++c) {
    CandEval<T> ev = eval_cand<T>(kind == 0 ? c_pt_cand[c] : c_ee_cand[c], x);
    if (ev.feasible && ev.d2 < best) {
      best = ev.d2;
      arg = c;
    }
  }
  if (which) *which = arg;
  return best;
}


// IPC log barrier and its first two derivatives in d.
template <class T> TC_D void barrier3(T d, T dhat, T* b, T* b1, T* b2) {
  const T L = log(d / dhat);
  const T e = d - dhat;
  *b = -e * e * L;
  *b1 = -T(2) * e * L - e * e / d;
  *b2 = -T(2) * L - T(4) * e / d + e * e / (d * d);
}


// Additive CCD for one pair moving linearly x(t) = x0 + t p: largest t found
// at which the distance is still >= s d0 (s = 0.1), or t_max when the pair
// cannot get that close before t_max.  Iterations are capped; at the cap the
// time reached so far (which is safe) is returned.
template <class T> TC_D T accd(int kind, const Vec3<T>* x0, const Vec3<T>* p_in, T t_max, int max_iter) {
  Vec3<T> p[4];
  Vec3<T> mean = v3<T>(0, 0, 0);
  for (int i = 0; i < 4; ++i) mean = mean + p_in[i];
  mean = T(0.25) * mean;
  for (int i = 0; i < 4; ++i) p[i] = p_in[i] - mean;
  T n[4];
  for (int i = 0; i < 4; ++i) n[i] = sqrt(dot(p[i], p[i]));
  T lp = kind == 0 ? n[0] + fmax(n[1], fmax(n[2], n[3])) : fmax(n[0], n[1]) + fmax(n[2], n[3]);
  if (!(lp > T(0))) return t_max;
  const T s = T(0.1);
  T d0 = sqrt(pair_dist2<T>(kind, x0, nullptr));
  if (!(d0 > T(0))) return T(0);
  const T g = s * d0;
  T t = T(0);
  T step = (T(1) - s) * d0 / lp;
  Vec3<T> x[4];
  for (int it = 0; it < max_iter; ++it) {
    const T tn = t + step;
    for (int i = 0; i < 4; ++i) x[i] = x0[i] + tn * p[i];  // distance is translation invariant
    const T d = sqrt(pair_dist2<T>(kind, x, nullptr));
    if (t > T(0) && d < g) return t;
    t = tn;
    if (t > t_max) return t_max;
    step = T(0.9) * d / lp;
  }
  return t;
}

}  // namespace tc
