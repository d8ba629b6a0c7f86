// Per-tet kinematics and the Cauchy stress of the rest-stable Neo-Hookean
// reading (Sec. III-B / III-C, Eq. 3-4), and the per-face traction of
// Algorithm 1 -- the device functions that the element pass, the stress
// kernel and the extraction kernels share, so that every path computes sigma
// and the face pressure with the same operations.
//
// Everything is written in terms of G = F - I = Du Dm^-1:
//   J - 1 = tr G + m2(G) + det G           (m2: sum of principal 2x2 minors)
//   sigma = (mu/J)(G + G^T + G G^T) + (lam_hat - mu/J)(J - 1) I      (Eq. 4)
// The full stable Neo-Hookean (log term) is that form with (mu, lam_hat) =
// (3 mu_s/4, lam_s) plus the part 2 kh h(x), kh = mu_s/4, h(x) = x - log(1 + x),
// x = (I_C - 3)/4 = tr(b - I)/4, whose first-order terms cancel those of the
// rest: sigma gains (kh/J) x/(1 + x) b.
#pragma once
#include "env.cuh"

namespace tc {

template <class R> struct Mat3 {
  R m[3][3];
};

template <class R> TC_D void cof3(const R A[3][3], R C[3][3]) {
  C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  C[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  C[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  C[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
  C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  C[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
  C[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  C[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
  C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
}

// The per-env arrays that sigma and the face traction read, held by value
// (for kernels that loop over the items of many envs and keep one env's
// fields in registers).  The functions below take it or an EnvView alike.
template <class R> struct KinView {
  int nv, nt, nfc;
  R mu, lam_hat, kh;
  const R* mat;
  const int4* tets;
  const double* X0;
  const R* Dminv;
  const R* u;
  const int32_t* cfaces;
};

template <class R> TC_D KinView<R> kin_view(const EnvView<R>& e) {
  return KinView<R>{e.nv, e.nt, e.nfc, e.mu, e.lam_hat, e.kh, e.mat, e.tets, e.X0, e.Dminv, e.u, e.cfaces};
}

// Load G = Du Dm^-1 for tet e at displacement u (SoA, stride nv).
template <class R, class V>
TC_D void load_G(const V& e, const R* u, int el, int4 t, R G[3][3], R Bm[3][3]) {
  const int nv = e.nv, nt = e.nt;
  const int v[4] = {t.x, t.y, t.z, t.w};
  R Du[3][3];
  for (int i = 0; i < 3; ++i) {
    const R u0 = u[i * nv + v[0]];
    for (int a = 0; a < 3; ++a) Du[i][a] = u[i * nv + v[a + 1]] - u0;
  }
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 3; ++j) Bm[a][j] = e.Dminv[(int64_t)(a * 3 + j) * nt + el];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = Du[i][0] * Bm[0][j] + Du[i][1] * Bm[1][j] + Du[i][2] * Bm[2][j];
}

template <class R> struct Kin {
  R trG, m2, detG, Jm1, J;
  R cG[3][3];
};

template <class R> TC_D Kin<R> kinematics(const R G[3][3]) {
  Kin<R> k;
  k.trG = G[0][0] + G[1][1] + G[2][2];
  k.m2 = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) + (G[0][0] * G[2][2] - G[0][2] * G[2][0]) +
         (G[1][1] * G[2][2] - G[1][2] * G[2][1]);
  cof3<R>(G, k.cG);
  k.detG = G[0][0] * k.cG[0][0] + G[0][1] * k.cG[0][1] + G[0][2] * k.cG[0][2];
  k.Jm1 = k.trG + k.m2 + k.detG;
  k.J = R(1) + k.Jm1;
  return k;
}

// Material of tet el: its own (mu, lam_hat, kh) when the env is
// heterogeneous (kh, the log-term coefficient, is 0 for the rest-stable law).
template <class R, class V> TC_D void tet_material(const V& e, int el, R& mu, R& lam_hat, R& kh) {
  if (e.mat) {
    mu = e.mat[el];
    lam_hat = e.mat[(int64_t)e.nt + el];
    kh = e.kh != R(0) ? e.mat[2 * (int64_t)e.nt + el] : R(0);
  } else {
    mu = e.mu;
    lam_hat = e.lam_hat;
    kh = e.kh;
  }
}

// h(x) = x - log(1 + x) for x >= -3/4 without cancellation near 0: with
// u = x / (2 + x), log(1 + x) = 2 atanh(u) = 2 (u + u^3/3 + u^5/5 + ...) and
// x - 2u = u x, so h = u x - 2 u^3 (1/3 + u^2/5 + ... + u^16/19) (|u| < 1/7
// for |x| < 1/4: the dropped terms are below 1e-16 relative); further out
// the direct difference loses at most a factor 10 to cancellation.
template <class R> TC_D R h_log(R x) {
  if (fabs(x) >= R(0.25)) return x - log1p(x);
  const R u = x / (R(2) + x), u2 = u * u;
  R s = R(1) / R(19);
#pragma unroll
  for (int k = 17; k >= 3; k -= 2) s = R(1) / R(k) + u2 * s;
  return u * x - R(2) * u * u2 * s;
}

// Cauchy stress (xx, yy, zz, xy, yz, zx) from G and its kinematics.
template <class R> TC_D void cauchy6(const R G[3][3], const Kin<R>& k, R mu, R lam_hat, R kh, R s6[6]) {
  const R muJ = mu / k.J;
  const R iso = (lam_hat - muJ) * k.Jm1;
  R bI[3][3];  // b - I = G + G^T + G G^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      bI[i][j] = G[i][j] + G[j][i] + G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2];
  s6[0] = muJ * bI[0][0] + iso;
  s6[1] = muJ * bI[1][1] + iso;
  s6[2] = muJ * bI[2][2] + iso;
  s6[3] = muJ * bI[0][1];
  s6[4] = muJ * bI[1][2];
  s6[5] = muJ * bI[2][0];
  if (kh != R(0)) {
    // log term: (kh/J) x/(1+x) b, x = tr(b - I)/4
    const R x = R(0.25) * (bI[0][0] + bI[1][1] + bI[2][2]);
    const R c = kh / k.J * (x / (R(1) + x));
    s6[0] += c * (R(1) + bI[0][0]);
    s6[1] += c * (R(1) + bI[1][1]);
    s6[2] += c * (R(1) + bI[2][2]);
    s6[3] += c * bI[0][1];
    s6[4] += c * bI[1][2];
    s6[5] += c * bI[2][0];
  }
}

// Algorithm 1 on contact face f: sigma of its parent tet, the unit outward
// normal n of the deformed face (stored winding is outward), t = sigma n
// (Eq. 5), pn = n.sigma.n (Eq. 7's p_n; the pressure is -pn) and the face
// area len / 2 (len = |e1 x e2|).
template <class R, class V>
TC_D void face_traction(const V& e, const int32_t* __restrict__ cparent, int f, R tv[3], R n[3], R& pn, R& len) {
  const int nv = e.nv, nfc = e.nfc;
  const int el = cparent[f];
  R G[3][3], Bm[3][3], s6[6];
  load_G<R>(e, e.u, el, e.tets[el], G, Bm);
  R mu, lh, kh;
  tet_material<R>(e, el, mu, lh, kh);
  cauchy6<R>(G, kinematics<R>(G), mu, lh, kh, s6);
  const int a = e.cfaces[f], b = e.cfaces[nfc + f], c = e.cfaces[2 * nfc + f];
  R e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = (R)(e.X0[d * nv + b] - e.X0[d * nv + a]) + (e.u[d * nv + b] - e.u[d * nv + a]);
    e2[d] = (R)(e.X0[d * nv + c] - e.X0[d * nv + a]) + (e.u[d * nv + c] - e.u[d * nv + a]);
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const R il = len > R(0) ? R(1) / len : R(0);
  for (int d = 0; d < 3; ++d) n[d] *= il;
  tv[0] = s6[0] * n[0] + s6[3] * n[1] + s6[5] * n[2];
  tv[1] = s6[3] * n[0] + s6[1] * n[1] + s6[4] * n[2];
  tv[2] = s6[5] * n[0] + s6[4] * n[1] + s6[2] * n[2];
  pn = tv[0] * n[0] + tv[1] * n[1] + tv[2] * n[2];
}

}  // namespace tc
