// Element pass (K1) and stress (K8).
//
// Material (Sec. III-B, rest-stable reading of Eq. 2/Eq. 4):
//   Psi = mu/2 (tr F^T F - 3) + lam_hat/2 (J - alpha)^2 - mu^2 / (2 lam_hat)
//   lam_hat = lam + mu, alpha = 1 + mu / lam_hat.
// Everything is written in terms of G = F - I = Du Dm^-1 so that FP32 keeps
// its relative accuracy at small strain (no O(1) cancellation):
//   J - 1 = tr G + m2(G) + det G           (m2: sum of principal 2x2 minors)
//   Psi   = mu/2 |G|^2 - mu (m2 + det G) + lam_hat/2 (J - 1)^2
//   P     = mu (G + G^T - tr G I - cof G) + lam_hat (J - 1) cof F
//   sigma = (mu/J)(G + G^T + G G^T) + (lam_hat - mu/J)(J - 1) I      (Eq. 4)
//   cof F = I + tr G I - G^T + cof G
// The tangent dP/dF is made PSD with its closed-form eigensystem in the
// singular basis F = U S V^T: twist modes mu + lam_hat (J - alpha) s_k,
// flip modes mu - lam_hat (J - alpha) s_k, and three scaling modes from the
// 3x3 Hessian of Psi in the singular values.  The full stable Neo-Hookean
// (log term, TC_MODEL_SNH_LOG) is this form with (mu, lam_hat) = (3 mu_s/4,
// lam_s) plus 2 kh h(x), kh = mu_s/4, h(x) = x - log(1 + x), x = (I_C - 3)/4:
// P gains kh x/(1+x) F, and the tangent kh x/(1+x) I (every mode) plus
// kh/(2 (1+x)^2) vec F vec F^T (the scaling modes: s_a s_b in the singular
// basis).  Negative eigenvalues are
// replaced by their absolute values (absolute eigenvalue filtering, Chen et
// al. 2024): under compression the twist modes turn negative, and clamping
// them to zero leaves the projected Newton method converging only linearly.
#include "env.cuh"
#include "kin.cuh"
#include "prof.cuh"
#include "solver.cuh"

namespace tc {

template <class R> TC_D R psi_of(const R G[3][3], const Kin<R>& k, R mu, R lam_hat, R kh) {
  R g2 = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g2 += G[i][j] * G[i][j];
  R psi = R(0.5) * mu * g2 - mu * (k.m2 + k.detG) + R(0.5) * lam_hat * k.Jm1 * k.Jm1;
  if (kh != R(0)) psi += R(2) * kh * h_log<R>(R(0.25) * (R(2) * k.trG + g2));
  return psi;
}

// 3x3 symmetric Jacobi eigen (A overwritten by eigenvalues on the diagonal).
template <class R> TC_D void eig3(R A[3][3], R V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? R(1) : R(0);
  for (int sweep = 0; sweep < (sizeof(R) == 4 ? 6 : 10); ++sweep) {
    const R off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const R dg = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off == R(0) || !(off > R(1e-36) * dg)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const R apq = A[p][q];
      if (apq == R(0)) continue;
      const R theta = (A[q][q] - A[p][p]) / (R(2) * apq);
      const R t = (theta >= R(0) ? R(1) : R(-1)) / (fabs(theta) + sqrt(theta * theta + R(1)));
      const R c = R(1) / sqrt(t * t + R(1));
      const R s = t * c;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

// Filtered tangent H9 = sum_m |lambda_m| q_m q_m^T in packed upper storage,
// vec index 3 i + j.
template <class R>
TC_D void psd_tangent(const R G[3][3], const Kin<R>& k, R mu, R lam_hat, R kh, R H[45]) {
  // S' = F^T F - I = G + G^T + G^T G: same eigenvectors as F^T F, accurate
  // s - 1 = c' / (1 + s) at small strain.
  R A[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      A[i][j] = G[i][j] + G[j][i] + G[0][i] * G[0][j] + G[1][i] * G[1][j] + G[2][i] * G[2][j];
  // log term: c1 on every mode, c2 s_a s_b on the scaling block (x = tr S' / 4)
  R c1 = R(0), c2 = R(0);
  if (kh != R(0)) {
    const R x = R(0.25) * (A[0][0] + A[1][1] + A[2][2]);
    const R ix = R(1) / (R(1) + x);
    c1 = kh * x * ix;
    c2 = R(0.5) * kh * ix * ix;
  }
  eig3<R>(A, V);
  R c[3] = {A[0][0], A[1][1], A[2][2]};
  // sort descending (columns of V follow)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2 - a; ++b)
      if (c[b] < c[b + 1]) {
        R t = c[b]; c[b] = c[b + 1]; c[b + 1] = t;
        for (int i = 0; i < 3; ++i) { R w = V[i][b]; V[i][b] = V[i][b + 1]; V[i][b + 1] = w; }
      }
  // proper rotation
  const R detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                 V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < R(0))
    for (int i = 0; i < 3; ++i) V[i][2] = -V[i][2];
  R s[3], sm1[3];
  for (int i = 0; i < 3; ++i) {
    const R ci = fmax(c[i], R(-1));
    s[i] = sqrt(R(1) + ci);
    sm1[i] = ci / (R(1) + s[i]);
  }
  // U = F V S^-1 with Gram-Schmidt; F = I + G
  R Fv[3][3];
  for (int i = 0; i < 3; ++i)
    for (int m = 0; m < 3; ++m) Fv[i][m] = V[i][m] + G[i][0] * V[0][m] + G[i][1] * V[1][m] + G[i][2] * V[2][m];
  R U[3][3];
  {
    R n0 = sqrt(Fv[0][0] * Fv[0][0] + Fv[1][0] * Fv[1][0] + Fv[2][0] * Fv[2][0]);
    n0 = n0 > R(0) ? n0 : R(1);
    for (int i = 0; i < 3; ++i) U[i][0] = Fv[i][0] / n0;
    const R pr = U[0][0] * Fv[0][1] + U[1][0] * Fv[1][1] + U[2][0] * Fv[2][1];
    R u1[3] = {Fv[0][1] - pr * U[0][0], Fv[1][1] - pr * U[1][0], Fv[2][1] - pr * U[2][0]};
    R n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    n1 = n1 > R(0) ? n1 : R(1);
    for (int i = 0; i < 3; ++i) U[i][1] = u1[i] / n1;
    U[0][2] = U[1][0] * U[2][1] - U[2][0] * U[1][1];
    U[1][2] = U[2][0] * U[0][1] - U[0][0] * U[2][1];
    U[2][2] = U[0][0] * U[1][1] - U[1][0] * U[0][1];
    const R s2 = U[0][2] * Fv[0][2] + U[1][2] * Fv[1][2] + U[2][2] * Fv[2][2];
    if (s2 < R(0)) {  // inverted element: signed smallest singular value
      s[2] = -s[2];
      sm1[2] = s[2] - R(1);
    }
  }
  const R cJ = lam_hat * k.Jm1 - mu;  // lam_hat (J - alpha)
  for (int i = 0; i < 45; ++i) H[i] = R(0);
  const R isq2 = R(0.70710678118654752440);
  // twist / flip for pairs (i, j), k the third index
#pragma unroll
  for (int pr = 0; pr < 3; ++pr) {
    const int i = pr == 2 ? 1 : 0, j = pr == 0 ? 1 : 2, kk = 3 - i - j;
    // twist: mu + cJ s_k = -mu (s_k - 1) + lam_hat (J - 1) s_k
    R lt = -mu * sm1[kk] + lam_hat * k.Jm1 * s[kk];
    R lf = R(2) * mu + mu * sm1[kk] - lam_hat * k.Jm1 * s[kk];  // mu - cJ s_k
    if (kh != R(0)) {
      lt += c1;
      lf += c1;
    }
#pragma unroll
    for (int mode = 0; mode < 2; ++mode) {
      const R lam = fabs(mode == 0 ? lt : lf);
      if (!(lam > R(0))) continue;
      const R sg = mode == 0 ? R(-1) : R(1);
      R q[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) q[3 * a + b] = isq2 * (U[a][i] * V[b][j] + sg * U[a][j] * V[b][i]);
      int idx = 0;
#pragma unroll
      for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = a; b < 9; ++b) H[idx++] += lam * q[a] * q[b];
    }
  }
  // scaling modes
  R Js[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
  R As[3][3], Av[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a == b) As[a][b] = mu + lam_hat * Js[a] * Js[a];
      else As[a][b] = lam_hat * Js[a] * Js[b] + cJ * s[3 - a - b];
      if (kh != R(0)) As[a][b] += (a == b ? c1 : R(0)) + c2 * s[a] * s[b];
    }
  eig3<R>(As, Av);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const R lam = fabs(As[m][m]);
    if (!(lam > R(0))) continue;
    R q[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        q[3 * a + b] = U[a][0] * Av[0][m] * V[b][0] + U[a][1] * Av[1][m] * V[b][1] + U[a][2] * Av[2][m] * V[b][2];
    int idx = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int b = a; b < 9; ++b) H[idx++] += lam * q[a] * q[b];
  }
}

// K1: energy (per-unit partial), gradient slots and the element's stiffness
// blocks (10 upper 3x3 corner blocks of V D^T H D, D = dF/dx).
template <class R, bool HESS>
__global__ void __launch_bounds__(kBlock) k_elem(const BatchView<R> bv, PartLayout L, int trial) {
  const Loc l = locate(bv.prefix, bv.nenv, K_TET, blockIdx.x);
  const EnvView<R>& e = bv.views[l.env];
  const R* __restrict__ u = trial ? e.ut : e.u;
  const int el = l.chunk * kBlock + threadIdx.x;
  double energy = 0.0;
  if (el < e.nt) {
    const int4 t = e.tets[el];
    R G[3][3], Bm[3][3];
    load_G<R>(e, u, el, t, G, Bm);
    const Kin<R> k = kinematics<R>(G);
    const R V = e.vol[el];
    R mu, lh, kh;
    tet_material<R>(e, el, mu, lh, kh);
    energy = (double)(V * psi_of<R>(G, k, mu, lh, kh));
    if (HESS) {
      const int nt = e.nt;
      // P = mu (G + G^T - trG I - cof G) + lam_hat (J-1) cof F
      R P[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const R cofF = (i == j ? R(1) + k.trG : R(0)) - G[j][i] + k.cG[i][j];
          P[i][j] = mu * (G[i][j] + G[j][i] - (i == j ? k.trG : R(0)) - k.cG[i][j]) + lh * k.Jm1 * cofF;
        }
      if (kh != R(0)) {
        // log term: + kh x/(1+x) F, x = (2 tr G + |G|^2)/4
        R g2 = 0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) g2 += G[i][j] * G[i][j];
        const R x = R(0.25) * (R(2) * k.trG + g2);
        const R c = kh * (x / (R(1) + x));
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) P[i][j] += c * ((i == j ? R(1) : R(0)) + G[i][j]);
      }
      // gradient: g_a = V P n_a, n_a = row (a-1) of Dm^-1, n_0 = -sum
      R gs[4][3];
      for (int i = 0; i < 3; ++i) {
        R s0 = 0;
        for (int a = 0; a < 3; ++a) {
          const R ga = V * (P[i][0] * Bm[a][0] + P[i][1] * Bm[a][1] + P[i][2] * Bm[a][2]);
          gs[a + 1][i] = ga;
          s0 += ga;
        }
        gs[0][i] = -s0;
      }
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) e.eslot[(int64_t)(3 * a + i) * nt + el] = gs[a][i];
      R H[45];
      psd_tangent<R>(G, k, mu, lh, kh, H);
      // stiffness blocks K_ab[i][k] = V sum_jl H[(i,j),(k,l)] n_a[j] n_b[l]
      // for corners a <= b (n_a: gradient of corner a's shape function)
      R n[4][3];
      for (int j = 0; j < 3; ++j) {
        n[1][j] = Bm[0][j];
        n[2][j] = Bm[1][j];
        n[3][j] = Bm[2][j];
        n[0][j] = -(Bm[0][j] + Bm[1][j] + Bm[2][j]);
      }
      R* K = e.kblk;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          R T[3][4];  // T[j][b] = sum_l H[(i,j),(kk,l)] n_b[l]
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              T[j][b] = H[sym_index(3 * i + j, 3 * kk + 0, 9)] * n[b][0] + H[sym_index(3 * i + j, 3 * kk + 1, 9)] * n[b][1] +
                        H[sym_index(3 * i + j, 3 * kk + 2, 9)] * n[b][2];
          int pidx = 0;
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a; b < 4; ++b) {
              K[kblk_index(el, pidx * 9 + 3 * i + kk)] = V * (n[a][0] * T[0][b] + n[a][1] * T[1][b] + n[a][2] * T[2][b]);
              ++pidx;
            }
        }
    }
  }
  energy = block_sum<kBlock>(energy);
  if (threadIdx.x == 0) bv.part[L.elem + blockIdx.x] = energy;
}

template <class R> void b_elem(const BatchHost<R>& b, bool hess, bool trial, cudaStream_t s) {
  if (b.units[K_TET] == 0) return;
  if (hess) TC_LAUNCH("k_elem_hess", s, k_elem<R, true><<<b.units[K_TET], kBlock, 0, s>>>(b.bv, b.L, trial ? 1 : 0));
  else TC_LAUNCH("k_elem_energy", s, k_elem<R, false><<<b.units[K_TET], kBlock, 0, s>>>(b.bv, b.L, trial ? 1 : 0));
}

// ---------------------------------------------------------------- stress (K8)

template <class R>
__global__ void __launch_bounds__(kBlock) k_stress(const EnvView<R> e, const R* __restrict__ u, float* __restrict__ sig) {
  const int el = blockIdx.x * blockDim.x + threadIdx.x;
  if (el >= e.nt) return;
  const int4 t = e.tets[el];
  R G[3][3], Bm[3][3];
  load_G<R>(e, u, el, t, G, Bm);
  R s6[6];
  R mu, lh, kh;
  tet_material<R>(e, el, mu, lh, kh);
  cauchy6<R>(G, kinematics<R>(G), mu, lh, kh, s6);
  const int64_t nt = e.nt;
#pragma unroll
  for (int c = 0; c < 6; ++c) sig[c * nt + el] = (float)s6[c];
}

template <class R> void launch_stress(const EnvView<R>& e, float* sigma, cudaStream_t s) {
  TC_LAUNCH("k_stress", s, k_stress<R><<<grid_for(e.nt), kBlock, 0, s>>>(e, e.u, sigma));
}

// Standalone sigma(F) over n deformation gradients (row-major n x 9 in,
// SoA 6 x n out): 36 B read and 24 B written per tet, streaming cache hints.
__global__ void __launch_bounds__(kBlock)
    k_stress_from_F(const float* __restrict__ F, int64_t n, float mu, float lam_hat, float* __restrict__ sig) {
  for (int64_t el = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; el < n; el += (int64_t)gridDim.x * blockDim.x) {
    float G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) G[i][j] = __ldcs(&F[el * 9 + 3 * i + j]) - (i == j ? 1.f : 0.f);
    const Kin<float> k = kinematics<float>(G);
    const float muJ = mu / k.J;
    const float iso = (lam_hat - muJ) * k.Jm1;
    float bI[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        bI[i][j] = G[i][j] + G[j][i] + G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2];
    __stcs(&sig[0 * n + el], muJ * bI[0][0] + iso);
    __stcs(&sig[1 * n + el], muJ * bI[1][1] + iso);
    __stcs(&sig[2 * n + el], muJ * bI[2][2] + iso);
    __stcs(&sig[3 * n + el], muJ * bI[0][1]);
    __stcs(&sig[4 * n + el], muJ * bI[1][2]);
    __stcs(&sig[5 * n + el], muJ * bI[2][0]);
  }
}

void launch_stress_from_F(const float* F, int64_t n, float mu, float lam_hat, float alpha, float* sigma,
                          cudaStream_t s) {
  (void)alpha;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  TC_LAUNCH("k_stress_from_F", s, k_stress_from_F<<<(unsigned)blocks, kBlock, 0, s>>>(F, n, mu, lam_hat, sigma));
}

template void b_elem<float>(const BatchHost<float>&, bool, bool, cudaStream_t);
template void b_elem<double>(const BatchHost<double>&, bool, bool, cudaStream_t);
template void launch_stress<float>(const EnvView<float>&, float*, cudaStream_t);
template void launch_stress<double>(const EnvView<double>&, float*, cudaStream_t);

}  // namespace tc
