// Stress extraction on the contact surface (Algorithm 1 and the pixel map).
//
// K9  per contact face: sigma of the parent tet (Eq. 4, recomputed from the
//     parent's displacements: contact faces are a small subset of tets, so this
//     is cheaper than streaming a stored sigma field), outward unit normal of
//     the deformed face, t = sigma n (Eq. 5), p = -n.sigma.n (Eq. 7, sign so
//     that compression is positive), t_tau = t - (t.n) n (Eq. 8), face area.
// K10a per contact vertex: p_v = sum_f A_f p_f / sum_f A_f over incident
//     contact faces (deformed areas), a fixed-order gather.
// K10b per pixel: barycentric interpolation of p_v over the covering face.
#include "env.cuh"
#include "prof.cuh"

namespace tc {

template <class R>
__global__ void __launch_bounds__(kBlock)
    k_traction(const EnvView<R> e, const int32_t* __restrict__ cparent, float* __restrict__ t_out,
               float* __restrict__ p_out, float* __restrict__ tt_out, float* __restrict__ face_p,
               float* __restrict__ face_A) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int nfc = e.nfc;
  if (f >= nfc) return;
  const int nv = e.nv, nt = e.nt;
  const int el = cparent[f];
  const int4 t = e.tets[el];
  const int v[4] = {t.x, t.y, t.z, t.w};
  R Du[3][3], Bm[3][3], G[3][3];
  for (int i = 0; i < 3; ++i) {
    const R u0 = e.u[i * nv + v[0]];
    for (int a = 0; a < 3; ++a) Du[i][a] = e.u[i * nv + v[a + 1]] - u0;
  }
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 3; ++j) Bm[a][j] = e.Dminv[(int64_t)(a * 3 + j) * nt + el];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G[i][j] = Du[i][0] * Bm[0][j] + Du[i][1] * Bm[1][j] + Du[i][2] * Bm[2][j];
  const R trG = G[0][0] + G[1][1] + G[2][2];
  const R m2 = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) + (G[0][0] * G[2][2] - G[0][2] * G[2][0]) +
               (G[1][1] * G[2][2] - G[1][2] * G[2][1]);
  const R detG = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                 G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
  const R Jm1 = trG + m2 + detG;
  const R muJ = e.mu / (R(1) + Jm1);
  const R iso = (e.lam_hat - muJ) * Jm1;
  R S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S[i][j] = muJ * (G[i][j] + G[j][i] + G[i][0] * G[j][0] + G[i][1] * G[j][1] + G[i][2] * G[j][2]) +
                (i == j ? iso : R(0));
  // deformed face (stored winding is outward), edge vectors as rest + displacement
  const int a = e.cfaces[f], b = e.cfaces[nfc + f], c = e.cfaces[2 * nfc + f];
  R e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = (R)(e.X0[d * nv + b] - e.X0[d * nv + a]) + (e.u[d * nv + b] - e.u[d * nv + a]);
    e2[d] = (R)(e.X0[d * nv + c] - e.X0[d * nv + a]) + (e.u[d * nv + c] - e.u[d * nv + a]);
  }
  R n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const R len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const R il = len > R(0) ? R(1) / len : R(0);
  for (int d = 0; d < 3; ++d) n[d] *= il;
  R tv[3];
  for (int i = 0; i < 3; ++i) tv[i] = S[i][0] * n[0] + S[i][1] * n[1] + S[i][2] * n[2];
  const R pn = tv[0] * n[0] + tv[1] * n[1] + tv[2] * n[2];
  if (t_out)
    for (int i = 0; i < 3; ++i) t_out[(int64_t)i * nfc + f] = (float)tv[i];
  if (p_out) p_out[f] = (float)(-pn);
  if (tt_out)
    for (int i = 0; i < 3; ++i) tt_out[(int64_t)i * nfc + f] = (float)(tv[i] - pn * n[i]);
  if (face_p) face_p[f] = (float)(-pn);
  if (face_A) face_A[f] = (float)(R(0.5) * len);
}

template <class R>
void launch_traction(const EnvView<R>& e, const int32_t* cparent, float* t, float* p, float* tt, float* face_p,
                     float* face_A, cudaStream_t s) {
  if (e.nfc > 0) TC_LAUNCH("k_traction", s, k_traction<R><<<grid_for(e.nfc), kBlock, 0, s>>>(e, cparent, t, p, tt, face_p, face_A));
}

__global__ void __launch_bounds__(kBlock)
    k_vertex_avg(int nvc, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                 const float* __restrict__ face_p, const float* __restrict__ face_A, float* __restrict__ vert_p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nvc) return;
  float num = 0.f, den = 0.f;
  for (int k = off[s]; k < off[s + 1]; ++k) {
    const int f = idx[k] >> 2;
    const float A = face_A[f];
    num += A * face_p[f];
    den += A;
  }
  vert_p[s] = den > 0.f ? num / den : 0.f;
}

void launch_vertex_avg(int nvc, const int32_t* off, const int32_t* idx, const float* face_p, const float* face_A,
                       float* vert_p, cudaStream_t s) {
  if (nvc > 0) TC_LAUNCH("k_vertex_avg", s, k_vertex_avg<<<grid_for(nvc), kBlock, 0, s>>>(nvc, off, idx, face_p, face_A, vert_p));
}

__global__ void __launch_bounds__(kBlock)
    k_splat(int npix, const int32_t* __restrict__ pix_face, const float* __restrict__ pix_w,
            const int32_t* __restrict__ cface_slot, int nfc, const float* __restrict__ vert_p, float* __restrict__ out,
            uint8_t* __restrict__ mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const int f = pix_face[i];
  float v = 0.f;
  if (f >= 0) {
    v = pix_w[i] * vert_p[cface_slot[f]] + pix_w[npix + i] * vert_p[cface_slot[nfc + f]] +
        pix_w[2 * npix + i] * vert_p[cface_slot[2 * nfc + f]];
  }
  out[i] = v;
  if (mask) mask[i] = f >= 0 ? 1 : 0;
}

void launch_splat(int npix, const int32_t* pix_face, const float* pix_w, const int32_t* cface_slot, int nfc,
                  const float* vert_p, float* out, uint8_t* mask, cudaStream_t s) {
  if (npix > 0) TC_LAUNCH("k_splat", s, k_splat<<<grid_for(npix), kBlock, 0, s>>>(npix, pix_face, pix_w, cface_slot, nfc, vert_p, out, mask));
}

template void launch_traction<float>(const EnvView<float>&, const int32_t*, float*, float*, float*, float*, float*,
                                     cudaStream_t);
template void launch_traction<double>(const EnvView<double>&, const int32_t*, float*, float*, float*, float*, float*,
                                      cudaStream_t);

}  // namespace tc
