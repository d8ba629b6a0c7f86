// Scene setup (once per env), all on the device:
//   rest shape Dm^-1 and volume per tet (Sec. III-B; F = Ds Dm^-1),
//   vertex -> (tet, corner) incidence, lumped masses,
//   boundary faces with parent tets (Algorithm 1, steps 1-3),
//   contact band (Sec. III-A: thinnest axis, 15 % of the thickness on the
//   side opposite the fixed set) and contact surface (faces, edges, vertices),
//   vertex -> face / edge incidence of the contact surface,
//   exact pixel binning of the contact faces,
//   indenter edges and a uniform grid over its body-frame bounding box.
#include <algorithm>
#include <cmath>
#include <vector>

#include "env.cuh"

namespace tc {

#define TC_TRY(x)                                   \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return TC_ERR_CUDA;      \
  } while (0)

// ------------------------------------------------------------- rest shape

template <class R>
__global__ void k_rest_shape(const int4* tets, const double* X0, int nv, int nt, R* Dminv, R* vol, Scalars* sc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nt) return;
  const int4 t = tets[e];
  const double* x = X0;
  const double* y = X0 + nv;
  const double* z = X0 + 2 * nv;
  double D[3][3];
  const int v[4] = {t.x, t.y, t.z, t.w};
  for (int a = 0; a < 3; ++a) {
    D[0][a] = x[v[a + 1]] - x[v[0]];
    D[1][a] = y[v[a + 1]] - y[v[0]];
    D[2][a] = z[v[a + 1]] - z[v[0]];
  }
  const double c00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
  const double c01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
  const double c02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
  const double det = D[0][0] * c00 + D[0][1] * c01 + D[0][2] * c02;
  if (!(det > 0.0)) {
    atomicOr(&sc->status, ST_INVALID_MESH);
    return;
  }
  const double id = 1.0 / det;
  double I[3][3];
  I[0][0] = c00 * id;
  I[1][0] = c01 * id;
  I[2][0] = c02 * id;
  I[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) * id;
  I[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) * id;
  I[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) * id;
  I[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) * id;
  I[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) * id;
  I[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) * id;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Dminv[(int64_t)(i * 3 + j) * nt + e] = (R)I[i][j];
  vol[e] = (R)(det / 6.0);
}

__global__ void k_mark_fixed(const int32_t* ids, int n, uint8_t* fixed, int nv, Scalars* sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = ids[i];
  if (v < 0 || v >= nv) {
    atomicOr(&sc->status, ST_INVALID_MESH);
    return;
  }
  fixed[v] = 1;
}

// keys (vertex << 32 | tet*4+corner) for the vertex -> tet CSR
__global__ void k_vt_keys(const int4* tets, int nt, uint64_t* keys, uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * nt) return;
  const int e = i >> 2, c = i & 3;
  const int4 t = tets[e];
  const int v = c == 0 ? t.x : (c == 1 ? t.y : (c == 2 ? t.z : t.w));
  keys[i] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)i;
  vals[i] = (uint32_t)i;
}

// counts of a CSR whose sorted keys carry the row in the high 32 bits
__global__ void k_row_counts(const uint64_t* keys, int64_t n, int32_t* counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicAdd(&counts[(int)(keys[i] >> 32)], 1);
}

__global__ void k_low32(const uint64_t* keys, int64_t n, int32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)(uint32_t)(keys[i] & 0xffffffffu);
}

template <class R>
__global__ void k_mass(const int32_t* off, const int32_t* idx, const R* vol, double rho, int nv, R* mass) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double m = 0.0;
  for (int k = off[v]; k < off[v + 1]; ++k) m += rho * (double)vol[idx[k] >> 2] * 0.25;
  mass[v] = (R)m;
}

// ---------------------------------------------------------- boundary faces
// Faces of tet (0,1,2,3): (1,2,3), (0,3,2), (0,1,3), (0,2,1) -- outward for a
// positively oriented tet.
__constant__ int c_tet_face[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

TC_HD uint64_t face_key(int a, int b, int c) {
  int lo = min(a, min(b, c)), hi = max(a, max(b, c));
  int mid = a + b + c - lo - hi;
  return ((uint64_t)lo << 42) | ((uint64_t)mid << 21) | (uint64_t)hi;
}

__global__ void k_face_keys(const int4* tets, int nt, uint64_t* keys, uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * nt) return;
  const int e = i >> 2, f = i & 3;
  const int4 t = tets[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  keys[i] = face_key(v[c_tet_face[f][0]], v[c_tet_face[f][1]], v[c_tet_face[f][2]]);
  vals[i] = (uint32_t)i;
}

__global__ void k_face_once(const uint64_t* keys, int64_t n, int32_t* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = keys[i];
  const bool uniq = (i == 0 || keys[i - 1] != k) && (i == n - 1 || keys[i + 1] != k);
  flag[i] = uniq ? 1 : 0;
}

// scatter boundary faces (outward winding rotated so the smallest id leads)
__global__ void k_face_emit(const uint32_t* vals, const int32_t* flag, const int32_t* pos, int64_t n,
                            const int4* tets, int32_t* faces, int32_t* parent, int nf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int o = pos[i];
  const uint32_t tf = vals[i];
  const int e = tf >> 2, f = tf & 3;
  const int4 t = tets[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  int a = v[c_tet_face[f][0]], b = v[c_tet_face[f][1]], c = v[c_tet_face[f][2]];
  while (a > b || a > c) {  // rotate (winding kept)
    const int tmp = a;
    a = b;
    b = c;
    c = tmp;
  }
  faces[0 * nf + o] = a;
  faces[1 * nf + o] = b;
  faces[2 * nf + o] = c;
  parent[o] = e;
}

// --------------------------------------------------------------- contact band

__global__ void k_fixed_coord_sum(const int32_t* ids, int n, const double* coord, double* part) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += coord[ids[i]];
  s = block_sum<kBlock>(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// band threshold with correctly rounded FP64 steps: thr = hi - 0.15 (hi - lo)
__global__ void k_band(const double* coord, int nv, double lo, double hi, int top, uint8_t* band) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double thick = __dsub_rn(hi, lo);
  const double c = coord[v];
  bool in;
  if (top) in = c >= __dsub_rn(hi, __dmul_rn(0.15, thick));
  else in = c <= __dadd_rn(lo, __dmul_rn(0.15, thick));
  band[v] = in ? 1 : 0;
}

__global__ void k_contact_flag(const int32_t* faces, int nf, const uint8_t* band, int32_t* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  flag[i] = (band[faces[i]] && band[faces[nf + i]] && band[faces[2 * nf + i]]) ? 1 : 0;
}

__global__ void k_contact_emit(const int32_t* faces, const int32_t* parent, int nf, const int32_t* flag,
                               const int32_t* pos, int32_t* cfaces, int32_t* cparent, int nfc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf || !flag[i]) return;
  const int o = pos[i];
  for (int k = 0; k < 3; ++k) cfaces[k * nfc + o] = faces[k * nf + i];
  cparent[o] = parent[i];
}

// edges of a face set: keys (min << 32 | max)
__global__ void k_edge_keys(const int32_t* faces, int nf, uint64_t* keys, uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nf) return;
  const int f = i / 3, k = i % 3;
  const int a = faces[k * nf + f], b = faces[((k + 1) % 3) * nf + f];
  keys[i] = ((uint64_t)(uint32_t)min(a, b) << 32) | (uint32_t)max(a, b);
  vals[i] = (uint32_t)i;
}

__global__ void k_unique_flag(const uint64_t* keys, int64_t n, int32_t* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flag[i] = (i == 0 || keys[i - 1] != keys[i]) ? 1 : 0;
}

__global__ void k_edge_emit(const uint64_t* keys, const int32_t* flag, const int32_t* pos, int64_t n, int32_t* edges,
                            int ne) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int o = pos[i];
  edges[o] = (int32_t)(keys[i] >> 32);
  edges[ne + o] = (int32_t)(keys[i] & 0xffffffffu);
}

__global__ void k_vert_keys(const int32_t* faces, int nf, uint64_t* keys, uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nf) return;
  keys[i] = (uint64_t)(uint32_t)faces[(i % 3) * nf + i / 3];
  vals[i] = (uint32_t)i;
}

__global__ void k_vert_emit(const uint64_t* keys, const int32_t* flag, const int32_t* pos, int64_t n, int32_t* verts,
                            int32_t* vslot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int v = (int)keys[i];
  verts[pos[i]] = v;
  vslot[v] = pos[i];
}

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_face_slots(const int32_t* cfaces, int nfc, const int32_t* vslot, int32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nfc) return;
  out[i] = vslot[cfaces[i]];
}

// keys (contact-vertex slot << 32 | prim*4 + local) of a primitive set with k vertices
__global__ void k_incidence_keys(const int32_t* prims, int n, int k, const int32_t* vslot, uint64_t* keys,
                                 uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k * n) return;
  const int p = i / k, l = i % k;
  const int s = vslot[prims[l * n + p]];
  keys[i] = ((uint64_t)(uint32_t)s << 32) | (uint32_t)(p * 4 + l);
  vals[i] = (uint32_t)i;
}

__global__ void k_edge_len2(const int32_t* edges, int ne, const double* X, int nx, double* out, double* part) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
    const int a = edges[i], b = edges[ne + i];
    const double dx = X[a] - X[b], dy = X[nx + a] - X[nx + b], dz = X[2 * nx + a] - X[2 * nx + b];
    const double l2 = dx * dx + dy * dy + dz * dz;
    out[i] = l2;
    s += sqrt(l2);
  }
  s = block_sum<kBlock>(s);
  if (part && threadIdx.x == 0) part[blockIdx.x] = s;
}

// ------------------------------------------------------------- pixel binning
// Coordinates snapped to integer nanometres (round half to even) and doubled
// so that pixel centres are integers; edge functions are exact in int64.

TC_D long long snap2(double x) { return 2ll * (long long)rint(__dmul_rn(x, 1e9)); }

TC_D long long edge_fn(long long au, long long av, long long bu, long long bv, long long pu, long long pv) {
  return (bu - au) * (pv - av) - (bv - av) * (pu - au);
}

TC_D long long floor_div(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

struct PixGrid {
  long long u0, v0, du, dv;  // doubled origin, single pixel steps (nm)
  int au, av, H, W;
};

__global__ void k_bin_faces(const int32_t* cfaces, int nfc, const double* X, int nv, PixGrid g, int32_t* best) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfc) return;
  long long U[3], V[3];
  for (int k = 0; k < 3; ++k) {
    const int v = cfaces[k * nfc + f];
    U[k] = snap2(X[g.au * nv + v]);
    V[k] = snap2(X[g.av * nv + v]);
  }
  const long long A2 = edge_fn(U[0], V[0], U[1], V[1], U[2], V[2]);
  if (A2 == 0) return;
  const long long umin = min(U[0], min(U[1], U[2])), umax = max(U[0], max(U[1], U[2]));
  const long long vmin = min(V[0], min(V[1], V[2])), vmax = max(V[0], max(V[1], V[2]));
  // centre of column c: u0 + (2c+1) du  (doubled)
  long long c0 = -floor_div(-(umin - g.u0 - g.du), 2 * g.du);  // ceil
  long long c1 = floor_div(umax - g.u0 - g.du, 2 * g.du);
  long long r0 = -floor_div(-(vmin - g.v0 - g.dv), 2 * g.dv);
  long long r1 = floor_div(vmax - g.v0 - g.dv, 2 * g.dv);
  c0 = max(c0, 0ll);
  r0 = max(r0, 0ll);
  c1 = min(c1, (long long)g.W - 1);
  r1 = min(r1, (long long)g.H - 1);
  for (long long r = r0; r <= r1; ++r) {
    const long long pv = g.v0 + (2 * r + 1) * g.dv;
    for (long long c = c0; c <= c1; ++c) {
      const long long pu = g.u0 + (2 * c + 1) * g.du;
      const long long ea = edge_fn(U[1], V[1], U[2], V[2], pu, pv);
      const long long eb = edge_fn(U[2], V[2], U[0], V[0], pu, pv);
      const long long ec = edge_fn(U[0], V[0], U[1], V[1], pu, pv);
      const bool in = A2 > 0 ? (ea >= 0 && eb >= 0 && ec >= 0) : (ea <= 0 && eb <= 0 && ec <= 0);
      if (in) atomicMin(&best[r * g.W + c], f);  // lowest face index wins
    }
  }
}

__global__ void k_bin_weights(const int32_t* cfaces, int nfc, const double* X, int nv, PixGrid g, int32_t* best,
                              float* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int npix = g.H * g.W;
  if (i >= npix) return;
  int f = best[i];
  float w0 = 0.f, w1 = 0.f, w2 = 0.f;
  if (f == 0x7fffffff) {
    f = -1;
  } else {
    long long U[3], V[3];
    for (int k = 0; k < 3; ++k) {
      const int v = cfaces[k * nfc + f];
      U[k] = snap2(X[g.au * nv + v]);
      V[k] = snap2(X[g.av * nv + v]);
    }
    const int r = i / g.W, c = i % g.W;
    const long long pu = g.u0 + (2ll * c + 1) * g.du, pv = g.v0 + (2ll * r + 1) * g.dv;
    const double A2 = (double)edge_fn(U[0], V[0], U[1], V[1], U[2], V[2]);
    w0 = (float)__ddiv_rn((double)edge_fn(U[1], V[1], U[2], V[2], pu, pv), A2);
    w1 = (float)__ddiv_rn((double)edge_fn(U[2], V[2], U[0], V[0], pu, pv), A2);
    w2 = (float)__ddiv_rn((double)edge_fn(U[0], V[0], U[1], V[1], pu, pv), A2);
  }
  best[i] = f;
  w[i] = w0;
  w[npix + i] = w1;
  w[2 * npix + i] = w2;
}

bool grid_valid(const tc_grid* g) {
  if (!g || g->H <= 0 || g->W <= 0 || (int64_t)g->H * g->W > (int64_t)INT32_MAX / 3) return false;
  if (g->axis_u < 0 || g->axis_u > 2 || g->axis_v < 0 || g->axis_v > 2 || g->axis_u == g->axis_v) return false;
  for (int k = 0; k < 2; ++k)
    if (!std::isfinite(g->origin[k]) || !std::isfinite(g->pixel[k])) return false;
  return std::nearbyint(g->pixel[0] * 1e9) > 0 && std::nearbyint(g->pixel[1] * 1e9) > 0;
}

bool same_grid(const tc_grid& a, const tc_grid& b) {
  return a.axis_u == b.axis_u && a.axis_v == b.axis_v && a.origin[0] == b.origin[0] && a.origin[1] == b.origin[1] &&
         a.pixel[0] == b.pixel[0] && a.pixel[1] == b.pixel[1] && a.H == b.H && a.W == b.W;
}

// Covering contact face and FP32 barycentric weights of every pixel of
// `grid` over the rest contact surface (the binning reading of the pixel
// map: nanometre-snapped coordinates, exact edge functions, lowest face wins).
// Allocates the two tables from the env's arena on the env's stream.
tc_status bin_pixel_grid(Env& env, const tc_grid* grid, int32_t** pix_face, float** pix_w) {
  if (!grid_valid(grid)) return TC_ERR_INVALID_ARG;
  Arena& a = env.arena;
  cudaStream_t s = env.stream;
  const int npix = grid->H * grid->W;
  PixGrid g;
  g.au = grid->axis_u;
  g.av = grid->axis_v;
  g.H = grid->H;
  g.W = grid->W;
  g.u0 = 2ll * (long long)std::nearbyint(grid->origin[0] * 1e9);
  g.v0 = 2ll * (long long)std::nearbyint(grid->origin[1] * 1e9);
  g.du = (long long)std::nearbyint(grid->pixel[0] * 1e9);
  g.dv = (long long)std::nearbyint(grid->pixel[1] * 1e9);
  int32_t* pf = a.alloc<int32_t>(npix);
  float* pw = a.alloc<float>(3 * (int64_t)npix);
  if (!pf || !pw) {
    if (pf) a.put(pf);
    if (pw) a.put(pw);
    return TC_ERR_OOM;
  }
  k_fill_i32<<<grid_for(npix), kBlock, 0, s>>>(pf, npix, 0x7fffffff);
  if (env.nfc > 0) k_bin_faces<<<grid_for(env.nfc), kBlock, 0, s>>>(env.cfaces, env.nfc, env.X0, env.nv, g, pf);
  k_bin_weights<<<grid_for(npix), kBlock, 0, s>>>(env.cfaces, env.nfc, env.X0, env.nv, g, pf, pw);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  *pix_face = pf;
  *pix_w = pw;
  return TC_OK;
}

// ----------------------------------------------------------- indenter grid

// FP32 hi/lo pair of each indenter coordinate (x = hi + lo to ~2^-48 relative)
__global__ void k_split_hilo(const double* x, int64_t n, float* hi, float* lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = __double2float_rn(x[i]);
  hi[i] = h;
  lo[i] = __double2float_rn(x[i] - (double)h);
}

// body-frame box per primitive, rounded outward to FP32
__global__ void k_prim_boxes(const double* V, int nvi, const int32_t* prims, int n, int k, float* box) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < 3; ++d) {
    double lo = 1e308, hi = -1e308;
    for (int l = 0; l < k; ++l) {
      const int v = prims ? prims[l * n + i] : i;
      lo = fmin(lo, V[d * nvi + v]);
      hi = fmax(hi, V[d * nvi + v]);
    }
    box[i * 6 + d] = __double2float_rd(lo);
    box[i * 6 + 3 + d] = __double2float_ru(hi);
  }
}

struct GridSpec {
  float org[3];
  float inv_cell;
  int dims[3];
};

__global__ void k_prim_cell_count(const float* box, int n, GridSpec g, int32_t* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c0[3], c1[3];
  for (int d = 0; d < 3; ++d) {
    c0[d] = grid_cell(box[i * 6 + d], g.org[d], g.inv_cell, g.dims[d]);
    c1[d] = grid_cell(box[i * 6 + 3 + d], g.org[d], g.inv_cell, g.dims[d]);
  }
  cnt[i] = (c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) * (c1[2] - c0[2] + 1);
}

__global__ void k_prim_cell_emit(const float* box, int n, GridSpec g, const int32_t* off, uint64_t* keys,
                                 uint32_t* vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c0[3], c1[3];
  for (int d = 0; d < 3; ++d) {
    c0[d] = grid_cell(box[i * 6 + d], g.org[d], g.inv_cell, g.dims[d]);
    c1[d] = grid_cell(box[i * 6 + 3 + d], g.org[d], g.inv_cell, g.dims[d]);
  }
  int o = off[i];
  for (int z = c0[2]; z <= c1[2]; ++z)
    for (int y = c0[1]; y <= c1[1]; ++y)
      for (int x = c0[0]; x <= c1[0]; ++x) {
        const int cell = x + g.dims[0] * (y + g.dims[1] * z);
        keys[o] = ((uint64_t)(uint32_t)cell << 32) | (uint32_t)i;
        vals[o] = (uint32_t)o;
        ++o;
      }
}

// --------------------------------------------------------------- host side

static int bits_for(int64_t n) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) <= n) ++b;
  return b;
}

// CSR from keys (row << 32 | value), rows in [0, nrows).
static tc_status build_csr(Arena& a, uint64_t* keys, uint32_t* vals, int64_t n, int nrows, int low_bits,
                           int32_t** off_out, int32_t** idx_out) {
  radix_sort(keys, vals, n, 32 + bits_for(nrows), a);
  (void)low_bits;
  int32_t* counts = a.alloc<int32_t>(nrows + 1);
  int32_t* off = a.alloc<int32_t>(nrows + 1);
  int32_t* idx = a.alloc<int32_t>(n);
  if (!counts || !off || !idx) return TC_ERR_OOM;
  TC_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (nrows + 1), a.stream));
  if (n > 0) {
    k_row_counts<<<grid_for(n), kBlock, 0, a.stream>>>(keys, n, counts);
    k_low32<<<grid_for(n), kBlock, 0, a.stream>>>(keys, n, idx);
  }
  scan_exclusive(counts, off, nrows + 1, a);
  a.put(counts);
  *off_out = off;
  *idx_out = idx;
  return TC_OK;
}

// unique sorted edges of a face set (faces: 3 x nf device) -> edges (2 x ne)
static tc_status unique_edges(Arena& a, const int32_t* faces, int nf, int32_t** edges_out, int* ne_out) {
  const int64_t n = 3 * (int64_t)nf;
  uint64_t* keys = a.alloc<uint64_t>(n);
  uint32_t* vals = a.alloc<uint32_t>(n);
  int32_t* flag = a.alloc<int32_t>(n);
  int32_t* pos = a.alloc<int32_t>(n);
  if (!keys || !vals || !flag || !pos) return TC_ERR_OOM;
  if (n > 0) k_edge_keys<<<grid_for(n), kBlock, 0, a.stream>>>(faces, nf, keys, vals);
  radix_sort(keys, vals, n, 64, a);
  if (n > 0) k_unique_flag<<<grid_for(n), kBlock, 0, a.stream>>>(keys, n, flag);
  const int ne = (int)scan_exclusive(flag, pos, n, a);
  int32_t* edges = a.alloc<int32_t>(2 * (int64_t)ne);
  if (!edges) return TC_ERR_OOM;
  if (n > 0) k_edge_emit<<<grid_for(n), kBlock, 0, a.stream>>>(keys, flag, pos, n, edges, ne);
  a.put(keys);
  a.put(vals);
  a.put(flag);
  a.put(pos);
  *edges_out = edges;
  *ne_out = ne;
  return TC_OK;
}

template <class R> static tc_status setup_typed(Env& env) {
  Arena& a = env.arena;
  env.Dminv = a.alloc<R>(9 * (int64_t)env.nt);
  env.vol = a.alloc<R>(env.nt);
  if (!env.Dminv || !env.vol) return TC_ERR_OOM;
  k_rest_shape<R><<<grid_for(env.nt), kBlock, 0, a.stream>>>(env.tets, env.X0, env.nv, env.nt, (R*)env.Dminv,
                                                             (R*)env.vol, env.sc);
  return TC_OK;
}

template <class R> static tc_status setup_mass(Env& env) {
  env.mass = env.arena.alloc<R>(env.nv);
  if (!env.mass) return TC_ERR_OOM;
  k_mass<R><<<grid_for(env.nv), kBlock, 0, env.arena.stream>>>(env.vt_off, env.vt_idx, (const R*)env.vol, env.rho,
                                                               env.nv, (R*)env.mass);
  return TC_OK;
}

static tc_status read_status(Env& env, int* st) {
  TC_TRY(cudaMemcpyAsync(env.sc_host, env.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, env.stream));
  TC_TRY(cudaStreamSynchronize(env.stream));
  *st = env.sc_host->status;
  return TC_OK;
}

static tc_status build_grid(Env& env) {
  Arena& a = env.arena;
  const int nvi = env.ind_nv;
  // per-kind boxes
  const int counts[3] = {env.ind_nv, env.ind_ne, env.ind_nf};
  const int32_t* prims[3] = {nullptr, env.IE, env.IF};
  const int kk[3] = {1, 2, 3};
  for (int kind = 0; kind < 3; ++kind) {
    env.prim_box[kind] = a.alloc<float>(6 * (int64_t)std::max(counts[kind], 1));
    if (!env.prim_box[kind]) return TC_ERR_OOM;
    if (counts[kind] > 0)
      k_prim_boxes<<<grid_for(counts[kind]), kBlock, 0, a.stream>>>(env.IV, nvi, prims[kind], counts[kind], kk[kind],
                                                                   env.prim_box[kind]);
  }
  double lo[3], hi[3];
  bbox(env.IV, env.IV + nvi, env.IV + 2 * nvi, nvi, lo, hi, a);
  // cell edge: twice the mean indenter edge length, at most 2^22 cells
  std::vector<double> l2(env.ind_ne);
  double mean_len = 0.0;
  if (env.ind_ne > 0) {
    cudaMemcpyAsync(l2.data(), env.ind_elen2, sizeof(double) * env.ind_ne, cudaMemcpyDeviceToHost, a.stream);
    cudaStreamSynchronize(a.stream);
    for (double v : l2) mean_len += std::sqrt(v);
    mean_len /= env.ind_ne;
  }
  double ext[3], vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    ext[d] = std::max(hi[d] - lo[d], 1e-9);
    vol *= ext[d];
  }
  double cell = std::max(2.0 * mean_len, std::cbrt(vol / 4194304.0));
  cell = std::max(cell, 1e-7);
  GridSpec g;
  for (int d = 0; d < 3; ++d) {
    g.org[d] = (float)(lo[d] - 0.5 * cell);
    g.dims[d] = (int)std::ceil((ext[d] + cell) / cell) + 1;
    env.grid_org[d] = g.org[d];
    env.grid_dims[d] = g.dims[d];
  }
  g.inv_cell = (float)(1.0 / cell);
  env.grid_inv_cell = g.inv_cell;
  const int64_t ncells = (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
  for (int kind = 0; kind < 3; ++kind) {
    const int n = counts[kind];
    int32_t* cnt = a.alloc<int32_t>(n + 1);
    int32_t* off = a.alloc<int32_t>(n + 1);
    if (!cnt || !off) return TC_ERR_OOM;
    TC_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (n + 1), a.stream));
    if (n > 0) k_prim_cell_count<<<grid_for(n), kBlock, 0, a.stream>>>(env.prim_box[kind], n, g, cnt);
    const int64_t total = scan_exclusive(cnt, off, n + 1, a);
    uint64_t* keys = a.alloc<uint64_t>(total);
    uint32_t* vals = a.alloc<uint32_t>(total);
    if (!keys || !vals) return TC_ERR_OOM;
    if (n > 0) k_prim_cell_emit<<<grid_for(n), kBlock, 0, a.stream>>>(env.prim_box[kind], n, g, off, keys, vals);
    int32_t *start = nullptr, *items = nullptr;
    tc_status st = build_csr(a, keys, vals, total, (int)ncells, 32, &start, &items);
    if (st != TC_OK) return st;
    env.grid_start[kind] = start;
    env.grid_items[kind] = items;
    a.put(cnt);
    a.put(off);
    a.put(keys);
    a.put(vals);
  }
  return TC_OK;
}

tc_status setup_scene(Env& env, const tc_mesh* mesh, const int32_t* fixed_ids, int32_t nfixed, const tc_trimesh* ind,
                      const tc_grid* grid) {
  Arena& a = env.arena;
  cudaStream_t s = env.stream;
  const int nv = env.nv, nt = env.nt;
  // --- upload inputs (row-major host -> SoA device)
  std::vector<double> Xs(3 * (size_t)nv);
  for (int v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) Xs[(size_t)d * nv + v] = mesh->X[3 * (size_t)v + d];
  std::vector<float> Xf(Xs.begin(), Xs.end());  // FP32 copy for conservative broad-phase boxes
  env.X0 = a.alloc<double>(3 * (int64_t)nv);
  env.X0f = a.alloc<float>(3 * (int64_t)nv);
  env.tets = a.alloc<int4>(nt);
  env.fixed = a.alloc<uint8_t>(nv);
  if (!env.X0 || !env.X0f || !env.tets || !env.fixed) return TC_ERR_OOM;
  TC_TRY(cudaMemcpyAsync(env.X0, Xs.data(), sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.X0f, Xf.data(), sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.tets, mesh->tets, sizeof(int4) * nt, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemsetAsync(env.fixed, 0, nv, s));
  int32_t* dfix = a.alloc<int32_t>(std::max(nfixed, 1));
  if (!dfix) return TC_ERR_OOM;
  if (nfixed > 0) {
    TC_TRY(cudaMemcpyAsync(dfix, fixed_ids, sizeof(int32_t) * nfixed, cudaMemcpyHostToDevice, s));
    k_mark_fixed<<<grid_for(nfixed), kBlock, 0, s>>>(dfix, nfixed, env.fixed, nv, env.sc);
  }
  // --- rest shape
  tc_status st = env.precision == TC_FP64 ? setup_typed<double>(env) : setup_typed<float>(env);
  if (st != TC_OK) return st;
  // --- vertex -> tet incidence
  {
    const int64_t n = 4 * (int64_t)nt;
    uint64_t* keys = a.alloc<uint64_t>(n);
    uint32_t* vals = a.alloc<uint32_t>(n);
    if (!keys || !vals) return TC_ERR_OOM;
    k_vt_keys<<<grid_for(n), kBlock, 0, s>>>(env.tets, nt, keys, vals);
    st = build_csr(a, keys, vals, n, nv, 32, &env.vt_off, &env.vt_idx);
    if (st != TC_OK) return st;
    a.put(keys);
    a.put(vals);
  }
  if (env.dynamic) {
    st = env.precision == TC_FP64 ? setup_mass<double>(env) : setup_mass<float>(env);
    if (st != TC_OK) return st;
  }
  int dstat = 0;
  if ((st = read_status(env, &dstat)) != TC_OK) return st;
  if (dstat & ST_INVALID_MESH) return TC_ERR_INVALID_MESH;
  // --- boundary faces
  int32_t *bfaces = nullptr, *bparent = nullptr;
  {
    const int64_t n = 4 * (int64_t)nt;
    uint64_t* keys = a.alloc<uint64_t>(n);
    uint32_t* vals = a.alloc<uint32_t>(n);
    int32_t* flag = a.alloc<int32_t>(n);
    int32_t* pos = a.alloc<int32_t>(n);
    if (!keys || !vals || !flag || !pos) return TC_ERR_OOM;
    k_face_keys<<<grid_for(n), kBlock, 0, s>>>(env.tets, nt, keys, vals);
    radix_sort(keys, vals, n, 63, a);
    k_face_once<<<grid_for(n), kBlock, 0, s>>>(keys, n, flag);
    env.nf = (int)scan_exclusive(flag, pos, n, a);
    bfaces = a.alloc<int32_t>(3 * (int64_t)env.nf);
    bparent = a.alloc<int32_t>(env.nf);
    if (!bfaces || !bparent) return TC_ERR_OOM;
    k_face_emit<<<grid_for(n), kBlock, 0, s>>>(vals, flag, pos, n, env.tets, bfaces, bparent, env.nf);
    a.put(keys);
    a.put(vals);
    a.put(flag);
    a.put(pos);
    std::vector<int32_t> soa(3 * (size_t)env.nf);
    env.h_bparent.resize(env.nf);
    TC_TRY(cudaMemcpyAsync(soa.data(), bfaces, sizeof(int32_t) * 3 * env.nf, cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaMemcpyAsync(env.h_bparent.data(), bparent, sizeof(int32_t) * env.nf, cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    env.h_bfaces.resize(3 * (size_t)env.nf);
    for (int f = 0; f < env.nf; ++f)
      for (int k = 0; k < 3; ++k) env.h_bfaces[3 * (size_t)f + k] = soa[(size_t)k * env.nf + f];
  }
  // --- contact band: thinnest axis; side opposite the fixed set
  {
    double lo[3], hi[3];
    bbox(env.X0, env.X0 + nv, env.X0 + 2 * nv, nv, lo, hi, a);
    int ax = env.thick_axis;
    if (ax < 0 || ax > 2) {
      ax = 0;
      for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] < hi[ax] - lo[ax]) ax = d;
    }
    env.thick_axis = ax;
    int top = 1;
    if (nfixed > 0) {
      const int nb = 32;
      double* part = a.alloc<double>(nb);
      k_fixed_coord_sum<<<nb, kBlock, 0, s>>>(dfix, nfixed, env.X0 + (int64_t)ax * nv, part);
      std::vector<double> h(nb);
      TC_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
      TC_TRY(cudaStreamSynchronize(s));
      double sum = 0.0;
      for (double v : h) sum += v;
      top = (sum / nfixed <= 0.5 * (lo[ax] + hi[ax])) ? 1 : 0;
      a.put(part);
    }
    env.out_sign = top ? 1.0 : -1.0;
    uint8_t* band = a.alloc<uint8_t>(nv);
    int32_t* flag = a.alloc<int32_t>(std::max(env.nf, 1));
    int32_t* pos = a.alloc<int32_t>(std::max(env.nf, 1));
    if (!band || !flag || !pos) return TC_ERR_OOM;
    k_band<<<grid_for(nv), kBlock, 0, s>>>(env.X0 + (int64_t)ax * nv, nv, lo[ax], hi[ax], top, band);
    if (env.nf > 0) k_contact_flag<<<grid_for(env.nf), kBlock, 0, s>>>(bfaces, env.nf, band, flag);
    env.nfc = (int)scan_exclusive(flag, pos, env.nf, a);
    env.cfaces = a.alloc<int32_t>(3 * (int64_t)std::max(env.nfc, 1));
    env.cparent = a.alloc<int32_t>(std::max(env.nfc, 1));
    if (!env.cfaces || !env.cparent) return TC_ERR_OOM;
    if (env.nf > 0)
      k_contact_emit<<<grid_for(env.nf), kBlock, 0, s>>>(bfaces, bparent, env.nf, flag, pos, env.cfaces, env.cparent,
                                                         env.nfc);
    a.put(band);
    a.put(flag);
    a.put(pos);
  }
  a.put(dfix);
  a.put(bfaces);
  a.put(bparent);
  const int nfc = env.nfc;
  // host copies of the contact faces
  {
    std::vector<int32_t> soa(3 * (size_t)nfc);
    env.h_cparent.resize(nfc);
    if (nfc > 0) {
      TC_TRY(cudaMemcpyAsync(soa.data(), env.cfaces, sizeof(int32_t) * 3 * nfc, cudaMemcpyDeviceToHost, s));
      TC_TRY(cudaMemcpyAsync(env.h_cparent.data(), env.cparent, sizeof(int32_t) * nfc, cudaMemcpyDeviceToHost, s));
      TC_TRY(cudaStreamSynchronize(s));
    }
    env.h_cfaces.resize(3 * (size_t)nfc);
    for (int f = 0; f < nfc; ++f)
      for (int k = 0; k < 3; ++k) env.h_cfaces[3 * (size_t)f + k] = soa[(size_t)k * nfc + f];
  }
  // --- contact edges and vertices
  st = unique_edges(a, env.cfaces, nfc, &env.cedges, &env.nec);
  if (st != TC_OK) return st;
  {
    const int64_t n = 3 * (int64_t)nfc;
    uint64_t* keys = a.alloc<uint64_t>(n);
    uint32_t* vals = a.alloc<uint32_t>(n);
    int32_t* flag = a.alloc<int32_t>(n);
    int32_t* pos = a.alloc<int32_t>(n);
    env.vslot = a.alloc<int32_t>(nv);
    if (!keys || !vals || !flag || !pos || !env.vslot) return TC_ERR_OOM;
    k_fill_i32<<<grid_for(nv), kBlock, 0, s>>>(env.vslot, nv, -1);
    if (n > 0) k_vert_keys<<<grid_for(n), kBlock, 0, s>>>(env.cfaces, nfc, keys, vals);
    radix_sort(keys, vals, n, 32, a);
    if (n > 0) k_unique_flag<<<grid_for(n), kBlock, 0, s>>>(keys, n, flag);
    env.nvc = (int)scan_exclusive(flag, pos, n, a);
    env.cverts = a.alloc<int32_t>(std::max(env.nvc, 1));
    if (!env.cverts) return TC_ERR_OOM;
    if (n > 0) k_vert_emit<<<grid_for(n), kBlock, 0, s>>>(keys, flag, pos, n, env.cverts, env.vslot);
    a.put(keys);
    a.put(vals);
    a.put(flag);
    a.put(pos);
  }
  env.cface_slot = a.alloc<int32_t>(3 * (int64_t)std::max(nfc, 1));
  if (!env.cface_slot) return TC_ERR_OOM;
  if (nfc > 0) k_face_slots<<<grid_for(3 * nfc), kBlock, 0, s>>>(env.cfaces, nfc, env.vslot, env.cface_slot);
  // vertex -> face and vertex -> edge incidence of the contact surface
  {
    const int64_t n = 3 * (int64_t)nfc;
    uint64_t* keys = a.alloc<uint64_t>(n);
    uint32_t* vals = a.alloc<uint32_t>(n);
    if (!keys || !vals) return TC_ERR_OOM;
    if (n > 0) k_incidence_keys<<<grid_for(n), kBlock, 0, s>>>(env.cfaces, nfc, 3, env.vslot, keys, vals);
    st = build_csr(a, keys, vals, n, env.nvc, 32, &env.cv_face_off, &env.cv_face_idx);
    if (st != TC_OK) return st;
    a.put(keys);
    a.put(vals);
  }
  {
    const int64_t n = 2 * (int64_t)env.nec;
    uint64_t* keys = a.alloc<uint64_t>(n);
    uint32_t* vals = a.alloc<uint32_t>(n);
    if (!keys || !vals) return TC_ERR_OOM;
    if (n > 0) k_incidence_keys<<<grid_for(n), kBlock, 0, s>>>(env.cedges, env.nec, 2, env.vslot, keys, vals);
    st = build_csr(a, keys, vals, n, env.nvc, 32, &env.cv_edge_off, &env.cv_edge_idx);
    if (st != TC_OK) return st;
    a.put(keys);
    a.put(vals);
  }
  // rest edge lengths; default barrier stiffness kappa = E * mean edge length
  {
    env.gel_elen2 = a.alloc<double>(std::max(env.nec, 1));
    const int nb = 32;
    double* part = a.alloc<double>(nb);
    if (!env.gel_elen2 || !part) return TC_ERR_OOM;
    k_edge_len2<<<nb, kBlock, 0, s>>>(env.cedges, env.nec, env.X0, nv, env.gel_elen2, part);
    std::vector<double> h(nb);
    TC_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    double sum = 0.0;
    for (double v : h) sum += v;
    if (env.kappa <= 0.0) env.kappa = env.nec > 0 ? env.E * sum / env.nec : env.E * 1e-3;
    a.put(part);
  }
  // --- pixel binning
  if (grid) {
    st = bin_pixel_grid(env, grid, &env.pix_face, &env.pix_w);
    if (st != TC_OK) return st;
    env.H = grid->H;
    env.W = grid->W;
    env.grid0 = *grid;
    const int npix = env.H * env.W;
    env.h_pix_face.resize(npix);
    env.h_pix_w.resize(3 * (size_t)npix);
    std::vector<float> soa(3 * (size_t)npix);
    TC_TRY(cudaMemcpyAsync(env.h_pix_face.data(), env.pix_face, sizeof(int32_t) * npix, cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaMemcpyAsync(soa.data(), env.pix_w, sizeof(float) * 3 * npix, cudaMemcpyDeviceToHost, s));
    TC_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < npix; ++i)
      for (int k = 0; k < 3; ++k) env.h_pix_w[3 * (size_t)i + k] = soa[(size_t)k * npix + i];
  }
  // --- indenter (body frame)
  {
    const int ni = ind->nv, nfi = ind->nf;
    env.ind_nv = ni;
    env.ind_nf = nfi;
    std::vector<double> Vs(3 * (size_t)ni);
    for (int v = 0; v < ni; ++v)
      for (int d = 0; d < 3; ++d) Vs[(size_t)d * ni + v] = ind->V[3 * (size_t)v + d];
    std::vector<int32_t> Fs(3 * (size_t)nfi);
    for (int f = 0; f < nfi; ++f)
      for (int k = 0; k < 3; ++k) {
        const int32_t id = ind->F[3 * (size_t)f + k];
        if (id < 0 || id >= ni) return TC_ERR_INVALID_ARG;
        Fs[(size_t)k * nfi + f] = id;
      }
    env.IV = a.alloc<double>(3 * (int64_t)ni);
    env.IF = a.alloc<int32_t>(3 * (int64_t)nfi);
    if (!env.IV || !env.IF) return TC_ERR_OOM;
    TC_TRY(cudaMemcpyAsync(env.IV, Vs.data(), sizeof(double) * 3 * ni, cudaMemcpyHostToDevice, s));
    TC_TRY(cudaMemcpyAsync(env.IF, Fs.data(), sizeof(int32_t) * 3 * nfi, cudaMemcpyHostToDevice, s));
    env.IVhi = a.alloc<float>(3 * (int64_t)ni);
    env.IVlo = a.alloc<float>(3 * (int64_t)ni);
    if (!env.IVhi || !env.IVlo) return TC_ERR_OOM;
    k_split_hilo<<<grid_for(3 * (int64_t)ni), kBlock, 0, s>>>(env.IV, 3 * (int64_t)ni, env.IVhi, env.IVlo);
    st = unique_edges(a, env.IF, nfi, &env.IE, &env.ind_ne);
    if (st != TC_OK) return st;
    env.ind_elen2 = a.alloc<double>(std::max(env.ind_ne, 1));
    if (!env.ind_elen2) return TC_ERR_OOM;
    k_edge_len2<<<32, kBlock, 0, s>>>(env.IE, env.ind_ne, env.IV, ni, env.ind_elen2, nullptr);
    st = build_grid(env);
    if (st != TC_OK) return st;
  }
  TC_TRY(cudaStreamSynchronize(s));
  return TC_OK;
}

}  // namespace tc
