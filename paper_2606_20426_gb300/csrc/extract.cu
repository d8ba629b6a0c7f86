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
//
// The per-env kernels (k_traction, k_vertex_avg, k_splat, and k_stress in
// elem.cu) serve the single-env calls.  k_extract does all of it for a whole
// batch of envs in one cooperative launch: the face pressure and area of every
// contact face, then the contact-vertex means, then the pixels, with a
// grid-wide barrier between these three phases, while sigma of every tet
// streams in the gaps (see k_extract).  Each item goes through the same
// device functions as in the per-env kernels, so the outputs are the same bit
// for bit.  (A two-phase form in which every pixel averaged its three
// vertices itself was measured slower: 45 us against 37 us for 8 bench envs.)
#include <algorithm>
#include <climits>
#include <mutex>

#include "env.cuh"
#include "kin.cuh"
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
  R tv[3], n[3], pn, len;
  face_traction<R>(e, cparent, f, tv, n, pn, len);
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

// area-weighted mean over the incident faces of contact vertex s
TC_D float vertex_mean(int s, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                       const float* __restrict__ face_p, const float* __restrict__ face_A) {
  float num = 0.f, den = 0.f;
  for (int k = off[s]; k < off[s + 1]; ++k) {  // explicit roundings: the same value in every kernel
    const int f = idx[k] >> 2;
    const float A = face_A[f];
    num = __fmaf_rn(A, face_p[f], num);
    den = __fadd_rn(den, A);
  }
  return den > 0.f ? __fdiv_rn(num, den) : 0.f;
}

// barycentric combination of the three vertex values (one expression, shared
// by every path, so that all of them round the same way)
TC_D float bary(float w0, float w1, float w2, float v0, float v1, float v2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(w0, v0), __fmul_rn(w1, v1)), __fmul_rn(w2, v2));
}

// barycentric interpolation at pixel i of npix (0 and mask 0 off the surface)
TC_D void splat_pixel(int i, int npix, const int32_t* __restrict__ pix_face, const float* __restrict__ pix_w,
                      const int32_t* __restrict__ cface_slot, int nfc, const float* __restrict__ vert_p,
                      float* __restrict__ out, uint8_t* __restrict__ mask) {
  const int f = pix_face[i];
  float v = 0.f;
  if (f >= 0) {
    v = bary(pix_w[i], pix_w[npix + i], pix_w[2 * npix + i], vert_p[cface_slot[f]], vert_p[cface_slot[nfc + f]],
             vert_p[cface_slot[2 * nfc + f]]);
  }
  out[i] = v;
  if (mask) mask[i] = f >= 0 ? 1 : 0;
}

__global__ void __launch_bounds__(kBlock)
    k_vertex_avg(int nvc, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                 const float* __restrict__ face_p, const float* __restrict__ face_A, float* __restrict__ vert_p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nvc) return;
  vert_p[s] = vertex_mean(s, off, idx, face_p, face_A);
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
  splat_pixel(i, npix, pix_face, pix_w, cface_slot, nfc, vert_p, out, mask);
}

void launch_splat(int npix, const int32_t* pix_face, const float* pix_w, const int32_t* cface_slot, int nfc,
                  const float* vert_p, float* out, uint8_t* mask, cudaStream_t s) {
  if (npix > 0) TC_LAUNCH("k_splat", s, k_splat<<<grid_for(npix), kBlock, 0, s>>>(npix, pix_face, pix_w, cface_slot, nfc, vert_p, out, mask));
}

// ------------------------------------------------------------ depth map
// Height of the deformed contact surface seen from the contact side (the
// depth the optical rendering of Sec. III-D is constrained to): each thread
// projects one deformed contact face on the grid plane, and every pixel
// centre inside the closed projected triangle gets the barycentric
// interpolation of the vertices' outward heights (thickness-axis coordinate
// times the outward sign); the largest value wins (a z-buffer: atomicMax on
// an order-preserving integer image of the FP32 value, so the result does
// not depend on the order of the faces).  Edge functions and interpolation
// are FP64 with explicitly rounded operations in a fixed order.

struct DepthGrid {
  int au, av, H, W, ax;
  double u0, v0, du, dv, sign;
};

TC_D int depth_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : (i ^ 0x7fffffff);
}
TC_D float depth_value(int k) { return __int_as_float(k >= 0 ? k : (k ^ 0x7fffffff)); }
TC_D double edge_rn(double au, double av, double bu, double bv, double pu, double pv) {
  return __dsub_rn(__dmul_rn(__dsub_rn(bu, au), __dsub_rn(pv, av)), __dmul_rn(__dsub_rn(bv, av), __dsub_rn(pu, au)));
}

template <class R>
__global__ void __launch_bounds__(kBlock) k_depth_faces(const EnvView<R> e, DepthGrid g, int* __restrict__ key) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= e.nfc) return;
  const int nv = e.nv;
  double U[3], V[3], Hh[3];
  for (int k = 0; k < 3; ++k) {
    const int v = e.cfaces[k * e.nfc + f];
    U[k] = __dadd_rn(e.X0[g.au * nv + v], (double)e.u[g.au * nv + v]);
    V[k] = __dadd_rn(e.X0[g.av * nv + v], (double)e.u[g.av * nv + v]);
    Hh[k] = __dmul_rn(g.sign, __dadd_rn(e.X0[g.ax * nv + v], (double)e.u[g.ax * nv + v]));
  }
  const double A2 = edge_rn(U[0], V[0], U[1], V[1], U[2], V[2]);
  if (A2 == 0.0) return;
  const double umin = fmin(U[0], fmin(U[1], U[2])), umax = fmax(U[0], fmax(U[1], U[2]));
  const double vmin = fmin(V[0], fmin(V[1], V[2])), vmax = fmax(V[0], fmax(V[1], V[2]));
  // candidate columns / rows around the box, each tested exactly below
  // (clamped in floating point first, so that the conversions stay in range)
  const long long c0 = (long long)fmax(0.0, floor((umin - g.u0) / g.du - 0.5) - 1.0);
  const long long c1 = (long long)fmin((double)g.W - 1.0, ceil((umax - g.u0) / g.du - 0.5) + 1.0);
  const long long r0 = (long long)fmax(0.0, floor((vmin - g.v0) / g.dv - 0.5) - 1.0);
  const long long r1 = (long long)fmin((double)g.H - 1.0, ceil((vmax - g.v0) / g.dv - 0.5) + 1.0);
  for (long long r = r0; r <= r1; ++r) {
    const double pv = __dadd_rn(g.v0, __dmul_rn((double)r + 0.5, g.dv));
    if (pv < vmin || pv > vmax) continue;
    for (long long c = c0; c <= c1; ++c) {
      const double pu = __dadd_rn(g.u0, __dmul_rn((double)c + 0.5, g.du));
      if (pu < umin || pu > umax) continue;
      const double ea = edge_rn(U[1], V[1], U[2], V[2], pu, pv);
      const double eb = edge_rn(U[2], V[2], U[0], V[0], pu, pv);
      const double ec = edge_rn(U[0], V[0], U[1], V[1], pu, pv);
      const bool in = (ea >= 0 && eb >= 0 && ec >= 0) || (ea <= 0 && eb <= 0 && ec <= 0);
      if (!in) continue;
      const double h = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(ea, Hh[0]), __dmul_rn(eb, Hh[1])), __dmul_rn(ec, Hh[2])), A2);
      atomicMax(&key[r * g.W + c], depth_key((float)h));
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_depth_init(int* key, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) key[i] = INT_MIN;
}

__global__ void __launch_bounds__(kBlock) k_depth_resolve(float* out, uint8_t* mask, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = reinterpret_cast<const int*>(out)[i];
  const bool hit = k != INT_MIN;
  out[i] = hit ? depth_value(k) : 0.f;
  if (mask) mask[i] = hit ? 1 : 0;
}

// The map is built in place: `out` holds the integer keys until resolved.
template <class R>
tc_status launch_depth_map(const Env& env, const tc_grid& grid, float* out, uint8_t* mask, cudaStream_t s) {
  const int npix = grid.H * grid.W;
  DepthGrid g{grid.axis_u, grid.axis_v, grid.H, grid.W, env.thick_axis, grid.origin[0], grid.origin[1],
              grid.pixel[0], grid.pixel[1], env.out_sign};
  int* key = reinterpret_cast<int*>(out);
  TC_LAUNCH("k_depth_init", s, k_depth_init<<<grid_for(npix), kBlock, 0, s>>>(key, npix));
  if (env.nfc > 0)
    TC_LAUNCH("k_depth_faces", s, k_depth_faces<R><<<grid_for(env.nfc), kBlock, 0, s>>>(env.view<R>(), g, key));
  TC_LAUNCH("k_depth_resolve", s, k_depth_resolve<<<grid_for(npix), kBlock, 0, s>>>(out, mask, npix));
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
template tc_status launch_depth_map<float>(const Env&, const tc_grid&, float*, uint8_t*, cudaStream_t);
template tc_status launch_depth_map<double>(const Env&, const tc_grid&, float*, uint8_t*, cudaStream_t);

// ------------------------------------------------------- batched extraction

template <class R> struct XEnv {
  EnvView<R> v;
  const int32_t* cparent;
  const int32_t* cface_slot;
  const int32_t* pix_face;
  const float* pix_w;
  float *face_p, *face_A, *vert_p;
  float* sigma;    // 6 x nt or null
  float* map;      // H x W or null (then no face / vertex / pixel work)
  uint8_t* mask;   // H x W or null
  int npix;
};

template <class R> struct XBatch {
  const XEnv<R>* env;
  const int64_t* off;  // 4 rows of nenv + 1 item offsets: tets, faces, contact vertices, pixels
  int nenv;
  unsigned* bar;       // grid barrier: arrivals, generation
  int* err;            // set when a barrier wait gave up
};

// env whose item range [row[e], row[e+1]) holds item i
TC_D int env_of(const int64_t* row, int n, int64_t i) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Grid-wide barrier of a cooperative launch, in two halves so that a block
// can do independent work between its arrival and its wait.  Every block is
// resident, so the last arrival always comes; the wait is bounded all the
// same: after ~2^22 polls a block records the failure in *err and goes on
// (the host turns it into TC_ERR_CUDA).  grid_arrive returns, in thread 0,
// the generation to wait past; grid_wait returns false once *err is set.
TC_D unsigned grid_arrive(unsigned* bar) {
  __syncthreads();
  unsigned g = 0;
  if (threadIdx.x == 0) {
    g = *(volatile unsigned*)(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    }
  }
  return g;
}

TC_D bool grid_wait(unsigned* bar, int* err, unsigned g) {
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    int polls = 0;
    while (*gen == g) {
      __nanosleep(32);
      if (++polls > (1 << 22)) {
        atomicExch(err, 1);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

// Block b's share [lo, hi) of `total` items: contiguous, in whole groups of 32.
TC_D void block_share(int64_t total, int64_t& lo, int64_t& hi) {
  const int64_t g = (total + 31) >> 5, b = blockIdx.x, nb = gridDim.x;
  lo = min(total, 32 * (g * b / nb));
  hi = min(total, 32 * (g * (b + 1) / nb));
}

// Walks the items [lo, hi) of one kind with stride blockDim.x and keeps the
// env of the current item in registers: the env is found by a binary search
// over the offsets once, then advanced in order (an item's env never comes
// before the previous one's), and its fields are loaded only when it changes.
template <class R, class Ctx, class Load, class Body>
TC_D void for_items(const XBatch<R>& xb, const int64_t* row, int64_t lo, int64_t hi, Load load, Body body) {
  int64_t i = lo + threadIdx.x;
  if (i >= hi) return;
  int e = env_of(row, xb.nenv, i);
  int64_t beg = row[e], end = row[e + 1];
  Ctx c = load(xb.env[e]);
  for (; i < hi; i += blockDim.x) {
    if (i >= end) {
      do {
        ++e;
        beg = row[e];
        end = row[e + 1];
      } while (i >= end);
      c = load(xb.env[e]);
    }
    body(c, (int)(i - beg));
  }
}

template <class R> struct SigmaCtx {
  KinView<R> k;
  float* sigma;
};
template <class R> struct FaceCtx {
  KinView<R> k;
  const int32_t* cparent;
  float *face_p, *face_A;
};
struct VertCtx {
  const int32_t *off, *idx;
  const float *face_p, *face_A;
  float* vert_p;
};
struct PixCtx {
  const int32_t *pix_face, *cface_slot;
  const float *pix_w, *vert_p;
  float* map;
  uint8_t* mask;
  int npix, nfc;
};

// sigma (K8) of the tets [lo, hi) of the flattened tet range
template <class R> TC_D void x_sigma(const XBatch<R>& xb, int64_t lo, int64_t hi) {
  for_items<R, SigmaCtx<R>>(
      xb, xb.off, lo, hi, [](const XEnv<R>& x) { return SigmaCtx<R>{kin_view(x.v), x.sigma}; },
      [](const SigmaCtx<R>& c, int el) {
        R G[3][3], Bm[3][3], s6[6];
        load_G<R>(c.k, c.k.u, el, c.k.tets[el], G, Bm);
        R mu, lh, kh;
        tet_material<R>(c.k, el, mu, lh, kh);
        cauchy6<R>(G, kinematics<R>(G), mu, lh, kh, s6);
        const int64_t nt = c.k.nt;
#pragma unroll
        for (int q = 0; q < 6; ++q) c.sigma[q * nt + el] = (float)s6[q];
      });
}

// One cooperative launch over a batch of envs.  Every block takes an equal
// contiguous share of each kind of item.  Without maps it streams sigma of
// its tets.  With maps: the face pressure and area of its contact faces
// (K9); arrive at a grid barrier; a third of its sigma share (K8) while the
// other blocks arrive; wait; the area-weighted means of its contact vertices
// (K10a); arrive; the second third of sigma; wait; the pixels (K10b); the
// last third of sigma.  The barriers order only the face -> vertex -> pixel
// chain, and the sigma streams fill the time a block would spend waiting.
template <class R> __global__ void __launch_bounds__(kBlock) k_extract(const XBatch<R> xb, int with_map) {
  const int n = xb.nenv;
  const int64_t* tet_off = xb.off;
  const int64_t* face_off = xb.off + (n + 1);
  const int64_t* cv_off = xb.off + 2 * (n + 1);
  const int64_t* pix_off = xb.off + 3 * (n + 1);
  int64_t slo, shi;
  block_share(tet_off[n], slo, shi);
  if (!with_map) {
    x_sigma<R>(xb, slo, shi);
    return;
  }
  const int64_t s1 = slo + ((shi - slo) / 3 & ~(int64_t)31), s2 = s1 + ((shi - slo) / 3 & ~(int64_t)31);
  int64_t lo, hi;
  // faces (K9)
  block_share(face_off[n], lo, hi);
  for_items<R, FaceCtx<R>>(
      xb, face_off, lo, hi,
      [](const XEnv<R>& x) { return FaceCtx<R>{kin_view(x.v), x.cparent, x.face_p, x.face_A}; },
      [](const FaceCtx<R>& c, int f) {
        R tv[3], nrm[3], pn, len;
        face_traction<R>(c.k, c.cparent, f, tv, nrm, pn, len);
        c.face_p[f] = (float)(-pn);
        c.face_A[f] = (float)(R(0.5) * len);
      });
  unsigned g = grid_arrive(xb.bar);
  x_sigma<R>(xb, slo, s1);
  if (!grid_wait(xb.bar, xb.err, g)) return;
  // contact vertices (K10a)
  block_share(cv_off[n], lo, hi);
  for_items<R, VertCtx>(
      xb, cv_off, lo, hi,
      [](const XEnv<R>& x) { return VertCtx{x.v.cv_face_off, x.v.cv_face_idx, x.face_p, x.face_A, x.vert_p}; },
      [](const VertCtx& c, int s) { c.vert_p[s] = vertex_mean(s, c.off, c.idx, c.face_p, c.face_A); });
  g = grid_arrive(xb.bar);
  x_sigma<R>(xb, s1, s2);
  if (!grid_wait(xb.bar, xb.err, g)) return;
  // pixels (K10b)
  block_share(pix_off[n], lo, hi);
  for_items<R, PixCtx>(
      xb, pix_off, lo, hi,
      [](const XEnv<R>& x) { return PixCtx{x.pix_face, x.cface_slot, x.pix_w, x.vert_p, x.map, x.mask, x.npix, x.v.nfc}; },
      [](const PixCtx& c, int i) { splat_pixel(i, c.npix, c.pix_face, c.pix_w, c.cface_slot, c.nfc, c.vert_p, c.map, c.mask); });
  x_sigma<R>(xb, s2, shi);
}

// Resident blocks per SM of k_extract<R> (for the cooperative grid), once per device.
template <class R> static int extract_blocks_per_sm(int dev) {
  static std::mutex m;
  static int cache[64] = {};
  std::lock_guard<std::mutex> g(m);
  if (dev < 0 || dev >= 64) return 1;
  if (!cache[dev]) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extract<R>, kBlock, 0) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    cache[dev] = b;
  }
  return cache[dev];
}

template <class R>
tc_status extract_batch(const std::vector<Env*>& envs, const std::vector<float*>& sigma,
                        const std::vector<float*>& map, const std::vector<uint8_t*>& mask, cudaStream_t s) {
  const int n = (int)envs.size();
  if (n == 0) return TC_OK;
  Env& lead = *envs[0];
  // device table: XEnv[n] | off[4 (n+1)] | barrier[2] + err (in the lead env's arena, grown on demand)
  const size_t env_bytes = ((sizeof(XEnv<R>) * n + 255) / 256) * 256;
  const size_t off_bytes = ((sizeof(int64_t) * 4 * (n + 1) + 255) / 256) * 256;
  const size_t need = env_bytes + off_bytes + 256;
  if (need > lead.x_cap) {
    if (lead.x_dev) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return TC_ERR_CUDA;
      lead.arena.put(lead.x_dev);
    }
    if (lead.x_host) cudaFreeHost(lead.x_host);
    lead.x_dev = nullptr;
    lead.x_host = nullptr;
    lead.x_cap = 0;
    lead.x_dev = lead.arena.alloc<unsigned char>((int64_t)need);
    if (!lead.x_dev) return TC_ERR_OOM;
    if (cudaMallocHost(&lead.x_host, need) != cudaSuccess) {
      lead.x_host = nullptr;
      return TC_ERR_OOM;
    }
    lead.x_cap = need;
  }
  unsigned char* h = (unsigned char*)lead.x_host;
  XEnv<R>* hx = (XEnv<R>*)h;
  int64_t* hoff = (int64_t*)(h + env_bytes);
  bool any_map = false;
  for (int r = 0; r < 4; ++r) hoff[r * (n + 1)] = 0;
  for (int e = 0; e < n; ++e) {
    Env& v = *envs[e];
    const bool m = map[e] != nullptr && v.H * v.W > 0;
    any_map |= m;
    XEnv<R>& x = hx[e];
    x.v = v.view<R>();
    x.cparent = v.cparent;
    x.cface_slot = v.cface_slot;
    x.pix_face = v.pix_face;
    x.pix_w = v.pix_w;
    x.face_p = v.face_p;
    x.face_A = v.face_A;
    x.vert_p = v.vert_p;
    x.sigma = sigma[e];
    x.map = m ? map[e] : nullptr;
    x.mask = m ? mask[e] : nullptr;
    x.npix = v.H * v.W;
    hoff[0 * (n + 1) + e + 1] = hoff[0 * (n + 1) + e] + (sigma[e] ? v.nt : 0);
    hoff[1 * (n + 1) + e + 1] = hoff[1 * (n + 1) + e] + (m ? v.nfc : 0);
    hoff[2 * (n + 1) + e + 1] = hoff[2 * (n + 1) + e] + (m ? v.nvc : 0);
    hoff[3 * (n + 1) + e + 1] = hoff[3 * (n + 1) + e] + (m ? (int64_t)v.H * v.W : 0);
  }
  unsigned char* d = (unsigned char*)lead.x_dev;
  if (cudaMemcpyAsync(d, h, env_bytes + off_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return TC_ERR_CUDA;
  unsigned* bar = (unsigned*)(d + env_bytes + off_bytes);
  int* err = (int*)(bar + 2);
  if (cudaMemsetAsync(bar, 0, 16, s) != cudaSuccess) return TC_ERR_CUDA;
  int64_t most = 0;
  for (int r = 0; r < 4; ++r) most = std::max(most, hoff[r * (n + 1) + n] + (r == 0 ? hoff[1 * (n + 1) + n] : 0));
  if (most == 0) return TC_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TC_ERR_CUDA;
  const int64_t resident = (int64_t)sms * extract_blocks_per_sm<R>(dev);
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(resident, (most + kBlock - 1) / kBlock));
  XBatch<R> xb{(const XEnv<R>*)d, (const int64_t*)(d + env_bytes), n, bar, err};
  int with_map = any_map ? 1 : 0;
  void* args[] = {(void*)&xb, (void*)&with_map};
  cudaError_t ce = cudaSuccess;
  TC_LAUNCH("k_extract", s, ce = cudaLaunchCooperativeKernel((const void*)k_extract<R>, dim3(blocks), dim3(kBlock), args, 0, s));
  if (ce != cudaSuccess) return TC_ERR_CUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TC_ERR_CUDA;
  return herr ? TC_ERR_CUDA : TC_OK;
}

template void launch_traction<float>(const EnvView<float>&, const int32_t*, float*, float*, float*, float*, float*,
                                     cudaStream_t);
template void launch_traction<double>(const EnvView<double>&, const int32_t*, float*, float*, float*, float*, float*,
                                      cudaStream_t);
template tc_status extract_batch<float>(const std::vector<Env*>&, const std::vector<float*>&,
                                        const std::vector<float*>&, const std::vector<uint8_t*>&, cudaStream_t);
template tc_status extract_batch<double>(const std::vector<Env*>&, const std::vector<float*>&,
                                         const std::vector<float*>&, const std::vector<uint8_t*>&, cudaStream_t);

}  // namespace tc
