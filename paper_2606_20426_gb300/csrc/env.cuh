// Device layout of one environment (gel pad + rigid indenter + pixel grid).
//
// Everything is structure-of-arrays in HBM so that per-tet and per-vertex
// passes are coalesced:
//   per tet   : tets (int4), Dm^-1 (9 x nt), vol, H9 (45 x nt, PSD dP/dF),
//               eslot (36 x nt: 12 gradient + 24 diagonal-block entries),
//               yslot (12 x nt: element share of H p in PCG)
//   per vertex: rest X (double, 3 x nv), displacement u, velocity v, Newton
//               and PCG vectors (3 x nv each), block-Jacobi inverse (6 x nv)
//   contact   : gel contact vertices / edges / faces with per-primitive
//               slots (gradient + packed symmetric Hessian block) filled by
//               the barrier kernels and gathered per vertex
//   indenter  : body-frame vertices (double), faces, edges, uniform grid
//   pixels    : covering face + barycentric weights per pixel
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <mutex>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "prims.cuh"
#include "prof.cuh"

namespace tc {

// Uniform grid over the indenter's body-frame bounding box.  Boxes are FP32,
// rounded outward from the FP64 geometry, and cells are computed with
// grid_cell() both when binning and when querying, so every query visits
// exactly the cells a primitive was binned into.
struct GridView {
  float org[3];
  float inv_cell;
  int dims[3];
  const int32_t* start[3];   // per primitive kind (0 vert, 1 edge, 2 face): ncells + 1
  const int32_t* items[3];   // primitive ids, ascending within a cell
  const float* box[3];       // per primitive body-frame AABB (lo xyz, hi xyz)
};

TC_HD int grid_cell(float x, float org, float inv_cell, int dim) {
  const float f = floorf((x - org) * inv_cell);
  int c = f < 0.f ? 0 : (f >= (float)dim ? dim - 1 : (int)f);
  return c;
}

// Entry q (0..89) of tet el's stiffness blocks: groups of 8 consecutive tets
// store each entry contiguously, so a warp writing entry q of 32 tets fills
// four 32-byte sectors, while the 9 entries of one block of one tet stay
// within 288 bytes for the assembly gather.
constexpr int kKblkGroup = 8;
TC_HD int64_t kblk_index(int el, int q) {
  return ((int64_t)(el / kKblkGroup) * 90 + q) * kKblkGroup + (el % kKblkGroup);
}
TC_HD int64_t kblk_size(int nt) { return (int64_t)90 * ((nt + kKblkGroup - 1) / kKblkGroup) * kKblkGroup; }

// Everything a kernel needs, passed by value.
template <class R> struct EnvView {
  int nv, nt, nfc, nec, nvc, ind_nv, ind_nf, ind_ne, npix;
  R mu, lam_hat, alpha;       // material (rest-stable Neo-Hookean part)
  R kh;                       // log-term coefficient mu_s / 4 (full stable Neo-Hookean) or 0
  const R* mat;               // per-tet (mu, lam_hat[, kh]) as 2 (3 with the log law) x nt, or null
  R inv_h2;                   // 1/dt^2 (dynamic) or 0
  double dhat, kappa;
  int pcg_max;                // this env's PCG iteration cap
  // lagged friction (mu_f = 0: off): friction ratio, smoothing width eps_v dt,
  // indenter pose at the step start, and per gel primitive kind the lagged
  // pairs: fr_n[k][prim] pairs, pair j's indenter primitive at
  // fr_ip[k][j * n_k + prim] and its 8 values (lambda, normal xyz, closest-point
  // weights of the 4 pair points) at fr_val[k][(8 j + q) * n_k + prim]
  R mu_f, eps_x;
  double Rm0[9], tr0[3];
  int32_t* fr_n[3];
  int32_t* fr_ip[3];
  R* fr_val[3];
  // topology
  const int4* tets;
  const double* X0;           // rest positions, SoA x|y|z, each nv
  const float* X0f;           // X0 rounded to FP32 (broad-phase boxes only)
  const uint8_t* fixed;       // 1 = fixed vertex
  const int32_t* vt_off;      // vertex -> (tet*4+corner), CSR
  const int32_t* vt_idx;
  // per tet
  const R* Dminv;             // 9 x nt (row-major entry k at k*nt + e)
  const R* vol;
  R* eslot;                   // 12 x nt element gradient per (corner, component)
  R* kblk;                    // the element's PSD 12x12 stiffness as its 10 upper 3x3
                              // corner blocks (a <= b, row-major): 90 entries per tet,
                              // interleaved by groups of 8 tets (kblk_index)
  // per vertex
  const R* mass;              // nv (dynamic) or null
  R* u;                       // 3 x nv displacement
  R* ut;                      // 3 x nv line-search trial displacement
  R* utilde;                  // 3 x nv inertial target u_t + h v (dynamic)
  R* u0;                      // 3 x nv displacement at the start of the step
  R* vel;                     // 3 x nv velocity (dynamic)
  double dt;                  // time step (<= 0: quasi-static)
  R* g;                       // 3 x nv gradient
  R* Minv;                    // 6 x nv block-Jacobi inverse (xx,yy,zz,xy,yz,zx)
  R *dx, *r, *z, *p, *q;      // 3 x nv PCG vectors
  R* p2;                      // 3 x nv second direction buffer (alternates with p)
  const R* wd;                // 3 x nv warm-start direction of the next solve (dx or dfirst)
  // contact surface
  const int32_t* cverts;      // nvc vertex ids
  const int32_t* cedges;      // 2 x nec
  const int32_t* cfaces;      // 3 x nfc vertex ids
  const int32_t* vslot;       // nv -> contact vertex slot or -1
  const int32_t* cv_face_off; // contact vertex -> face*4+local
  const int32_t* cv_face_idx;
  const int32_t* cv_edge_off; // contact vertex -> edge*4+local
  const int32_t* cv_edge_idx;
  const double* gel_elen2;    // nec rest squared lengths
  R* cv_slot;                 // 9 x nvc  (3 g + 6 H)
  R* ce_slot;                 // 27 x nec (6 g + 21 H)
  R* cf_slot;                 // 54 x nfc (9 g + 45 H)
  // block-sparse (BSR, 3x3 blocks) Newton matrix over the free vertices
  int nnzb;
  const int32_t* bsr_rp;      // nv + 1 row offsets (fixed rows are empty)
  const int32_t* bsr_ci;      // nnzb column vertex ids, ascending per row
  const int32_t* bsr_diag;    // nv: position of the diagonal block, -1 if fixed
  const int32_t* be_off;      // nnzb + 1: element contributions of each block
  const int32_t* be_idx;      //   tet*16 + a*4 + b (corner a's row, corner b's column)
  const int32_t* bc_off;      // nnzb + 1: contact contributions of each block
  const int32_t* bc_idx;      //   kind<<30 | a<<28 | b<<26 | primitive
  // The block entries are stored sliced (SELL-32): the free rows (non-empty
  // rows, ascending) form slices of 32; slice s owns slots
  // [sell_off[s], sell_off[s + 1]), 32 per block position, so block kk of
  // the row with free index f sits in slot sell_off[f / 32] + 32 kk + f % 32
  // (a slice is as wide as its longest row; shorter rows leave their tail
  // slots unused).  A warp reading block kk of 32 consecutive rows reads 32
  // consecutive slots.
  int nfree;                  // free rows
  int nsell;                  // slots (>= nnzb)
  const int32_t* free_v;      // nfree: vertex of each free row, ascending
  const int32_t* free_of;     // nv: free index of each vertex, -1 for an empty row
  const int32_t* sell_off;    // nfree / 32 (rounded up) + 1 slot offsets
  const int32_t* sell_ci;     // nsell column vertex ids (unused slots: the row itself)
  R* bsr_val;                 // 9 x nsell block entries (entry r*3+c of slot t at (r*3+c)*nsell + t)
  // indenter (body frame)
  const double* IV;           // 3 x ind_nv SoA
  const float* IVhi;          // IV as FP32 hi + lo pairs (hi = fl(IV), lo = fl(IV - hi))
  const float* IVlo;
  const int32_t* IF;          // 3 x ind_nf
  const int32_t* IE;          // 2 x ind_ne
  const double* ind_elen2;    // ind_ne
  GridView grid;
  // candidate indenter primitives per gel contact primitive (kind 0 vertex,
  // 1 edge, 2 face): cand[k][j * n_k + prim], j < min(cand_n[k][prim], cand_cap)
  int32_t* cand[3];
  int32_t* cand_n[3];
  int cand_cap;
  double Rm[9], tr[3];        // current indenter pose (world = R body + t)
  Scalars* sc;                // this env's scalars (per phase in a batch)
};

// ------------------------------------------------------------ batching
//
// Every Newton phase runs as one launch over all envs taking part in it.
// Work is cut into units (one block each) of one item kind; per kind, a
// prefix table over the batch's envs maps a block to (env, chunk).  Per-unit
// partial sums are folded per env, in unit order, by per-env finalize kernels,
// so results do not depend on scheduling or on the batch composition.

enum Kind : int {
  K_TET = 0,   // tets, 256 per unit
  K_VERT,      // vertices, 256 per unit
  K_VGRP,      // vertices gathered by 8-lane groups, 32 per unit
  K_CV,        // contact vertices, 128 per unit
  K_CE,        // contact edges, 128 per unit
  K_CF,        // contact faces, 128 per unit
  K_NKIND
};

TC_HD int unit_items(int kind) {
  return kind == K_VGRP ? 32 : (kind >= K_CV ? 128 : 256);
}

// Indenter motion of one env for a CCD pass: gel positions (moved by dx when
// use_dir) seen from pose (Ra, ta) at the start and (Rb, tb) at the end.
struct Motion {
  double Ra[9], ta[3], Rb[9], tb[3];
  float Raf[9], taf[3], Rbf[9], tbf[3];  // FP32 copies for the broad phase
  int use_dir;
};

template <class R> struct BatchView {
  const EnvView<R>* views;   // nenv device views
  int nenv;
  const int* prefix;         // K_NKIND rows of nenv + 1 unit offsets
  double* part;              // per-unit partials (layout chosen by the launcher)
  const double* param;       // per-env scalar parameter (eta, alpha), or null
  const Motion* motion;      // per-env CCD motion, or null
};

struct Loc {
  int env, chunk;
};

// block -> (env, chunk) for one kind (binary search over the prefix row)
TC_D Loc locate(const int* prefix, int nenv, int kind, int unit) {
  const int* p = prefix + kind * (nenv + 1);
  int lo = 0, hi = nenv - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p[mid] <= unit) lo = mid;
    else hi = mid - 1;
  }
  return {lo, unit - p[lo]};
}

TC_HD int units_for(int count, int kind) { return (count + unit_items(kind) - 1) / unit_items(kind); }

struct EnvStats {
  int64_t newton = 0, pcg = 0, substeps = 0, steps = 0, halvings = 0;
  int64_t pcg_capped = 0;  // PCG solves that stopped at pcg_max above their tolerance
};

// Host-side environment.
struct Env {
  int device = 0;
  int precision = TC_FP64;
  cudaStream_t stream = nullptr;
  Arena arena;
  // sizes
  int nv = 0, nt = 0, nf = 0, nfc = 0, nec = 0, nvc = 0;
  int ind_nv = 0, ind_nf = 0, ind_ne = 0, H = 0, W = 0;
  // material / options
  double E = 0, nu = 0, rho = 0, mu = 0, lam = 0, lam_hat = 0, alpha = 0;
  int model = 0;              // TC_MODEL_SNH or TC_MODEL_SNH_LOG
  double kh = 0;              // log-term coefficient (mu_s / 4) of the full stable Neo-Hookean, else 0
  double dhat = 0, kappa = 0, dt = 0, rtol = 1e-6, gabs = 0, ptol = 0;
  int newton_max = 1024, pcg_max = 1000, thick_axis = 2;
  bool dynamic = false;
  double mu_f = 0.0, eps_v = 0.01;
  double out_sign = 1.0;      // outward direction of the contact side along thick_axis
  bool friction = false;      // dynamic and mu_f > 0
  tc_pose pose{};
  tc_pose pose_start{};       // indenter pose at the start of the current step
  // lagged friction pairs (allocated on first use, capacity fr_cap = the
  // candidate capacity per primitive); see EnvView
  int32_t* fr_n[3] = {nullptr, nullptr, nullptr};
  int32_t* fr_ip[3] = {nullptr, nullptr, nullptr};
  void* fr_val[3] = {nullptr, nullptr, nullptr};
  int fr_cap = 0;
  EnvStats stats;
  // device integer topology
  int4* tets = nullptr;
  double* X0 = nullptr;
  float* X0f = nullptr;
  uint8_t* fixed = nullptr;
  int32_t *vt_off = nullptr, *vt_idx = nullptr;
  int32_t *cverts = nullptr, *cedges = nullptr, *cfaces = nullptr, *cparent = nullptr, *vslot = nullptr;
  int32_t *cface_slot = nullptr;  // 3 x nfc contact-vertex slots of each face
  int32_t *cv_face_off = nullptr, *cv_face_idx = nullptr, *cv_edge_off = nullptr, *cv_edge_idx = nullptr;
  double* gel_elen2 = nullptr;
  int32_t* pix_face = nullptr;   // binning of the grid given at create time (grid0)
  float* pix_w = nullptr;
  tc_grid grid0{};
  // binnings of other grids passed to tc_pressure_map, least recently used
  // first out once more than kGridCache are held
  struct GridTable {
    tc_grid key;
    int32_t* pix_face;
    float* pix_w;
    uint64_t last_use;
  };
  static constexpr int kGridCache = 4;
  std::vector<GridTable> grid_tables;
  uint64_t grid_clock = 0;
  // indenter
  double* IV = nullptr;
  float *IVhi = nullptr, *IVlo = nullptr;
  int32_t *IF = nullptr, *IE = nullptr;
  int32_t* cand[3] = {nullptr, nullptr, nullptr};
  int32_t* cand_n[3] = {nullptr, nullptr, nullptr};
  int cand_cap = 0;
  bool cand_valid = false;    // lists cover the current state (see the CCD pass)
  double* ind_elen2 = nullptr;
  float grid_org[3] = {0, 0, 0}, grid_inv_cell = 1;
  int grid_dims[3] = {1, 1, 1};
  int32_t* grid_start[3] = {nullptr, nullptr, nullptr};
  int32_t* grid_items[3] = {nullptr, nullptr, nullptr};
  float* prim_box[3] = {nullptr, nullptr, nullptr};
  // typed fields (one of the two sets is allocated)
  void* mat_tet = nullptr;    // per-tet (mu, lam_hat[, kh]), 2 (3 with the log law) x nt, or null
  void* Dminv = nullptr;
  void* vol = nullptr;
  void* mass = nullptr;
  void *u = nullptr, *ut = nullptr, *vel = nullptr, *utilde = nullptr;
  void *eslot = nullptr, *kblk = nullptr, *bsr_val = nullptr;
  int nnzb = 0, nfree = 0, nsell = 0;
  int32_t *bsr_rp = nullptr, *bsr_ci = nullptr, *bsr_diag = nullptr;
  int32_t *free_v = nullptr, *free_of = nullptr, *sell_off = nullptr, *sell_ci = nullptr;
  int32_t *be_off = nullptr, *be_idx = nullptr, *bc_off = nullptr, *bc_idx = nullptr;
  void *g = nullptr, *Minv = nullptr, *dx = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  void* p2 = nullptr;
  void* dfirst = nullptr;     // solution of the last substep's first Newton solve (warm start)
  bool warm_first = false;    // the next solve is a substep's first: warm-start from dfirst
  void *cv_slot = nullptr, *ce_slot = nullptr, *cf_slot = nullptr;
  void* utrial = nullptr;
  // extraction scratch (float)
  float *sigma = nullptr, *face_p = nullptr, *face_A = nullptr, *vert_p = nullptr;
  // tables of a batched extraction led by this env (device from the arena,
  // pinned host staging), grown on demand
  void* x_dev = nullptr;
  void* x_host = nullptr;
  size_t x_cap = 0;
  Scalars* sc = nullptr;      // device (setup checks)
  Scalars* sc_host = nullptr; // pinned host mirror
  // host copies of integer outputs
  std::vector<int32_t> h_bfaces, h_bparent, h_cfaces, h_cparent, h_pix_face;
  std::vector<float> h_pix_w;
  int last_status = TC_OK;
  Profiler* prof = nullptr;  // per-kernel timing, null unless enabled
  void* exec = nullptr;      // BatchExec<R> of this env (batches of one)
  // working set (see acquire_working): resident or released, and its size
  bool work_resident = false;
  size_t work_bytes = 0;
  std::mutex api_mu;             // held by every public call on the env (and by a server releasing its working set)
  void* server = nullptr;        // the step server that meters this env's working set, if any
  uint64_t server_tick = 0;      // its last use by that server (least recently used first out)
  std::atomic<int> busy{0};      // step requests of this env queued or in flight on a server
  std::atomic<int> in_flight{0}; // 1 while one of them is admitted

  template <class R> EnvView<R> view() const;
};

template <class R> EnvView<R> Env::view() const {
  EnvView<R> e{};
  e.nv = nv; e.nt = nt; e.nfc = nfc; e.nec = nec; e.nvc = nvc;
  e.ind_nv = ind_nv; e.ind_nf = ind_nf; e.ind_ne = ind_ne; e.npix = H * W;
  e.mu = (R)mu; e.lam_hat = (R)lam_hat; e.alpha = (R)alpha; e.kh = (R)kh;
  e.mat = (const R*)mat_tet;
  e.inv_h2 = dynamic ? (R)(1.0 / (dt * dt)) : (R)0;
  e.dhat = dhat; e.kappa = kappa; e.pcg_max = pcg_max;
  e.mu_f = friction ? (R)mu_f : R(0);
  e.eps_x = friction ? (R)(eps_v * dt) : R(1);
  for (int k = 0; k < 9; ++k) e.Rm0[k] = pose_start.R[k];
  for (int k = 0; k < 3; ++k) e.tr0[k] = pose_start.t[k];
  for (int k = 0; k < 3; ++k) { e.fr_n[k] = fr_n[k]; e.fr_ip[k] = fr_ip[k]; e.fr_val[k] = (R*)fr_val[k]; }
  e.tets = tets; e.X0 = X0; e.X0f = X0f; e.fixed = fixed; e.vt_off = vt_off; e.vt_idx = vt_idx;
  e.Dminv = (const R*)Dminv; e.vol = (const R*)vol; e.eslot = (R*)eslot; e.kblk = (R*)kblk;
  e.nnzb = nnzb; e.bsr_rp = bsr_rp; e.bsr_ci = bsr_ci; e.bsr_diag = bsr_diag; e.bsr_val = (R*)bsr_val;
  e.nfree = nfree; e.nsell = nsell; e.free_v = free_v; e.free_of = free_of; e.sell_off = sell_off;
  e.sell_ci = sell_ci;
  e.be_off = be_off; e.be_idx = be_idx; e.bc_off = bc_off; e.bc_idx = bc_idx;
  e.mass = (const R*)mass; e.u = (R*)u; e.ut = (R*)utrial; e.utilde = (R*)utilde; e.g = (R*)g; e.Minv = (R*)Minv;
  e.u0 = (R*)ut; e.vel = (R*)vel; e.dt = dynamic ? dt : 0.0;
  e.dx = (R*)dx; e.r = (R*)r; e.z = (R*)z; e.p = (R*)p; e.q = (R*)q; e.p2 = (R*)p2;
  e.wd = (const R*)(warm_first && dfirst ? dfirst : dx);
  e.cverts = cverts; e.cedges = cedges; e.cfaces = cfaces; e.vslot = vslot;
  e.cv_face_off = cv_face_off; e.cv_face_idx = cv_face_idx; e.cv_edge_off = cv_edge_off; e.cv_edge_idx = cv_edge_idx;
  e.gel_elen2 = gel_elen2;
  e.cv_slot = (R*)cv_slot; e.ce_slot = (R*)ce_slot; e.cf_slot = (R*)cf_slot;
  e.IV = IV; e.IVhi = IVhi; e.IVlo = IVlo; e.IF = IF; e.IE = IE; e.ind_elen2 = ind_elen2;
  for (int k = 0; k < 3; ++k) { e.cand[k] = cand[k]; e.cand_n[k] = cand_n[k]; }
  e.cand_cap = cand_cap;
  for (int d = 0; d < 3; ++d) {
    e.grid.org[d] = grid_org[d];
    e.grid.dims[d] = grid_dims[d];
    e.grid.start[d] = grid_start[d];
    e.grid.items[d] = grid_items[d];
    e.grid.box[d] = prim_box[d];
  }
  e.grid.inv_cell = grid_inv_cell;
  for (int k = 0; k < 9; ++k) e.Rm[k] = pose.R[k];
  for (int k = 0; k < 3; ++k) e.tr[k] = pose.t[k];
  e.sc = sc;
  return e;
}

// ------------------------------------------------------------ entry points
// (defined in the .cu files; all return tc_status)

tc_status setup_scene(Env& env, const tc_mesh* mesh, const int32_t* fixed, int32_t nfixed,
                      const tc_trimesh* ind, const tc_grid* grid);
// The per-step working buffers of an env (element blocks and slots, Newton
// matrix values, gradient, block-Jacobi inverse, PCG vectors, line-search
// trial, contact slots, candidate lists): allocated if released (no-op when
// resident), and released.  Release only when no work of the env is pending.
tc_status acquire_working(Env& env);
void release_working(Env& env);
// A step server that meters the env's working set stops doing so (env destroyed).
void server_forget(Env& env);
// Pixel binning of a sensor grid over the env's rest contact surface
// (device tables allocated from the env's arena); grid checks.
tc_status bin_pixel_grid(Env& env, const tc_grid* grid, int32_t** pix_face, float** pix_w);
bool grid_valid(const tc_grid* g);
bool same_grid(const tc_grid& a, const tc_grid& b);
// BSR pattern and fixed-order contribution lists of the Newton matrix
// (host build from the host tets, after setup_scene)
tc_status build_bsr(Env& env, const int32_t* tets, const int32_t* fixed_ids, int32_t nfixed);

// Extraction.
template <class R> void launch_stress(const EnvView<R>& e, float* sigma, cudaStream_t s);
template <class R> void launch_traction(const EnvView<R>& e, const int32_t* cparent, float* t, float* p, float* tt,
                                        float* face_p, float* face_A, cudaStream_t s);
template <class R> int intersect_test(const EnvView<R>& e, int* dflag, cudaStream_t s);
void launch_vertex_avg(int nvc, const int32_t* off, const int32_t* idx, const float* face_p, const float* face_A,
                       float* vert_p, cudaStream_t s);
void launch_splat(int npix, const int32_t* pix_face, const float* pix_w, const int32_t* cface_slot, int nfc,
                  const float* vert_p, float* out, uint8_t* mask, cudaStream_t s);
void launch_stress_from_F(const float* F, int64_t n, float mu, float lam_hat, float alpha, float* sigma,
                          cudaStream_t s);
// Depth map of the deformed contact surface on a grid (Sec. III-D's depth).
template <class R>
tc_status launch_depth_map(const Env& env, const tc_grid& grid, float* out, uint8_t* mask, cudaStream_t s);
// Algorithm 2's per-contact-vertex force decomposition from the contact slots
// (run a contact pass at the current state first).
template <class R>
void launch_vertex_forces(const EnvView<R>& e, float* f, float* fn, float* ft, float* p, cudaStream_t s);
// sigma (K8) and the pressure map (K9-K10) of several envs of one precision in
// one cooperative launch on stream s; per env, sigma / map / mask may be null
// (a map needs the env's create-time grid).  Synchronises s.
template <class R>
tc_status extract_batch(const std::vector<Env*>& envs, const std::vector<float*>& sigma,
                        const std::vector<float*>& map, const std::vector<uint8_t*>& mask, cudaStream_t s);

}  // namespace tc

// The opaque handle of the C ABI.
struct tc_env {
  tc::Env impl;
};
