/*
 * tacauchy.h -- C ABI of the GB300 (sm_103a) TaCauchy hot-path library.
 *
 * One implicit step of a tetrahedral hyperelastic gel pad under
 * incremental-potential contact (IPC) with a rigid indenter, followed by the
 * paper's stress extraction:
 *   - Sec. III-B: Lame parameters (Eq. 1), stable Neo-Hookean material (Eq. 2),
 *     IPC barrier distance dhat, at most 1024 Newton iterations per step;
 *   - Sec. III-C: Cauchy stress per tet (Eq. 3, Eq. 4), traction t = sigma n
 *     (Eq. 5-6), normal pressure (Eq. 7), tangential traction (Eq. 8),
 *     Algorithm 1 (surface extraction + per-face decomposition);
 *   - Algorithm 2: the simulation loop (step, stress, traction, contact force
 *     f_k = -g_k / dt^2).
 *
 * Conventions
 *   - Units are SI (metres, pascals, newtons, seconds).
 *   - Every call returns tc_status (0 = TC_OK); nothing aborts or throws
 *     across the ABI.  Device-side failures are collected in a per-env status
 *     word and reported by the call that observes them.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the env's device (for example PyTorch tensors).
 *     Caller-owned buffers are only read or written during the call
 *     (device outputs: enqueued on the env's stream, complete when the call
 *     returns because every public call synchronises that stream).
 *   - The library owns all env state; it stays resident on the device between
 *     calls.  Inputs are copied at create time.
 *   - An env may be used by one host thread at a time.
 *   - Sizes are counts of elements, not bytes.
 */
#ifndef TACAUCHY_H
#define TACAUCHY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tc_status;
enum {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,          /* null pointer, negative size, bad enum    */
  TC_ERR_INVALID_MESH = 2,         /* tet with det(Dm) <= 0, index out of range */
  TC_ERR_INITIAL_PENETRATION = 3,  /* indenter touches or crosses the gel      */
  TC_ERR_NEWTON_MAXITER = 4,       /* Newton (or indenter substeps) hit the cap */
  TC_ERR_PCG_MAXITER = 5,          /* reserved, never returned: a PCG solve that
                                      reaches pcg_max is not an error; its
                                      iterate is still a descent direction and
                                      the Newton loop goes on with it
                                      (tc_info.pcg_capped counts such solves) */
  TC_ERR_LINESEARCH = 6,           /* no energy decrease after 60 halvings     */
  TC_ERR_NONFINITE = 7,            /* NaN/Inf in a pose, energy or direction   */
  TC_ERR_CUDA = 8,                 /* a CUDA runtime call failed               */
  TC_ERR_OOM = 9,                  /* device allocation failed                 */
  TC_ERR_ADMISSION = 10,           /* serving: env does not fit the HBM budget */
  TC_ERR_TIMEOUT = 11,             /* serving: wait ran out                    */
  TC_ERR_CAPACITY = 12             /* an internal fixed-size table overflowed  */
};

enum { TC_FP64 = 0, TC_FP32_MIXED = 1 };

/* Gel mesh (Algorithm 1 input (V, T)).  X: host, nv x 3 row-major rest
 * positions; tets: host, nt x 4 vertex ids, positively oriented
 * (det[X1-X0, X2-X0, X3-X0] > 0, else TC_ERR_INVALID_MESH). */
typedef struct { const double* X; int32_t nv; const int32_t* tets; int32_t nt; } tc_mesh;

/* Material laws (Sec. III-B): TC_MODEL_SNH, the rest-stable Neo-Hookean
 * Psi = mu/2 (I_C - 3) + lam_hat/2 (J - alpha)^2 - mu^2/(2 lam_hat) with
 * lam_hat = lam + mu, alpha = 1 + mu/lam_hat (the paper's Eq. 2 / Eq. 4
 * corrected to a stress-free rest state); TC_MODEL_SNH_LOG, the full stable
 * Neo-Hookean of Smith et al. 2018 that Sec. III-B cites,
 * Psi = mu_s/2 (I_C - 3) + lam_s/2 (J - alpha_s)^2 - mu_s/2 log(I_C + 1) - Psi(I)
 * with mu_s = 4/3 mu, lam_s = lam + 5/6 mu, alpha_s = 1 + 3 mu_s/(4 lam_s).
 * Both take Eq. 1's (mu, lam) and linearise to the same linear elasticity. */
enum { TC_MODEL_SNH = 0, TC_MODEL_SNH_LOG = 1 };

/* Material (Sec. III-B, Eq. 1).  Young's modulus E (Pa), Poisson ratio nu in
 * (-1, 0.5), density (kg/m^3, used only when dt > 0).  per_tet_E_nu: NULL
 * (homogeneous) or host nt x 2 row-major (E_t, nu_t) per tet, for
 * heterogeneous gels such as the dual-layer 9DTact pad of Sec. IV-D; each tet
 * then takes Eq. 1 and the law's parameters from its own pair (E and nu
 * above still set the default barrier stiffness).  Copied at create time.
 * model: TC_MODEL_SNH (0, the default of a zero-initialised struct) or
 * TC_MODEL_SNH_LOG; another value gives TC_ERR_INVALID_ARG.  The
 * standalone tc_stress_from_F evaluates TC_MODEL_SNH only. */
typedef struct { double E, nu, density; const double* per_tet_E_nu; int32_t model; } tc_material;

/* Solver options.
 *   dhat        IPC barrier distance (m), Sec. III-B.
 *   kappa       barrier stiffness (N/m); <= 0 selects E * mean rest length of
 *               the contact-surface edges.
 *   dt          time step (s); <= 0 selects the quasi-static problem.
 *   newton_rtol Newton stops when |g| <= newton_rtol * |g_0| (g_0: gradient at
 *               the first iterate of each indenter substep), or when
 *               |g| <= 1e-12 E L^2, or when the Newton step's max-norm is
 *               <= 1e-4 dhat (TC_FP64) / 1e-3 dhat (TC_FP32_MIXED), or when
 *               that step is below 10x those bounds and its predicted energy
 *               decrease is below the rounding level of the energy (1e-14 |E|
 *               in FP64, 1e-7 |E| in FP32 mixed).
 *   newton_max  Newton iterations per substep (1024 in Sec. III-B).
 *   pcg_max     PCG iterations per Newton iteration (per env, also when it
 *               runs in a batch with envs of other caps).
 *   precision   TC_FP64 (all device arithmetic in double) or TC_FP32_MIXED
 *               (element, barrier, PCG in float; energies, line-search and
 *               PCG dot-product accumulators in double; barrier distance in
 *               double for pairs closer than 1e-2 dhat).
 *   contact_axis thickness axis 0/1/2; -1 = thinnest bounding-box axis
 *               (Sec. III-A).
 *   friction_mu friction ratio of the lagged IPC friction (Sec. III-B gives
 *               0.5); 0 = frictionless.  Acts only when dt > 0.
 *   friction_eps_v velocity threshold of the friction smoothing in m/s
 *               (Sec. III-B gives 0.01); <= 0 selects 0.01.
 * Friction (IPC lagged friction, Li et al. 2020): at the start of each
 * indenter substep every contact pair within dhat fixes its normal force
 * lambda = kappa m(c) |b'(d)|, the normal of its closest-point vector and its
 * closest-point weights; the substep's potential adds
 * sum_k mu lambda_k f0(|P_k rel_k|), rel_k the relative displacement of the
 * pair's closest points since the step start (indenter points moving with the
 * kinematic pose), P_k the projection on the lagged tangent plane, f0 the C1
 * smoothing of |.| below eps_v dt. */
typedef struct {
  double dhat, kappa, dt, newton_rtol;
  int32_t newton_max, pcg_max, precision, contact_axis;
  double friction_mu, friction_eps_v;
} tc_scene_opts;

/* Rigid indenter surface in its body frame.  V: host nv x 3; F: host nf x 3. */
typedef struct { const double* V; int32_t nv; const int32_t* F; int32_t nf; } tc_trimesh;

/* Rigid pose: world = R * body + t, R row-major 3 x 3 (a rotation). */
typedef struct { double R[9]; double t[3]; } tc_pose;

/* Sensor pixel grid in the rest contact plane.  Pixel (r, c) has its centre
 * at (origin[0] + (c + 1/2) pixel[0], origin[1] + (r + 1/2) pixel[1]) in the
 * (axis_u, axis_v) coordinates of the rest configuration.  Coordinates are
 * snapped to whole nanometres for binning. */
typedef struct { int32_t axis_u, axis_v; double origin[2], pixel[2]; int32_t H, W; } tc_grid;

/* Optional device-memory provider (for example a PyTorch caching allocator).
 * alloc returns a device pointer aligned to 256 bytes or NULL; free releases
 * it.  With a NULL tc_allocator the library uses cudaMallocAsync/cudaFreeAsync
 * on the env's stream. */
typedef struct {
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*release)(void* ctx, void* ptr, size_t bytes, void* stream);
  void* ctx;
} tc_allocator;

typedef struct tc_env tc_env;

/* Counts and counters of an env (host struct filled by tc_env_info). */
typedef struct {
  int32_t nv, nt;            /* gel vertices, tets                          */
  int32_t nf;                /* boundary faces (Algorithm 1, step 2)        */
  int32_t nfc, nec, nvc;     /* contact faces, edges, vertices              */
  int32_t ind_nv, ind_nf, ind_ne;
  int32_t H, W;              /* pixel grid                                   */
  int64_t newton_iters, pcg_iters, substeps, steps, line_search_halvings;
  double kappa;              /* barrier stiffness in use (N/m)              */
  size_t device_bytes;       /* device memory held by the env               */
  int64_t nnzb;              /* 3x3 blocks of the Newton matrix (free rows)  */
  int64_t pcg_capped;        /* PCG solves that stopped at pcg_max above     */
                             /* their tolerance (not an error, see TC_ERR_PCG_MAXITER) */
  size_t working_bytes;      /* device bytes of the per-step working set      */
  int32_t working_resident;  /* 1 while the working set is allocated          */
} tc_info;

/* Scene setup (row a0): rest shape Dm^-1 and volumes, lumped masses, boundary
 * faces with parent tets, contact band and contact surface, vertex/face
 * incidence, pixel binning, indenter grid.  fixed: host, nfixed vertex ids
 * held at their rest positions.  start_pose: indenter pose at time 0 (must not
 * touch the gel: TC_ERR_INITIAL_PENETRATION).  grid may be NULL (no pressure
 * map).  cuda_stream: cudaStream_t the env's work is enqueued on (NULL = the
 * legacy default stream).  On success *out owns a new env. */
tc_status tc_create_scene(const tc_mesh* mesh, const tc_material* material,
                          const int32_t* fixed, int32_t nfixed,
                          const tc_trimesh* indenter, const tc_pose* start_pose,
                          const tc_scene_opts* opts, const tc_grid* grid,
                          const tc_allocator* allocator, void* cuda_stream,
                          tc_env** out);

/* One step (Algorithm 2, physics line): move the indenter from its current
 * pose to *target in CCD-limited substeps and minimise the incremental
 * potential of the gel at each substep.  Each Newton system is solved by
 * block-Jacobi PCG started from an earlier solve's solution d kept with the
 * env (the previous solve's; for the first solve of a substep, the previous
 * substep's first), scaled by the minimiser -g.d / d.A d of the quadratic
 * model along d; a fresh env starts from zero.  A step that fails
 * (TC_ERR_NEWTON_MAXITER, TC_ERR_LINESEARCH, TC_ERR_NONFINITE) leaves the env
 * as it was before the call: positions, velocities and indenter pose of the
 * step start. */
tc_status tc_step(tc_env* env, const tc_pose* target);

/* One step of each of n independent envs (Algorithm 2, physics line, applied
 * to every env), run together: each Newton phase (element pass, barrier pass,
 * assembly, PCG, CCD, line-search energy) is one launch over all envs still
 * iterating, so small envs share the GPU instead of running one after another.
 * Each env's result is the one tc_step would give it alone (the per-env
 * reductions are folded in the same order).  envs: host array of n distinct
 * envs of one precision and device; targets: host array of n poses;
 * statuses: host array of n, receiving each env's own status (a non-finite
 * target gives TC_ERR_NONFINITE for that env and leaves it unchanged).  The
 * work runs on the first env's stream after every other env's stream has
 * drained.  Returns TC_OK unless the call as a whole failed (invalid
 * arguments, CUDA error, allocation failure); n = 0 is a no-op. */
tc_status tc_step_batch(tc_env** envs, int32_t n, const tc_pose* targets,
                        tc_status* statuses);

/* Launch shape of the PCG (one thread-block cluster per env):
 * cluster_ctas in 1 .. 16 CTAs per env (clusters above 8 CTAs are a
 * non-portable size the GPU may not co-schedule), threads in {512, 1024} per
 * CTA.
 * Process-wide for the given precision (TC_FP64 or TC_FP32_MIXED), so an
 * env's result does not depend on the batch it runs in; changing it changes
 * the rounding of later steps.  TC_ERR_CAPACITY if the GPU cannot co-schedule
 * such a cluster.  Not in the paper. */
tc_status tc_pcg_shape(int32_t precision, int32_t cluster_ctas, int32_t threads);

typedef struct {
  int32_t cluster_ctas, threads;  /* the shape tried                         */
  int32_t coresident;             /* clusters of it the GPU holds at once    */
  double us_per_env_iter;         /* device time per CG iteration of one env  */
  int64_t env_iters;              /* CG iterations timed (all envs)           */
} tc_pcg_tune;

/* Autotuner: assemble the Newton systems of the n envs at their current
 * state (positions are not changed), time their PCG solves under every
 * co-schedulable shape of {16, 8} CTAs x {1024, 512} threads, and select the
 * shape with the least device time per CG iteration of one env.  mode 0 launches each env's solve alone, one
 * after another (the latency of one env's solve: requests on their own
 * server workers); mode 1 launches one solve over all n envs (the
 * throughput of a full batch).  results (host, up to max_results entries,
 * may be NULL when max_results is 0) receives one entry per shape tried and
 * *n_results their count.  The envs must share precision and device and have
 * no server request pending.  The timed solves start from zero and leave
 * their solution as the envs' next PCG warm start.  Not in the paper. */
tc_status tc_autotune_pcg(tc_env** envs, int32_t n, int32_t mode, tc_pcg_tune* results,
                          int32_t max_results, int32_t* n_results);

/* Cauchy stress per tet (Eq. 4 with the rest-stable reading):
 * sigma_out device float 6 x nt, component-major (component k of tet e at
 * k * nt + e), components in the order (xx, yy, zz, xy, yz, zx). */
tc_status tc_stress(tc_env* env, float* sigma_out);

/* Algorithm 1 per contact face (in tc_surface_faces order): traction
 * t = sigma n (device float 3 x nfc, component-major), pressure
 * p = -n.sigma.n (compression positive; Eq. 7's p_n = -p) (device float nfc),
 * tangential traction t_tau = t - (t.n) n (Eq. 8) (device float 3 x nfc).
 * n is the unit outward normal of the deformed face.  Any pointer may be NULL
 * to skip that output. */
tc_status tc_traction(tc_env* env, float* t, float* p, float* t_tau);

/* Pressure map on a sensor pixel grid (Sec. III-C: the traction field of
 * Algorithm 1 splatted onto the sensor's pixels): per-face pressure
 * area-weighted to contact vertices (deformed areas), interpolated
 * barycentrically at every pixel of `grid`.  grid: host tc_grid, or NULL for
 * the grid given at create time (TC_ERR_INVALID_ARG if there was none).  A
 * grid is binned over the rest contact surface on its first use and the
 * binning is kept with the env (the four most recently used grids besides
 * the create-time one); invalid grids (H or W <= 0, equal or out-of-range
 * axes, pixel sizes below 1 nm, non-finite values) give TC_ERR_INVALID_ARG.
 * out: device float H x W; mask: device uint8 H x W (1 = pixel covered by a
 * contact face) or NULL. */
tc_status tc_pressure_map(tc_env* env, const tc_grid* grid, float* out, uint8_t* mask);

/* Stress and pressure maps of several envs at once (Sec. III-C, Eq. 4 and
 * Algorithm 1 over every env): one launch computes sigma of every tet and the
 * pressure and area of every contact face of all the envs, averages to their
 * contact vertices and splats to their pixel grids (the create-time grids),
 * with a grid-wide barrier between those three phases.  The outputs equal,
 * bit for bit, what tc_stress and tc_pressure_map(env, NULL, ...) write for
 * each env.  envs: host array of n distinct envs of one precision and device
 * (none with a server request pending); sigma_out, map_out, mask_out: host
 * arrays of n device pointers (layouts as tc_stress and tc_pressure_map), each
 * array and each entry may be NULL to skip that output (a mask needs its map,
 * a map needs an env created with a grid: else TC_ERR_INVALID_ARG).  The work
 * runs on the first env's stream after every other env's stream has drained;
 * n = 0 is a no-op.  Not in the paper (which extracts one env per call). */
tc_status tc_extract_batch(tc_env** envs, int32_t n, float* const* sigma_out, float* const* map_out,
                           uint8_t* const* mask_out);

/* Depth map of the deformed contact surface (the depth that constrains the
 * optical rendering of Sec. III-D): at every pixel centre of `grid` (host, or
 * NULL for the create-time grid) covered by a deformed contact face projected
 * on the grid plane, the face's outward height (coordinate along the thickness
 * axis, sign-flipped when the contact side is the low side), interpolated
 * barycentrically in FP64 and rounded to FP32; where several faces cover a
 * centre the largest height wins (the surface nearest the indenter).
 * height: device float H x W (0 where uncovered); mask: device uint8 H x W
 * (1 = covered) or NULL.  No graphics API: one thread per contact face. */
tc_status tc_depth_map(tc_env* env, const tc_grid* grid, float* height, uint8_t* mask);

/* Algorithm 2's contact decomposition at every contact-surface vertex k (in
 * increasing vertex id: the vertices of tc_surface_faces' faces), at the
 * current state: the contact force f_k = -g_k / dt^2 (minus the barrier and
 * friction part of the gradient of the potential, which is scaled by dt^2),
 * the unit normal n_k (area-weighted mean of the incident deformed contact
 * faces' outward normals), the area A_k (a third of those faces' deformed
 * areas), f_n = (f.n) n, f_tau = f - f_n and the pressure p_k = |f_k| / A_k.
 * f, f_n, f_tau: device float 3 x nvc (component-major); p: device float nvc;
 * any may be NULL. */
tc_status tc_vertex_forces(tc_env* env, float* f, float* f_n, float* f_tau, float* p);

/* The contact-force pressure p_k = |f_k| / A_k of tc_vertex_forces on a pixel
 * grid, by the barycentric interpolation of tc_pressure_map (grid: host, or
 * NULL for the create-time grid; out device float H x W; mask device uint8
 * H x W or NULL).  A second pressure map beside the stress-based one. */
tc_status tc_force_pressure_map(tc_env* env, const tc_grid* grid, float* out, uint8_t* mask);

/* Incremental potential at the current positions and indenter pose
 * (Algorithm 2's minimisation objective: elastic energy + kappa * barrier
 * sum, plus the inertia term in the dynamic case) and its gradient w.r.t. the
 * gel positions with fixed vertices zeroed.  energy: host double or NULL;
 * grad: host double nv x 3 (row-major) or NULL; not both NULL. */
tc_status tc_energy_gradient(tc_env* env, double* energy, double* grad);

/* Total contact force on the gel, sum_k f_k with f_k = -kappa dB/dx_k
 * (Algorithm 2: f_k = -g_k / dt^2).  out: host double[3]. */
tc_status tc_contact_force(tc_env* env, double* out);

/* Contact faces (Algorithm 1, steps 1-3, restricted to the contact band):
 * faces host int32 nfc x 3 (outward winding, smallest id first, ordered by
 * sorted vertex triple), parent host int32 nfc.  Either may be NULL. */
tc_status tc_surface_faces(tc_env* env, int32_t* faces, int32_t* parent);

/* All boundary faces and parents (host int32 nf x 3 and nf), same order rules. */
tc_status tc_boundary_faces(tc_env* env, int32_t* faces, int32_t* parent);

/* Pixel binning table: face index per pixel (-1 = uncovered) host int32 H*W,
 * barycentric weights host float H*W x 3.  Either may be NULL. */
tc_status tc_pixel_table(tc_env* env, int32_t* pix_face, float* pix_w);

/* Current gel positions, host double nv x 3 (get) / set (for evaluating the
 * extraction on externally supplied positions). */
tc_status tc_get_positions(tc_env* env, double* x);
tc_status tc_set_positions(tc_env* env, const double* x);

tc_status tc_env_info(tc_env* env, tc_info* info);

/* Per-kernel timing with CUDA events on the env's stream (off by default).
 * on != 0 enables it and clears the totals; on == 0 disables it.  While on,
 * every kernel an API call launches for this env is bracketed by two events
 * (a small launch overhead).  tc_profile_read fills up to max entries
 * (kernel name, total milliseconds, launches) and sets *n to the number of
 * distinct kernels seen. */
typedef struct { char name[32]; double ms; int64_t launches; } tc_kernel_time;
tc_status tc_profile_enable(tc_env* env, int32_t on);
tc_status tc_profile_read(tc_env* env, tc_kernel_time* out, int32_t max, int32_t* n);
void tc_destroy(tc_env* env);
const char* tc_status_str(tc_status s);

/* Standalone stress kernel over deformation gradients (no env): sigma of
 * Eq. 4 (rest-stable reading) for n tets.  F: device float n x 9 (one
 * row-major 3 x 3 matrix per tet); sigma_out: device float 6 x n,
 * component-major as in tc_stress; stream: cudaStream_t or NULL. */
tc_status tc_stress_from_F(const float* F, int64_t n, double E, double nu,
                           float* sigma_out, void* stream);

/* Pressure map that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers, not for the method).  It is for callers
 * that cannot obtain device memory at the time of the call -- for example a
 * real-time control loop that forbids allocator calls after start-up, or code
 * running inside a foreign memory pool -- so it never calls cudaMalloc,
 * cudaFree or an allocating library routine.  It computes what
 * tc_pressure_map computes, from caller-supplied device arrays:
 *   x          float 3 x nv   deformed positions, component-major
 *   sigma      float 6 x nt   Cauchy stress as written by tc_stress
 *   cfaces     int32 3 x nfc  contact faces (outward winding), component-major
 *   cparent    int32 nfc      parent tet of each face
 *   cface_slot int32 3 x nfc  index of each face vertex among the nvc contact
 *                             vertices (sorted by vertex id)
 *   cv_face_off int32 nvc+1, cv_face_idx int32: per contact vertex, the
 *                             incident contact faces encoded face*4 + corner
 *   pix_face int32 npix, pix_w float 3 x npix: the binning of tc_pixel_table
 *   out float npix, mask uint8 npix (nullable)
 * Per-face and per-vertex intermediates live in one file-scope device array
 * of fixed size, shared by every call: at most 262,144 contact faces and
 * 262,144 contact vertices (TC_ERR_CAPACITY beyond), about 3 MB held on every
 * GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * keeps it; if the lookup fails the call returns TC_ERR_CUDA and the next call
 * tries again.  Make that first call on each device before any stream
 * capture.  With no contact face (nfc = 0) every pix_face entry must be -1;
 * out and mask are then all 0.  Calls that overlap on the
 * GPU (different streams, or different host threads) race on the shared
 * array; serialise them.  Synchronises `stream` before returning. */
tc_status tc_pressure_map_noalloc(const float* x, int32_t nv, const float* sigma, int32_t nt,
                                  const int32_t* cfaces, const int32_t* cparent,
                                  const int32_t* cface_slot, int32_t nfc,
                                  const int32_t* cv_face_off, const int32_t* cv_face_idx, int32_t nvc,
                                  const int32_t* pix_face, const float* pix_w, int32_t npix,
                                  float* out, uint8_t* mask, void* stream);

/* ------------------------------------------------------------------------
 * Step server: continuous batching of step requests from many envs.
 *
 * Not in the paper, which steps one env per call.  A server owns a pool of
 * worker threads, each with its own CUDA stream, on the device current at
 * creation.  tc_submit queues a request (env, target pose, optional output
 * buffers) and returns a ticket at once.  Device memory: an env's state is
 * a persistent part (rest shape, topology, positions, velocities, PCG warm
 * starts, pixel tables -- held from tc_create_scene to tc_destroy) and a
 * working set that only a step needs (element stiffness blocks, Newton
 * matrix values, gradient, PCG vectors, contact slots and candidate lists,
 * about two thirds of the env's memory).  The server meters the working sets
 * of the envs submitted to it against hbm_budget_bytes: a working set stays
 * resident after its request (the next request of that env reuses it), and
 * when a request needs room, the working sets of that server's envs with no
 * request in flight are released, least recently used first (an env being
 * used by a caller at that moment is skipped), and acquired again by their
 * next call that needs them (results do not change).  Before every
 * scheduling round a worker admits queued requests in FIFO order while it and
 * the server have free slots and the request's working set fits the budget;
 * a request waits while an earlier request of the same env is in flight, a
 * lone request is always admitted, and a request whose env's working set
 * alone exceeds the budget completes with TC_ERR_ADMISSION.  Each round advances every request of the worker by one phase
 * group of the implicit step (Algorithm 2, physics line) with one launch set
 * per phase over all of them, so requests that arrive while others are on the
 * GPU join at the next round boundary, and workers overlap on the device.
 * A request's result equals tc_step on the same env and pose (bit for bit).
 * When it finishes, its stress (as tc_stress) and pressure map (as
 * tc_pressure_map) are written to the buffers given at submit, and the
 * ticket completes.  While a request is queued or in flight its env belongs
 * to the server: tc_step, tc_step_batch and tc_set_positions on it return
 * TC_ERR_INVALID_ARG, and no other call may use it.  All calls are
 * thread-safe; tc_server_destroy must not overlap any other call on the
 * same server.
 * ---------------------------------------------------------------------- */
typedef struct tc_server tc_server;

typedef struct {
  tc_status status;   /* the step's status (TC_ERR_ADMISSION: the env never
                         fits the budget, or the server shut down first) */
  double queue_us;    /* submit -> admitted into the running batch          */
  double latency_us;  /* submit -> step done and outputs written            */
  int32_t rounds;     /* scheduling rounds the request took part in         */
} tc_result;

typedef struct {
  int64_t submitted, completed, rounds;
  int32_t queued, inflight, peak_inflight, max_slots, workers;
  size_t inflight_bytes;   /* working-set bytes resident for the server's envs */
  size_t budget_bytes;
  int64_t evictions;       /* working sets released to make room            */
  int32_t known_envs;      /* envs whose working sets the server meters      */
} tc_server_stats;

/* hbm_budget_bytes > 0: bound on the summed working sets resident for the
 * server's envs (see above);
 * max_slots > 0: bound on the number of requests in flight; workers: worker
 * threads, each with its own CUDA stream and scheduler holding up to
 * ceil(max_slots / workers) requests (<= 0: one worker per slot, so every
 * request iterates independently; 1: a single batch over all requests). */
tc_status tc_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t workers, tc_server** out);

/* Queue one step of env toward *target (host pose; non-finite:
 * TC_ERR_NONFINITE).  sigma_out (device float 6 x nt), map_out (device float
 * H x W) and mask_out (device uint8 H x W) may each be NULL; mask_out needs
 * map_out, and map_out needs an env created with a grid.  *ticket receives
 * the request's id.  Never blocks on the GPU. */
tc_status tc_submit(tc_server* server, tc_env* env, const tc_pose* target,
                    float* sigma_out, float* map_out, uint8_t* mask_out,
                    uint64_t* ticket);

/* *done = 1 once the request has finished; then *result (nullable) is
 * filled and the ticket is released (a later call with it returns
 * TC_ERR_INVALID_ARG).  Unknown ticket: TC_ERR_INVALID_ARG. */
tc_status tc_poll(tc_server* server, uint64_t ticket, int32_t* done, tc_result* result);

/* Block up to timeout_us (>= 0) microseconds for the request to finish.
 * Finished: TC_OK, *result (nullable) filled, ticket released.  Not finished
 * in time: TC_ERR_TIMEOUT (the request keeps running; wait or poll again). */
tc_status tc_wait(tc_server* server, uint64_t ticket, int64_t timeout_us, tc_result* result);

tc_status tc_server_info(tc_server* server, tc_server_stats* out);

/* *stream = the cudaStream_t of worker `worker` (0 <= worker < workers), for
 * callers that order their own work or events after the server's. */
tc_status tc_server_stream(tc_server* server, int32_t worker, void** stream);

/* Cancel queued requests (their status becomes TC_ERR_ADMISSION), finish the
 * ones in flight, stop the worker and free the server. */
void tc_server_destroy(tc_server* server);

#ifdef __cplusplus
}
#endif
#endif /* TACAUCHY_H */
