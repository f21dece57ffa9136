/*
 * lc_lb.h -- C ABI of the GB300 (sm_103a) hybrid lattice Boltzmann /
 * Beris-Edwards solver for colloids in nematic and cholesteric liquid crystals
 * (Lintuvuori, Marenduzzo, Stratford & Cates, "Colloids in liquid crystals: a
 * lattice Boltzmann study", Sec. 2).
 *
 * Conventions (every entry point):
 *   - returns an int status (LC_OK or a negative LC_ERR_*); nothing throws or
 *     aborts across the ABI; the message of the last failure on a handle is
 *     available from lc_lb_last_error(handle) (and lc_lb_last_error(NULL) for
 *     failures that happened before a handle existed);
 *   - device work is queued on the handle's CUDA stream (the one given to
 *     lc_lb_create; NULL = a non-blocking stream the handle creates, since
 *     the step is captured in a CUDA graph); calls that return data to the
 *     host synchronise that stream;
 *   - a handle is not thread-safe; distinct handles are independent;
 *   - the handle owns its device memory, taken from the allocator installed
 *     with lc_lb_set_allocator (cudaMalloc/cudaFree when none is installed);
 *   - fields exchanged with the caller are FP64, structure-of-arrays
 *     [component][z][y][x] with node index x + nx*(y + ny*z), whatever the
 *     storage precision.  Q has 5 components (xx, xy, xz, yy, yz), zz = -xx-yy.
 *   - D3Q19 populations use the order: rest; +x,-x,+y,-y,+z,-z; (1,1,0),
 *     (-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),
 *     (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1); weights 1/3, 1/18, 1/36.
 */
#ifndef LC_LB_H
#define LC_LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LC_OK = 0,
  LC_ERR_ARG = -1,       /* bad argument (size, pointer, value range) */
  LC_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  LC_ERR_OOM = -3,       /* the allocator returned NULL */
  LC_ERR_OVERLAP = -4,   /* colloid touches another colloid or a wall (add_colloid, or a move refused in a step) */
  LC_ERR_NONFINITE = -5, /* a reduction met NaN/Inf */
  LC_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
  LC_ERR_STATE = -7      /* call not valid in the handle's state */
};
enum { LC_FP32 = 0, LC_FP64 = 1 };
enum { LC_NORMAL = 0, LC_PLANAR = 1 };
/* field selectors for lc_lb_get_fields / lc_lb_set_fields */
enum {
  LC_Q = 0,     /* 5 x N order parameter */
  LC_U = 1,     /* 3 x N velocity u = (sum f c + F/2)/rho of the current state */
  LC_RHO = 2,   /* 1 x N density */
  LC_F_PRE = 3, /* 19 x N pre-collision (post-stream) populations f (full, not deviation) */
  LC_FORCE = 4, /* 3 x N body force: discrete divergence of the LC stress of the current Q */
  LC_SOLID = 5  /* 1 x N: -1 fluid, c >= 0 inside colloid c (stored as double) */
};

typedef struct lc_lb lc_lb;
typedef struct lc_lb_batch lc_lb_batch;

/* Box: nx*ny*nz nodes, periodic in x and y; periodic in z unless wall_z = 1,
 * which puts no-slip walls at z = -1/2 and z = nz - 1/2 carrying strong
 * homeotropic anchoring along z. */
typedef struct {
  int nx, ny, nz;
  int wall_z;
} lc_grid;

/* Constants of the model (Sec. 2.1, Eqs. 1-4) and of the LB:
 *   rho0  reference density;  tau  BGK relaxation time (viscosity (tau-1/2)/3);
 *   A0, gamma, K, q0  Landau-de Gennes constants of Eq. 1 (q0 = 2 pi / pitch);
 *   xi  flow-alignment parameter of Eq. 4;  Gamma  rotational diffusion of Eq. 2;
 *   S0  surface order of Eq. 7 (<= 0: the bulk uniaxial order
 *       1/4 + 3/4 sqrt(1 - 8/(3 gamma)));
 *   body_force  uniform force density on fluid nodes (0 for the paper's runs);
 *   precision  LC_FP32 (FP32 storage, FP64 reductions) or LC_FP64;
 *   lc_enabled  0: Q frozen, no LC stress;  flow_enabled  0: LB frozen, u = 0. */
typedef struct {
  double rho0, tau;
  double A0, gamma, K, q0, xi, Gamma;
  double S0;
  double body_force[3];
  int precision;
  int lc_enabled;
  int flow_enabled;
  int reserved;
} lc_params;

/* FP64 diagnostics of the current state. */
typedef struct {
  double mass;        /* sum of f over fluid nodes */
  double momentum[3]; /* sum of f c over fluid nodes (pre-collision) */
  double free_energy; /* sum of f' over fluid nodes + (w/2)|Qs-Q0|^2 over weak-anchoring faces */
  double resid_rms;   /* RMS over fluid nodes of the 9 entries of the last Q increment */
  double resid_max;   /* largest |entry| of the last Q increment */
  long long n_fluid;
  long long n_defect; /* fluid nodes with 3/2 lambda_max(Q) < 0.435 (Sec. 3.1 threshold) */
  long long step;
} lc_diag;

/* Optional allocator for all device memory of the library (e.g. a framework's
 * caching allocator).  alloc returns a device pointer or NULL; free releases
 * it.  Applies to handles created after the call.  NULL, NULL restores
 * cudaMalloc / cudaFree. */
typedef void* (*lc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*lc_free_fn)(void* ptr, void* stream, void* ctx);
int lc_lb_set_allocator(lc_alloc_fn alloc, lc_free_fn free_fn, void* ctx);

/* Create a box (Sec. 2: one LB/FD domain).  The state starts as the
 * uniaxial bulk order along z with f at rest equilibrium.  stream is a
 * cudaStream_t other than the legacy default stream (NULL = the handle
 * creates one).  Errors: LC_ERR_ARG for
 * nx,ny,nz < 1, N >= 2^31, tau <= 1/2, unknown precision; LC_ERR_OOM;
 * LC_ERR_CUDA. */
int lc_lb_create(const lc_grid* grid, const lc_params* params, void* stream, lc_lb** out);
void lc_lb_destroy(lc_lb* h);

/* Uniaxial Q = S0 (n n - delta/3) (uniaxial form, Sec. 2.1) plus noise of
 * amplitude noise_amp on each of the 5 stored components, drawn from the
 * counter-based SplitMix64 generator: r = splitmix64(seed ^ (5*node + comp)),
 * noise = amp * (2 * (r >> 11) * 2^-53 - 1), evaluated in FP64 and rounded to
 * the storage precision.  f is reset to rest equilibrium. */
int lc_lb_init_uniaxial(lc_lb* h, const double n[3], double noise_amp, uint64_t seed);

/* Cholesteric helix (Sec. 3.2) along axis a (0,1,2): n_b = cos(q0 r_a),
 * n_c = sin(q0 r_a), (a,b,c) cyclic, amplitude S0, plus the same noise. */
int lc_lb_init_helix(lc_lb* h, int axis, double noise_amp, uint64_t seed);

/* Replace a field: LC_Q (5 x N) or LC_F_PRE (19 x N full pre-collision
 * populations).  src is host memory unless src_is_device (then an FP64
 * device buffer).  bytes must equal the field size in FP64. */
int lc_lb_set_fields(lc_lb* h, int which, const void* src, size_t bytes, int src_is_device);

/* Add a spherical colloid (Sec. 2.2) of nominal radius a0 at X: nodes with
 * |r - X|^2 < a0^2 (minimum image, FP64, no fused multiply-add) are solid.
 * anchoring LC_NORMAL (homeotropic) or LC_PLANAR; w = anchoring strength
 * (INFINITY or <= 0: the paper's fixed surface Q0); mobile = 1 lets the
 * colloid move under F_hyd + F_LC + F_ext.  Errors: LC_ERR_ARG (a0 <= 0,
 * more than 126 colloids), LC_ERR_OVERLAP (its centre is closer to another
 * colloid's current centre than the sum of the radii, minimum image, or its
 * surface passes a wall plane z = -1/2 or nz - 1/2).  *id_out receives its
 * index. */
int lc_lb_add_colloid(lc_lb* h, const double X[3], double a0, int anchoring, double w, int mobile,
                      const double F_ext[3], int* id_out);
int lc_lb_set_colloid_velocity(lc_lb* h, int id, const double V[3], const double W[3]);
int lc_lb_set_colloid_force(lc_lb* h, int id, const double F_ext[3]);
/* External torque T_ext on colloid id (a rotating colloid: the paper's
 * colloids feel only the hydrodynamic and LC torques, Sec. 2.2); a mobile
 * colloid's update then takes W' = W + (I + zw)^{-1} (T_hyd + T_LC + T_ext).
 * Errors: LC_ERR_ARG (no colloid id, T_ext NULL).  Synchronises. */
int lc_lb_set_colloid_torque(lc_lb* h, int id, const double T_ext[3]);

/* Advance nsteps coupled steps (Sec. 2.2 step order): LC stress and body
 * force, density/velocity, Q update (Eq. 2), collide + bounce-back + stream,
 * colloid update.  Asynchronous on the handle's stream; replays a captured
 * CUDA graph per step after the first call.
 * Contact (the paper treats none): a mobile colloid whose move would bring
 * it closer to another colloid than the sum of the radii, or its surface
 * past a wall plane, is not moved in that step (its velocities are updated);
 * the first such contact is reported as LC_ERR_OVERLAP, with the step, box
 * and colloids in lc_lb_last_error, by the next call that synchronises
 * (lc_lb_synchronize, lc_lb_relax, lc_lb_get_fields, lc_lb_get_colloid,
 * lc_lb_get_forces, lc_lb_diagnostics), which clears it.  The state stays
 * valid: no node is ever inside two colloids. */
int lc_lb_step(lc_lb* h, int nsteps);

/* Relax: steps in chunks of check_every until the residual (RMS of the Q
 * increment) is <= tol or max_steps is reached.  Synchronises once per
 * chunk.  steps_out / resid_out may be NULL. */
int lc_lb_relax(lc_lb* h, double tol, long long max_steps, int check_every, long long* steps_out,
                double* resid_out);

/* Copy a field (see LC_*) as FP64 into dst (host unless dst_is_device).
 * bytes must be >= the field size.  Synchronises the stream. */
int lc_lb_get_fields(lc_lb* h, int which, void* dst, size_t bytes, int dst_is_device);

/* Forces of the last completed step on colloid id: F = F_hyd + F_LC, T the
 * torque, and the current V, W (angular velocity) and X.  Any pointer may be
 * NULL.  Synchronises. */
int lc_lb_get_forces(lc_lb* h, int id, double F[3], double T[3], double V[3], double W[3], double X[3]);

/* Full colloid record (27 doubles): X V W F_hyd T_hyd F_lc T_lc impulse
 * angular_impulse (impulse = total momentum received). */
int lc_lb_get_colloid(lc_lb* h, int id, double out[27]);

/* Boundary links (Sec. 2.2, Fig. 1): (fluid node, direction b, colloid) with
 * node + c_b inside the colloid, sorted by (colloid, node, b).  Writes at
 * most cap entries; *n_out receives the total count. */
int lc_lb_get_links(lc_lb* h, int32_t* node, int8_t* dir, int16_t* colloid, size_t cap, size_t* n_out);

/* Defect analytics (Sec. 3.1: defects are where the order parameter is below
 * 0.435; Sec. 3.2: the disclination loops around a colloid in a cholesteric).
 * A defect node is a fluid node whose scalar order 3/2 lambda_max(Q), taken
 * in FP64 from the stored Q, is below thr (> 0; the paper's value is 0.435).
 * Components are the connected sets of defect nodes under face adjacency,
 * periodic in x and y, and in z unless the box has walls; each is named by
 * its smallest node index x + nx (y + ny z) ("root") and listed in root
 * order.  Per component: the node count; the centroid [x, y, z], per
 * periodic axis the circular mean (angle of the mean of exp(2 pi i x / L),
 * times L / 2 pi, moved into [0, L)), along a walled z axis the plain mean;
 * the gyration tensor (xx, xy, xz, yy, yz, zz), the mean of d d^T over the
 * component, d the minimum-image displacement from the centroid.
 * Writes at most cap components into the caller's host arrays (any may be
 * NULL: root, size cap entries; centroid 3 cap, gyration 6 cap doubles);
 * *n_defect and *n_comp receive the totals (either may be NULL).  Labels
 * and counts are exact; the FP64 sums are accumulated in an unspecified
 * order.  Device memory: 3 N + N/256 + 2 ints kept by the handle, plus
 * 64 bytes per component during the call.  Synchronises the stream.
 * LC_ERR_ARG for a threshold that is not positive and finite;
 * LC_ERR_TIMEOUT if a bounded device loop gave up (not expected). */
int lc_lb_defects(lc_lb* h, double thr, size_t cap, long long* n_defect, long long* n_comp, long long* root,
                  long long* size, double* centroid, double* gyration);

/* Per-node component labels of lc_lb_defects: labels[i] = root of node i's
 * component, or -1 for a node that is not a defect node (solid nodes
 * included); n >= N entries, host memory unless dst_is_device.
 * Synchronises the stream. */
int lc_lb_defect_labels(lc_lb* h, double thr, int32_t* labels, size_t n, int dst_is_device);

int lc_lb_diagnostics(lc_lb* h, lc_diag* out);

/* Allocation-free diagnostics: the paper has no counterpart; this exists for
 * callers that cannot allocate device memory at the point of the call --
 * allocator or out-of-memory handlers that must not re-enter an allocator,
 * code that runs under a fixed device-memory budget, and loops that cannot
 * afford the device-wide synchronisation of cudaMalloc/cudaFree.  It fills
 * mass, momentum, n_fluid, n_defect and step of *out exactly as
 * lc_lb_diagnostics does (the other fields are set to 0) and calls no
 * cudaMalloc, cudaFree or allocating library routine.  Its scratch is a
 * static device array of 384 KiB + 64 B that every GPU loading this library
 * holds until the process exits; it serves boxes of at most 2,097,152 nodes
 * (a 128^3 box) and returns LC_ERR_ARG for larger ones.  The first call on a
 * device looks up the array's device address (once per device, with that
 * device current) and keeps it for the process: the call assumes the
 * device's primary context (the runtime's default) and must not be used
 * after cudaDeviceReset on that device.  The device current at the call must
 * be the one the handle was created on (LC_ERR_ARG otherwise).  All calls on
 * a device share the array, which keeps the last call's contents (each call
 * overwrites every record it reads), so two calls whose GPU work overlaps --
 * e.g. two handles on different streams -- race.  Synchronises the handle's
 * stream. */
int lc_lb_diagnostics_noalloc(lc_lb* h, lc_diag* out);

/* Profiling: run nsteps steps without the graph and with every kernel on
 * the handle's stream, with CUDA events around each, and return the mean
 * milliseconds per step of: [0] LC stress + body force + LB collide/stream
 * (the force + LB part, in the variant the autotuner chose), [1] Q update,
 * [2] link momentum exchange, [3] colloid update, [4] the whole step.  The
 * _detail forms add [5] the variant (0 fused: one kernel; 1 split: stress/
 * force kernel and LB kernel, run one after the other here; 2 stored: the
 * stress kernel stores H and P, the LB kernel takes the face divergence of
 * the stored P) and [6], [7] the milliseconds of its two kernels (fused:
 * [7] = 0).  LCLB_VARIANT=fused|split|stored in the environment overrides the
 * tuned variant.  The state advances by nsteps.  Synchronises. */
int lc_lb_profile(lc_lb* h, int nsteps, double ms_out[5]);
int lc_lb_batch_profile(lc_lb_batch* b, int nsteps, double ms_out[5]);
int lc_lb_profile_detail(lc_lb* h, int nsteps, double ms_out[8]);
int lc_lb_batch_profile_detail(lc_lb_batch* b, int nsteps, double ms_out[8]);
/* Number of kernel launches in one step as captured in the step's CUDA
 * graph (autotunes and captures first if needed; the state does not
 * advance). */
int lc_lb_step_launches(lc_lb* h, int* n_out);
int lc_lb_batch_step_launches(lc_lb_batch* b, int* n_out);
int lc_lb_synchronize(lc_lb* h);
const char* lc_lb_last_error(const lc_lb* h);
const char* lc_lb_version(void);

/* Batched boxes: n independent boxes of possibly different size and
 * constants (all with the same precision), advanced together by one
 * persistent launch per phase over a work list of (box, tile), captured in
 * one CUDA graph per step.  lc_lb_batch_box returns a borrowed handle to box
 * i for the single-box calls (init, set/get fields, add_colloid, forces,
 * links, diagnostics); lc_lb_step on a borrowed handle is LC_ERR_STATE. */
int lc_lb_batch_create(int n, const lc_grid* grids, const lc_params* params, void* stream, lc_lb_batch** out);
void lc_lb_batch_destroy(lc_lb_batch* b);
int lc_lb_batch_box(lc_lb_batch* b, int i, lc_lb** box);
int lc_lb_batch_step(lc_lb_batch* b, int nsteps);
/* Relax every box until all residuals are <= tol (boxes that reach it keep
 * stepping with the rest).  resid_out (n doubles) may be NULL. */
int lc_lb_batch_relax(lc_lb_batch* b, double tol, long long max_steps, int check_every, long long* steps_out,
                      double* resid_out);
const char* lc_lb_batch_last_error(const lc_lb_batch* b);

/* Autotuner: time the candidate tile shapes of each phase kernel on a
 * scratch box of the given size and precision, and keep the fastest (cached
 * per size and precision for the process; LCLB_TUNE_CACHE names a file to
 * persist it).  Called automatically on first use of a size; exposed to
 * force a retune.  out_desc (may be NULL) receives a short text of the
 * choice. */
int lc_lb_autotune(const lc_grid* grid, int precision, void* stream, char* out_desc, size_t desc_len);

#ifdef __cplusplus
}
#endif
#endif /* LC_LB_H */
