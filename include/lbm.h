/*
 * liblbm: GB300 (sm_103a) library for the time step of the D2Q9
 * multiple-relaxation-time pseudopotential (Shan-Chen) lattice Boltzmann
 * model with fluid-solid interaction, after Li, Luo, Kang & Chen,
 * "Contact angles in the pseudopotential lattice Boltzmann modeling of
 * wetting" (Sec. II: Eqs. (1)-(11), (14); Sec. III: Eq. (15), wall rule,
 * initial droplet Eq. (16)).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: nx * ny nodes, node (x, y) at index y * nx + x (x fastest),
 * periodic in x and in y; solid nodes (switch function s = 1) form walls.
 * Velocities e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 * e6=(-1,1) e7=(-1,-1) e8=(1,-1); populations f_alpha laid out [9][ny][nx]
 * whenever they cross this interface.  Lattice units: c = delta_t = 1,
 * cs^2 = 1/3.
 *
 * Pointers: every array argument is a plain pointer.  Inputs are host
 * pointers unless the call takes a *_is_device flag; they are copied during
 * the call and may be freed afterwards.  Outputs are caller-owned buffers of
 * the stated length.  The context owns all device memory it allocates.
 *
 * Errors: every call returns an lbm_status; nothing aborts or throws across
 * this boundary.  lbm_last_error() returns a message for the calling thread.
 * Errors found on the device during lbm_step (non-finite density, a timed-out
 * grid barrier) latch in the context and are returned by the next call that
 * synchronises (lbm_diagnostics, lbm_get_fields, lbm_sync).
 *
 * Streams: a context enqueues all its work on the CUDA stream given at
 * creation (NULL = the legacy default stream).  Calls on different contexts
 * may come from different threads; calls on one context must not overlap.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,       /* invalid argument or configuration */
  LBM_ERR_OOM = 2,       /* device or host allocation failed */
  LBM_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  LBM_ERR_NONFINITE = 4, /* non-finite or non-positive density on a fluid node */
  LBM_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
  LBM_ERR_STATE = 6      /* call not valid in the context's current state */
} lbm_status;

/* Fluid-solid interaction F_ads: Eq. (10) density-based, Eq. (11)
   pseudopotential-based, Eq. (14) the paper's modified pseudopotential-based
   interaction with phi(x) = psi(x). */
typedef enum { LBM_FSI_DENSITY = 0, LBM_FSI_PSI = 1, LBM_FSI_MODIFIED = 2 } lbm_fsi;

/* Equation of state: the piecewise-linear EOS of Eq. (15) (the paper's), or
   the Carnahan-Starling EOS p = rho R T (1 + e + e^2 - e^3) / (1 - e)^3 -
   a rho^2, e = b rho / 4, as an option the paper does not use (its G_w
   ranges and sigma are those of Eq. (15)).  Either way psi^2 = 2 (p -
   rho cs^2) / G (Sec. II.B).  With LBM_FP32_SHIFTED the Carnahan-Starling
   psi^2 is evaluated in FP64 from the compensated density.  lbm_adjoint
   supports Eq. (15) only. */
typedef enum { LBM_EOS_PIECEWISE_LINEAR = 0, LBM_EOS_CARNAHAN_STARLING = 1 } lbm_eos;

/* Wall treatment.  LBM_WALL_NEQ_ONNODE: the rule quoted in Sec. III.A for a
   wall below the node (f2 = f4, f5 = f7 - (f1 - f3)/2 - (Fx + Fy)/4,
   f6 = f8 + (f1 - f3)/2 + (Fx - Fy)/4, with F the node's force of the same
   step), mirrored in y for a wall above; walls must be whole solid rows.
   LBM_WALL_HALFWAY_BB: halfway bounce-back on every fluid-solid link, any
   solid mask. */
typedef enum { LBM_WALL_NEQ_ONNODE = 0, LBM_WALL_HALFWAY_BB = 1 } lbm_wall;

/* How Eq. (7) treats solid neighbours.  Sec. III.A applies Eq. (7) at the
   wall through a ghost layer: COPY gives a solid node the psi of the fluid
   node next to it along the wall normal, MIRROR the psi of the fluid node
   two rows away (both need whole solid rows).  ZERO gives solid nodes
   psi = 0.  SKIP does not apply Eq. (7) at fluid nodes that have a solid
   neighbour (Sec. III.B, rough surfaces); any mask.  MEAN gives a solid
   node the mean psi of the fluid nodes next to it along the axes (up, down,
   right, left), a ghost layer for walls of any shape such as the pillars of
   Sec. III.B; on a flat wall it equals COPY.  lbm_adjoint supports COPY,
   MIRROR, ZERO and SKIP. */
typedef enum {
  LBM_GHOST_COPY = 0,
  LBM_GHOST_MIRROR = 1,
  LBM_GHOST_ZERO = 2,
  LBM_GHOST_SKIP = 3,
  LBM_GHOST_MEAN = 4
} lbm_ghost;

/* Weights omega_alpha of Eqs. (10), (11), (14).  LBM_OMEGA_W: w_alpha of
   Eq. (7), 1/3 and 1/12, under which the G_w values printed with Figs. 2-4
   give the printed contact angles (default).  LBM_OMEGA_CS2W: cs^2 w_alpha,
   1/9 and 1/36, the sentence after Eq. (10) read literally. */
typedef enum { LBM_OMEGA_W = 0, LBM_OMEGA_CS2W = 1 } lbm_omega;

/* Storage and arithmetic.  LBM_FP64: populations stored and collided in
   FP64.  LBM_FP32_SHIFTED: populations stored and collided in FP32 as
   f - w_alpha rho_ref; density summed with error-free FP32 transformations
   (FP64-grade, no FP64 instructions on the step path); psi evaluated from
   that density and rounded once.  LBM_FP32_SHIFTED_F64: as LBM_FP32_SHIFTED
   but density summed and psi evaluated in IEEE FP64 instructions. */
typedef enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1, LBM_FP32_SHIFTED_F64 = 2 } lbm_precision;

/* tau_nu between the phases when tau_nu_L != tau_nu_V (Sec. III.C gives
   the liquid and vapour viscosities only).  LBM_VISC_TAU_LINEAR: tau_nu
   linear in rho (equivalently the kinematic viscosity nu = (tau_nu - 1/2)
   cs^2 linear in rho) (default).  LBM_VISC_MU_LINEAR: the dynamic
   viscosity mu = rho nu linear in rho, tau_nu = 1/2 + mu(rho) / (rho cs^2).
   Both clamped to [min, max] of the two end values. */
typedef enum { LBM_VISC_TAU_LINEAR = 0, LBM_VISC_MU_LINEAR = 1 } lbm_visc;

typedef struct {
  lbm_eos eos;
  /* Eq. (15): theta_V, theta_M, theta_L in units of cs^2, then rho_1, rho_2;
     Carnahan-Starling: a, b, R, T (all > 0; the density must stay below
     4 / b) */
  double eos_p[6];
  double G;     /* interaction strength of Eq. (7); psi needs G < 0 */
  double sigma; /* Eq. (9) */
  /* relaxation times of Eq. (2) */
  double tau_rho, tau_e, tau_zeta, tau_j, tau_q;
  /* tau_nu in liquid and vapour (Sec. III.C); when they differ tau_nu varies
     between rho_V and rho_L as `visc` says, clamped to the two values.
     rho_L and rho_V also set the contact-angle level (rho_L + rho_V) / 2. */
  double tau_nu_L, tau_nu_V, rho_L, rho_V;
  lbm_wall wall;
  lbm_ghost ghost;
  lbm_omega omega;
  lbm_precision prec;
  double rho_ref; /* shift of the FP32 storage (ignored for LBM_FP64) */
  lbm_visc visc;  /* tau_nu between the phases (used when tau_nu_L != tau_nu_V) */
} lbm_params;

/* One lattice of a batch (lbm_create_batch). */
typedef struct {
  int nx, ny;
  const lbm_params* params; /* all instances of a batch share params->prec */
  const uint8_t* solid;     /* [ny][nx], nonzero = solid; NULL = no solid */
  lbm_fsi fsi;
  const double* gw_field;   /* [ny][nx] G_w read on solid nodes; NULL = uniform */
  double gw_uniform;
} lbm_instance_desc;

typedef struct {
  long step;
  double mass;      /* sum of rho over fluid nodes (FP64) */
  double rho_max;   /* over fluid nodes (Sec. III.B, Table I) */
  double rho_min;
  double u_max;     /* max |v| over fluid nodes, v of Eq. (6) (Sec. III.C) */
  double theta_deg; /* contact angle of the circle fitted to rho = (rho_L + rho_V)/2 */
  double fit_rms;   /* rms distance of the contour points from the circle */
  double xc, yc, radius;
  int n_contour;    /* contour points used by the fit */
  lbm_status status;
} lbm_diag;

/* Fills *p with the parameters of Sec. III: theta_V = 0.64 cs^2,
   theta_M = -0.04 cs^2, theta_L = cs^2, rho_1 = 1.36, rho_2 = 481.04, G = -1,
   sigma = 0.084, tau_rho = tau_j = 1, 1/tau_e = 1/tau_zeta = 0.8,
   1/tau_q = 1.1, tau_nu = 1.1, rho_L = 500, rho_V = 1, NEQ wall, COPY ghost,
   LBM_OMEGA_W, LBM_FP64, rho_ref = rho_V, LBM_VISC_TAU_LINEAR. */
lbm_status lbm_default_params(lbm_params* p);

/* Creates a context holding one lattice.  solid: [ny][nx] host array (NULL =
   no solid); gw_field: [ny][nx] host array of G_w read on solid nodes (NULL =
   gw_uniform on every solid node).  The populations start at zero: call
   lbm_init_droplet or lbm_set_density before stepping.  stream: a
   cudaStream_t or NULL.  LBM_ERR_ARG for nx < 3, ny < 4, tau <= 0.5, G >= 0,
   a non-flat mask with the NEQ wall or a COPY/MIRROR ghost, or a fluid node
   with solid directly above and below. */
lbm_status lbm_create(int nx, int ny, const lbm_params* p, const uint8_t* solid, lbm_fsi fsi,
                      const double* gw_field, double gw_uniform, void* stream, lbm_ctx** out);

/* Creates a context holding count independent lattices of possibly different
   sizes, parameters, interactions and G_w; lbm_step advances all of them in
   one launch per time step (or one persistent launch, lbm_set_launch). */
lbm_status lbm_create_batch(int count, const lbm_instance_desc* descs, void* stream,
                            lbm_ctx** out);

void lbm_destroy(lbm_ctx* ctx);

/* Number of instances and the size of instance inst. */
lbm_status lbm_instance_size(const lbm_ctx* ctx, int inst, int* nx, int* ny);

/* Initial droplet (Sec. III.A, Eq. (16) with a smooth interface):
   rho = rho_V + (rho_L - rho_V)/2 * (1 - tanh(2 (r - R) / width)), r the
   distance to (x0, y0) with the minimum image in x; f_alpha = w_alpha rho
   (fluid at rest) on fluid nodes.  Resets the step counter. */
lbm_status lbm_init_droplet(lbm_ctx* ctx, int inst, double x0, double y0, double R,
                            double width);

/* Fluid at rest with the density field rho [ny][nx] (host or device FP64).
   Resets the step counter.  Synchronises. */
lbm_status lbm_set_density(lbm_ctx* ctx, int inst, const double* rho, int src_is_device);

/* lbm_set_density without synchronising: the copy and the initialisation
   are enqueued on the context's stream and the call returns.  rho must stay
   valid and unchanged until the copy has run (lbm_sync); page-locked host
   memory lets the copy run asynchronously (a pageable buffer is copied
   before the call returns).  Errors of the enqueued work surface at the next
   synchronising call. */
lbm_status lbm_set_density_async(lbm_ctx* ctx, int inst, const double* rho, int src_is_device);

/* Advances every instance by n time steps of the method of Sec. II: per
   node, streaming (Eq. 5, pull form) with the wall treatment of Sec. III.A
   folded into the pull, density and velocity (Eq. 6), psi from the EOS
   (Eq. 15, or the Carnahan-Starling option), the fluid-fluid force (Eq. 7),
   the fluid-solid force (Eq. 10, 11 or 14), and the MRT collision (Eqs. 2-4)
   with the forcing of Eq. 9.  Asynchronous: returns after enqueueing on the
   context's stream; n = 0 is a no-op, n < 0 is LBM_ERR_ARG.  Device-side
   errors (non-finite density, a timed-out persistent wait) latch in the
   context and are returned by the next synchronising call. */
lbm_status lbm_step(lbm_ctx* ctx, long n);

/* Waits for the context's stream and for the host copies of the batch
   calls below (an implementation call; the paper has no counterpart);
   returns a latched device error if any (LBM_ERR_NONFINITE,
   LBM_ERR_TIMEOUT, or LBM_ERR_STATE for an index that the checked build
   caught); the error stays latched, so every later lbm_sync returns it. */
lbm_status lbm_sync(lbm_ctx* ctx);

long lbm_time(const lbm_ctx* ctx);

/* rho and v of Eq. (6) at the current time, FP64 [ny][nx] each (NULL skips
   one).  Solid nodes read 0.  dst_is_device: the pointers are device memory.
   Synchronises. */
lbm_status lbm_get_fields(lbm_ctx* ctx, int inst, double* rho, double* ux, double* uy,
                          int dst_is_device);

/* lbm_get_fields without synchronising: the field kernels and the copies
   are enqueued on the context's stream; the outputs hold the fields after
   lbm_sync.  Calls for several instances may be queued back to back (the
   context's scratch fields are reused in stream order).  Page-locked host
   outputs let the copies overlap the caller. */
lbm_status lbm_get_fields_async(lbm_ctx* ctx, int inst, double* rho, double* ux, double* uy,
                                int dst_is_device);

/* The whole batch at once, without synchronising (one kernel per stage for
   all instances, one copy per field).  Fields are concatenated in instance
   order: instance k occupies the nx_k ny_k values that follow those of
   instances 0 .. k-1, each in the [ny][nx] layout of lbm_get_fields.
   lbm_set_density_all_async: fluid at rest with those densities, every
   instance (resets the step counter).  lbm_get_fields_all_async: rho and v
   of Eq. (6) of every instance (NULL skips a field); valid after lbm_sync.
   Buffers hold sum_k nx_k ny_k doubles.  Device buffers are read or written
   in the context's stream order (a device density source is read in place).
   Host buffers go through two copy streams of the context's own, ordered
   against its stream by events: the upload of host densities into a staging
   buffer starts at once, beside the steps already queued, and the read-back
   to the host runs beside the steps queued after it.  A host buffer must
   stay valid and unchanged (inputs) or unread (outputs) until lbm_sync;
   page-locked host memory lets the copies run asynchronously. */
lbm_status lbm_set_density_all_async(lbm_ctx* ctx, const double* rho, int src_is_device);
lbm_status lbm_get_fields_all_async(lbm_ctx* ctx, double* rho, double* ux, double* uy,
                                    int dst_is_device);

/* Populations f_alpha(x, t) after streaming and the wall rule (the state
   Eq. (6) is evaluated on), FP64 [9][ny][nx]; FP32 storage is shifted back.
   Solid nodes read 0.  Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, int inst, double* f, int dst_is_device);

/* Diagnostics of instance inst: mass, rho_max, rho_min, max |v|, and the
   contact angle of the circle fitted (algebraic least squares) to the
   points where rho crosses (rho_L + rho_V)/2 on edges between fluid nodes,
   x unwrapped about x_ref, points closer than d_min to the wall height y_w
   dropped; theta = 90 deg + asin((yc - y_w)/R).  Synchronises. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, int inst, double y_w, double x_ref, double d_min,
                           lbm_diag* out);

/* Spreading (contact) radius of a droplet on a wall (dynamic wetting,
   Sec. III.A, Fig. 7), from the density of instance inst at the current
   time along node row `row` (the first fluid row above a bottom wall).
   From the column nearest x_ref the row is walked right and left to the
   first node below `level`; each crossing is interpolated linearly between
   that node and the one before it, and solid nodes count as below the
   level.  *r_out = (x_right - x_left) / 2 in lattice units: 0 when rho at
   the start column is below the level (no contact), nx / 2 when the whole
   row is above it.  level <= 0 means (rho_L + rho_V) / 2 of the instance.
   LBM_ERR_ARG for a row outside [0, ny) or a non-finite x_ref.
   Synchronises. */
lbm_status lbm_contact_radius(lbm_ctx* ctx, int inst, int row, double level, double x_ref,
                              double* r_out);

/* Replaces the G_w field of instance inst ([ny][nx] host, read on solid
   nodes) and rebuilds the wall vectors of the fluid-solid force. */
lbm_status lbm_set_gw_field(lbm_ctx* ctx, int inst, const double* gw);

/* Gradient of a contact-angle loss with respect to the G_w field, by a
   hand-written reverse mode of the FP64 time step (every stage of Sec. II:
   Eqs. (5)-(7), (9)-(11), (14), (15), the wall rule of Sec. III.A).
   Runs T steps from the context's current state (leaving it T steps
   later), measures theta as lbm_diagnostics does (circle fitted to the
   (rho_L + rho_V)/2 contour, points below y_w + d_min dropped, x unwrapped
   about x_ref), sets *loss_out = (theta - theta_target)^2 (deg^2) and
   *theta_out = theta, and writes dL/dG_w into grad_gw ([ny][nx] host
   array, nonzero on solid nodes only).  The loss is differentiated with the
   set of contour edges held fixed (it is smooth while no edge changes
   sides).  Memory: checkpoints of the state every ceil(sqrt(T)) steps plus
   one recomputed segment, O(sqrt(T) * nx * ny).  Needs a single-lattice
   LBM_FP64 context with tau_nu_L == tau_nu_V; synchronises. */
lbm_status lbm_adjoint(lbm_ctx* ctx, long T, double theta_target, double y_w, double x_ref,
                       double d_min, double* loss_out, double* theta_out, double* grad_gw);

/* Launch shape of lbm_step (an implementation call; the paper has no
   counterpart, and the step it runs is the one of lbm_step whatever the
   shape): bx threads per block along x (a block covers
   bx - 2 columns), h rows per block or strip segment (0 = choose
   automatically: balanced segments of at most 32 rows for warp strips, 64
   for blocks; for warp strips the limit is halved, down to 2 rows, while
   the whole batch gives fewer strips than two per resident warp, and for
   persistent warp strips it is the height that gives the most strips not
   exceeding one per resident warp),
   persistent = 1 runs all n steps in one cooperative launch: block
   pipelines with a bounded grid barrier between steps, warp strips (the
   FP32 column pairs of stages 4 where they apply, else one row per lane)
   with no barrier (a strip starts a step once the strips within four nodes
   of it have finished the previous one; every wait is bounded and a
   time-out returns LBM_ERR_TIMEOUT at the next synchronising call),
   graph = 1 captures the n per-step launches (or
   the one persistent launch) in a CUDA graph, reused for every later call
   with the same n.  stages selects the step pipeline: 1 = blocks marching up
   rows with loads prefetched into registers; 2 = independent warps, each
   marching up a 30-column strip (no block barriers),
   with FP32 storage two rows at a time on the paired FP32 instructions;
   3 = the same warp strips one row at a time; 4 = independent warps, each
   marching up a 60-column strip one row at a time with two columns per lane
   on the paired FP32 instructions (FP32 storage, every lattice width a
   multiple of 4; otherwise as 2); 8 or 16 = blocks marching
   up rows with a TMA ring of that many source rows in shared memory (FP32
   storage, every lattice width a multiple of 4); 0 = automatic (4 where it
   applies, else warp strips as 2).  Results do not depend on any of these
   choices.  A persistent launch needs one parameter set across the batch
   (LBM_ERR_ARG otherwise). */
lbm_status lbm_set_launch(lbm_ctx* ctx, int bx, int h, int persistent, int graph, int stages);

/* The launch shape lbm_step uses now (an implementation detail; the paper
   has no counterpart): threads per block, and the pipeline as a code: 1 =
   block rows, 2 = FP32 warp strips two rows per lane, 3 = warp strips one
   row per lane (FP64 and FP32 with FP64 density, stages 3, and the
   persistent launch of the warp strips of stages 2), 4 = FP32 warp strips
   two columns per lane (per step or persistent),
   8 or 16 = block rows with a TMA ring; and
   the persistent flag as set.  Outputs may be NULL. */
lbm_status lbm_get_launch(const lbm_ctx* ctx, int* bx, int* pipeline, int* persistent);

/* Writes the state of every lattice (post-collision populations, wall
   forces, step counter) to `path`, with a hash of the lattices, parameters,
   masks and G_w fields.  Synchronises. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);

/* Restores a state written by lbm_save into a context created with the same
   lattices, parameters, masks and G_w fields (LBM_ERR_ARG otherwise).
   Stepping on from the loaded state is bitwise identical to never having
   stopped. */
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* (An implementation call; the paper has no counterpart.)  Times lbm_step
   over `steps` steps for a fixed list of launch shapes
   (pipeline, block width, rows per block, per-step or persistent launch)
   on the context's own lattices and keeps the fastest; the persistent
   shapes are tried only where the batch has one parameter set.  The state
   and the step counter are restored after every trial, so the call changes
   nothing but the launch shape (lbm_get_launch reports it, persistent flag
   included); results do not depend on the shape.  The graph setting is
   kept.  Outputs (any may be NULL): the chosen bx, h and stages (as in
   lbm_set_launch; h = 0 is the automatic height) and its time per step in
   ms. */
lbm_status lbm_autotune(lbm_ctx* ctx, int steps, int* bx, int* h, int* stages, double* ms);

/* Self-test of the bounded device-side wait used by the persistent step
   kernel's grid barrier: one block waits for an arrival that never comes and
   must give up after `seconds` (0 < seconds <= 10).  Returns LBM_ERR_TIMEOUT
   when the wait gave up as designed; any other status means it did not. */
lbm_status lbm_selftest_wait_timeout(void* stream, double seconds);

/* Self-test of the FP32 reciprocal and square root of the FP32 step (a
   hardware approximation refined by one Newton-Raphson step) against the
   correctly rounded CUDA ones.  x: n host floats; out: 4 n host floats,
   out[4 i + 0..3] = step reciprocal, correctly rounded reciprocal, step
   square root, correctly rounded square root of x[i].  Synchronises the
   default stream.  LBM_ERR_ARG for NULL pointers or n < 1. */
lbm_status lbm_selftest_fp32_math(long n, const float* x, float* out);

/* Self-test of the FP64 reciprocal of the FP64 step (the hardware
   approximation refined by two Newton-Raphson steps): for n values x (host
   array), out[2 i], out[2 i + 1] = step reciprocal, correctly rounded
   reciprocal of x[i].  Synchronises the default stream.  LBM_ERR_ARG for
   NULL pointers or n < 1. */
lbm_status lbm_selftest_fp64_math(long n, const double* x, double* out);

/* Throughput of the FP64 pipe of the current device (an implementation
   detail; the paper has no counterpart): a probe kernel of eight
   independent chains of dependent FMAs per thread, 8 blocks of 256 threads
   per SM, timed with CUDA events on its second launch; *ops_per_s receives
   the DFMA instructions per second.  The FP64 step's roofline is reported
   against it.  Synchronises the device's default stream; LBM_ERR_ARG for a
   NULL pointer, LBM_ERR_CUDA if the probe cannot run. */
lbm_status lbm_selftest_fp64_rate(double* ops_per_s);

/* The dependency lists of the persistent warp strips (lbm_set_launch with
   persistent = 1), for inspection; host only, no GPU needed.  One nx x ny
   lattice cut into 30-column strips and h-row segments (segments outer,
   strips inner): item i covers columns [x0, min(nx, x0 + 30)) and rows
   [y0, y1), written as items3[3 i .. 3 i + 2] = x0, y0, y1.  Item i starts a
   step once the items nbr[off[i] .. off[i+1]) have finished the previous
   one: every item with a node within 4 nodes of one of its own along x and
   along y, periodic (itself included).  *n_items and *n_nbr receive the
   counts; with items3, off or nbr NULL only the counts are returned.  cap
   is the capacity of each of items3, off (n_items + 1) and nbr, in ints;
   LBM_ERR_ARG if one is too small, for NULL counts, nx or ny < 3, h < 1. */
lbm_status lbm_strip_neighbours(int nx, int ny, int h, int* n_items, int* items3, int* off,
                                int* nbr, int cap, int* n_nbr);

/* The work items of a context's lbm_step as built now (an implementation
   detail; the paper has no counterpart), for inspection: item i is the
   column strip [x0, x0 + width) of instance inst over rows [y0, y1), written
   as items4[4 i .. 4 i + 3] = inst, x0, y0, y1.  With persistent warp strips
   (lbm_set_launch persistent = 1) nbr[off[i] .. off[i+1]) lists the items
   item i waits for between steps, by the rule of lbm_strip_neighbours;
   otherwise every list is empty.  The items are listed in the order the
   even steps launch them (per parameter set; FP32 column-pair strips per
   step: tall segments first, then short ones, and odd steps take each of
   the two parts in reverse).  *n_items and *n_nbr receive the counts;
   with items4, off or nbr NULL only the counts are returned.  cap is the
   capacity of each of items4, off (n_items + 1) and nbr, in ints; LBM_ERR_ARG
   if one is too small or a count pointer is NULL. */
lbm_status lbm_get_work_items(const lbm_ctx* ctx, int* n_items, int* items4, int* off, int* nbr,
                              int cap, int* n_nbr);

/* Diagnostics without any device allocation, for callers that cannot call
   cudaMalloc: a host program whose device memory is owned entirely by its
   own allocator or budget, or a time-critical loop that must not pay the
   device-wide synchronisation cudaMalloc/cudaFree can imply.  The paper has
   no counterpart; this is a variant of lbm_diagnostics for fields the
   caller already holds.
   Inputs (all device memory, [ny][nx], FP64 unless stated): rho, ux, uy
   (e.g. from lbm_get_fields with dst_is_device = 1); solid: uint8 mask,
   nonzero = solid, or NULL for none.  level, y_w, x_ref, d_min as in
   lbm_diagnostics (level is normally (rho_L + rho_V)/2).  Work is enqueued
   on `stream` (a cudaStream_t or NULL) and the call waits for it.
   Scratch: a fixed 77,952-byte device array inside the library, kept by
   every GPU that loads it until the process exits.  The first call on a
   device looks up that array's device address (cudaGetSymbolAddress) with
   the device current.  Every call copies its result to the host and
   synchronises `stream`, so no call can be part of a stream capture.  All
   calls share the array: calls whose work overlaps on a GPU (other streams
   or threads) race and must be serialised by the caller; each call
   overwrites all the scratch it reads, so nothing carries over.
   Limit: nx * ny <= LBM_NOALLOC_MAX_NODES, else LBM_ERR_ARG.  out->step is
   -1 (no context).  Never calls cudaMalloc, cudaFree or an allocating
   library routine. */
#define LBM_NOALLOC_MAX_NODES (1LL << 28)
lbm_status lbm_diagnostics_noalloc(int nx, int ny, const double* rho, const double* ux,
                                   const double* uy, const uint8_t* solid, double level,
                                   double y_w, double x_ref, double d_min, void* stream,
                                   lbm_diag* out);

/* Message of the last error on the calling thread ("" if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
