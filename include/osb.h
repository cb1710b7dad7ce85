/*
 * osb.h -- C ABI of libosb: the explicit time step of the 3D compressible
 * Navier-Stokes equations on a periodic structured grid, as solved for the
 * Taylor-Green vortex in OpenSBLI (Jacobs, Jammy & Sandham, arXiv:1609.01277,
 * Section 3.3), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an osb_status; nothing throws across the ABI.  On an
 *    error, osb_last_error() returns a short message for the calling thread.
 *  - Conserved state layout: structure of arrays [field][z][y][x], x fastest,
 *    fields (rho, rho*u0, rho*u1, rho*u2, rho*E), FP64, no padding; N = nx*ny*nz
 *    points per field, so a host state is 5*N doubles.
 *  - Grid: domain [0, 2*pi)^3, x_i = i*h_a with h_a = 2*pi/n_a per axis, periodic
 *    in every direction (Section 2.2 grid, Section 2.6 periodic boundaries),
 *    unless osb_set_boundaries puts symmetry planes on an axis (that axis is
 *    then [0, pi] with x_i = (i + 1/2) pi/n_a).
 *  - Device memory is owned by the caller (for example allocated by PyTorch):
 *    the library never allocates or frees device memory.  The caller passes
 *    one state buffer and one workspace buffer per grid, sized by
 *    osb_state_bytes() and osb_workspace_bytes(), 256-byte aligned.
 *  - Stream: every kernel of a grid runs on the stream given at creation.
 *    Calls that return host data synchronise that stream.  One grid must not
 *    be used from two threads at once.
 */
#ifndef OSB_H
#define OSB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OSB_OK = 0,
    OSB_ERR_INVALID_ARG = 1, /* bad size, order, parameter or null pointer      */
    OSB_ERR_UNSUPPORTED = 2, /* valid request that the library does not provide */
    OSB_ERR_CUDA = 3,        /* a CUDA runtime call or a kernel launch failed   */
    OSB_ERR_NONFINITE = 4,   /* the state holds NaN or Inf                      */
    OSB_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up              */
    OSB_ERR_BUFFER = 6,      /* a buffer is too small or misaligned             */
    OSB_ERR_BOUNDS = 7       /* bounds-check build only: a kernel computed an
                                index outside its buffer (the access was
                                skipped; the state is invalid)                  */
} osb_status;

/* Arithmetic of the stencil path.  OSB_FP64: everything FP64.  OSB_FP32:
 * stencils, products and residual in FP32 with FP32 accumulation, while the
 * RK accumulator register and all diagnostics reductions stay FP64.
 * OSB_DF64: stencils, products and residual in double-float arithmetic (each
 * value the unevaluated sum of two FP32 numbers, about 48 significant bits,
 * computed with error-free FP32 transformations), the RK accumulator and the
 * reductions in FP64; it meets the FP64 path's accuracy bar at the FP32
 * pipes' rate.  Learned closures take FP64 or FP32 grids only. */
enum { OSB_FP64 = 0, OSB_FP32 = 1, OSB_DF64 = 2 };

/* Discretisation of the viscous work d_j(u_i tau_ij) in the energy equation
 * (Section 3.3, energy equation).  OSB_VISC_A differentiates the point-wise
 * product u_i tau_ij (discretely conservative: total energy is kept to
 * roundoff).  OSB_VISC_B is the product-rule expansion that the Der operator
 * of Section 2.1.1 produces. */
enum { OSB_VISC_A = 0, OSB_VISC_B = 1 };

typedef struct {
    int nx, ny, nz;  /* points per axis, each >= 1                            */
    int order;       /* central-difference order 2r: 2, 4, 6, 8, 10 or 12      */
    int precision;   /* OSB_FP64, OSB_FP32 or OSB_DF64                         */
    int visc_form;   /* OSB_VISC_A or OSB_VISC_B                               */
} osb_grid_desc;

/* Non-dimensional parameters (Section 3.3): Reynolds, Mach, ratio of specific
 * heats, Prandtl number, and the time-step size.  All must be > 0, gamma > 1. */
typedef struct {
    double Re, Mach, gamma, Pr, dt;
} osb_params;

/* Grid means (rho_ref = 1, Omega = the whole box), Section 3.3:
 *   ke        = <(1/2) rho u_j u_j>
 *   enstrophy = <(1/2) rho (eps_ijk d_j u_k)^2>, d_j the first-derivative stencil
 *   total[m]  = <Q_m> for the five conserved fields
 *   nonfinite = number of points with a non-finite conserved value
 *   max_cfl   = dt * max over points of sum_j (|u_j| + c)/h_j, c^2 = gamma p/rho
 * t and step are the simulated time and the number of RK3 steps taken. */
typedef struct {
    double t;
    long long step;
    double ke, enstrophy;
    double total[5];
    long long nonfinite;
    double max_cfl;
} osb_diag;

typedef struct osb_grid osb_grid; /* opaque; owns host metadata only */
typedef struct osb_closure osb_closure; /* opaque; learned residual correction */

/* Bytes of device memory the caller must provide for the state registers of
 * the low-storage RK3 scheme (two FP64 accumulators, two stage registers in
 * the grid's precision).  Returns 0 for an invalid descriptor. */
size_t osb_state_bytes(const osb_grid_desc *desc);

/* Bytes of device scratch for the point-wise intermediate fields of a stage
 * and the diagnostics partial sums.  Returns 0 for an invalid descriptor. */
size_t osb_workspace_bytes(const osb_grid_desc *desc);

/* Creates a grid over caller-owned device buffers.
 *  state_dev / workspace_dev: device pointers, 256-byte aligned, at least
 *    osb_state_bytes / osb_workspace_bytes long (else OSB_ERR_BUFFER).
 *  cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 *  The state is undefined until osb_init_taylor_green or osb_set_state.
 *  Errors: OSB_ERR_INVALID_ARG (sizes < 1, odd order, order outside 2..12,
 *  non-positive Re, Mach, Pr, dt, or gamma <= 1), OSB_ERR_UNSUPPORTED (an order
 *  or form without compiled kernels), OSB_ERR_BUFFER. */
osb_status osb_grid_create(const osb_grid_desc *desc, const osb_params *params,
                           void *state_dev, size_t state_bytes,
                           void *workspace_dev, size_t workspace_bytes,
                           void *cuda_stream, osb_grid **out);

/* Frees the host metadata of a grid; never touches the caller's buffers. */
osb_status osb_grid_destroy(osb_grid *grid);

/* Per-step diagnostics series (Section 3.3 grid means), fused into the first
 * RK stage: with a series attached, every osb_rk3_step / osb_euler_step step
 * appends the kinetic energy <(1/2) rho u.u> and the enstrophy
 * <(1/2) rho |omega|^2> (omega_i = eps_ijk d_j u_k, first-derivative stencil)
 * of the state at the START of the step, i.e. the step's stencil source.  The
 * stage kernel that forms the velocity gradient sums both over its thread
 * blocks (warp shuffles, FP64 block sums); one small kernel adds the block
 * sums in a fixed order, so the values are deterministic.  The FP64 and
 * double-float paths equal osb_diagnostics' ke and enstrophy up to rounding;
 * the FP32 path evaluates them from its FP32 stencil source (relative
 * error ~1e-7).
 *  series_dev: device FP64 ring of 2*capacity values, caller-owned: entry k
 *    (the k-th step after this call) goes to series_dev[2 (k mod capacity)],
 *    ke first.  NULL detaches.  Resets the step counter to 0.
 * osb_diag_series_count returns the number of steps recorded (synchronises
 * the stream).  osb_batch_step refuses grids with a series
 * (OSB_ERR_UNSUPPORTED).  Errors: OSB_ERR_INVALID_ARG (capacity < 1, or a
 * buffer not 8-byte aligned). */
osb_status osb_set_diag_series(osb_grid *grid, double *series_dev, int capacity);
osb_status osb_diag_series_count(osb_grid *grid, long long *count);

/* Boundary conditions per axis (Section 2.6, "Boundary conditions").
 *  OSB_BC_PERIODIC (every axis after osb_grid_create): the axis is [0, 2 pi),
 *    points x_i = 2 pi i / n, halos wrap around.
 *  OSB_BC_SYMMETRIC: symmetry planes at both ends of the axis, at 0 and pi
 *    (two of the Taylor-Green vortex's own mirror planes); points
 *    x_i = (i + 1/2) pi / n.  The halo beyond the plane after the last point
 *    mirrors the points before it, phi(x_{n+k}) = phi(x_{n-1-k}), and likewise
 *    phi(x_{-1-k}) = phi(x_k) at the first point; the momentum component
 *    normal to the plane changes sign there.  Every derived quantity a stage
 *    differentiates takes the parity of its factors, so the result equals the
 *    periodic scheme on the doubled, mirror-extended grid restricted to this
 *    one.  osb_init_taylor_green and osb_diagnostics use these coordinates
 *    and spacings.
 * Symmetric grids step with the three-kernel stage in every precision; they
 * take no learned closure and no ensemble stepping (OSB_ERR_UNSUPPORTED).
 * Errors: OSB_ERR_INVALID_ARG (a kind other than the two above). */
enum { OSB_BC_PERIODIC = 0, OSB_BC_SYMMETRIC = 1 };
osb_status osb_set_boundaries(osb_grid *grid, int bc_x, int bc_y, int bc_z);

/* Sets the Taylor-Green initial state of Section 3.3 (L = 1):
 *   u0 = sin x cos y cos z, u1 = -cos x sin y cos z, u2 = 0,
 *   p  = 1/(gamma M^2) + (cos 2x + cos 2y)(2 + cos 2z)/16, T = 1 (rho = gamma M^2 p),
 * then, if noise_dev is not NULL, u_i += noise_amp * noise_dev[i][z][y][x]
 * at fixed rho and p.  noise_dev: device FP64, 3*N values, caller-owned (the
 * caller draws the random numbers).  Resets t and step to 0. */
osb_status osb_init_taylor_green(osb_grid *grid, const double *noise_dev, double noise_amp);

/* Copies a conserved state (5*N FP64, layout above) from host memory in, or
 * out to host memory.  Both synchronise the grid's stream.  set_state resets
 * t and step to 0. */
osb_status osb_set_state(osb_grid *grid, const double *host_src);
osb_status osb_get_state(osb_grid *grid, double *host_dst);

/* Device-to-device variants of the two calls above (stream-ordered, no sync). */
osb_status osb_set_state_device(osb_grid *grid, const double *dev_src);
osb_status osb_get_state_device(osb_grid *grid, double *dev_dst);

/* Semi-discrete residual R(Q) = dQ/dt of the current state (no update):
 * skew-symmetric convective terms (Section 3.3, skew-symmetric form),
 * pressure, viscous stress with the Laplacian by the second-derivative
 * stencil, heat flux and viscous work.  R_dev: device FP64, 5*N values,
 * caller-owned.  In OSB_FP32 (OSB_DF64) grids the residual is computed in FP32
 * (double-float) and widened. */
osb_status osb_residual(osb_grid *grid, double *R_dev);

/* Advances the state by nsteps steps of the low-storage third-order
 * Runge-Kutta scheme (Section 2.4): for k = 1..3,
 *   q_k = U_{k-1} + alpha_k dt R(q_{k-1}),  U_k = U_{k-1} + beta_k dt R(q_{k-1}),
 * alpha = (2/3, 5/12, 3/5), beta = (1/4, 3/20, 3/5), q_0 = U_0 = Q^n,
 * Q^{n+1} = U_3.  Stream-ordered, no sync.  nsteps >= 0.  Runs of two or more
 * steps (no closure attached, no profiling) replay a CUDA graph of one step,
 * captured on first use on a library-owned stream (set OSB_GRAPHS=0 to
 * launch the kernels directly); results are identical either way. */
osb_status osb_rk3_step(osb_grid *grid, int nsteps);

/* Forward Euler, the first-order scheme the paper offers beside RK3
 * (Section 2.4): nsteps steps of U^{n+1} = U^n + dt R(U^n), one residual
 * evaluation per step, on the same grid, state and precision as
 * osb_rk3_step (the two may be mixed).  Queued on the grid's stream.
 * Errors: NULL grid or nsteps < 0 -> OSB_ERR_INVALID_ARG; launch failure ->
 * OSB_ERR_CUDA. */
osb_status osb_euler_step(osb_grid *grid, int nsteps);

/* Computes the diagnostics of the current state into *out (FP64 reductions,
 * deterministic order).  Synchronises the stream.  Returns
 * OSB_ERR_NONFINITE (with *out filled) if any conserved value is NaN/Inf. */
osb_status osb_diagnostics(osb_grid *grid, osb_diag *out);

/* Advances n independent grids (an ensemble of uneven sizes, Reynolds and
 * Mach numbers and time steps; an extension of the paper's Section
 * 3.3 solver) by nsteps RK3 steps each.  Two ways, chosen by precision
 * (environment OSB_BATCH_MODE = persistent | streams overrides):
 *  - FP64 and FP32 (default "persistent"): ONE persistent kernel launch for all steps,
 *    captured into a CUDA graph on first use and replayed on later calls with
 *    the same grids, parities and nsteps.  Work items (step, stage phase,
 *    instance, tile) are taken in order by resident CTAs; a per-instance
 *    completion count orders the phases of each instance.  Each tile is 32 x 8
 *    points by tz planes, tz chosen per grid shape by osb_autotune (default 4).
 *  - double-float (default "streams"; FP32 on request): each grid's own one-step CUDA
 *    graph (the kernels osb_rk3_step runs) replayed step by step on one of up
 *    to 8 library-owned streams (grids spread over them by size, largest
 *    first), so small grids run side by side; the streams wait for earlier
 *    work on the grids' stream and the grids' stream waits for them.
 * Requirements: 1 <= n <= 128 distinct grids on one stream with the same
 * order, precision and viscous form (else OSB_ERR_INVALID_ARG /
 * OSB_ERR_UNSUPPORTED).  Synchronises the stream.
 * OSB_ERR_TIMEOUT (persistent kernel only): a device-side wait exceeded its
 * limit (osb_batch_configure); the kernel stopped and the grids' states are
 * undefined, the CUDA context stays usable.  OSB_ERR_CUDA in the stream mode
 * (a step graph that could not be captured or launched): the streams are
 * joined back into the grids' stream and synchronised, and the grids' states
 * are undefined.  Results equal those of osb_rk3_step on each grid (bit for bit in FP64 and in the stream mode; FP32
 * work items of the persistent kernel to FP32 rounding). */
osb_status osb_batch_step(osb_grid *const *grids, int n, int nsteps);

/* Ensemble controls (tooling; no counterpart in the paper).  wait_limit_seconds
 * bounds every per-instance wait of osb_batch_step's persistent kernel
 * (default 2 s; must be in
 * (0, 3600]).  test_stall != 0 makes the first wait of the next batches target
 * a count that nothing reaches, so the wait runs out and the call returns
 * OSB_ERR_TIMEOUT -- used to test the failure path without faulting a GPU
 * (while set, every ensemble runs the persistent kernel).
 * Process-wide settings. */
osb_status osb_batch_configure(double wait_limit_seconds, int test_stall);

/* Times osb_batch_step's persistent kernel on this grid alone for each candidate tile depth
 * (1, 2, 4, 8, 16 z planes), trial_steps steps each, and keeps the fastest for
 * the grid's shape (nx, ny, nz, order, precision, form) in a process-wide table,
 * also written to the file named by $OSB_AUTOTUNE_CACHE when set (read back
 * on first use).  The grid's state, time and step count are restored
 * afterwards (through a host copy).  *best_tz receives the choice (may be NULL). */
osb_status osb_autotune(osb_grid *grid, int trial_steps, int *best_tz);

/* Tile depths for an ensemble, tuned in place: for each distinct grid shape
 * in turn (largest total points first; the others held at their current
 * depths), the candidate depths of osb_autotune are timed on
 * osb_batch_step's persistent kernel over the whole ensemble, trial_steps
 * steps each, and the fastest is kept in the process-wide table (and the
 * $OSB_AUTOTUNE_CACHE file).  A grid timed alone favours short z chunks for
 * parallelism; inside a large ensemble the others supply it, and longer
 * chunks save the z-queue warm-up planes (64 grids of 32^3..128^3, FP32:
 * 1.48e10 -> 1.65e10 point-stages/s).  The grids' states, times and step
 * counts are restored afterwards (through host copies).  Requirements as
 * osb_batch_step's; errors: OSB_ERR_INVALID_ARG (NULL grids, n outside
 * 1..128, trial_steps < 1), and those of osb_batch_step. */
osb_status osb_autotune_batch(osb_grid *const *grids, int n, int trial_steps);

/* The z planes per work item that osb_batch_step's persistent kernel uses for
 * grids of this descriptor's shape (the tuned depth, else the default: 8 for
 * FP32, 4 otherwise).  0 for an invalid descriptor. */
int osb_tile_depth(const osb_grid_desc *desc);

/* Diagnostics of a caller-provided state without any device allocation and
 * without a grid object.  The state is read as a fully periodic box
 * [0, 2 pi)^3 (h = 2 pi / n, wrapped stencils); states of grids with symmetry
 * planes (osb_set_boundaries) must use osb_diagnostics instead, since this
 * call has no boundary argument and would return wrong enstrophy and CFL.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory at the point where they need
 * the diagnostics -- for example code running while a stream is captured into
 * a CUDA graph in global capture mode (where cudaMalloc is an error that
 * invalidates the capture), loops that must not take the implicit device
 * synchronisation an allocation can cause, or hosts whose device memory is
 * entirely pre-reserved by their own allocator.
 *
 *  Q_dev:   device, 5*nx*ny*nz FP64 values in the conserved layout above (no
 *           padding between fields), caller-owned, read only.
 *  out_dev: device, 9 FP64 values, caller-owned, written: ke, enstrophy,
 *           total[0..4], the non-finite point count (as a double), max_cfl --
 *           the same quantities as osb_diag.
 *  params:  gamma, Mach and dt are used (gamma > 1, Mach > 0, dt > 0).
 *  cuda_stream: stream the two kernels run on; the call does not synchronise.
 * Scratch: a fixed device array of 1216 partial-sum records (155,648 bytes)
 * inside the library, held on every device that loads the library until the
 * process exits.  Every admissible grid (nx*ny*nz < 2^31, each >= 1) fits it;
 * larger or invalid sizes are rejected with OSB_ERR_INVALID_ARG, pointers not
 * 8-byte aligned with OSB_ERR_BUFFER, both before any GPU work.  Every call
 * looks up the array's device address on the current device (no allocation);
 * the first call on a device may load the library's device code, so make it
 * before any stream capture begins.  All
 * calls share the one array, so calls whose kernels overlap on the GPU (for
 * example on two streams at once) race and give wrong results; serialise them.
 * No allocation of any kind: no cudaMalloc, cudaFree or allocating library
 * routine is called. */
osb_status osb_diagnostics_noalloc(const double *Q_dev, int nx, int ny, int nz, int order,
                                   const osb_params *params, double *out_dev, void *cuda_stream);

/* ------------------------------------------------------------------------
 * z-slab domain decomposition.  The paper runs its largest Taylor-Green case
 * (Section 3.3) with the box split over many processes, the periodic
 * boundaries and the subdomain faces kept up to date by halo transfers
 * (Section 2.6).  Here one grid holds a slab of consecutive z planes of a
 * periodic box; the caller moves the halo planes between slabs (on one GPU by
 * device copies, across GPUs e.g. by NCCL send/recv) through staging buffers
 * it owns, and advances the slabs one RK stage at a time:
 *
 *     for each step, for k = 0, 1, 2:
 *         every slab: osb_halo_pack(slab, k, send_lo, send_hi)
 *         exchange:   slab s receives recv_lo = send_hi of slab s-1 and
 *                     recv_hi = send_lo of slab s+1 (periodic in s)
 *         every slab: osb_halo_unpack(slab, k, recv_lo, recv_hi)
 *         every slab: osb_rk3_stage(slab, k)
 *
 * A slab's array has nz = n_own + 2H planes: H = order ghost planes at each
 * end (the nested first derivatives of viscous form A reach 2R = order planes)
 * around the n_own planes it owns.  Each owned plane then evolves exactly as
 * in the undivided box (bit for bit: the same operands in the same order).
 * ------------------------------------------------------------------------ */

/* Makes a grid a z-slab of a periodic box of nz_domain planes along z (the z
 * spacing is 2 pi / nz_domain).  Requires nz >= 3 * order (two ghost widths
 * and one owned width), a periodic z axis, no diagnostics series and no
 * closure; osb_rk3_step, osb_euler_step and osb_batch_step then refuse the
 * grid (OSB_ERR_UNSUPPORTED), osb_diagnostics reduces the owned planes only
 * (means over those planes: combine slabs weighted by n_own, after exchanging
 * source 3).  The grid's state is read and written with osb_set_state /
 * osb_get_state as before, ghost planes included. */
osb_status osb_set_z_slab(osb_grid *grid, int nz_domain);

/* Bytes of one staging buffer (send_lo, send_hi, recv_lo or recv_hi) of a
 * z-slab grid: 5 fields x order planes x nx x ny x 8 bytes (large enough for
 * every source); 0 if the grid is not a slab. */
size_t osb_halo_bytes(const osb_grid *grid);

/* Packs the order planes next to each face of the slab's owned planes of one
 * source into two staging buffers, layout [field][plane][y][x] in the source's
 * element type (FP64, FP32 or double-float), contiguous:
 *   source 0..2: the stencil source of RK stage `source` of the step in
 *                progress (must equal the next stage osb_rk3_stage runs);
 *   source 3:    the FP64 accumulator holding Q^n (before osb_diagnostics).
 *  send_lo_dev / send_hi_dev: device, osb_halo_bytes bytes each, caller-owned,
 *   8-byte aligned; written with the planes next to the low / high z face.
 * Queued on the grid's stream (no synchronisation).  Errors: NULL arguments, a
 * grid that is not a slab, a source out of order -> OSB_ERR_INVALID_ARG;
 * unaligned buffers -> OSB_ERR_BUFFER; a failed launch -> OSB_ERR_CUDA. */
osb_status osb_halo_pack(osb_grid *grid, int source, void *send_lo_dev, void *send_hi_dev);

/* Unpacks the buffers received from the z neighbours into the ghost planes of
 * the same source: recv_lo_dev (the low neighbour's send_hi) into the order
 * planes below the owned planes, recv_hi_dev (the high neighbour's send_lo)
 * into those above.  Same arguments, ownership and errors as osb_halo_pack. */
osb_status osb_halo_unpack(osb_grid *grid, int source, const void *recv_lo_dev, const void *recv_hi_dev);

/* One stage k (0, 1, 2, in this order) of the RK3 step (Section 2.4) on the
 * grid's stream; after stage 2 the step is complete (time and step count
 * advance).  Any grid can be stepped this way; a z-slab must be.  Errors: a
 * stage out of order -> OSB_ERR_INVALID_ARG; a failed launch -> OSB_ERR_CUDA. */
osb_status osb_rk3_stage(osb_grid *grid, int k);

/* Measurement utility (no counterpart in the paper): the FP64 fused
 * multiply-add rate of the device, the roofline denominator of the FP64 stage
 * kernels.  One launch of `blocks` blocks of 256 threads; each thread runs 8
 * independent FMA chains for 16*iters steps and writes one double to out_dev.
 * flops = blocks * 256 * 8 * 16 * iters * 2; the caller times the launch on
 * cuda_stream (the call does not synchronise).
 *  out_dev: device, blocks*256 FP64 values, caller-owned, overwritten.
 * Errors: NULL or unaligned out_dev, blocks < 1 or iters < 1 ->
 * OSB_ERR_INVALID_ARG; a failed launch -> OSB_ERR_CUDA. */
osb_status osb_fp64_rate_probe(double *out_dev, int blocks, int iters, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Scalar advection-diffusion on the periodic box [0, 2 pi)^3: the equation of
 * the paper's verification tests -- the wave equation of Section 3.1
 * (k = 0, no source) and the manufactured-solution advection-diffusion test
 * of Section 3.2:
 *     d phi/dt + d_j(phi a_j - k d_j phi) + S = 0,   a_j, k constant,
 * discretised with the central first- and second-derivative stencils of the
 * given order (Section 2.4, h = 2 pi / n per axis; an axis with one point
 * carries no derivative) and advanced nsteps steps of the low-storage RK3
 * scheme used by osb_rk3_step.  FP64 throughout.
 *
 *  phi_dev:  device, nx*ny*nz FP64 values, x fastest; read as phi(t), written
 *            with phi(t + nsteps dt).  Caller-owned.
 *  work_dev: device scratch of 2*nx*ny*nz FP64 values, caller-owned, clobbered.
 *  src_dev:  device, nx*ny*nz FP64 values of S, or NULL for S = 0.
 *  adv:      host, the 3 velocity components a_0, a_1, a_2.
 *  diff:     the diffusivity k >= 0.
 *  cuda_stream: the stream the kernels (and, for odd nsteps, one device-to-
 *            device copy of the result) are queued on; the call does not
 *            synchronise and allocates nothing.
 * Errors: NULL pointers, sizes below 1 or above 2^31 points, an order outside
 * 2..12 or odd, dt <= 0, k < 0 or nsteps < 0 -> OSB_ERR_INVALID_ARG; buffers
 * not 8-byte aligned -> OSB_ERR_BUFFER; a failed launch -> OSB_ERR_CUDA.
 * nsteps = 0 does nothing. */
osb_status osb_scalar_rk3(double *phi_dev, double *work_dev, const double *src_dev, int nx, int ny, int nz,
                          int order, const double *adv, double diff, double dt, int nsteps, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Learned residual correction ("closure") for coarse grids.  Not in the paper
 * (its future work lists LES models, Section 1); an extension.
 * Network: three 3x3x3 periodic convolutions 5 -> 32 -> 32 -> 5 with ReLU
 * after the first two; input: the 5 conserved fields normalised per channel
 * ((Q_c - mean_c)/std_c); output y scaled per channel by out_std_c and added
 * to the residual R in every RK stage.  BF16 weights and activations, FP32
 * accumulation on the tensor cores.  Grid sizes must be multiples of (8,4,4).
 * ------------------------------------------------------------------------ */

/* FP32 master parameters: W1[32][5][27] b1[32] W2[32][32][27] b2[32]
 * W3[5][32][27] b3[5] (tap k = (dz+1)*9 + (dy+1)*3 + (dx+1), cross-correlation
 * y(p) = b + sum_k W[k] x(p + offset_k)).  36,357 values. */
size_t osb_closure_param_count(void);
/* Device scratch for a closure on an nx x ny x nz grid; 0 if unsupported. */
size_t osb_closure_workspace_bytes(int nx, int ny, int nz);
/* params_dev: caller-owned FP32 device array of 3 * osb_closure_param_count()
 * values (parameters, then the two Adam moment arrays), 16-byte aligned.
 * ws_dev: caller-owned, 256-byte aligned, osb_closure_workspace_bytes long.
 * After writing parameters, call osb_closure_sync_weights. */
osb_status osb_closure_create(int nx, int ny, int nz, float *params_dev, void *ws_dev, size_t ws_bytes,
                              void *cuda_stream, osb_closure **out);
osb_status osb_closure_destroy(osb_closure *closure);
/* Per-channel input mean/std and output scale (arrays of 5; stds > 0). */
osb_status osb_closure_set_normalization(osb_closure *closure, const float *in_mean, const float *in_std,
                                         const float *out_std);
/* Which equations receive the correction (apply[5], nonzero = yes; default all
 * five).  Training always fits all five outputs; the mask only selects what
 * is added to R.  Correcting only the momentum equations (1,1,1 for rho u_i,
 * 0 for rho and rho E) plays the role of a subgrid-stress model. */
osb_status osb_closure_set_channels(osb_closure *closure, const int *apply);
/* on != 0: the momentum part of the correction may not feed kinetic energy at
 * any point -- where u . C_m > 0 (u = m / rho of the state being corrected)
 * the component of C_m along u is removed, the clipping of backscatter used
 * by eddy-viscosity subgrid models.  Default off.  Training is unaffected. */
osb_status osb_closure_set_dissipative(osb_closure *closure, int on);
/* Weight w > 0 multiplying the loss and every gradient of the following
 * osb_closure_loss_grad calls (default 1): per-sample weighting of the
 * training loss. */
osb_status osb_closure_set_loss_weight(osb_closure *closure, float w);
/* Rebuilds the BF16 tensor-core weight layouts from the FP32 parameters. */
osb_status osb_closure_sync_weights(osb_closure *closure);
/* C_dev (device FP32, 5*N SoA) = out_std * net(normalised Q); Q_dev device
 * FP64 fields with the given field stride (>= N).  Stream-ordered. */
osb_status osb_closure_forward(osb_closure *closure, const double *Q_dev, size_t field_stride, float *C_dev);
/* MSE between the normalised output for input X and the normalised target
 * Cstar (both device FP64 fields, strides >= N); writes the loss (device FP32
 * scalar) and the gradient of every parameter (device FP32, layout of the
 * parameters; written, not accumulated).  Deterministic. */
osb_status osb_closure_loss_grad(osb_closure *closure, const double *X_dev, size_t x_stride, const double *Cstar_dev,
                                 size_t c_stride, float *grad_dev, float *loss_dev);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step >= 1)
 * on the parameters with the given gradient, then osb_closure_sync_weights. */
osb_status osb_closure_adam_step(osb_closure *closure, const float *grad_dev, float lr, int step);
/* Synchronises the closure's stream and reports OSB_ERR_TIMEOUT if a bounded
 * wait of a tensor-core convolution ever ran out (results then invalid). */
osb_status osb_closure_status(osb_closure *closure);
/* Attaches a closure to a grid of the same size (NULL detaches): every RK
 * stage and osb_residual then add its correction to R.  Grids with a closure
 * are stepped singly (osb_batch_step returns OSB_ERR_UNSUPPORTED). */
osb_status osb_grid_set_closure(osb_grid *grid, osb_closure *closure);
/* Box filter (training data for the closure): coarse = mean over factor^3
 * blocks of a fine state.  Both device FP64, 5 fields, no padding; fine sizes
 * multiples of factor.  Stream-ordered. */
osb_status osb_box_filter(const double *fine_dev, int fnx, int fny, int fnz, int factor, double *coarse_dev,
                          void *cuda_stream);

/* Per-kernel timing (tooling, no counterpart in the paper).  profile_start
 * creates 4 CUDA events per stage for up to max_stages stage launches; each
 * subsequent RK stage records them around its three kernels (primitives,
 * gradient fluxes, residual+update) on the grid's stream.  profile_stop
 * synchronises the stream, writes for kind k = 0, 1, 2 the summed event time
 * total_ms[k] and launch count launches[k] (arrays of 3), and frees the
 * events.  Stages beyond max_stages are not recorded. */
osb_status osb_profile_start(osb_grid *grid, int max_stages);
osb_status osb_profile_stop(osb_grid *grid, double *total_ms, long long *launches);

const char *osb_status_string(osb_status status);
const char *osb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OSB_H */
