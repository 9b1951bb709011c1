/*
 * hydro.h -- C ABI of libhydro, a GB300 (sm_103a) library that advances the
 * compressible Euler equations of a gamma-law gas with a constant-gravity
 * source on a uniform Cartesian grid.
 *
 * The paper this library serves ("Modeling Astrophysical Explosions with
 * Sustained Exascale Computing", introduction) describes the star as a fluid
 * on a domain-decomposed Cartesian grid, and ("Capabilities needed") says
 * that every time step needs nearest-neighbour communication plus a global
 * one.  Here the nearest-neighbour part is the depth-2 stencil halo read
 * inside one GPU and the global part is the CFL time-step min-reduction and
 * the conserved-total sums.  The paper prints no scheme; the update is the
 * unsplit finite-volume step:
 *   - primitive variables W = (rho, u_0 .. u_{ndim-1}, p), p = (gamma-1)(E - |m|^2/(2 rho));
 *   - PLM slopes with the MC limiter (van Leer 1977);
 *   - single-stage unsplit MUSCL-Hancock half step in primitive variables
 *     (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
 *     3rd ed., sec. 14.4), all axes and gravity at once; a cell whose
 *     predicted face density or pressure is not positive uses zero slopes;
 *   - an HLLC flux at every face (Toro sec. 10.4-10.6, Davis wave speeds);
 *   - conservative update: density first, momentum source g (rho^n +
 *     rho^{n+1})/2, energy source g . (low-face + high-face mass flux)/2;
 *   - dt = cfl / max_cells sum_d (|u_d| + c)/dx_d in FP64, taken from the
 *     state each step starts from, clamped to land exactly on a target time.
 * Boundaries: outflow (zero gradient), periodic, reflecting (mirror with the
 * normal momentum negated; the far side of a wall face is the mirror of the
 * near side's predicted state, so no mass crosses a wall).
 *
 * Memory and ownership.  The caller owns all device memory and the stream:
 * two state buffers (ping-pong) of hydro_state_bytes() each and one workspace
 * of hydro_workspace_bytes(), all device pointers with 256-byte alignment.
 * The library allocates no device memory; it owns only the host-side handle.
 * A state is nvar = ndim + 2 planes of nx*ny*nz values, plane q at offset
 * q*nx*ny*nz, x fastest: (rho, rho u_0 .. rho u_{ndim-1}, E), in FP64, or in
 * FP32 for HYDRO_FP32.  With hse_subtract the stored state is the
 * perturbation U - U0(z) from the hydrostatic background U0 = (rho0, 0, 0, 0,
 * p0/(gamma-1)).
 *
 * Errors.  Every call returns a hydro_status; nothing traps, exits or throws
 * across the ABI.  CUDA failures are reported as HYDRO_ERR_CUDA.  Device-side
 * detection of a non-positive or non-finite density or pressure puts the
 * handle in an error state (further steps leave the state unchanged) that is
 * reported as HYDRO_ERR_NONPHYSICAL by the next call that synchronises, until
 * hydro_set_state or hydro_destroy.  One host thread per handle.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYDRO_OK = 0,
    HYDRO_ERR_INVALID_ARG = -1,   /* bad pointer, size, enum or alignment */
    HYDRO_ERR_OOM = -2,           /* a caller buffer is too small */
    HYDRO_ERR_CUDA = -3,          /* a CUDA call failed */
    HYDRO_ERR_NONPHYSICAL = -4,   /* rho or p <= 0 or non-finite was produced */
    HYDRO_ERR_TIMEOUT = -5,       /* a bounded device wait ran out */
    HYDRO_ERR_STATE = -6          /* call not valid in the handle's state */
} hydro_status;

enum { HYDRO_BC_OUTFLOW = 0, HYDRO_BC_PERIODIC = 1, HYDRO_BC_REFLECT = 2 };
enum { HYDRO_FP64 = 0, HYDRO_FP32 = 1 /* FP32 state and update, FP64 dt, time and totals */ };
/* Time integrators.  HANCOCK: single-stage unsplit MUSCL-Hancock (Toro, 3rd
   ed., sec. 14.4), one kernel per step.  SSPRK2: method of lines with the
   two-stage SSP Runge-Kutta method of Shu and Osher (1988), U1 = U + dt L(U),
   U^{n+1} = (U + U1 + dt L(U1)) / 2, L the same PLM-MC/HLLC operator
   without the half-step predictor; two kernels per step and one more state
   in the workspace.  SSPRK2 is available through hydro_init only (not in
   batches or slab decompositions). */
enum { HYDRO_SCHEME_HANCOCK = 0, HYDRO_SCHEME_SSPRK2 = 1, HYDRO_SCHEME_CTU = 2 };
/* CTU: the unsplit corner transport upwind method (Colella 1990): per axis a
   one-dimensional MUSCL-Hancock predictor, first-pass HLLC fluxes, face
   states corrected by the transverse flux differences, final HLLC fluxes;
   one kernel per step; PLM only.  With hse_subtract = 1 the step is written
   on the perturbations: the z predictor advects the background and takes
   g rho'/rho - B_k/rho, the x and y predictors take g, face states are
   corrected as total states, and the x and y states' z-momentum correction
   adds the background's pressure difference across the cell (the first-pass
   z fluxes carry p'). */
/* Face-state reconstruction.  PLM: MC-limited piecewise linear (van Leer
   1977).  PPM: the piecewise parabolic method (Colella and Woodward 1984):
   interface values from the MC-limited slopes, parabola limited to be
   monotone; needs HYDRO_SCHEME_SSPRK2, hse_subtract = 0 and n[d] >= 3. */
enum { HYDRO_RECON_PLM = 0, HYDRO_RECON_PPM = 1 };
enum {
    HYDRO_RED_TOTALS = 1,    /* out[nvar]: sum over cells of (rho, m_d, E) * cell volume, FP64, fixed order */
    HYDRO_RED_DT = 2,        /* out[1]: CFL dt of the current state */
    HYDRO_RED_TIME = 3,      /* out[1]: current time */
    HYDRO_RED_MAXSPEED = 4,  /* out[1]: max_cells sum_d (|u_d| + c)/dx_d of the current state */
    HYDRO_RED_STEP = 5,      /* out[1]: steps taken since init or set_state */
    HYDRO_RED_DT_LAST = 6    /* out[1]: dt taken by the last step */
};

/* Problem description.  ndim 2 or 3; n[d] >= 2 for d < ndim and n[d] == 1
   for d >= ndim; lo < hi; bc_* per axis; gamma > 1; cfl > 0; grav is the
   constant acceleration.  hse_subtract = 1 needs ndim = 3 and gravity along
   z only, and the background tables of hydro_init. */
typedef struct {
    int ndim;
    int n[3];
    double lo[3], hi[3];
    int bc_lo[3], bc_hi[3];
    double gamma, cfl;
    double grav[3];
    int precision;       /* HYDRO_FP64 or HYDRO_FP32 */
    int hse_subtract;
    int scheme;          /* HYDRO_SCHEME_HANCOCK (0), HYDRO_SCHEME_SSPRK2 or HYDRO_SCHEME_CTU */
    int recon;           /* HYDRO_RECON_PLM (0) or HYDRO_RECON_PPM */
} hydro_problem;

typedef struct hydro_sim hydro_sim;

/* Bytes of one state buffer: nvar * nx*ny*nz * (8 or 4).  0 if invalid. */
size_t hydro_state_bytes(const hydro_problem *prob);

/* Bytes of the workspace: time-control block, per-CTA partials, FP64
   background tables.  0 if invalid. */
size_t hydro_workspace_bytes(const hydro_problem *prob);

/* Bind caller buffers and set the initial state.
   Ua, Ub: device state buffers (hydro_state_bytes each); work: device
   workspace (hydro_workspace_bytes).  W0: HOST array of total primitive
   variables (rho, u_0 .. u_{ndim-1}, p), FP64, nvar planes, converted to the
   stored form on the device (Ub is used as staging).  bg: HOST FP64
   background tables when hse_subtract (else NULL): rho0 and p0 at the
   centres of planes k = -2 .. nz+1 (2 arrays of nz+4, in that order), then
   rho0 and p0 at the faces z_lo + f dz, f = -2 .. nz+2 (2 arrays of nz+5).
   stream: a cudaStream_t (NULL = legacy default stream).  Computes the
   first dt on the device; t = 0, step = 0.  *out receives the handle. */
int hydro_init(const hydro_problem *prob, void *Ua, void *Ub, void *work,
               const double *W0, const double *bg, void *stream, hydro_sim **out);

/* hydro_init with the initial state given as HOST FP64 total conserved
   variables U0 = (rho, rho u_0 .. rho u_{ndim-1}, E), nvar planes of
   nx*ny*nz values.  The device rounds them to the stored precision (FP32
   for HYDRO_FP32) and, with hse_subtract, first subtracts the background
   U0(z) = (rho0, 0, 0, 0, p0/(gamma-1)) in FP64.  Every other argument,
   the set-up and the errors are those of hydro_init.  (hydro_init takes
   primitives because initial conditions are specified as density,
   velocity and pressure at cell centres; this entry serves restarts and
   couplings that hold conserved variables.) */
int hydro_init_conserved(const hydro_problem *prob, void *Ua, void *Ub, void *work,
                         const double *U0, const double *bg, void *stream, hydro_sim **out);

/* One step on the handle's stream.  dt_taken (nullable): when given, the
   call synchronises and returns the dt used; when NULL nothing is read back
   and errors surface at the next synchronising call. */
int hydro_step(hydro_sim *sim, double *dt_taken);

/* Steps until t reaches t_end exactly (the last dt is clamped) or max_steps
   steps have been taken.  Reads the device time block once per batch of
   launches.  nsteps_out, t_out nullable. */
int hydro_advance_to(hydro_sim *sim, double t_end, long max_steps, long *nsteps_out,
                     double *t_out);

/* Reductions of the current state (see HYDRO_RED_*); synchronises. */
int hydro_reduce(hydro_sim *sim, int what, double *out);

/* Device pointer of the buffer that holds the current state.  Launches
   made after time reached a target (hydro_advance_to) or after an error
   move nothing, so the current buffer follows the device's step count; it
   is exact after any call that synchronises (hydro_advance_to,
   hydro_reduce, hydro_step with dt_taken, the state and field calls). */
void *hydro_current(hydro_sim *sim);

/* Raw stored state (hydro_state_bytes) to / from HOST memory, for
   checkpoint and restart.  set_state also sets t and step, recomputes dt and
   clears the error state. */
int hydro_get_state(hydro_sim *sim, void *host_dst);
int hydro_set_state(hydro_sim *sim, const void *host_src, double t, long step);

/* Current state as FP64 total conserved variables (what = 0) or total
   primitive variables (what = 1) into a HOST array of nvar*N doubles; the
   spare ping-pong buffer is used as device staging. */
int hydro_get_fields(hydro_sim *sim, int what, double *host_dst);

/* Test hook: overwrite one stored value of the current state with v
   (converted to the stored precision).  Used to inject a non-physical cell
   from the host. */
int hydro_debug_poke(hydro_sim *sim, int var, long cell, double v);

/* Select the 3D z-chunk length (planes per CTA); 0 restores the default.
   A negative value selects the balanced grid instead: as many CTAs as the
   device holds resident at once, the (tile, z-chunk) pieces taken in whole
   waves of neighbouring tiles at the same heights while at least one wave
   remains, and the planes of the last, partial wave split evenly, so that
   every CTA marches the same number of planes and the launch has no partial
   last wave.  HYDRO_ZCHUNK_BALANCED (-1) uses whole columns as the pieces,
   -Z pieces of Z planes.  MUSCL-Hancock and SSP-RK2 steps of tile variants
   0..7 only: HYDRO_ERR_INVALID_ARG for 2D, the corner transport upwind step
   and the paired-cell variants, and selecting a paired-cell variant returns
   to z-chunks.  Results do not depend on the choice. */
#define HYDRO_ZCHUNK_BALANCED (-1)
int hydro_set_zchunk(hydro_sim *sim, int zchunk);

/* Select the 3D tile shape and staging depth: variant index of
   hydro_batch_variant_shape.  Variants 0..3 load each staged plane
   synchronously, 4..7 (the same shapes) copy the next plane asynchronously
   one plane ahead (MUSCL-Hancock step; the other integrators use the shape
   only).  Default: variant 7 (32 x 16) for FP32, 6 (16 x 16) for FP64, the
   autotuner's usual choices on GB300.  Variants 3
   and 7 (32 x 16) are FP32 only.  Results do not depend on the choice
   among 0..7; the paired-cell FP32 variants 8..10 are described below. */
int hydro_set_tile(hydro_sim *sim, int variant);

/* Paired-cell FP32 tiles: variants 8, 9, 10 (32 x 16, 32 x 8 and 16 x 16
   cells) run the FP32 MUSCL-Hancock step with each thread owning two
   x-adjacent cells, in packed f32x2 arithmetic (FP32, HYDRO_SCHEME_HANCOCK,
   3D single solves only).  Their results do not depend on the choice among
   8..10, and differ from those of variants 0..7 by FP32 rounding only (the
   same formulas, grouped into other instructions).  hydro_tile_shape gives
   the cell tile (tx x ty) of any single-solve variant 0..10. */
int hydro_tile_shape(int variant, int *tx, int *ty);

/* Number of kernels launched by this handle so far. */
long hydro_launch_count(hydro_sim *sim);

/* Checkpoint to / restart from a file: a header (magic "HYDROCK1", version
   1, the problem, t, step, state size, FNV-1a checksum of the state) and
   the raw stored state (hydro_get_state's layout).  Load needs a handle
   made with the same problem (and background tables); it rejects any
   mismatch, short or corrupted file with HYDRO_ERR_INVALID_ARG and leaves
   the handle unchanged, else sets state, t and step as hydro_set_state.
   Both synchronise the handle's stream. */
int hydro_checkpoint_save(hydro_sim *sim, const char *path);
int hydro_checkpoint_load(hydro_sim *sim, const char *path);

/* Test hook, needs no GPU: the column pieces (tile, first plane, end plane)
   one CTA of a 3D step marches, in marching order -- the chunked grid's CTA
   (tile, chunk) for zchunk > 0, else CTA b of a balanced grid of G CTAs
   (hydro_set_zchunk's negative settings) -- for `tiles` tiles of nz planes.
   Writes up to max_pieces triples to out and returns the number of pieces,
   or HYDRO_ERR_INVALID_ARG. */
int hydro_debug_pieces(int zchunk, long long tiles, int nz, int tile, int chunk, long long G, long long b,
                       int *out, int max_pieces);

/* Test hook: evaluate the update's FP64 arithmetic helpers on n device
   values, out[i] = 1/x[i] (which = 0), y[i]/x[i] (1), 1/sqrt(x[i]) (2) or
   the MC-limited slope of (x[i], y[i]) (3), so that they can be checked
   against CUDA's IEEE operations.  x, y, out: device pointers.  Synchronises
   the stream. */
int hydro_selftest_math(int which, const double *x, const double *y, double *out, long n,
                        void *stream);

/* Test hook, needs no GPU: drives the per-device one-time set-up guards
   that the kernel launchers use (kernel attributes such as the
   shared-memory limit, and occupancy-derived persistent grid sizes, are
   per device, so one process driving several devices must configure each)
   with a fake sequence of device ordinals devs[0..n) in [0, ndev) instead
   of real devices, walked by `threads` host threads at once.  The set-up
   for device fail_dev (-1: none) fails on its first attempt and must be
   retried.  On return once_calls[d] and value_calls[d] count the set-up
   attempts for device d of the run-once guard and of the cached-value
   guard, and values[d] holds the cached value (100 + d once computed).
   Returns HYDRO_ERR_STATE if a thread saw a wrong cached value. */
int hydro_selftest_device_once(const int *devs, int n, int fail_dev, int threads, int ndev,
                               int *once_calls, int *value_calls, int *values);

/* Throughput probe of the fused multiply-add pipe of one precision
   (HYDRO_FP64 or HYDRO_FP32), the denominator of the step kernels'
   arithmetic roofline: `ctas` CTAs of `threads` threads (a multiple of 32,
   at most 256) each run 8 independent chains x <- x * a + b for `iters`
   rounds and store their sums into `out` (device, ctas * threads values of
   the precision).  Launches on `stream` without synchronising: the caller
   times it with events.  hydro_fma_probe_flops gives the floating-point
   operations of one launch (2 per FMA). */
int hydro_fma_probe(int precision, long long iters, int ctas, int threads, void *out, void *stream);
double hydro_fma_probe_flops(long long iters, int ctas, int threads);

int hydro_destroy(hydro_sim *sim);
const char *hydro_strerror(int status);

/* ---------------------------------------------------------------------
   Batched solves.  Many independent instances of different sizes (2D and
   3D, one precision; one hydrostatic-background flag for the 3D ones) step
   together: each step is one persistent launch for the 3D instances and one
   for the 2D instances, whose CTAs claim work items (instance, tile,
   z-chunk) from a device-resident queue, largest first; the launches are
   replayed from a captured CUDA graph when the stream is not the legacy
   default stream.  Each instance keeps its own time-control block and CFL
   dt (the last item of an instance to finish sets it) and its own step
   limit, after which the kernels skip it.  Instances may join and leave
   between steps: the queue, the instance table and the item lists live in
   device memory and are rewritten by stream-ordered copies from pinned host
   staging, so membership changes need no synchronisation and no new graph
   (hydro_batch_add_async / hydro_batch_remove_async; the plain add and
   remove synchronise).  The paper motivates such suites as capacity
   computing for parameter studies and uncertainty quantification
   ("Increasing computing power", "Capabilities needed").  All device
   buffers are caller-owned, 256-byte aligned: per instance two state
   buffers (hydro_state_bytes) and one instance work buffer
   (hydro_instance_work_bytes), plus one batch work buffer
   (hydro_batch_create_bytes).  The handle keeps a pinned host staging
   buffer for the uploads. */
typedef struct hydro_batch hydro_batch;

/* Per-instance work buffer (time control, partial slots, background
   tables) and the largest number of work items the instance can produce. */
size_t hydro_instance_work_bytes(const hydro_problem *prob);
long hydro_problem_max_items(const hydro_problem *prob);

/* Batch work buffer for up to max_instances instances whose work items
   (hydro_problem_max_items summed over the 3D / the 2D instances present at
   one time) stay within max_items3d / max_items2d. */
size_t hydro_batch_create_bytes(int max_instances, long max_items3d, long max_items2d);
int hydro_batch_create(int max_instances, long max_items3d, long max_items2d, int precision, void *work,
                       void *stream, hydro_batch **out);

/* Add an instance: Ua/Ub its state buffers, inst_work its work buffer, W0
   its HOST FP64 total primitives, bg its HOST background tables (hse) or
   NULL; it stops advancing after step_end steps (< 0: never).  *id receives
   its index.  Returns HYDRO_ERR_OOM when max_instances or the item
   capacity would be exceeded, HYDRO_ERR_INVALID_ARG for a precision or 3D
   mode different from the batch's.  Synchronises. */
int hydro_batch_add(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                    const double *W0, const double *bg, long step_end, int *id);
/* hydro_batch_add without synchronisation: W0_device is a DEVICE array of
   the FP64 total primitives (nvar planes of N), which the conversion
   kernel, enqueued on the batch stream, reads; it and the host tables bg
   (copied before return) may be released once the work enqueued so far has
   run (record an event on the stream).  Errors of the initial state surface
   through the instance's control block (hydro_batch_reduce). */
int hydro_batch_add_async(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                          const double *W0_device, const double *bg, long step_end, int *id);
/* Remove an instance (synchronises; its buffers are free on return). */
int hydro_batch_remove(hydro_batch *b, int id);
/* Remove an instance without synchronisation: launches enqueued before the
   call still use its buffers, so the caller releases them only after that
   work has run (an event recorded on the stream after this call). */
int hydro_batch_remove_async(hydro_batch *b, int id);
/* Graph capture on (default) or off (direct launches). */
int hydro_batch_set_graph(hydro_batch *b, int on);

/* Convenience: one work buffer of hydro_batch_workspace_bytes holding the
   batch buffer and every instance buffer; instance i gets id i. */
size_t hydro_batch_workspace_bytes(const hydro_problem *probs, int count);
int hydro_batch_init(const hydro_problem *probs, int count, void *const *Ua, void *const *Ub,
                     void *work, const double *const *W0, const double *const *bg, void *stream,
                     hydro_batch **out);

/* Select the 3D tile shape and staging depth (variant index, see
   hydro_set_tile; variants 3 and 7 are FP32 only) and the longest z-chunk
   of an instance's column (0 = default, 64 planes; each column is cut into
   chunks of nearly equal length); rebuilds the work lists (and the graph
   when the kernel changes).  Results do not depend on this choice.
   hydro_batch_variant_shape gives a variant's tile shape (tx x ty);
   variants v and v + 4 share it. */
int hydro_batch_configure(hydro_batch *b, int variant, int zchunk);
int hydro_batch_variant_shape(int variant, int *tx, int *ty);

/* nsteps steps of every instance (no synchronisation). */
int hydro_batch_step(hydro_batch *b, long nsteps);

/* Per-instance reductions (HYDRO_RED_*) and FP64 field export (as
   hydro_reduce / hydro_get_fields); both synchronise. */
int hydro_batch_reduce(hydro_batch *b, int id, int what, double *out);
int hydro_batch_get_fields(hydro_batch *b, int id, int what, double *host_dst);
/* Raw stored state of an instance to HOST memory (synchronises); device
   pointer of the buffer holding it (synchronises). */
int hydro_batch_get_state(hydro_batch *b, int id, void *host_dst);
void *hydro_batch_current(hydro_batch *b, int id);
/* Enqueue the copy of an instance's state, as it will be once the launches
   enqueued so far have run, to host_dst (pinned host memory for a truly
   asynchronous copy); no synchronisation.  Meaningful for an instance that
   did not enter its error state. */
int hydro_batch_get_state_async(hydro_batch *b, int id, void *host_dst);

/* Kernel launches so far; work-list sizes and persistent grid sizes. */
long hydro_batch_launch_count(hydro_batch *b);
int hydro_batch_items(hydro_batch *b, int *items3d, int *items2d, int *grid3d, int *grid2d);
int hydro_batch_destroy(hydro_batch *b);

/* Conserved totals of a state without any allocation.  The paper has no
   counterpart to this call; it exists for callers that must not allocate
   device memory themselves, e.g. a host application whose memory manager has
   already reserved the device's memory for its own pool (a cudaMalloc would
   fail or fragment that pool), or a time-critical loop that cannot afford the
   device-wide synchronisation that cudaMalloc and cudaFree can cause.
   It computes the same FP64 fixed-order sums as hydro_reduce with
   HYDRO_RED_TOTALS (out[q] = sum over cells of the total conserved variable q
   times the cell volume, q < ndim + 2) for the state U (device pointer, the
   layout and precision of prob; with hse_subtract the stored perturbation,
   and bg the HOST background tables in hydro_init's order, which must be
   finite).  Its scratch is one fixed array of about 420 KB in device memory,
   part of the library image: every GPU that loads the library holds it
   until the process exits.  Limits: hse problems need nz + 5 <= 4096;
   larger ones are rejected with HYDRO_ERR_INVALID_ARG before anything is
   launched.  Every call looks up the array's device address on the current
   device, copies the background from pageable host memory and synchronises
   `stream`, so it cannot be called while a stream is being captured.  All
   calls share the one array: calls whose GPU work can overlap race and give
   wrong sums -- calls on different streams, and calls from different host
   threads even on one stream (their clears, kernels and read-backs can
   interleave).  Calls no allocating routine. */
int hydro_totals_noalloc(const hydro_problem *prob, const void *U, const double *bg,
                         void *stream, double *out);

/* ---- Domain decomposition into z slabs (virtual ranks) ----------------
   The paper's codes split the domain across nodes and exchange boundary
   data with their neighbours every step, with one global reduction for the
   time step (introduction, "Capabilities needed").  These calls cut a 3D
   problem into R slabs along z (rank r holds planes [z0, z0 + nz) with
   R's extra planes given to the lowest ranks) and advance all of them on
   the current device: every step is (1) the halo exchange, two planes of
   every variable from each neighbour (periodic z wraps; a physical z end
   keeps its boundary condition), (2) the step kernel on every slab, (3) a
   max-reduction of the slabs' CFL signal speeds giving every slab the same
   next dt.  The result is bitwise the undivided solve's.  On a machine with
   one GPU per rank, (1) becomes point-to-point copies and (3) an allreduce;
   hydro_slabs_exchange_plan gives the copy list for either.  Requires
   ndim == 3 and n[2] / R >= 2.  No time control: every step takes the CFL
   dt (t_end is not clamped). */
typedef struct hydro_slabs hydro_slabs;

/* Planes of rank `rank`: first global plane and count. */
int hydro_slab_extent(const hydro_problem *global, int nranks, int rank, int *z0, int *nz);
/* Bytes of one state buffer of rank `rank` (its nz + 4 planes, halos
   included) and of its workspace; 0 when the decomposition is invalid. */
size_t hydro_slab_state_bytes(const hydro_problem *global, int nranks, int rank);
size_t hydro_slab_workspace_bytes(const hydro_problem *global, int nranks, int rank);
/* The halo copies of one step as (src rank, src first interior plane,
   dst rank, dst first stored plane: -2 or nz) quadruples into out (up to
   max_copies; out may be NULL to count).  Each copy moves two planes of
   every variable.  Returns the number of copies or a negative status. */
int hydro_slabs_exchange_plan(const hydro_problem *global, int nranks, int *out, int max_copies);
/* Ua[r], Ub[r], work[r]: device buffers of hydro_slab_state_bytes /
   hydro_slab_workspace_bytes (256-byte aligned, caller owned, kept until
   hydro_slabs_destroy).  W0 and bg: the GLOBAL host arrays of hydro_init
   (each rank reads its own planes).  Synchronises `stream`. */
int hydro_slabs_init(const hydro_problem *global, int nranks, void *const *Ua, void *const *Ub,
                     void *const *work, const double *W0, const double *bg, void *stream,
                     hydro_slabs **out);
/* Choose the 3D tile shape and z-chunk (0: default; HYDRO_ZCHUNK_BALANCED:
   each slab's step on the balanced grid) of the slabs' steps. */
int hydro_slabs_configure(hydro_slabs *s, int variant, int zchunk);
/* Enqueue nsteps full steps (exchange, R step kernels, dt reduction each).
   The R step kernels run concurrently on internal streams forked from and
   joined back into `stream`; everything is ordered on `stream`. */
int hydro_slabs_step(hydro_slabs *s, long nsteps);
/* Gather the interior state of all slabs into one GLOBAL host array in
   hydro_get_state's layout (synchronises). */
int hydro_slabs_get_state(hydro_slabs *s, void *host_dst);
/* FP64 total conserved (what = 0) or primitive (1) fields of the whole
   domain into a GLOBAL host array, as hydro_get_fields (synchronises). */
int hydro_slabs_get_fields(hydro_slabs *s, int what, double *host_dst);
/* hydro_reduce over the whole domain (totals summed over slabs in rank
   order; scalars from rank 0, identical on all ranks). */
int hydro_slabs_reduce(hydro_slabs *s, int what, double *out);
long hydro_slabs_launch_count(hydro_slabs *s);
int hydro_slabs_destroy(hydro_slabs *s);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
