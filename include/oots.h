/*
 * oots.h -- C ABI of the GB300 (sm_103a) on-the-spot photoionisation library.
 *
 * The library advances the neutral fraction of hydrogen on a uniform 3D grid
 * lit by point sources, with the explicit and implicit raytracing /
 * microphysics schemes of Mackey (2012), "Accuracy and efficiency of
 * raytracing photoionisation algorithms" (arXiv:1201.5651):
 *   A1  implicit: cells are integrated inside the raytrace and pass on a
 *       time-averaged column (Sect. 2.1, Eq. 3);
 *   A2  first-order explicit: trace, timestep, integrate (Sect. 2.2);
 *   A3  second-order explicit: trace, timestep, half step, trace on the
 *       time-centred state, full step (Sect. 2.2, Fig. 1).
 * Columns come from short characteristics traced outward from each source's
 * vertex, octant by octant (Sect. 2, Sect. 5); the per-cell rate is the
 * photon-conserving absorbed-photon rate; the cell ODE is Eq. 2 with the
 * temperature fixed and collisional ionisation off.
 *
 * Conventions
 *   - Every function returns an int status: OOTS_OK (0) or a negative error.
 *     After an error, oots_last_error(ctx) describes it (thread-local text,
 *     valid until the next call on that thread).
 *   - Arrays are x-fastest: index = X + nx*(Y + ny*Z).  Units are CGS.
 *   - "x" is the NEUTRAL fraction (1 - y of the paper).
 *   - The caller owns every host buffer.  Host copies are synchronous with
 *     respect to the calling thread (they complete before the call returns).
 *   - The library owns the device memory of a context; the *_device variants
 *     read or write caller-owned device memory on the context's stream and
 *     never keep or free the pointer.
 *   - A context is not thread-safe; use one context per thread.
 *   - Device waits are bounded: a wavefront tile that waits too long for its
 *     upstream neighbours gives up, the call returns OOTS_E_DEVICE_TIMEOUT and
 *     the context stays usable after oots_reset_error().
 */
#ifndef OOTS_H
#define OOTS_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define OOTS_OK                 0
#define OOTS_E_INVAL           -1   /* bad argument (null pointer, size, range)        */
#define OOTS_E_STATE           -2   /* call out of order (e.g. stepping without grid)  */
#define OOTS_E_NOMEM           -3   /* device or host allocation failed                */
#define OOTS_E_CUDA            -4   /* CUDA runtime error (text in oots_last_error)     */
#define OOTS_E_DEVICE_TIMEOUT  -5   /* a bounded device wait gave up                   */
#define OOTS_E_UNSUPPORTED     -6   /* valid but not supported (e.g. A1 with 2 sources) */

/* ---- enumerations ---------------------------------------------------------- */
#define OOTS_FP64       0   /* state, rates, columns in FP64                               */
#define OOTS_MIXED      1   /* FP32 state and rates, float-float (~48-bit) columns,
                               FP64 photon budget                                         */
#define OOTS_A1         1
#define OOTS_A2         2
#define OOTS_A3         3
#define OOTS_MONO       0   /* all photons at the threshold nu0                           */
#define OOTS_BLACKBODY  1   /* blackbody photon spectrum on [nu0, 40 nu0], sigma ~ nu^-3  */

typedef struct oots_ctx oots_ctx;
typedef struct oots_batch oots_batch;

/* Timestep criteria of Eq. 4 (Table 1).  A factor <= 0 switches its
 * criterion off.  K1: dt <= K1 t_rec, t_rec = 1/(alpha n) of every cell;
 * K3: dt <= K3 max(0.05, x)/|dx/dt|; K4: dt <= K4/|dx/dt| (minimum over all
 * cells).  K2 (energy) does not apply: the temperature is fixed.
 * dt_fixed > 0 overrides the criteria.  Every substep is capped at t_end - t. */
typedef struct {
    double K1, K2, K3, K4;
    double dt_fixed;
} oots_dtcrit;

/* Photon budget, summed over every substep since the last oots_reset_budget:
 * emitted = sum Q dt; absorbed = photons absorbed in the grid; ions = new
 * ions (sum n V (x_old - x_new)); recombinations = sum n V int alpha n (1-x)^2 dt.
 * absorbed = ions + recombinations holds per substep. */
typedef struct {
    double emitted, absorbed, ions, recombinations;
} oots_budget;

/* ---- context ----------------------------------------------------------------- */

/* Create a context on CUDA device `device` (0-based) with the given precision
 * (OOTS_FP64 or OOTS_MIXED).  *out receives the context; its stream is a new
 * non-blocking stream owned by the context.  Errors: E_INVAL (null out, bad
 * precision), E_CUDA (no such device). */
int oots_create(oots_ctx **out, int device, int precision);

/* Destroy a context and free its device memory.  NULL is accepted. */
int oots_destroy(oots_ctx *ctx);

/* Use a caller-owned CUDA stream (a cudaStream_t passed as void*) for all
 * later work of this context; NULL returns to the context's own stream. */
int oots_set_stream(oots_ctx *ctx, void *stream);

/* Text of the last error raised on the calling thread (never NULL). */
const char *oots_last_error(const oots_ctx *ctx);

/* Clear a sticky device error (after OOTS_E_DEVICE_TIMEOUT). */
int oots_reset_error(oots_ctx *ctx);

/* ---- grid and state ------------------------------------------------------------ */

/* Define the grid: nx*ny*nz cells of side dx_cm (> 0).  Allocates the state
 * (released by a later oots_set_grid or oots_destroy) and resets time,
 * substep count and budget; the state starts neutral (x = 1 - 1e-6) with
 * n = 1 until set.  Errors: E_INVAL (non-positive sizes), E_NOMEM. */
int oots_set_grid(oots_ctx *ctx, int nx, int ny, int nz, double dx_cm);

/* Hydrogen number density [cm^-3]: n_H (ncell doubles, host) or, if n_H is
 * NULL, the uniform value uniform_n (> 0).  Values must be > 0. */
int oots_set_density(oots_ctx *ctx, const double *n_H, double uniform_n);

/* Neutral fraction: x (ncell doubles in [0,1], host) or, if x is NULL,
 * uniform_x.  Values outside [0,1] are rejected (E_INVAL). */
int oots_set_neutral_fraction(oots_ctx *ctx, const double *x, double uniform_x);

/* Physics constants: case-B recombination coefficient alpha_B [cm^3/s],
 * threshold cross-section sigma0 [cm^2], SC weighting floor tau0 (the
 * optical-depth floor of the Mellema et al. weights; 0.6 by default), and
 * the (fixed) temperature T [K], recorded for information.
 * Defaults: 2.59e-13, 6.3e-18, 0.6, 1e4. */
int oots_set_physics(oots_ctx *ctx, double alpha_B, double sigma0, double tau0, double T);

/* ---- sources ---------------------------------------------------------------------- */

/* Add a point source at pos_cells (position in cell units from the grid
 * corner; it is moved to the nearest cell vertex, halves rounded up, clamped
 * to [0, n], Sect. 5), emitting Q ionising photons per second with spectrum
 * OOTS_MONO or OOTS_BLACKBODY (temperature T_bb [K], tables of the
 * frequency-integrated rate against column, Sect. 2).  *id (optional)
 * receives the source index.  At most 64 sources.  Errors: E_INVAL. */
int oots_add_source(oots_ctx *ctx, const double pos_cells[3], double Q, int spectrum, double T_bb, int *id);

/* Add a plane-parallel source: a source at infinity whose rays run parallel
 * to grid axis `axis` (0: x, 1: y, 2: z), along +axis (direction = +1,
 * entering through the face at index 0) or -axis (direction = -1, entering
 * through the face at index n-1), with photon flux F [photons cm^-2 s^-1]
 * across that face and spectrum OOTS_MONO or OOTS_BLACKBODY (T_bb [K]).  This
 * is the source of the slab test of Sect. 3.1.  A cell's entry column is the
 * sum of n x dx over the cells before it on its row; its rate shares the
 * photons the row loses in it over the cell volume per unit face area, dx.
 * The photon budget counts F times the face area as emitted.  Plane and point
 * sources mix freely (A1 takes a single source of either kind).  *id
 * (optional) receives the source index.  Errors: E_INVAL (axis, direction,
 * F <= 0 or not finite, spectrum, T_bb outside [1e3, 1e6], more than 64
 * sources), E_STATE (no grid). */
int oots_add_plane_source(oots_ctx *ctx, int axis, int direction, double F, int spectrum, double T_bb, int *id);

/* Remove all sources. */
int oots_clear_sources(oots_ctx *ctx);

/* ---- scheme -------------------------------------------------------------------------- */

/* Choose the scheme (OOTS_A1, OOTS_A2, OOTS_A3) and its timestep criteria.
 * A1 supports a single source (E_UNSUPPORTED otherwise, checked when
 * stepping).  crit may be NULL to keep the current criteria. */
int oots_set_scheme(oots_ctx *ctx, int scheme, const oots_dtcrit *crit);

/* Fill *out with the criteria of Table 1 ID `id` (0..12) for `scheme`, with
 * the energy criterion dropped (T fixed): explicit dt00-04 K4 = 1..1/16,
 * dt05-08 K4 = 1/2..1/16, dt09-12 K3 = 1/2..1/16; implicit dt00-04
 * K1 = 1, 0.3, 0.1, 0.03, 0.003, dt05-08 K4, dt09-12 K3. */
int oots_dtcrit_preset(int id, int scheme, oots_dtcrit *out);

/* ---- stepping -------------------------------------------------------------------------- */

/* The timestep interface (Sect. 2.1): trace the current state and return the
 * dt the criteria allow (not capped by an end time; +inf encoded as a huge
 * value if nothing limits it).  Does not change the state. */
int oots_compute_dt(oots_ctx *ctx, double *dt);

/* The microphysics interface: one substep of the scheme with timestep dt
 * (> 0), advancing time by dt. */
int oots_step(oots_ctx *ctx, double dt);

/* Advance to t_end with the scheme's criteria (substeps replayed from a
 * CUDA graph, dt kept on the device).  *t_out and *nsub_out (optional)
 * receive the final time and the number of substeps taken by this call. */
int oots_advance(oots_ctx *ctx, double t_end, double *t_out, long long *nsub_out);

/* Enqueue exactly n substeps toward t_end on the context's stream (graph
 * replays, dt kept on the device; substeps after t_end is reached do no work)
 * and return without waiting.  Pair with oots_synchronize. */
int oots_run_substeps(oots_ctx *ctx, long long n, double t_end);

/* Run one substep eagerly with a CUDA event around every kernel launch and
 * report, for each launch in order, its kind (OOTS_K_* below) and duration
 * in milliseconds.  nmax: capacity of kinds/ms; *n_out: launches reported. */
#define OOTS_K_SWEEP1    1   /* first trace (columns of x^n)             */
#define OOTS_K_RATEDT    2   /* Eq. 4 criterion, minimum over cells      */
#define OOTS_K_FINAL0    3   /* choose dt                                */
#define OOTS_K_HALF      4   /* half-step integration (A3)               */
#define OOTS_K_SWEEP2    5   /* second trace on the half-step state (A3) */
#define OOTS_K_FULL      6   /* full-step integration and photon budget  */
#define OOTS_K_FINAL1    7   /* close the substep                        */
#define OOTS_K_IMPLICIT  8   /* implicit sweep (A1)                      */
#define OOTS_K_HALF_GENERAL 9  /* half step, cells no closed form settles (one warp each) */
#define OOTS_K_FULL_GENERAL 10 /* full step, cells no closed form settles (one warp each) */
#define OOTS_K_PLANE_TRACE 11  /* columns of the plane-parallel sources (either trace) */
#define OOTS_K_PLANE_IMPLICIT 12 /* A1 row integration of a plane-parallel source */
#define OOTS_K_PACK      13  /* n x of the traced state into tile bricks (before each throughput trace) */
#define OOTS_K_RATEDT_VERIFY 14 /* several sources: re-run of the Eq. 4 pass when the step hint was too short */
int oots_profile_substep(oots_ctx *ctx, int *kinds, double *ms, int nmax, int *n_out);

/* ---- read-back --------------------------------------------------------------------------- */

/* Neutral fraction of every cell (ncell doubles; FP32 state is widened). */
int oots_get_neutral_fraction(oots_ctx *ctx, double *out);

/* Column density to the entry of every cell from source `source` at the
 * start of the last substep (its first trace), ncell doubles [cm^-2]. */
int oots_get_column_density(oots_ctx *ctx, int source, double *out);

/* Photon budget since the last reset, and reset it. */
int oots_get_budget(oots_ctx *ctx, oots_budget *out);
int oots_reset_budget(oots_ctx *ctx);

/* Current simulation time [s] and the substeps taken since oots_set_grid. */
int oots_get_time(oots_ctx *ctx, double *t, long long *nsub);

/* Set time (for restarts) without touching the state. */
int oots_set_time(oots_ctx *ctx, double t);

/* ---- caller-owned device memory --------------------------------------------------------- */

/* Copy the neutral fraction from / to caller-owned device memory on the
 * context's stream (enqueued; not synchronised).  dtype 0: float64, 1: float32
 * (converted as needed). */
int oots_set_neutral_fraction_device(oots_ctx *ctx, const void *x_dev, int dtype);
int oots_get_neutral_fraction_device(oots_ctx *ctx, void *x_dev, int dtype);

/* Block until the context's stream is idle; returns a pending device error. */
int oots_synchronize(oots_ctx *ctx);

/* ---- partitioned runs (one process per GPU) -------------------------------------------------- */

/* The paper decomposes its domain and traces each source's rays outward from
 * the source, passing columns between subdomains (Sect. 5).  Here a run over
 * several GPUs splits the work of every substep two ways: each process
 * traces only the sources whose bit is set in src_mask (bit s = source s;
 * ~0 for all), and integrates, and takes the Eq. 4 minimum over, only the
 * cells with z in [z0, z1) (z1 <= 0: to nz).  Every process keeps the whole
 * state and all columns; the caller exchanges them between the phases below
 * (a trace's columns of every source on every process's cells; the half-step
 * and full-step states of every process's cells; the minimum of the dt
 * values).  Point sources and the explicit schemes A2/A3 only.  The default
 * partition (all sources, all cells) makes the phases one substep.
 * Errors: E_INVAL (z-range), E_STATE (no grid). */
int oots_set_partition(oots_ctx *ctx, unsigned long long src_mask, int z0, int z1);

/* One phase of a substep on this context's partition, in the scheme's order:
 *   OOTS_PH_TRACE1  trace x into the first columns (the partition's sources);
 *   OOTS_PH_DT      Eq. 4 minimum over the partition's cells into *value (not
 *                   capped by an end time; 1e300 when nothing limits it); it
 *                   needs the first columns of every source on those cells;
 *   OOTS_PH_STEP1   take the step *value (> 0): A3 the half step into
 *                   x_half, A2 the whole step into x (time += *value);
 *   OOTS_PH_TRACE2  (A3) trace x_half into the second columns;
 *   OOTS_PH_FULL    (A3) the full step into x with the second columns of every
 *                   source, time += the step.
 * Each call finishes its work before it returns.  Errors: E_INVAL (phase out
 * of order for the scheme, value NULL or dt not positive), E_UNSUPPORTED (A1
 * or plane sources), E_DEVICE_TIMEOUT, E_CUDA. */
#define OOTS_PH_TRACE1  0
#define OOTS_PH_DT      1
#define OOTS_PH_STEP1   2
#define OOTS_PH_TRACE2  3
#define OOTS_PH_FULL    4
int oots_run_phase(oots_ctx *ctx, int phase, double *value);

/* Device address and size in bytes of one of the context's arrays, for
 * exchanges between processes (e.g. NCCL broadcasts into it): kind 0 the
 * state x, 1 the half-step state x_half, 2 the first columns of source
 * `source`, 3 its second columns; ncell values each, x-fastest, in the
 * context's precision (double for OOTS_FP64, float for OOTS_MIXED).  The
 * memory stays owned by the context and valid until its grid, sources or
 * partition change.  Errors: E_INVAL, E_STATE. */
int oots_array_device(oots_ctx *ctx, int kind, int source, void **ptr, unsigned long long *bytes);

/* ---- batches ------------------------------------------------------------------------------- */

/* Group n contexts (1 <= n <= 65535) of the same device and precision, each
 * with its grid, sources, scheme (A2 or A3) and criteria, so that every
 * substep of all of them runs as one persistent sweep launch and one launch
 * per per-cell pass.  The contexts stay owned by the caller and must outlive
 * the batch; they must not be stepped individually while batched.  Errors:
 * E_INVAL (arguments, n out of range, contexts that differ in device,
 * precision or fixed/adaptive dt), E_UNSUPPORTED (A1 or mixed schemes),
 * E_STATE (a context already batched). */
int oots_batch_create(oots_batch **out, oots_ctx *const *ctxs, int n);

/* Advance every context of the batch to its own end time t_end_each[i];
 * each grid keeps its own dt.  nsub_out (optional, n entries) receives the
 * substeps each context took. */
int oots_batch_advance(oots_batch *b, const double *t_end_each, long long *nsub_out);

/* Enqueue exactly n substeps of every context of the batch toward its own
 * end time t_end_each[i] (graph replays on the first context's stream; a grid
 * that reaches its end time does no further work) and return without
 * waiting.  Pair with oots_synchronize on the first context. */
int oots_batch_run_substeps(oots_batch *b, long long n, const double *t_end_each);

int oots_batch_destroy(oots_batch *b);

/* ---- tuning and diagnostics ----------------------------------------------------------------- */

/* Choose the sweep tile shape (0..6, see oots_tile_shape_info; -1 = automatic) -- the autotuner's hook. */
int oots_set_tile_shape(oots_ctx *ctx, int shape);

/* Number of tile shapes and the dimensions of one. */
int oots_tile_shape_info(int shape, int dims[3]);

/* Debug and tuning controls: key 1 = spin limit of the bounded tile waits
 * (iterations, > 0); key 2 = index of a tile that never publishes its
 * progress (-1 = none), which makes its downstream waits run out and the call
 * return OOTS_E_DEVICE_TIMEOUT without faulting the device; key 3 = planes a
 * sweep tile completes between two progress publications (1..64; 0 = the
 * default of 4); key 4 = where the sweep's tiles start: 0 (default) at
 * multiples of the tile size in global coordinates (rows of x aligned to
 * memory), 1 at the octant's origin (the octant's diagonal planes then cut
 * only the tiles on the tile diagonals); key 5 = threads per block of the
 * closed-form per-cell passes (the dt criterion, the half and full steps):
 * 128, 256, or 0 for the default (128 with several sources per grid, 256
 * with one).  OOTS_E_INVAL for an unknown key or a value out of range. */
int oots_debug_set(oots_ctx *ctx, int key, long long value);

/* ---- allocation-free trace --------------------------------------------------------------- */

/* The column-density trace of one source, for callers that cannot allocate
 * device memory: code that works inside a pre-sized memory pool or arena
 * that owns the whole device, or a host process whose allocator must not be
 * re-entered (a cudaMalloc there can fail, fragment the arena or deadlock).
 * No counterpart in the paper: it exposes the library's wavefront sweep on
 * its own.
 *
 * Inputs and outputs are caller-owned device buffers (x-fastest, ncell
 * values each): x_dev the neutral fraction, n_dev the density (NULL: the
 * uniform uniform_n), Nin_dev receives the entry column of every cell
 * [cm^-2] from a source at pos_cells (snapped to a vertex as in
 * oots_add_source).  precision: OOTS_FP64 (double buffers) or OOTS_MIXED
 * (float buffers).  The call enqueues on `stream` (NULL: the default stream)
 * and returns when the trace has finished.
 *
 * Nothing is allocated: the scratch (tile work list, published tile faces,
 * descriptors) is one 64 MiB static device array that every GPU
 * loading the library holds until the process exits.  A grid that needs more
 * tiles of 16x8x8 cells than fit in it (about 5400 in FP64, 7200 mixed, i.e.
 * roughly 5 million cells) is rejected with OOTS_E_INVAL, *status_detail
 * (optional) set to the tiles needed and the limit in oots_last_error.
 * The first call on a device sets that device up (looks up the scratch's
 * device address and opts the kernel into its shared memory); that set-up
 * is serialised across host threads, and the first call should come before
 * any stream capture.  All calls share the one scratch array and leave it
 * holding the last call's contents (the call clears what must start at
 * zero); calls that overlap on the GPU (different streams or threads at the
 * same time) race and must not be made.  The call synchronises `stream`
 * before it returns, to read the sweep's error word.
 * Returns OOTS_OK, OOTS_E_INVAL, OOTS_E_CUDA or OOTS_E_DEVICE_TIMEOUT. */
int oots_trace_noalloc(int device, int precision, int nx, int ny, int nz, double dx_cm,
                       const void *n_dev, double uniform_n, const void *x_dev, const double pos_cells[3],
                       double sigma0, double tau0, void *Nin_dev, void *stream, int *status_detail);

/* Library version string. */
const char *oots_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OOTS_H */
