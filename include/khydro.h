/*
 * khydro.h -- C ABI of the GB300 Godunov hydrodynamics step library
 * (libkhydro.so, sm_103a).
 *
 * The library advances the Euler equations (arXiv:2501.02317, Sec. 3, Eq. 2)
 * on uniform Cartesian meshes in 1D, 2D and 3D with one explicit Godunov
 * finite-volume scheme: conserved->primitive recovery and the CFL time step
 * (Sec. 3.1), ghost zones from the physical boundary rules (Sec. 3.1.1),
 * minmod-limited piecewise-linear reconstruction (Eq. 3, Sec. 3.2.2), the
 * HLLC Riemann flux with the subtraction-safe wave speeds (Eq. 4, Eq. 5,
 * Sec. 3.2.2) and the conservative update inside the Heun predictor-corrector
 * or the memory-optimized van Leer predictor-corrector (Sec. 3.3).  Three
 * precisions: all-FP64; mixed (FP32 reconstruction and Riemann flux, FP64
 * conserved state, recovery and flux-difference accumulation; Sec. 3.2.2);
 * all-FP32.
 *
 * Conventions for every call:
 *   - Every call returns a khy_status; nothing throws across the ABI.
 *     khy_last_error() gives a thread-local message for the last failure.
 *   - State arrays are field-major [nvar][nz][ny][nx], x fastest, float64,
 *     interior cells only; nvar = 2 + ndim.  Conserved fields are
 *     (rho, m_1..m_ndim, E); primitive fields are (rho, v_1..v_ndim, p).
 *   - "count" arguments are element counts and must equal nvar * ncell,
 *     otherwise KHY_ERR_ARG.
 *   - Host pointers are owned by the caller and are only read or written
 *     during the call.  Device pointers (the *_dev calls) must point to
 *     device memory of the current CUDA device, 16-byte aligned.
 *   - A khy_sim owns its device memory (allocated in khy_create, released in
 *     khy_destroy) and runs on the CUDA stream given at creation (NULL = the
 *     library creates a private non-blocking stream).  Calls on one khy_sim
 *     must not overlap.
 *   - Device-side anomalies (a non-positive density, a negative internal
 *     energy or a NaN before the floors) latch in a device status word; the
 *     next call that synchronises returns KHY_ERR_NONPHYSICAL.  Kernels never
 *     trap.
 */
#ifndef KHYDRO_H
#define KHYDRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KHY_OK = 0,
    KHY_ERR_ARG = -1,          /* invalid argument (sizes, enums, pointers) */
    KHY_ERR_OOM = -2,          /* device allocation failed */
    KHY_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    KHY_ERR_NONPHYSICAL = -4,  /* rho <= 0, E - ke < 0 or NaN seen by the recovery */
    KHY_ERR_DT_UNDERFLOW = -5, /* the CFL step fell below 1e-300 or is not finite */
    KHY_ERR_TIMEOUT = -6,      /* a bounded wait gave up (khy_server_wait; no kernel waits on another) */
    KHY_ERR_BUDGET = -7        /* serving: the job does not fit the HBM budget */
} khy_status;

/* Precision (Sec. 3.2.2): all-FP64; mixed (FP32 reconstruction and Riemann
 * flux, FP64 conserved state); all-FP32 (FP32 state and flux: the paper's
 * "Single", conservation to FP32 round-off; single grids only). */
typedef enum { KHY_PREC_FP64 = 0, KHY_PREC_MIXED = 1, KHY_PREC_FP32 = 2 } khy_prec;

/* Physical boundary rules of Sec. 3.1.1 plus periodic wrap, per axis side. */
typedef enum {
    KHY_BC_PERIODIC = 0, /* wrap; must be set on both sides of an axis */
    KHY_BC_OUTFLOW = 1,  /* copy the first interior cell, normal velocity clamped outward */
    KHY_BC_FREE = 2,     /* copy the first interior cell */
    KHY_BC_REFLECT = 3   /* mirror the interior, normal velocity negated */
} khy_bc;

/* Time integrator (Sec. 3.3).
 *   KHY_INT_HEUN: U^1 = U^n + dt L(U^n); U^{n+1} = (U^n + (U^1 + dt L(U^1))) / 2.
 *                 A single grid also keeps the primitives of U^n and U^1 in
 *                 device memory (flux precision), so the stage kernels read
 *                 them instead of recovering every halo cell again: state
 *                 memory 120 B per 3D cell in the mixed path (160 B FP64).
 *   KHY_INT_HEUN_LEAN: the same Heun step, bit for bit, without the stored
 *                 primitives (halo cells are recovered on the fly): 80 B per
 *                 3D cell in the mixed path, slower.
 *   KHY_INT_VL2 : memory-optimized van Leer predictor-corrector: the
 *                 predictor U^{n+1/2} = U^n + (dt/2) L_1(U^n) uses first-order
 *                 (piecewise-constant) face states and only its primitives
 *                 W^{n+1/2} are kept, in the flux precision (FP32 in the mixed
 *                 path); the corrector U^{n+1} = U^n + dt L(W^{n+1/2}) uses PLM
 *                 face states of W^{n+1/2}.  The second state array (U^1, FP64)
 *                 becomes a primitive array (FP32 in the mixed and FP32 paths),
 *                 and the result is U^n plus flux differences only, so it is
 *                 conservative to round-off.  Single grids only. */
typedef enum { KHY_INT_HEUN = 0, KHY_INT_VL2 = 1, KHY_INT_HEUN_LEAN = 2 } khy_integrator;

/* Mesh and method parameters.  n[d] >= 2 for d < ndim and n[d] == 1 for
 * d >= ndim; hi[d] > lo[d]; gamma > 1; 0 < cfl <= 1; floors >= 0.  A zeroed
 * integrator field selects Heun. */
typedef struct khy_mesh_desc {
    int ndim;         /* 1, 2 or 3 */
    int n[3];         /* interior cells per axis */
    double lo[3];     /* domain lower corner */
    double hi[3];     /* domain upper corner */
    double gamma;     /* adiabatic index */
    double cfl;       /* Courant number C of dt = C min dx_d / (|v_d| + c_s) */
    int prec;         /* khy_prec */
    int bc[3][2];     /* khy_bc per axis, [0] = low side, [1] = high side */
    int integrator;   /* khy_integrator */
    double rho_floor; /* floor on the recovered density (primitive only) */
    double p_floor;   /* floor on the recovered pressure (primitive only) */
} khy_mesh_desc;

typedef struct khy_sim khy_sim;

/* ------------------------------------------------------------ single grid */

/* Validates *desc, allocates the state (U^n, and U^1 or the van Leer
 * primitives W^{n+1/2}; for KHY_INT_HEUN the primitives of U^n and U^1) and
 * the device clock on the current CUDA device, and binds the stream
 * (cudaStream_t, may be NULL).
 * On success *out receives the simulation, time t = 0, state zero.
 * A valid desc has ndim in 1..3, at least 2 cells on every active axis and
 * n = 1 on the others, at most 2^31 cells in all, finite lo < hi on every
 * active axis, gamma > 1, 0 < cfl <= 1, non-negative floors, and khy_bc,
 * khy_prec and khy_integrator values in range.
 * Errors: KHY_ERR_ARG (invalid desc), KHY_ERR_OOM, KHY_ERR_CUDA. */
khy_status khy_create(const khy_mesh_desc *desc, void *cuda_stream, khy_sim **out);

/* Releases everything khy_create allocated.  NULL is ignored. */
void khy_destroy(khy_sim *sim);

/* Sets the boundary rule of one axis side (Sec. 3.1.1); axis < ndim,
 * side 0 = low, 1 = high.  Periodic must end up on both sides of an axis or
 * neither (checked at the next step).  Allowed between steps. */
khy_status khy_set_boundary(khy_sim *sim, int axis, int side, int bc);

/* Copies conserved U (host, count = nvar*ncell doubles) to the device state. */
khy_status khy_set_conserved(khy_sim *sim, const double *U, size_t count);

/* Copies primitive W (host) and converts it on the device to conserved
 * variables: m_d = rho v_d, E = p/(gamma-1) + rho |v|^2/2 (Eq. 2). */
khy_status khy_set_primitive(khy_sim *sim, const double *W, size_t count);

/* Device-pointer variants: U_dev / W_dev is device memory with count doubles;
 * the copy is stream-ordered on the simulation's stream (no host sync). */
khy_status khy_set_conserved_dev(khy_sim *sim, const double *U_dev, size_t count);
khy_status khy_set_primitive_dev(khy_sim *sim, const double *W_dev, size_t count);

/* Sets the simulation time t. */
khy_status khy_set_time(khy_sim *sim, double t);

/* Advances by steps of the descriptor's integrator (Sec. 3.3) until t reaches
 * t_end or max_steps steps were taken (max_steps < 0: no limit).  Each step:
 * dt = C min over cells and directions of dx_d/(|v_d| + c_s) from U^n (first
 * sub-step only, Sec. 3.1), clipped so that the last step lands on t_end;
 * then the two sub-steps of khy_integrator.  The loop runs on the device in
 * captured CUDA graphs; the host polls a device flag between graph chunks.
 * steps_taken / t_out may be NULL.  Synchronises the stream. */
khy_status khy_step_to(khy_sim *sim, double t_end, long max_steps, long *steps_taken, double *t_out);

/* Enqueues exactly nsteps steps toward t_end on the stream without any
 * host synchronisation (steps past t_end are no-ops on the device).  Used for
 * timing and for overlapping several simulations. */
khy_status khy_enqueue_steps(khy_sim *sim, double t_end, long nsteps);

/* Profiling: enqueues nsteps steps toward t_end without graphs, with a
 * CUDA event pair around each launch, synchronises, and writes the average
 * duration in milliseconds of the clock launch (ms[0]), the first sub-step
 * launch (ms[1]: Heun stage 1 or van Leer predictor) and the second (ms[2]).
 * nsteps >= 1. */
khy_status khy_profile_steps(khy_sim *sim, double t_end, long nsteps, float ms[3]);

/* Copies the conserved state to host U (count doubles).  Synchronises. */
khy_status khy_get_conserved(khy_sim *sim, double *U, size_t count);

/* Stream-ordered copy of the conserved state to device memory U_dev. */
khy_status khy_get_conserved_dev(khy_sim *sim, double *U_dev, size_t count);

/* Copies the primitive state (rho, v_1..v_ndim, p) of the current conserved
 * state to host W (count = nvar*ncell doubles, field-major like U), as the
 * library recovers it for the fluxes (Sec. 3.1): floors applied to the
 * primitives, values in the flux precision (FP32 in the mixed and all-FP32
 * paths, widened to double on the host; FP64 in the all-FP64 path).  Works
 * for every integrator (the Heun step's stored primitives, otherwise a
 * recovery pass into the step's scratch buffer between steps).
 * Synchronises.  Errors: KHY_ERR_ARG (NULL, wrong count), KHY_ERR_CUDA; a
 * non-physical state is flagged as by a step (khy_get_flags). */
khy_status khy_get_primitive(khy_sim *sim, double *W, size_t count);

/* Current time, steps taken since creation and the last dt.  Synchronises. */
khy_status khy_get_time(khy_sim *sim, double *t, long *steps, double *last_dt);

/* Conservation totals (diagnostic): Neumaier-compensated sum of every
 * conserved field over the interior cells, out[0..nvar-1].  Synchronises. */
khy_status khy_totals(khy_sim *sim, double out[5]);

/* Latched device status bits (1 = non-physical state seen, 2 = a floor was
 * applied) and the number of floor applications; clears them when clear != 0. */
khy_status khy_get_flags(khy_sim *sim, unsigned *flags, unsigned long long *floor_hits, int clear);

/* Device memory held by the simulation, in bytes: *state_bytes for the state
 * arrays (U^n and U^1 or W^{n+1/2}, and the stored primitives of KHY_INT_HEUN),
 * *total_bytes including the clock and reduction buffers.  Either pointer may
 * be NULL. */
khy_status khy_device_bytes(khy_sim *sim, size_t *state_bytes, size_t *total_bytes);

/* ------------------------------------------------------------ many grids */

/* A batch: many independent grids of one dimensionality and one precision,
 * stepped together (the batched workload; also the engine of the server).
 * State arrays of a batch are the grids' field-major arrays concatenated in
 * grid order (count = sum over grids of nvar * ncell).  Every grid keeps its
 * own clock: its own CFL dt (Sec. 3.1), its own target time and step limit.
 * One batch step is one Heun step (Sec. 3.3) of every grid that has not
 * reached its target; finished grids idle.  Each grid's result is bitwise
 * equal to the same grid stepped alone with khy_step_to. */
typedef struct khy_batch khy_batch;

/* Validates every descriptor (same ndim and prec for all; KHY_PREC_FP64 or
 * KHY_PREC_MIXED; KHY_INT_HEUN or KHY_INT_HEUN_LEAN, both run as the Heun
 * step with stored primitives), allocates the pooled states (U, U^1 and their
 * primitives) and the clocks,
 * binds the stream (NULL: a private stream)
 * and builds the segment schedule for the tile variant remembered for this
 * batch shape (variant 0 if none was tuned).  Targets start at t_end = 0, so
 * nothing steps until khy_batch_set_target. */
khy_status khy_batch_create(const khy_mesh_desc *descs, int ngrids, void *cuda_stream, khy_batch **out);
void khy_batch_destroy(khy_batch *b);

/* Host copies of the whole batch state (concatenated, see above).
 * set_primitive converts on the device as khy_set_primitive does.  Sync. */
khy_status khy_batch_set_primitive(khy_batch *b, const double *W, size_t count);
khy_status khy_batch_set_conserved(khy_batch *b, const double *U, size_t count);
khy_status khy_batch_get_conserved(khy_batch *b, double *U, size_t count);

/* Target time and step limit (counted from now; < 0: none) of one grid, or
 * of every grid when grid == -1.  Stream-ordered. */
khy_status khy_batch_set_target(khy_batch *b, int grid, double t_end, long max_steps);

/* Enqueues nsteps batch steps (CUDA graph replays), no host sync. */
khy_status khy_batch_enqueue_steps(khy_batch *b, long nsteps);

/* Steps until every grid reached its target or step limit; *batch_steps
 * receives the number of batch steps enqueued.  Synchronises. */
khy_status khy_batch_run(khy_batch *b, long *batch_steps);

/* Time, steps taken and last dt of one grid.  Synchronises. */
khy_status khy_batch_get_clock(khy_batch *b, int grid, double *t, long *steps, double *dt);

/* Autotuner: times every schedule -- tile variant x CTAs per resident CTA
 * slot in {0 (queue), 1, 4, 16, 32} -- for trial_steps steps on the current state
 * (state and clocks are restored afterwards), keeps the fastest and
 * remembers it for batches of the same shape class (ndim, prec, grid count
 * and cell-weighted mean grid side, each to a power of two); new batches of
 * that class start with it.  *variant receives the tile variant (the CTAs
 * per slot: khy_batch_get_schedule).  Synchronises. */
khy_status khy_batch_autotune(khy_batch *b, int trial_steps, int *variant, float *ms_per_step);

/* Selects a schedule explicitly: tile variant (as khy_batch_set_variant)
 * and ctas_per_slot in [1, 256], the number of equal-cost pieces the tile
 * runs are cut into per resident CTA slot (default 16: more pieces than
 * slots, which the hardware balances), or 0: one persistent CTA per
 * resident slot, each taking whole tile runs (cut only where the batch has
 * too few) from a counter, longest first.  Results do not depend on the
 * schedule.  Errors: KHY_ERR_ARG. */
khy_status khy_batch_set_schedule(khy_batch *b, int variant, int ctas_per_slot);

/* Current tile variant and CTAs per resident slot (either may be NULL). */
khy_status khy_batch_get_schedule(khy_batch *b, int *variant, int *ctas_per_slot);

/* Selects a tile variant explicitly (keeping the CTAs per slot): 1D 0..1
 * (rows of 128, 256), 2D 0..4 (rows of 64, 128, 256, 124, 252), 3D 0..2
 * (32x8, 32x16, 64x8); see khy_batch_info.  Other values: KHY_ERR_ARG. */
khy_status khy_batch_set_variant(khy_batch *b, int variant);

/* Like khy_profile_steps for a batch: average ms of the clock, stage-1 and
 * stage-2 launches over nsteps un-graphed steps. */
khy_status khy_batch_profile_steps(khy_batch *b, long nsteps, float ms[3]);

/* Total cells, pooled doubles per state (every grid at a 32-element offset:
 * at least the sum of nvar*ncell), current variant, CTAs of the schedule. */
khy_status khy_batch_info(khy_batch *b, long long *cells, size_t *pool_doubles, int *variant, int *nblocks);

/* ------------------------------------------------------------ serving */

/* A server runs simulation jobs with continuous batching: jobs (2D or 3D
 * grids, mixed precision, each with its own size, initial state and target
 * time) are submitted from any thread; a server thread admits each one as
 * soon as a slot and HBM for its two states are free in the server's arena,
 * steps all admitted jobs together (one launch per stage per dimensionality,
 * the batch engine), and retires each job the moment it reaches its target
 * (result copied to the host, memory and slot freed for the next job).
 * Every job's result is bitwise equal to the same grid stepped alone. */
typedef struct khy_server khy_server;

/* Job states reported by khy_server_poll. */
enum { KHY_JOB_QUEUED = 0, KHY_JOB_ACTIVE = 1, KHY_JOB_DONE = 2, KHY_JOB_FAILED = 3 };

/* Allocates the arena (hbm_budget_bytes of device memory: U and U^1 in FP64
 * and their primitives in FP32, 24 bytes per state element), the per-slot
 * clocks (max_slots) and starts the server thread on the current device.
 * Errors: KHY_ERR_ARG, KHY_ERR_OOM. */
khy_status khy_server_create(size_t hbm_budget_bytes, int max_slots, void *cuda_stream, khy_server **out);

/* Stops the server thread (jobs still queued or running are dropped) and
 * frees everything. */
void khy_server_destroy(khy_server *s);

/* Queues a job: mesh desc (ndim 2 or 3, KHY_PREC_MIXED, a Heun integrator), primitive initial
 * state W (host, count = nvar*ncell doubles, copied), target time t_end > 0.
 * *job_id receives the job's id.  KHY_ERR_BUDGET if the job's state arrays
 * cannot fit the arena even when it is empty. */
khy_status khy_server_submit(khy_server *s, const khy_mesh_desc *desc, const double *W, size_t count, double t_end,
                             long *job_id);

/* State (KHY_JOB_*), times in seconds since khy_server_create (submitted,
 * admitted, finished) and steps taken of a job.  times may be NULL. */
khy_status khy_server_poll(khy_server *s, long job_id, int *state, double times[3], long *steps);

/* Blocks until the job finished (KHY_OK), failed (KHY_ERR_NONPHYSICAL) or
 * timeout_s seconds passed (KHY_ERR_TIMEOUT). */
khy_status khy_server_wait(khy_server *s, long job_id, double timeout_s);

/* Copies a finished job's conserved state to host U (count = nvar*ncell);
 * release != 0 forgets the job afterwards. */
khy_status khy_server_result(khy_server *s, long job_id, double *U, size_t count, int release);

/* Completed jobs, active jobs, queued jobs, cell-updates of completed jobs
 * and seconds since creation. */
khy_status khy_server_stats(khy_server *s, long *completed, int *active, int *queued,
                            unsigned long long *cell_updates, double *elapsed_s);

/* ------------------------------------------------------------ no allocation */

/* Capacity, in bytes, of the stage-1 scratch state that khy_step_noalloc
 * keeps in a file-scope device array: it steps meshes with
 * nvar * ncell * 8 <= KHY_NOALLOC_SCRATCH_BYTES (e.g. up to 1024^2 cells in
 * 2D, exactly at the limit, or 94^3 in 3D; 95^3 is refused). */
#define KHY_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* One Heun step that allocates nothing (the paper has no counterpart: this
 * is an interface for callers that cannot call cudaMalloc when they step --
 * a host program that reserves all device memory for its own pool, a
 * real-time loop that cannot take the device synchronisation cudaMalloc and
 * cudaFree may cause, or a plug-in whose host application owns every
 * allocation).
 *
 * Advances the conserved state U_dev (device memory, nvar*ncell doubles,
 * field-major, in and out) by one Heun step from time t toward t_end, exactly
 * as one step of khy_step_to: dt from the CFL condition on U_dev, clipped so
 * the step lands on t_end; no step when t >= t_end.  Writes three doubles to
 * the device buffer out_dev: the new time, the dt taken (0 if none) and the
 * status bits (1 = non-physical state seen, 2 = a floor was applied, 4 = the
 * CFL step (or the remaining t_end - t) was below 1e-300 or not finite: no
 * step was taken, the state and time are unchanged, and a caller that loops
 * until t_end must stop on this bit instead of calling again).
 * Stream-ordered on cuda_stream (may be NULL), no host synchronisation.
 *
 * Scratch: U^1 and the step clock live in one file-scope __device__ array of
 * KHY_NOALLOC_SCRATCH_BYTES + 256 bytes that every GPU which loads the library
 * holds until the process exits; no cudaMalloc, cudaFree or allocating
 * library routine is called.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: it assumes the device's primary context is not
 * destroyed and re-created meanwhile (no cudaDeviceReset while the library
 * is in use).  Every call shares the
 * array: calls whose work overlaps on the GPU (other streams or threads)
 * race.  Errors: KHY_ERR_ARG for an invalid descriptor, KHY_PREC_FP32,
 * KHY_INT_VL2, NULL pointers, NaN times, or a state larger than the scratch (the message gives
 * both sizes);
 * KHY_ERR_CUDA if a launch fails. */
khy_status khy_step_noalloc(const khy_mesh_desc *desc, double *U_dev, double t, double t_end, double *out_dev,
                            void *cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char *khy_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int khy_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KHYDRO_H */
