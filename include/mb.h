/*
 * mb.h -- C ABI of the GB300 moving-boundary cut-cell library (libmbcut.so).
 *
 * One directional sweep of the dimensionally split, flux-stabilised
 * Cartesian cut-cell method for the 2-D compressible Euler equations (and
 * linear advection) around a moving rigid body, after Bennett, Nikiforakis &
 * Klein, arXiv 1711.11361.  A sweep is: (1) cut-cell geometry at the sweep's
 * start, middle and end poses; (2) MUSCL-Hancock + HLLC standard fluxes on
 * every face; (3) stabilised cut-cell fluxes and the moving-wall term;
 * (4) the conservative alpha*Q update with covering / uncovering; (5) the
 * CFL wave-speed reduction.
 *
 * Conventions for every entry point:
 *   - Return an mb_status; nothing aborts.  mb_last_error() gives text.
 *   - Host pointers are caller-owned and only read/written during the call.
 *   - Device memory is owned by the library (allocated in mb_*create, freed
 *     in mb_destroy).
 *   - Work is issued on the simulation's stream (default: a stream the
 *     library creates; see mb_set_stream).  Calls returning host data
 *     synchronise that stream.
 *   - States are conserved variables, SoA planes of nx*ny doubles, x fastest:
 *     Euler [rho, rho*u, rho*v, E]; advection [u].  Solid cells read as NaN.
 *   - One mb_sim holds a batch of independent instances (n >= 1) that advance
 *     together; kernels are launched once per sweep for the whole batch.
 */
#ifndef MB_H
#define MB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mb_sim mb_sim;

typedef enum {
    MB_OK = 0,
    MB_E_INVAL = -1,     /* bad argument or unsupported configuration */
    MB_E_NOMEM = -2,     /* device allocation failed */
    MB_E_CUDA = -3,      /* CUDA runtime error (see mb_last_error) */
    MB_E_UNSTABLE = -4,  /* a fluid cell became non-finite or rho/p <= 0, or
                            a covered/uncovered cell had no fluid neighbour */
    MB_E_TIMEOUT = -5,   /* reserved for a bounded device wait that gives up;
                            never returned: no kernel of this library waits
                            on another kernel or on the host */
    MB_E_STATE = -6,     /* call order (e.g. second sweep with another dt) */
    MB_E_CAPACITY = -7   /* a fixed-size device work list overflowed */
} mb_status;

enum { MB_BC_TRANSMISSIVE = 0, MB_BC_REFLECTIVE = 1, MB_BC_PERIODIC = 2 };
/* Equations.  MB_EULER_AXISYM: the Euler equations in axisymmetric form
 * about the line y = y0 (x axial, y - y0 the radius; Sec. III.E models the
 * open-ended tube this way): the planar sweeps of MB_EULER, and after every
 * y sweep the geometric source -(1/r) [rho v, rho u v, rho v^2, v (E + p)]
 * applied explicitly over the sweep's dt to every fluid cell, r at the cell
 * centre (a reading: the paper does not state how it integrates the
 * source).  Set y0 = 0 and a reflective y-low side for the axis.  It may
 * share a batch with MB_EULER instances. */
enum { MB_EULER = 0, MB_ADVECTION = 1, MB_EULER_AXISYM = 2 };
enum { MB_UNCOVER_DONOR = 0, MB_UNCOVER_FLUX_GCL = 1 };
enum { MB_FP64 = 0, MB_FP32 = 1 };

/* Uniform cell-centred grid on [x0,x1] x [y0,y1] (Sec. II.A). */
typedef struct {
    int nx, ny;                 /* cells; 8 <= nx, ny <= 16384 */
    double x0, y0, x1, y1;
    int bc[4];                  /* x-low, x-high, y-low, y-high; periodic in pairs */
    int equation;               /* MB_EULER, MB_ADVECTION or MB_EULER_AXISYM */
    double adv[2];              /* advection velocity (MB_ADVECTION) */
    double cfl;                 /* CFL number on regular cells (Sec. III) */
    int uncover_mode;           /* MB_UNCOVER_DONOR: volume-weighted donor
                                   initialisation (Sec. II.C.5, eqs.
                                   volumeWeighting..DonorCellUpdate);
                                   MB_UNCOVER_FLUX_GCL: the new cell fills
                                   through its swept apertures */
    int precision;              /* MB_FP64, or MB_FP32 bulk arithmetic with
                                   FP64 geometry and stabilisation weights */
} mb_grid;

/* Rigid body: union of simple polygons with disjoint interiors, each listed
 * counter-clockwise, vertices at t = 0 (copied at create).  Sec. II.A. */
typedef struct {
    int npoly;
    const int *poly_start;      /* npoly+1 offsets into vx/vy */
    const int *poly_moving;     /* npoly flags: 1 moves with the motion, 0 fixed */
    const double *vx, *vy;
} mb_body;

/* Prescribed motion of the moving polygons: translation U*t plus rotation
 * theta(t) = a0 + a1*sin(omega*t) about `pivot` (which translates too). */
typedef struct {
    double U[2];
    double pivot[2];
    double a0, a1, omega;
} mb_motion;

/* Create a single instance (Sec. II.A-C).  gamma: ratio of specific heats
 * (ignored for advection).  The state starts undefined: call mb_write_state. */
mb_status mb_create(const mb_grid *grid, double gamma, const mb_body *body,
                    const mb_motion *motion, mb_sim **out);

/* Create a batch of n independent instances (arrays of length n) that every
 * mb_step / mb_sweep advances together in one set of kernel launches. */
mb_status mb_batch_create(int n, const mb_grid *grids, const double *gammas,
                          const mb_body *bodies, const mb_motion *motions, mb_sim **out);

/* Free every device buffer, stream, event and cached graph of the sim
 * (waits for its work first); NULL is a no-op.  No paper counterpart. */
void mb_destroy(mb_sim *sim);

/* Text of the last error on this sim (or of the last failed create if sim is
 * NULL).  Valid until the next call on the same sim. */
const char *mb_last_error(const mb_sim *sim);

/* Run subsequent work on `stream` (a cudaStream_t, or NULL for the library's
 * own stream).  The caller keeps ownership of the stream. */
mb_status mb_set_stream(mb_sim *sim, void *stream);

/* Overlap of a sweep's bulk update with its geometry and band fluxes (FP32
 * Euler batches; on by default).  With overlap on, the cells whose update
 * needs no band data (no cell within three positions along the sweep touched
 * by the body at the sweep's start pose) are updated by a pass that runs
 * concurrently with the geometry and band-flux kernels on a second,
 * higher-priority stream; the remaining cells are listed and updated after
 * the band fluxes.  Rotating bodies and sweeps that move a body by 0.9 cells
 * or more take the second pass whole.  enable = 0: every cell waits for the
 * band fluxes.  Results are the same bits either way.  Not in the middle of a
 * step. */
mb_status mb_set_overlap(mb_sim *sim, int enable);

/* Set instance `inst`'s state (host array, nc*nx*ny doubles as above) at time
 * t with the body at its pose of time t (translation U*t).  Values in cells
 * that are solid at that pose are ignored.  Called between the two sweeps of
 * a step it abandons that step: the next sweep starts a new one. */
mb_status mb_write_state(mb_sim *sim, int inst, const double *Q, double t);

/* Copy instance `inst`'s state to host arrays.  Q: nc*nx*ny doubles (solid
 * cells NaN); alpha (optional): nx*ny volume fractions at the current pose;
 * clock (optional): {t, X, Y, step}.  Synchronises; returns the first error
 * any kernel has flagged for this instance since the last write. */
mb_status mb_read_state(mb_sim *sim, int inst, double *Q, double *alpha, double *clock);

/* mb_write_state of every instance in one call (the initial data of the
 * method's update, Sec. II): Q is an array of n host pointers, Q[k] instance
 * k's state (nc*nx*ny doubles, layout as above, caller-owned); t (optional,
 * n doubles) their times, all 0 when NULL.  Same result as n mb_write_state
 * calls.  The arrays are copied into a device buffer that holds every
 * instance's FP64 state (library-owned, allocated on the first batched call)
 * while the classification of the new poses runs beside the copies; arrays
 * in page-locked host memory (cudaHostAlloc, cudaMallocHost,
 * cudaHostRegister) copy at the full speed of the host link.  Returns
 * MB_E_INVAL (nothing written) if sim, Q or any Q[k] is NULL, MB_E_NOMEM if
 * the buffer cannot be allocated, MB_E_CUDA on a failed copy or launch.
 * Synchronises: the arrays may be reused on return. */
mb_status mb_write_states(mb_sim *sim, const double *const *Q, const double *t);

/* mb_read_state of every instance in one call: Q is an array of n host
 * pointers (caller-owned); Q[k] (NULL entries skipped) receives instance k's
 * state (nc*nx*ny doubles, solid cells NaN), clocks (optional, 4n doubles)
 * the clocks {t, X, Y, step} of each.  One conversion launch into the
 * batch's device buffer, then one copy per instance.  Synchronises; returns
 * MB_E_INVAL if sim or Q is NULL, MB_E_NOMEM / MB_E_CUDA as
 * mb_write_states, else the first error a kernel has flagged, in instance
 * order (the states are read either way). */
mb_status mb_read_states(mb_sim *sim, double *const *Q, double *clocks);

/* mb_write_states and mb_read_states with FP32 host states (nc*nx*ny floats
 * per instance, same layout): half the bytes on the host link.  On an FP32
 * batch the device state written from FP32 host values has the same bits as
 * the one written from the FP64 values they were rounded from (the device
 * rounds FP64 input to FP32 the same way), and mb_read_states_f32 returns
 * the device values exactly; on an FP64 batch the FP32 values are widened
 * on writing and rounded on reading.  Same arguments, errors, staging and
 * synchronisation as the FP64 calls. */
mb_status mb_write_states_f32(mb_sim *sim, const float *const *Q, const double *t);
mb_status mb_read_states_f32(mb_sim *sim, float *const *Q, double *clocks);

/* One time step of every instance: two sweeps, x then y on even steps and
 * y then x on odd steps (Sec. II.A, II.C.4).  dt > 0: that step for all
 * instances; dt <= 0: each instance's own CFL step (Sec. III), computed on
 * the device.  dt_used (optional, n doubles) synchronises to report them. */
mb_status mb_step(mb_sim *sim, double dt, double *dt_used);

/* One directional sweep (dir 0: x, 1: y) of every instance with time step dt
 * (> 0): the five stages of the split update along dir, Sec. II.C.4 (eqs.
 * Klein2DcompleteMovingMethod2a-b with the stabilised fluxes of eqs.
 * Klein2DtotalfluxaMethod2, Klein2shieldedFluxMethod2 and the wall term of
 * eq. Klein2DMovingResultantFluxes) and Sec. II.C.5 (covering and
 * uncovering).  Two calls make a step; the second must use the same dt
 * (MB_E_STATE otherwise).  The body moves along dir by U_dir*dt and through
 * half the step's rotation.  Asynchronous: errors flagged by the kernels are
 * reported by mb_sync / mb_read_state. */
mb_status mb_sweep(mb_sim *sim, int dir, double dt);

/* Run nsteps steps (as mb_step with the same dt rule), replaying one CUDA
 * graph per step.  Does not synchronise. */
mb_status mb_run(mb_sim *sim, int nsteps, double dt);

/* Kernel launches of one step as captured by mb_run: the kernel nodes of the
 * step graph captured last (0 before the first capture).  No paper
 * counterpart: launch accounting for callers. */
mb_status mb_graph_kernels(const mb_sim *sim, int *kernels_per_step);

/* Record the caller's CUDA event (a cudaEvent_t; NULL: none) on the sim's
 * stream between the two sweeps of every later step, so that the caller can
 * time each sweep.  The caller owns the event and keeps it alive while it is
 * set.  Drops the cached step graphs; not in the middle of a step.  No paper
 * counterpart: measurement support. */
mb_status mb_set_sweep_event(mb_sim *sim, void *event);

/* Wait for the sim's stream and report flagged errors (any instance). */
mb_status mb_sync(mb_sim *sim);

/* Sizes: number of instances, and for instance inst its nx, ny and number of
 * components (any output pointer may be NULL). */
mb_status mb_info(const mb_sim *sim, int inst, int *n_inst, int *nx, int *ny, int *nc);

/* Diagnostics of instance inst's last sweep: out[0..3] = sum over cells of the
 * wall terms (content per unit cell area, eq. Klein2DcompleteMovingMethod2a),
 * out[4] = cells merged by the positivity safeguard, out[5] = band cells. */
mb_status mb_diagnostics(mb_sim *sim, int inst, double *out);

/* Measured FP64 rate of this GPU: fused multiply-adds per second of a plain
 * kernel of independent FP64 FMA chains filling every SM (best of three
 * launches, CUDA events on `stream`, a cudaStream_t or NULL), the peak the
 * FP64 path's roofline is reported against.  Allocates a few KB of device
 * memory for the duration of the call and synchronises `stream`.  No paper
 * counterpart: measurement support. */
mb_status mb_fp64_rate(void *stream, double *fma_per_s);

/* State of instance inst at n cells (ij: n pairs i, j) between steps: out
 * receives nc planes of n doubles (solid cells NaN), in the batch's
 * precision rounded to double.  Synchronises the sim's stream; MB_E_INVAL for
 * a cell outside the grid.  No paper counterpart: probes such as the
 * pressure history of Sec. III.E. */
mb_status mb_probe(mb_sim *sim, int inst, int n, const int *ij, double *out);

/* Cells merged by the positivity safeguard (a reading; the paper has none)
 * in all sweeps of instance inst since its state was last written, counted
 * once per merge a cell takes part in.  Synchronises the sim's stream. */
mb_status mb_merge_count(mb_sim *sim, int inst, long long *cells);

/* Copy the band records (cells cut at the start or end pose) of instance
 * inst's last sweep into `out` (an array of max_records records of
 * mb_band_record_size() bytes each, library-internal layout for debugging);
 * *count receives the number of records of that sweep. */
mb_status mb_band_records(mb_sim *sim, int inst, void *out, int max_records, int *count);

/* Size in bytes of one band record as copied by mb_band_records. */
int mb_band_record_size(void);

/* Pick the bulk kernels' launch shapes for this batch by timing candidates
 * on the device (between steps; the simulation is not changed): the CTA size
 * of each sweep direction's kernel, its register budget (registers for 4 or
 * 5 resident CTAs per SM), the depth of the x sweep's row ring and the rows
 * per thread of the y sweep.  report (optional, 8 doubles): x CTA size, y CTA
 * size, y rows per thread, the best x and y kernel times in ms, the x and y
 * register budgets (resident CTAs per SM) and the x ring depth (chunks of 64
 * cells).  Later mb_batch_add calls use the chosen shapes. */
mb_status mb_autotune(mb_sim *sim, double *report);

/* Kernel timing.  enable != 0 brackets every launch of the bulk sweep kernel
 * with CUDA events on the sim's stream (mb_run then launches without graphs).
 * mb_kernel_time returns the bulk kernel's total milliseconds and launch
 * count since timing was enabled (synchronises). */
mb_status mb_enable_timing(mb_sim *sim, int enable);
mb_status mb_kernel_time(mb_sim *sim, double *total_ms, int *launches);

/* Add one instance to a batch between steps (not between the two sweeps of
 * a step); it gets the next index, with state undefined until mb_write_state.
 * It takes the batch's current sweep order (x first when the batch has taken
 * an even number of steps since its last mb_write_state of instance 0).
 * Same checks as mb_batch_create; precision and equation must be the batch's.
 * The other instances keep their device-resident state. */
mb_status mb_batch_add(mb_sim *sim, const mb_grid *grid, double gamma, const mb_body *body,
                       const mb_motion *motion, int *inst);

/* Remove instance inst between steps, releasing its device memory; the
 * instances after it move down one index. */
mb_status mb_batch_remove(mb_sim *sim, int inst);

/* Device bytes instance inst holds (its buffers and its share of the batch's
 * shared arrays); 0 for a bad index. */
size_t mb_instance_bytes(const mb_sim *sim, int inst);

/* The same figure for an instance not yet created (0 if the description is
 * invalid); allocates nothing. */
size_t mb_request_bytes(const mb_grid *grid, const mb_body *body, const mb_motion *motion);

/* ---- request loop (continuous batching; not a construct of the paper) ----
 * A server keeps one batch.  Submitted requests queue; mb_server_tick admits
 * queued requests (first come, first served) while the device-memory budget
 * and the slot limit allow, advances every admitted simulation by one CFL
 * step in the batch's shared launches, and retires those that reached their
 * step count: the final state goes to the request's Qout and the memory is
 * released for the next requests.  Admission waits for an even batch step so
 * that each simulation alternates its sweep order exactly as it would alone;
 * a request's result is therefore the same alone and in any mix. */
typedef struct mb_server mb_server;

typedef struct {
    mb_grid grid;               /* precision and equation must be the server's */
    double gamma;
    mb_body body;               /* copied at submit */
    mb_motion motion;
    const double *Q0;           /* initial state, nc*nx*ny host doubles (copied at submit) */
    double t0;                  /* time of Q0 (body posed at t0) */
    int nsteps;                 /* CFL steps to take */
    double *Qout;               /* final state, nc*nx*ny host doubles, caller-owned,
                                   written by the tick that retires the request; may be NULL */
} mb_request;

mb_status mb_server_create(int precision, int equation, double budget_bytes, int max_active, mb_server **out);
void mb_server_destroy(mb_server *srv);
const char *mb_server_last_error(const mb_server *srv);
mb_status mb_server_submit(mb_server *srv, const mb_request *req, int *id);
/* One tick (admit, step, retire).  Outputs (optional): simulations on the
 * device, requests waiting, requests finished (including failed ones). */
mb_status mb_server_tick(mb_server *srv, int *n_active, int *n_queued, int *n_done);
/* state: 0 queued, 1 running, 2 done, < 0 the mb_status it failed with;
 * info (optional, 5 doubles): submit, admit and completion times (seconds,
 * host steady clock), steps taken, device bytes held while running. */
mb_status mb_server_query(mb_server *srv, int id, int *state, double *info);
/* Text of the error a failed request ended with ("" otherwise). */
const char *mb_server_request_error(const mb_server *srv, int id);

/* Allocation-free cut-cell classification (the paper has no counterpart: it
 * exists for callers that may not allocate device memory -- code running
 * where the application forbids cudaMalloc, such as real-time loops or
 * plugins whose host framework owns all device memory).
 *
 * Computes, for the grid `grid` and the polygons of `body` posed with
 * translation (X, Y) and rotation theta about motion->pivot (moving polygons
 * only), the volume fraction of every cell into alpha_dev (nx*ny doubles,
 * x fastest) and its class byte into class_dev (nx*ny bytes: 1 solid,
 * 2 cut, 8 touched by the body boundary, 16 touched by a moving polygon).
 * Both outputs are caller-owned DEVICE arrays; the body arrays are host
 * arrays and may be reused when the call returns.  Work is queued on
 * `stream` (a cudaStream_t, NULL for the legacy default stream).
 *
 * Allocates nothing: its scratch is a fixed 0.7 MB device array inside the
 * library, held by every GPU that loads it until the process exits.  Limits:
 * at most 16384 polygon vertices, nx and ny at most 8192 (larger requests
 * return MB_E_INVAL); per grid column at most 192 polygon edges meeting the
 * column and at most 32 edges crossing each of its two grid lines (a body
 * sampled more finely than that on a coarse grid returns MB_E_CAPACITY, and
 * the outputs are then not valid).  Polygons need at least 3 vertices and
 * the domain a positive extent (MB_E_INVAL otherwise); every argument is
 * checked before the first CUDA call.  mb_noalloc_last_error() gives the
 * message of the calling host thread's last failure.
 *
 * The call blocks the host: it synchronises `stream` once its copies into
 * the scratch array are queued, and again after the kernels to read their
 * error word back.  The first call on each device looks up the scratch
 * array's device address (once, safe from several host threads) and should
 * come before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU (for example from two host threads on two streams of one
 * device) race: serialise them. */
mb_status mb_cut_cells_noalloc(const mb_grid *grid, const mb_body *body, const mb_motion *motion,
                               double X, double Y, double theta, double *alpha_dev,
                               unsigned char *class_dev, void *stream);

/* Text of the calling host thread's last error of mb_cut_cells_noalloc. */
const char *mb_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MB_H */
