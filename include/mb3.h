/* Three-dimensional moving-boundary cut-cell sweep (arXiv 1711.11361,
 * Sec. II.C.4, eqs. Klein2DcompleteMovingMethod2a-c): x, y and z sweeps of
 * the compressible Euler equations (5 conserved variables) around one
 * convex polyhedral body translating at constant velocity, in FP64 on the
 * GPU (with an FP32 option for the flow arithmetic, mb3_set_precision).
 * The same readings as the two-dimensional library (mb.h), extended
 * to three dimensions:
 *   - volume fractions, face apertures and the time-averaged apertures of a
 *     sweep's faces (the fluid fraction of the box a face sweeps through the
 *     body, eq. timeAveragedBeta) are exact for the polyhedron;
 *   - shielded distance and wall normal from the mid pose's apertures; the
 *     wall state is the exact wall Riemann problem (eq. riemann_wallvel);
 *   - covering and uncovering (Sec. II.C.5) over the face neighbours, else
 *     those sharing an edge, else a vertex; the positivity safeguard over the
 *     face neighbours, seeded also by cells keeping less than 1% of their
 *     volume over a sweep;
 *   - a step runs x, y, z on even steps and z, y, x on odd steps.
 *
 * Layout: a state is 5 planes (rho, rho u, rho v, rho w, E) of nx*ny*nz
 * doubles, x fastest, then y, then z; solid cells read NaN.  All pointers in
 * this header are HOST pointers; the caller owns them.  Calls on one mb3_sim
 * are not thread-safe; they queue work on the simulation's own stream and
 * return when it has finished (each call synchronises). */
#ifndef MB3_H
#define MB3_H

#include "mb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mb3_sim mb3_sim;

typedef struct {
    int nx, ny, nz;         /* cells per axis, each >= 1 (>= 2 unless the axis is periodic) */
    double lo[3], hi[3];    /* domain corners, hi > lo */
    int bc[6];              /* MB_BC_* of x-low, x-high, y-low, y-high, z-low, z-high;
                               periodic sides come in pairs */
} mb3_grid;

typedef struct {
    int nplane;             /* 0 (no body) .. MB3_MAX_PLANES */
    const double *normals;  /* nplane x 3 outward unit normals, body coordinates */
    const double *offsets;  /* nplane: the body is {x : n . x <= offset} */
    double bbox[6];         /* its bounding box, body coordinates: x0 x1 y0 y1 z0 z1 */
    double U[3];            /* translation velocity */
} mb3_body;

#define MB3_MAX_PLANES 32

/* A simulation on the current CUDA device; gamma > 1, 0 < cfl <= 1,
 * uncover_mode MB_UNCOVER_DONOR (the paper's) or MB_UNCOVER_FLUX_GCL.
 * Returns MB_E_INVAL for a bad argument, MB_E_NOMEM / MB_E_CUDA when device
 * memory cannot be had. */
mb_status mb3_create(const mb3_grid *grid, double gamma, double cfl, const mb3_body *body, int uncover_mode,
                     mb3_sim **out);
void mb3_destroy(mb3_sim *sim);
const char *mb3_last_error(const mb3_sim *sim);

/* state Q (layout above) at time t with the body at translation T[3];
 * solid cells become NaN */
mb_status mb3_write_state(mb3_sim *sim, const double *Q, double t, const double *T);
/* state (optional), volume fractions at the current pose (optional,
 * nx*ny*nz), clock {t, X, Y, Z, step} (optional); returns the first error
 * a kernel flagged since the last write (MB_E_UNSTABLE, MB_E_CAPACITY) */
mb_status mb3_read_state(mb3_sim *sim, double *Q, double *alpha, double *clock);

/* one sweep along d (0: x, 1: y, 2: z) with time step dt > 0; three sweeps
 * make a step and must share dt */
mb_status mb3_sweep(mb3_sim *sim, int d, double dt);
/* one step (three sweeps); dt <= 0: the CFL step on the device (Sec. III),
 * written to *dt_used (optional) */
mb_status mb3_step(mb3_sim *sim, double dt, double *dt_used);
/* the CFL step of the current state */
mb_status mb3_cfl_dt(mb3_sim *sim, double *dt);
/* the last sweep's summed wall terms (5 doubles, optional) and cells merged
 * by the safeguard (optional) */
mb_status mb3_last_sweep(mb3_sim *sim, double *wall, int *merged);
/* the flow arithmetic's precision: MB_FP64 (the default; every kernel in
 * FP64, the path the parity tests hold to the oracle) or MB_FP32 (the
 * MUSCL-Hancock evolved states, the HLLC fluxes of faces without a wall
 * part and the CFL wave speeds in FP32, from an FP32 copy of the state kept
 * beside it).  Geometry, wall states and shielded fluxes, the update of the
 * contents, covering and uncovering, the safeguard and the state stay FP64,
 * and fluxes are stored in FP64, so the update stays conservative to FP64
 * rounding.  Allocates the copy (4 bytes x 5 per cell) on first use;
 * MB_E_STATE in the middle of a step, MB_E_INVAL for another value. */
mb_status mb3_set_precision(mb3_sim *sim, int precision);
/* device time (ms) of the last sweep's face-flux kernel (MUSCL-Hancock +
 * HLLC + stabilised flux of every face along the sweep), from CUDA events
 * recorded around it on the simulation's stream */
mb_status mb3_flux_time(mb3_sim *sim, double *ms);

#ifdef __cplusplus
}
#endif

#endif
