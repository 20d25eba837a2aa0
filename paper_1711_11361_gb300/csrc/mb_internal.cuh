// mb_internal.cuh -- device data structures and physics shared by the
// libmbcut kernels (moving-boundary cut-cell sweep, arXiv 1711.11361).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mb {

constexpr int MAXC = 4;
constexpr int NBULK = 32;              // non-physical bulk cells listed per sweep
constexpr int GEO_GC = 16;            // grid columns per geometry group (one CTA each)
constexpr double ALPHA_MIN = 1e-10;   // smaller volume fractions count as solid
// launch shape of the FP32x2 bulk kernels: bits 0-9 CTA threads (64 or 128),
// bit 10 registers budgeted for 4 resident CTAs per SM (else 5), bit 11 an
// x-sweep ring of 8 chunks (else 4)
constexpr int SHAPE_MINB4 = 1024, SHAPE_RING8 = 2048;

// cell class byte (state at the current pose A of the sweep)
constexpr uint8_t CLS_SOLID = 1;      // alpha == 0
constexpr uint8_t CLS_CUT = 2;        // touched by the body boundary, alpha > 0
constexpr uint8_t CLS_BAND = 4;       // has a band record this sweep
constexpr uint8_t CLS_TOUCH = 8;      // touched by the body boundary (any alpha)
constexpr uint8_t CLS_MOVT = 16;      // touched by an edge of a moving polygon

// band record flags
constexpr int RF_TOUCH_A = 1, RF_TOUCH_B = 2, RF_TOUCH_M = 4, RF_MOVING = 8;
constexpr int RF_FLUID_A = 16;        // takes part in this sweep's fluxes (alpha_A > 0 or flux-GCL uncovered)
constexpr int RF_FLUID_B = 32;        // alpha_B > 0
constexpr int RF_UNCOV = 64;          // alpha_A == 0, alpha_B > 0
constexpr int RF_COVER = 128;         // alpha_A > 0, alpha_B == 0
constexpr int RF_WALL = 256;          // wall data valid
constexpr int RF_USE8 = 512;          // event uses the 8-neighbourhood
constexpr int RF_BAD = 1024;          // positivity safeguard triggered
// a cell that keeps less than this fraction of its volume over a sweep seeds
// the positivity safeguard's first merge (its state is content / alpha_B)
constexpr double MIX_COLLAPSE = 0.01;
constexpr int RF_NONBR = 2048;        // event without fluid neighbour
constexpr int RF_MOV_B = 4096;        // a moving edge meets the cell at the end pose

// instance error flags
constexpr int ERR_UNSTABLE = 1, ERR_EDGE_CAP = 2, ERR_BAND_CAP = 4, ERR_NONBR = 8, ERR_STATE = 16;
constexpr int ERR_MIX_CAP = 32;     // more non-physical cells than the safeguard's lists hold
constexpr int ERR_MIX_BULK = 64;    // a merged cluster still non-physical (non-band cell)
constexpr int ERR_MIX_BAND = 128;   // a band cell still non-physical after merging
constexpr int ERR_DEFER_CAP = 256;  // the list of deferred bulk cells overflowed

struct BandRec {
    int cell;            // j*pitch + i
    int i, j;
    int flags;
    double aA, aB, aM;   // volume fractions at start, end, middle pose
    double bown;         // time-averaged aperture of the owned face along the sweep
    double d;            // average shielded distance (mid pose)
    double nx, ny;       // wall normal (unit, into the body) at the mid pose
    double wx, wy;       // wall velocity at the cell centre
    double FB[MAXC];     // boundary flux along the sweep
    double QB[MAXC];     // boundary state
    double Qp[MAXC];     // provisional state (flux-GCL uncovered cells)
    double Flo[MAXC];    // beta_lo * F2D_lo (stabilised face flux times aperture)
    double Fhi[MAXC];    // beta_hi * F2D_hi
    double C[MAXC];      // content alpha_B Q' after the update
    double C2[MAXC];     // content after covering / uncovering
    double den;          // event weight denominator
    int mix;             // safeguard cluster root (record index) or -1
    int aux;             // k_geom: moving flag of the mid pose (then 0); k_band_prep: next to an event
    float Flof[MAXC];    // Flo and Fhi rounded to FP32, for the FP32 bulk kernels' band faces
    float Fhif[MAXC];
};

// list of the cell pairs whose bulk update waits for the band fluxes (FP32
// Euler sweeps; written by the concurrent bulk pass, read by k_bulk_def_*)
struct DeferList {
    int2 *item;     // (instance, first cell of the pair | cells to store << 28)
    int *count;
    int cap;
};

struct InstDesc {
    int nx, ny, pitch, nc;
    double x0, y0, dx, dy;
    double rdx, rdy;            // 1/dx, 1/dy (candidate row and column ranges only)
    float rdxf, rdyf;           // the same in FP32
    const double *xn, *yn;      // grid-line coordinates x_0..x_nx, y_0..y_ny (device)
    int bc[4];
    int eq;
    int axisym;          // Euler in axisymmetric form: geometric source after every y sweep
    int ucov;
    double adv[2];
    double gamma, cfl;
    void *Q[3];          // state buffers (T*), plane stride pitch*ny
    uint8_t *cls;
    int *rec;
    double *alpha;       // volume fraction at the current pose (pitch layout)
    int nv, voff;        // vertices [voff, voff+nv) of the global pools
    int rotating;
    double U[2], pivot[2], a0, a1, omega;
    double wall_bound[2];
    int rec_base, rec_cap;
    int gcol_max, gcol_off;     // geometry columns reserved for this instance
    int serial_bulk;            // 1: no bulk cell is updated before the sweep's band fluxes
    int yseg;                   // rows per thread of the y sweep (tuned)
    int tile_off[2];            // first bulk tile (per direction)
    int ntiles[2];
    int tiles_x[2];             // tiles along x per direction
};

struct InstDyn {
    double t, X, Y, dt;
    double th;                  // rotation angle of the current pose
    long long step;
    int sweep_in_step;
    int err;
    unsigned long long S[2];    // max wave speeds (bits of positive doubles)
    // current sweep
    double XA, YA, XM, YM, XB, YB;
    double thA, thM, thB;
    double cA, sA, cM, sM, cB, sB;
    double Om;                  // rotation rate at the mid time
    double delta;               // translation along the sweep (world units)
    int col0, col1;
    int row0, row1;             // rows of the body's extent over the sweep's poses
    float lamf;                 // dt / h along the sweep (FP32 kernels)
    int defer_all;              // every bulk cell waits for the band fluxes (see k_pose)
    double lam;                 // dt / h along the sweep
    int band_count;
    int nbad;
    int mixed;
    long long mixed_total;      // cells merged by the safeguard in every sweep since the state was written
    int nbadlist;
    int badlist[16];            // first records flagged by the positivity check
    int nbulk;                  // non-band cells found non-physical by the bulk update
    int bulkbad[NBULK];         // their cell indices (first NBULK)
    double wall_sum[MAXC];
    // k_pose: body extent over the sweep's poses merged across its CTAs
    // (order-preserving keys of xmin, xmax, ymin, ymax; the minima stored
    // complemented), and the count of its CTAs done; both back to 0 after use
    unsigned long long bbkey[4];
    int pose_done;
    int pad3;
};

// ---------------------------------------------------------------------------
// physics (Sec. II.A equations of state and flux; Sec. II.C.5 last paragraph)
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T fdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
template <class T> __device__ __forceinline__ T tsqrt(T a) { return sqrt(a); }
template <> __device__ __forceinline__ float tsqrt<float>(float a) { return sqrtf(a); }

template <class T>
__device__ __forceinline__ T pressure(T g, const T *q) {
    return (g - T(1)) * (q[3] - T(0.5) * fdiv(q[1] * q[1] + q[2] * q[2], q[0]));
}

// physical flux along direction d
template <class T>
__device__ __forceinline__ void euler_flux(T g, int d, const T *q, T *f) {
    T rho = q[0];
    T inv = fdiv(T(1), rho);
    T un = (d == 0 ? q[1] : q[2]) * inv;
    T p = (g - T(1)) * (q[3] - T(0.5) * (q[1] * q[1] + q[2] * q[2]) * inv);
    f[0] = rho * un;
    f[1] = q[1] * un + (d == 0 ? p : T(0));
    f[2] = q[2] * un + (d == 1 ? p : T(0));
    f[3] = un * (q[3] + p);
}

// HLLC with Davis wave-speed estimates (Toro, ch. 10)
template <class T>
__device__ __forceinline__ void hllc(T g, int d, const T *qL, const T *qR, T *F) {
    const int in = d == 0 ? 1 : 2, it = 3 - in;
    T rL = qL[0], rR = qR[0];
    T iL = fdiv(T(1), rL), iR = fdiv(T(1), rR);
    T uL = qL[in] * iL, uR = qR[in] * iR;
    T pL = (g - T(1)) * (qL[3] - T(0.5) * (qL[1] * qL[1] + qL[2] * qL[2]) * iL);
    T pR = (g - T(1)) * (qR[3] - T(0.5) * (qR[1] * qR[1] + qR[2] * qR[2]) * iR);
    T cL = tsqrt(g * pL * iL), cR = tsqrt(g * pR * iR);
    T SL = fmin(uL - cL, uR - cR), SR = fmax(uL + cL, uR + cR);
    if (SL >= T(0)) { euler_flux(g, d, qL, F); return; }
    if (SR <= T(0)) { euler_flux(g, d, qR, F); return; }
    T num = pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR);
    T den = rL * (SL - uL) - rR * (SR - uR);
    T Ss = fdiv(num, den);
    const T *q = Ss >= T(0) ? qL : qR;
    T r = Ss >= T(0) ? rL : rR, iv = Ss >= T(0) ? iL : iR, u = Ss >= T(0) ? uL : uR;
    T p = Ss >= T(0) ? pL : pR, S = Ss >= T(0) ? SL : SR;
    T f[4];
    euler_flux(g, d, q, f);
    T fac = fdiv(r * (S - u), S - Ss);
    T qs[4];
    qs[0] = fac;
    qs[in] = fac * Ss;
    qs[it] = fac * (q[it] * iv);
    qs[3] = fac * (q[3] * iv + (Ss - u) * (Ss + fdiv(p, r * (S - u))));
    for (int k = 0; k < 4; ++k) F[k] = f[k] + S * (qs[k] - q[k]);
}

template <class T>
__device__ __forceinline__ T vanleer(T dm, T dp) {
    T pr = dm * dp;
    return pr > T(0) ? fdiv(T(2) * pr, dm + dp) : T(0);
}

// MUSCL-Hancock boundary extrapolation and half-step evolution of one cell
// (conserved variables, van Leer slopes; zero slope when a stencil
// neighbour is solid; first order if an evolved state is not physical).
template <class T>
__device__ __forceinline__ void evolve(int eq, T g, int d, T lam, T a0, T a1, const T *qm, const T *q0,
                                       const T *qp, bool lim, T *QL, T *QR) {
    if (eq == 1) {  // linear advection, a = velocity along d
        T a = d == 0 ? a0 : a1;
        T sl = lim ? vanleer(q0[0] - qm[0], qp[0] - q0[0]) : T(0);
        T qL = q0[0] - T(0.5) * sl, qR = q0[0] + T(0.5) * sl;
        T dfl = T(0.5) * lam * (a * qL - a * qR);
        QL[0] = qL + dfl;
        QR[0] = qR + dfl;
        return;
    }
    T qL[4], qR[4], fL[4], fR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T sl = lim ? vanleer(q0[k] - qm[k], qp[k] - q0[k]) : T(0);
        qL[k] = q0[k] - T(0.5) * sl;
        qR[k] = q0[k] + T(0.5) * sl;
    }
    euler_flux(g, d, qL, fL);
    euler_flux(g, d, qR, fR);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T dfl = T(0.5) * lam * (fL[k] - fR[k]);
        QL[k] = qL[k] + dfl;
        QR[k] = qR[k] + dfl;
    }
    bool ok = QL[0] > T(0) && QR[0] > T(0) && pressure(g, QL) > T(0) && pressure(g, QR) > T(0);
    if (!ok) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { QL[k] = q0[k]; QR[k] = q0[k]; }
    }
}

template <class T>
__device__ __forceinline__ void riemann_flux(int eq, T g, int d, T a0, T a1, const T *qL, const T *qR, T *F) {
    if (eq == 1) {
        T a = d == 0 ? a0 : a1;
        F[0] = a > T(0) ? a * qL[0] : a * qR[0];
        return;
    }
    hllc(g, d, qL, qR, F);
}

// Exact solution of the moving-wall Riemann problem (eq. riemann_wallvel):
// the ghost mirrors the normal velocity about the wall's; the contact moves
// with the wall; shock branch in closed form, rarefaction isentropic.  R is
// the arithmetic type: double on the FP64 path; the FP32-bulk path solves the
// wall problem in float (it is flux arithmetic, like the bulk fluxes).
template <class R>
__device__ __forceinline__ void wall_state(R g, const R *q, R nx, R ny, R wx, R wy, R *rs, R *ps, R *usx, R *usy) {
    R rho = q[0], u = q[1] / rho, v = q[2] / rho;
    R p = (g - R(1)) * (q[3] - R(0.5) * (q[1] * q[1] + q[2] * q[2]) / rho);
    R un = u * nx + v * ny, wn = wx * nx + wy * ny;
    R du = un - wn;
    R mu = (g - R(1)) / (g + R(1));
    R pst, rst;
    if (du > R(0)) {
        R A = R(2) / ((g + R(1)) * rho), B = mu * p;
        pst = p + du / (R(2) * A) * (du + sqrt(du * du + R(4) * A * (p + B)));
        R pr = pst / p;
        rst = rho * (pr + mu) / (mu * pr + R(1));
    } else {
        R c = sqrt(g * p / rho);
        R x = R(1) + R(0.5) * (g - R(1)) * du / c;
        if (x > R(0)) {
            pst = p * pow(x, R(2) * g / (g - R(1)));
            rst = rho * pow(pst / p, R(1) / g);
        } else {
            pst = R(0);
            rst = R(0);
        }
    }
    R fp = R(1e-12) * p;
    *ps = pst > fp ? pst : fp;
    *rs = rst > R(1e-12) * rho ? rst : R(1e-12) * rho;
    *usx = u - du * nx;
    *usy = v - du * ny;
}

// node coordinates x_i = x0 + i*dx (no contraction: geometry is bit-reproducible)
__device__ __forceinline__ double node_coord(double o, int i, double h) { return __dadd_rn(o, __dmul_rn((double)i, h)); }

// index helpers along a line: cell k of line l in direction d
__device__ __forceinline__ int cell_index(const InstDesc &I, int d, int l, int k) {
    return d == 0 ? l * I.pitch + k : k * I.pitch + l;
}

// map a position k (possibly outside [0,n)) onto a real cell for boundary
// condition bc; returns the cell position and whether the normal component
// flips (reflective)
__device__ __forceinline__ int ghost_map(int k, int n, int bclo, int bchi, bool *flip) {
    *flip = false;
    if (k >= 0 && k < n) return k;
    int bc = k < 0 ? bclo : bchi;
    if (bc == 2) { k %= n; return k < 0 ? k + n : k; }
    *flip = (bc == 1);
    int m = k < 0 ? -1 - k : 2 * n - 1 - k;
    // positions more than n cells outside (tile slack beyond a small grid)
    // are never used for a real update; keep them inside the grid
    return m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
}

// atomic max for non-negative doubles through their bit patterns
__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
    if (!(v >= 0.0)) v = 1e300;   // NaN or negative: force the smallest dt
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace mb
