// Three-dimensional moving-boundary cut-cell sweep (Sec. II.C.4, eqs.
// Klein2DcompleteMovingMethod2a-c) for one convex polyhedral body in
// translation, FP64.  One simulation, its own stream; per sweep a fixed
// sequence of kernels over the body's region R (the cells meeting the
// body's bounding box at the sweep's two poses, widened by two cells) and
// over all cells and faces:
//   k3_cells  volume fractions at poses A, M, B and the touch flags (R)
//   k3_faces  apertures at M of the x-, y- and z-faces, time-averaged
//             apertures of the sweep's faces (R)
//   k3_wall   flux-GCL provisional states, shielded distance, wall normal,
//             wall state and flux of the band cells (R)
//   k3_evolve MUSCL-Hancock evolved boundary states of every cell along d
//   k3_flux   HLLC + stabilised flux of every d-face
//   k3_update the conservative update alpha_B Q' of every cell
//   k3_events covering / uncovering, gathered per cell in cell order (R)
//   k3_bad / k3_mix  the positivity safeguard (one block merges in shared memory)
//   k3_final  Q = content / alpha_B, solid cells NaN, error checks
// Geometry: the volume of a box inside the body by the divergence theorem
// over the faces of box ∩ body, each face the plane's polygon clipped by all
// other half-spaces in its own plane; apertures by clipping the face
// rectangle.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mb3.h"

namespace mb3 {

constexpr int NC = 5;
constexpr int MAXP = MB3_MAX_PLANES;
static_assert(MAXP <= 32, "one plane per lane and per mask bit");
constexpr int MAXH = 6 + MAXP;          // half-spaces of a box inside the body
constexpr int MAXPV = MAXH + 4;         // polygon vertices
constexpr double ALPHA_MIN = 1e-10;
constexpr double COLLAPSE = 0.01;
constexpr int MIX_LAYERS = 8;
constexpr int SEEDCAP = 4096;           // safeguard seeds per sweep
constexpr int NODECAP = 1 << 16;        // safeguard nodes per merge

constexpr int E_UNSTABLE = 1, E_NONBR = 2, E_SEEDCAP = 4, E_NODECAP = 8;

struct Body3 {
    int np;
    double n[3 * MAXP];
    double c[MAXP];     // offsets of the posed planes
};

__host__ __device__ inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// area of {p : p = o + s e1 + t e2} clipped by the half-spaces a_m s + b_m t
// <= r_m, starting from the square [-L, L]^2 (a 2-D Sutherland-Hodgman)
// (each vertex's signed distance is evaluated once per half-plane, and a
// half-plane holding every vertex leaves the polygon as it is)
__device__ double clipped_area(const double *a, const double *b, const double *r, int nh, double L) {
    double px[MAXPV], py[MAXPV], qx[MAXPV], qy[MAXPV], s[MAXPV];
    int n = 4;
    px[0] = -L; py[0] = -L; px[1] = L; py[1] = -L; px[2] = L; py[2] = L; px[3] = -L; py[3] = L;
    for (int m = 0; m < nh && n > 0; ++m) {
        bool out = false;
        for (int k = 0; k < n; ++k) {
            s[k] = a[m] * px[k] + b[m] * py[k] - r[m];
            if (!(s[k] <= 0.0)) out = true;
        }
        if (!out) continue;
        int k2 = 0;
        for (int k = 0; k < n; ++k) {
            const int k1 = k + 1 < n ? k + 1 : 0;
            const double sa = s[k], sb = s[k1];
            const bool ina = sa <= 0.0, inb = sb <= 0.0;
            if (ina && k2 < MAXPV) { qx[k2] = px[k]; qy[k2] = py[k]; ++k2; }
            if (ina != inb && k2 < MAXPV) {
                const double t = sa / (sa - sb);
                qx[k2] = px[k] + t * (px[k1] - px[k]);
                qy[k2] = py[k] + t * (py[k1] - py[k]);
                ++k2;
            }
        }
        n = k2;
        for (int k = 0; k < n; ++k) { px[k] = qx[k]; py[k] = qy[k]; }
    }
    if (n < 3) return 0.0;
    double A = 0.0;
    for (int k = 0; k < n; ++k) {
        const int k1 = k + 1 < n ? k + 1 : 0;
        A += px[k] * py[k1] - px[k1] * py[k];
    }
    return 0.5 * A;
}

// volume of the box [lo, lo + h] inside the body; *touch: the body
// boundary cuts the box.  Coordinates relative to lo.  V = (1/3) sum over
// the faces of box ∩ body of offset x area (divergence theorem).  Called by
// all 32 lanes of a warp for the same box: lane l takes faces l, l + 32;
// the sums are reduced over the warp (every exit depends on the box only).
__device__ double box_solid_volume(const Body3 &B, const double *lo, const double *h, bool *touch) {
    const int lane = threadIdx.x & 31;
    double hn[MAXH][3], hc[MAXH];
    int nh = 0;
    for (int a = 0; a < 3; ++a) {   // the box: -x_a <= 0, x_a <= h_a
        for (int s = 0; s < 2; ++s) {
            hn[nh][0] = hn[nh][1] = hn[nh][2] = 0.0;
            hn[nh][a] = s ? 1.0 : -1.0;
            hc[nh] = s ? h[a] : 0.0;
            ++nh;
        }
    }
    const int nbox = nh;
    // the body's planes against the box, lane f taking plane f: over the
    // box's vertices v, n . v is least at v_a = h_a where n_a < 0 (else 0)
    // and greatest at v_a = h_a where n_a > 0, and the rounded sums keep
    // that order; the box lies outside plane f when its lowest vertex does,
    // and plane f cuts it when its highest vertex lies outside
    bool outside = false, cuts = false;
    if (lane < B.np) {
        const double *n = &B.n[3 * lane];
        const double c = B.c[lane] - dot3(n, lo);
        const double vl[3] = {n[0] < 0.0 ? h[0] : 0.0, n[1] < 0.0 ? h[1] : 0.0, n[2] < 0.0 ? h[2] : 0.0};
        const double vh[3] = {n[0] > 0.0 ? h[0] : 0.0, n[1] > 0.0 ? h[1] : 0.0, n[2] > 0.0 ? h[2] : 0.0};
        outside = !(dot3(n, vl) <= c);
        cuts = !outside && !(dot3(n, vh) <= c);
    }
    if (__ballot_sync(0xffffffffu, outside)) { *touch = false; return 0.0; }
    for (unsigned m = __ballot_sync(0xffffffffu, cuts); m; m &= m - 1) {   // the cutting planes in order
        const int f = __ffs(m) - 1;
        const double *n = &B.n[3 * f];
        hn[nh][0] = n[0]; hn[nh][1] = n[1]; hn[nh][2] = n[2];
        hc[nh] = B.c[f] - dot3(n, lo);
        ++nh;
    }
    const double vol = h[0] * h[1] * h[2];
    if (nh == nbox) { *touch = false; return vol; }
    // half-width of the starting square: the polygon of box ∩ plane lies
    // within |h| + |c| of the plane's origin c n
    const double L = 2.0 * sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double V = 0.0, body_area = 0.0;
    for (int f = lane; f < nh; f += 32) {
        // in-plane basis e1, e2 (e1 x e2 = n), origin o = c n
        const double *n = hn[f];
        double t[3] = {1.0, 0.0, 0.0};
        if (fabs(n[0]) > 0.9) { t[0] = 0.0; t[1] = 1.0; }
        double e1[3] = {n[1] * t[2] - n[2] * t[1], n[2] * t[0] - n[0] * t[2], n[0] * t[1] - n[1] * t[0]};
        const double l1 = sqrt(dot3(e1, e1));
        for (int q = 0; q < 3; ++q) e1[q] /= l1;
        const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
        const double o[3] = {hc[f] * n[0], hc[f] * n[1], hc[f] * n[2]};
        double a[MAXH], b[MAXH], r[MAXH];
        int m2 = 0;
        for (int m = 0; m < nh; ++m) {
            if (m == f) continue;
            a[m2] = dot3(hn[m], e1);
            b[m2] = dot3(hn[m], e2);
            r[m2] = hc[m] - dot3(hn[m], o);
            ++m2;
        }
        const double A = clipped_area(a, b, r, m2, L + fabs(hc[f]));
        V += hc[f] * A;
        if (f >= nbox) body_area += A;
    }
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_xor_sync(0xffffffffu, V, o);
        body_area += __shfl_xor_sync(0xffffffffu, body_area, o);
    }
    *touch = body_area > 0.0;
    return fmin(vol, fmax(0.0, V / 3.0));
}

// solid area of the rectangle {x_a = v} x [lb, lb + wb] x [lc, lc + wc]
// (b, c the axes after a, cyclically): the rectangle clipped by the body's
// planes, in coordinates relative to (lb, lc)
__device__ double rect_solid_area(const Body3 &B, int a, double v, double lb, double wb, double lc, double wc) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    // the planes against the rectangle's corners first: none inside one
    // plane leaves no solid, all inside one leaves that plane out
    unsigned cut = 0;
    for (int f = 0; f < B.np; ++f) {
        const double *nn = &B.n[3 * f];
        const double cc = B.c[f] - nn[a] * v - nn[b] * lb - nn[c] * lc;
        const double lo_ = (nn[b] < 0.0 ? nn[b] * wb : 0.0) + (nn[c] < 0.0 ? nn[c] * wc : 0.0) - cc;
        const double hi_ = (nn[b] > 0.0 ? nn[b] * wb : 0.0) + (nn[c] > 0.0 ? nn[c] * wc : 0.0) - cc;
        if (lo_ > 0.0) return 0.0;
        if (hi_ > 0.0) cut |= 1u << f;
    }
    double px[MAXPV], py[MAXPV], qx[MAXPV], qy[MAXPV], s[MAXPV];
    int n = 4;
    px[0] = 0.0; py[0] = 0.0; px[1] = wb; py[1] = 0.0; px[2] = wb; py[2] = wc; px[3] = 0.0; py[3] = wc;
    for (; cut && n > 0; cut &= cut - 1) {
        const int f = __ffs(cut) - 1;
        const double *nn = &B.n[3 * f];
        const double cc = B.c[f] - nn[a] * v - nn[b] * lb - nn[c] * lc;
        bool out = false;   // (as in clipped_area)
        for (int k = 0; k < n; ++k) {
            s[k] = nn[b] * px[k] + nn[c] * py[k] - cc;
            if (!(s[k] <= 0.0)) out = true;
        }
        if (!out) continue;
        int k2 = 0;
        for (int k = 0; k < n; ++k) {
            const int k1 = k + 1 < n ? k + 1 : 0;
            const double sa = s[k], sb = s[k1];
            const bool ina = sa <= 0.0, inb = sb <= 0.0;
            if (ina && k2 < MAXPV) { qx[k2] = px[k]; qy[k2] = py[k]; ++k2; }
            if (ina != inb && k2 < MAXPV) {
                const double t = sa / (sa - sb);
                qx[k2] = px[k] + t * (px[k1] - px[k]);
                qy[k2] = py[k] + t * (py[k1] - py[k]);
                ++k2;
            }
        }
        n = k2;
        for (int k = 0; k < n; ++k) { px[k] = qx[k]; py[k] = qy[k]; }
    }
    if (n < 3) return 0.0;
    double A = 0.0;
    for (int k = 0; k < n; ++k) {
        const int k1 = k + 1 < n ? k + 1 : 0;
        A += px[k] * py[k1] - px[k1] * py[k];
    }
    return fmin(wb * wc, fmax(0.0, 0.5 * A));
}

// ---------------------------------------------------------------------------
// device descriptor: the grid, the region R and the buffers
// ---------------------------------------------------------------------------
struct Desc {
    int nx, ny, nz, n;
    double lo[3], h[3];
    int bc[6];
    double gamma, U[3];
    int gcl;
    int d;                  // the sweep's direction
    double lam;             // dt / h_d
    int r0[3], rn[3];       // region R: first cell and extent per axis
    double *Q, *Qn, *C, *Cn, *F;
    double *E;              // evolved boundary states along d, 2 NC planes
    int f32;                // FP32 flux option: Qf, and E read as floats
    float *Qf;              // the state in FP32 (FP32 flux option)
    float gammaf, hlamf;    // gamma and lam / 2 in FP32 (no conversion per thread)
    double *aA, *aM, *aB;   // over R
    unsigned char *tA, *tB; // over R
    double *aP;             // alpha at the sweep's pose A over the region P
    unsigned char *tP;      // (the previous sweep's R), with its touch flags
    int p0[3], pn[3];
    double *bM[3];          // mid-pose apertures of R's faces, per axis
    double *bt;             // time-averaged apertures of R's d-faces
    unsigned char *whas;    // wall data over R
    double *wdist, *wFB, *wQB;
    unsigned char *evt;     // event type over R: 0 none, 1 covered, 2 uncovered donor, 3 covered, leaves
    unsigned *emask;        // recipients / donors (bit (dk+1)*9 + (dj+1)*3 + (di+1))
    double *easum;
    unsigned char *upd;
    int *err;
    double *wall;           // 5 summed wall terms
    int *seeds, *nseed;
    int *lab, *par_;        // full grid, -1 where no node (safeguard)
    int *nodes;
    double *ntot;           // (NC + 1) per node
    int *mixed;
    double *smax;           // 3 wave speed maxima (CFL)
};

__device__ __forceinline__ int cidx(const Desc &D, int i, int j, int k) { return (k * D.ny + j) * D.nx + i; }
__device__ __forceinline__ bool in_r(const Desc &D, int i, int j, int k) {
    return i >= D.r0[0] && i < D.r0[0] + D.rn[0] && j >= D.r0[1] && j < D.r0[1] + D.rn[1] && k >= D.r0[2] &&
           k < D.r0[2] + D.rn[2];
}
__device__ __forceinline__ int ridx(const Desc &D, int i, int j, int k) {
    return ((k - D.r0[2]) * D.rn[1] + (j - D.r0[1])) * D.rn[0] + (i - D.r0[0]);
}
// the low a-face of cell (i, j, k) in R's face array of axis a (the cell's
// index along a may be r0 + rn: the high face of R's last cell)
__device__ __forceinline__ bool in_rf(const Desc &D, int a, int i, int j, int k) {
    const int ijk[3] = {i, j, k};
    for (int q = 0; q < 3; ++q) {
        const int hi = D.r0[q] + D.rn[q] + (q == a ? 1 : 0);
        if (ijk[q] < D.r0[q] || ijk[q] >= hi) return false;
    }
    return true;
}
__device__ __forceinline__ int rfidx(const Desc &D, int a, int i, int j, int k) {
    const int m0 = D.rn[0] + (a == 0), m1 = D.rn[1] + (a == 1);
    return ((k - D.r0[2]) * m1 + (j - D.r0[1])) * m0 + (i - D.r0[0]);
}
__device__ __forceinline__ double alphaA(const Desc &D, int i, int j, int k) {
    return in_r(D, i, j, k) ? D.aA[ridx(D, i, j, k)] : 1.0;
}
__device__ __forceinline__ double alphaB(const Desc &D, int i, int j, int k) {
    return in_r(D, i, j, k) ? D.aB[ridx(D, i, j, k)] : 1.0;
}
__device__ __forceinline__ double swept(const Desc &D, int i, int j, int k) {
    return in_rf(D, D.d, i, j, k) ? D.bt[rfidx(D, D.d, i, j, k)] : 1.0;
}
// (outside R without a floating-point test: alpha_A = 1 there)
__device__ __forceinline__ bool fluid_a(const Desc &D, int i, int j, int k) {
    if (!in_r(D, i, j, k)) return true;
    const int r = ridx(D, i, j, k);
    const double a = D.aA[r];
    return a > 0.0 || (D.gcl && a == 0.0 && D.aB[r] > 0.0);
}
// float to double exactly by moving the bit fields: integer work, off
// GB300's narrow FP64 pipe, which takes conversions too.  Normal numbers
// rebias the exponent (127 -> 1023); a subnormal m 2^-149 is normalised
// at its highest set bit p; infinities and NaN keep an all-ones exponent
// and the shifted payload
__device__ __forceinline__ double widen(float x) {
    const unsigned u = __float_as_uint(x), e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const unsigned long long s = (unsigned long long)(u >> 31) << 63;
    unsigned long long b;
    if (e == 0u) {
        if (m == 0u) {
            b = s;
        } else {
            const int p = 31 - __clz((int)m);
            b = s | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffULL);
        }
    } else if (e == 0xffu) {
        b = s | (0x7ffULL << 52) | ((unsigned long long)m << 29);
    } else {
        b = s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    }
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double node(const Desc &D, int a, int i) { return D.lo[a] + (double)i * D.h[a]; }
// x is neither infinite nor NaN: its exponent field is not all ones (an
// integer test, off GB300's narrow FP64 pipe)
__device__ __forceinline__ bool finite64(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// the state content / alpha_B is physical iff the content is (alpha_B > 0):
// rho > 0 and 2 rho E > |m|^2, no division
__device__ __forceinline__ bool content_bad(const double *q) {
    bool bad = false;
    for (int m = 0; m < NC; ++m) if (!finite64(q[m])) bad = true;   // alpha_B >= 1e-10: the quotient is finite with it
    return bad || !(q[0] > 0.0) || !(2.0 * q[0] * q[4] > q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}
__device__ __forceinline__ void add_seed(const Desc &D, int c) {
    const int s = atomicAdd(D.nseed, 1);
    if (s < SEEDCAP) D.seeds[s] = c;
    else atomicOr(D.err, E_SEEDCAP);
}
// neighbour (i+di, j+dj, k+dk) under the periodic sides, -1 outside
__device__ __forceinline__ int nbr(const Desc &D, int i, int j, int k, int di, int dj, int dk, int *ii, int *jj,
                                   int *kk) {
    int a = i + di, b = j + dj, c = k + dk;
    if (D.bc[0] == MB_BC_PERIODIC) { a %= D.nx; if (a < 0) a += D.nx; }
    if (D.bc[2] == MB_BC_PERIODIC) { b %= D.ny; if (b < 0) b += D.ny; }
    if (D.bc[4] == MB_BC_PERIODIC) { c %= D.nz; if (c < 0) c += D.nz; }
    if (a < 0 || a >= D.nx || b < 0 || b >= D.ny || c < 0 || c >= D.nz) return -1;
    *ii = a; *jj = b; *kk = c;
    return cidx(D, a, b, c);
}

__device__ __forceinline__ void r_cell(const Desc &D, int t, int *i, int *j, int *k) {
    *i = D.r0[0] + t % D.rn[0];
    *j = D.r0[1] + (t / D.rn[0]) % D.rn[1];
    *k = D.r0[2] + t / (D.rn[0] * D.rn[1]);
}

// the item of a warp-per-item kernel: item v * gridDim.x + b for warp v of
// block b, so that neighbouring items (cut cells cluster along the body's
// surface) land on different blocks, and so on different SMs
__device__ __forceinline__ int warp_item() { return (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x; }

// volume fractions at the three poses and the touch flags of R's cells,
// one warp per cell and pose (pose B first, then M, then A, so that a
// costly cell's poses run side by side).  CELLS_ALL: poses A, M and B;
// CELLS_REUSE_A: pose A is the previous sweep's pose B, whose values P
// holds (a cell outside P lies two cells or more from the body's bounding
// box: alpha 1, no touch, as computing it gives), copied by the pose-B
// warp; CELLS_ONE: pose B only, into all three
enum { CELLS_ALL = 0, CELLS_REUSE_A = 1, CELLS_ONE = 2 };
__device__ __forceinline__ double fraction(double V, double vol) {
    const double a = fmin(1.0, fmax(0.0, 1.0 - V / vol));
    return a < ALPHA_MIN ? 0.0 : a;
}
__global__ void k3_cells(Desc D, Body3 BA, Body3 BM, Body3 BB, int mode) {
    const int rc = D.rn[0] * D.rn[1] * D.rn[2];
    const int w = warp_item();
    const int npose = mode == CELLS_ALL ? 3 : mode == CELLS_REUSE_A ? 2 : 1;
    if (w >= npose * rc) return;
    const int t = w % rc, pose = w / rc;   // 0: B, 1: M, 2: A
    int i, j, k;
    r_cell(D, t, &i, &j, &k);
    const double lo[3] = {node(D, 0, i), node(D, 1, j), node(D, 2, k)};
    const double hi[3] = {node(D, 0, i + 1), node(D, 1, j + 1), node(D, 2, k + 1)};
    const double h[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    const double vol = h[0] * h[1] * h[2];
    bool touch;
    const double a = fraction(box_solid_volume(pose == 0 ? BB : pose == 1 ? BM : BA, lo, h, &touch), vol);
    if ((threadIdx.x & 31) != 0) return;
    if (pose == 0) {
        D.aB[t] = a;
        D.tB[t] = touch;
        if (mode == CELLS_ONE) {
            D.aM[t] = a;
            D.aA[t] = a;
            D.tA[t] = touch;
        } else if (mode == CELLS_REUSE_A) {
            const bool inP = i >= D.p0[0] && i < D.p0[0] + D.pn[0] && j >= D.p0[1] && j < D.p0[1] + D.pn[1] &&
                             k >= D.p0[2] && k < D.p0[2] + D.pn[2];
            const int q = inP ? ((k - D.p0[2]) * D.pn[1] + (j - D.p0[1])) * D.pn[0] + (i - D.p0[0]) : 0;
            D.aA[t] = inP ? D.aP[q] : 1.0;
            D.tA[t] = inP ? D.tP[q] : 0;
        }
    } else if (pose == 1) {
        D.aM[t] = a;
    } else {
        D.aA[t] = a;
        D.tA[t] = touch;
    }
}

// apertures at M of R's x-, y- and z-faces, then the time-averaged
// apertures of R's d-faces (the fluid fraction of [x_f - delta, x_f] with
// the body at A), one face per thread over the four index ranges
__global__ void k3_faces(Desc D, Body3 BM, Body3 BA, double delta) {
    int t = warp_item() * 32 + (int)(threadIdx.x & 31);   // whole warps spread over blocks
    for (int a = 0; a < 4; ++a) {
        const int ax = a < 3 ? a : D.d;
        const int m0 = D.rn[0] + (ax == 0), m1 = D.rn[1] + (ax == 1), m2 = D.rn[2] + (ax == 2);
        const int cnt = m0 * m1 * m2;
        if (t >= cnt) { t -= cnt; continue; }
        const int ijk[3] = {D.r0[0] + t % m0, D.r0[1] + (t / m0) % m1, D.r0[2] + t / (m0 * m1)};
        const int b = (ax + 1) % 3, c = (ax + 2) % 3;
        if (a < 3) {
            const double lb = node(D, b, ijk[b]), wb = node(D, b, ijk[b] + 1) - lb;
            const double lc = node(D, c, ijk[c]), wc = node(D, c, ijk[c] + 1) - lc;
            const double A = rect_solid_area(BM, ax, node(D, ax, ijk[ax]), lb, wb, lc, wc);
            D.bM[ax][t] = fmin(1.0, fmax(0.0, 1.0 - A / (wb * wc)));
        } else if (delta == 0.0) {
            const double lb = node(D, b, ijk[b]), wb = node(D, b, ijk[b] + 1) - lb;
            const double lc = node(D, c, ijk[c]), wc = node(D, c, ijk[c] + 1) - lc;
            const double A = rect_solid_area(BA, ax, node(D, ax, ijk[ax]), lb, wb, lc, wc);
            D.bt[t] = fmin(1.0, fmax(0.0, 1.0 - A / (wb * wc)));
        }
        return;
    }
}

// time-averaged apertures of R's d-faces for delta != 0: the fluid fraction
// of [x_f - delta, x_f] with the body at A, one warp per face
__global__ void k3_swept(Desc D, Body3 BA, double delta) {
    const int t = warp_item();
    const int ax = D.d;
    const int m0 = D.rn[0] + (ax == 0), m1 = D.rn[1] + (ax == 1), m2 = D.rn[2] + (ax == 2);
    if (t >= m0 * m1 * m2) return;
    const int ijk[3] = {D.r0[0] + t % m0, D.r0[1] + (t / m0) % m1, D.r0[2] + t / (m0 * m1)};
    double lo[3], h[3];
    for (int q = 0; q < 3; ++q) { lo[q] = node(D, q, ijk[q]); h[q] = node(D, q, ijk[q] + 1) - lo[q]; }
    const double xf = node(D, ax, ijk[ax]);
    const double s0 = delta > 0.0 ? xf - delta : xf, s1 = delta > 0.0 ? xf : xf - delta;
    lo[ax] = s0;
    h[ax] = s1 - s0;
    bool tch;
    const double V = box_solid_volume(BA, lo, h, &tch);
    if ((threadIdx.x & 31) == 0) D.bt[t] = fmin(1.0, fmax(0.0, 1.0 - V / (h[0] * h[1] * h[2])));
}

// exact wall Riemann problem (eq. riemann_wallvel), normal n into the body
__device__ void wall_state3(double g, const double *q, const double *n, const double *w, double *rs, double *ps,
                            double *us) {
    const double rho = q[0];
    const double u[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
    const double p = (g - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / rho);
    const double du = (u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) - (w[0] * n[0] + w[1] * n[1] + w[2] * n[2]);
    const double mu = (g - 1.0) / (g + 1.0);
    double pst, rst;
    if (du > 0.0) {
        const double A = 2.0 / ((g + 1.0) * rho), Bc = mu * p;
        pst = p + du / (2.0 * A) * (du + sqrt(du * du + 4.0 * A * (p + Bc)));
        const double pr = pst / p;
        rst = rho * (pr + mu) / (mu * pr + 1.0);
    } else {
        const double c = sqrt(g * p / rho);
        const double x = 1.0 + 0.5 * (g - 1.0) * du / c;
        if (x > 0.0) {
            pst = p * pow(x, 2.0 * g / (g - 1.0));
            rst = rho * pow(pst / p, 1.0 / g);
        } else {
            pst = 0.0;
            rst = 0.0;
        }
    }
    *ps = pst > 1e-12 * p ? pst : 1e-12 * p;
    *rs = rst > 1e-12 * rho ? rst : 1e-12 * rho;
    for (int m = 0; m < 3; ++m) us[m] = u[m] - du * n[m];
}

// flux-GCL provisional states of uncovered cells (in place in Q), then the
// wall data of R's band cells (Sec. II.B, II.C.3, II.C.4)
__global__ void k3_wall(Desc D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.rn[0] * D.rn[1] * D.rn[2]) return;
    int i, j, k;
    r_cell(D, t, &i, &j, &k);
    const int c = cidx(D, i, j, k);
    const double aA = D.aA[t], aB = D.aB[t];
    if (D.gcl && aA == 0.0 && aB > 0.0) {
        double acc[NC] = {0, 0, 0, 0, 0}, wsum = 0.0;
        for (int pass = 0; pass < 3 && wsum == 0.0; ++pass)
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int nzc = (di != 0) + (dj != 0) + (dk != 0);
                        if (nzc == 0 || nzc > pass + 1) continue;
                        int ii, jj, kk;
                        const int cc = nbr(D, i, j, k, di, dj, dk, &ii, &jj, &kk);
                        if (cc < 0) continue;
                        const double w = alphaA(D, ii, jj, kk);
                        if (!(w > 0.0)) continue;
                        wsum += w;
                        for (int q = 0; q < NC; ++q) acc[q] += w * D.Q[(size_t)q * D.n + cc];
                    }
        if (wsum == 0.0) atomicOr(D.err, E_NONBR);
        else for (int q = 0; q < NC; ++q) {
            D.Q[(size_t)q * D.n + c] = acc[q] / wsum;
            if (D.f32) D.Qf[(size_t)q * D.n + c] = float(acc[q] / wsum);
        }
    }
    const bool fl = aA > 0.0 || (D.gcl && aA == 0.0 && aB > 0.0);
    D.whas[t] = 0;
    if (!fl || !(D.tA[t] || D.tB[t])) return;
    const int d = D.d;
    int hi[3] = {i, j, k};
    hi[d] += 1;
    const double blo = D.bM[d][rfidx(D, d, i, j, k)], bhi = D.bM[d][rfidx(D, d, hi[0], hi[1], hi[2])];
    const double db = fabs(blo - bhi);
    const double ahat = D.aM[t] - fmin(blo, bhi);
    D.wdist[t] = db > 1e-12 ? fmin(1.0, fmax(0.0, ahat / db)) : 1.0;
    double nL[3];
    for (int a = 0; a < 3; ++a) {
        int up[3] = {i, j, k};
        up[a] += 1;
        const double bl = D.bM[a][rfidx(D, a, i, j, k)], bu = D.bM[a][rfidx(D, a, up[0], up[1], up[2])];
        nL[a] = (bl - bu) * D.h[(a + 1) % 3] * D.h[(a + 2) % 3];
    }
    const double L = sqrt(nL[0] * nL[0] + nL[1] * nL[1] + nL[2] * nL[2]);
    double nn[3];
    for (int a = 0; a < 3; ++a) nn[a] = L > 0.0 ? nL[a] / L : 0.0;
    double qc[NC], qn[NC];
    const bool fresh = isnan(D.Qn[c]);
    for (int q = 0; q < NC; ++q) {
        qc[q] = D.Q[(size_t)q * D.n + c];
        qn[q] = fresh ? qc[q] : D.Qn[(size_t)q * D.n + c];
    }
    const double g = D.gamma;
    double rs, ps_step, us[3], rs2, ps_sw, us2[3];
    wall_state3(g, qn, nn, D.U, &rs, &ps_step, us);
    wall_state3(g, qc, nn, D.U, &rs2, &ps_sw, us2);
    const double Eadv = ps_step / (g - 1.0) + 0.5 * rs * (us[0] * us[0] + us[1] * us[1] + us[2] * us[2]);
    const double ud = us[d];
    double *FB = &D.wFB[(size_t)NC * t], *QB = &D.wQB[(size_t)NC * t];
    QB[0] = rs;
    for (int m = 0; m < 3; ++m) QB[1 + m] = rs * us[m];
    QB[4] = Eadv;
    FB[0] = rs * ud;
    for (int m = 0; m < 3; ++m) FB[1 + m] = rs * ud * us[m] + (m == d ? ps_sw : 0.0);
    FB[4] = ud * (Eadv + ps_step);
    D.whas[t] = 1;
}

// ---------------------------------------------------------------------------
// fluxes, update, events, safeguard, new states
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pressure5(double g, const double *q) {
    return (g - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}
// (GB300's FP64 pipe is narrow: each quotient costs a Newton sequence, so
// the kernels share one reciprocal of rho where they can.  The flow
// arithmetic below takes its type T as a template argument: double for the
// FP64 path, float for the FP32 flux option; every literal is a T, so the
// float instances stay in float and the double ones are the FP64 path's
// arithmetic unchanged)
// a b + c with one rounding (the file is built without contraction, so
// the flow arithmetic fuses where it says so)
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <typename T> __device__ __forceinline__ T sq3(const T *m) { return fmad(m[0], m[0], fmad(m[1], m[1], m[2] * m[2])); }
// the physical flux along d of a state with 1/rho given
template <typename T>
__device__ __forceinline__ void flux5(T g, int d, const T *q, T ir, T *f) {
    const T rho = q[0], un = q[1 + d] * ir;
    const T p = (g - T(1)) * fmad(T(-0.5) * sq3(q + 1), ir, q[4]);
    f[0] = rho * un;
    for (int m = 0; m < 3; ++m) f[1 + m] = m == d ? fmad(q[1 + m], un, p) : q[1 + m] * un;
    f[4] = un * (q[4] + p);
}
// HLLC, Davis wave speeds (Toro, Riemann Solvers ch. 10)
template <typename T>
__device__ __forceinline__ void hllc5(T g, int d, const T *qL, const T *qR, T *F) {
    const int in = 1 + d;
    // 1/rho of both states from one reciprocal of their product
    const T rL = qL[0], rR = qR[0], rr2 = T(1) / (rL * rR), iL = rR * rr2, iR = rL * rr2;
    const T uL = qL[in] * iL, uR = qR[in] * iR;
    const T pL = (g - T(1)) * fmad(T(-0.5) * sq3(qL + 1), iL, qL[4]);
    const T pR = (g - T(1)) * fmad(T(-0.5) * sq3(qR + 1), iR, qR[4]);
    const T cL = sqrt(g * pL * iL), cR = sqrt(g * pR * iR);
    const T SL = fmin(uL - cL, uR - cR), SR = fmax(uL + cL, uR + cR);
    if (SL >= T(0)) { flux5(g, d, qL, iL, F); return; }
    if (SR <= T(0)) { flux5(g, d, qR, iR, F); return; }
    const T num = fmad(-(rR * uR), SR - uR, fmad(rL * uL, SL - uL, pR - pL));
    const T den = fmad(rL, SL - uL, -(rR * (SR - uR)));
    const T Ss = num / den;
    const bool left = Ss >= T(0);
    const T *q = left ? qL : qR;
    const T r = left ? rL : rR, ir = left ? iL : iR, u = left ? uL : uR, p = left ? pL : pR;
    const T S = left ? SL : SR;
    T f[NC], qs[NC];
    f[0] = r * u;
    for (int m = 0; m < 3; ++m) f[1 + m] = m == d ? fmad(q[1 + m], u, p) : q[1 + m] * u;
    f[4] = u * (q[4] + p);
    // fac = a / dS and p / a with a = rho (S - u), dS = S - S*, from one
    // reciprocal of a dS
    const T a = r * (S - u), dS = S - Ss, rr = T(1) / (a * dS);
    const T fac = a * a * rr;
    qs[0] = fac;
    for (int m = 0; m < 3; ++m) qs[1 + m] = m == d ? fac * Ss : fac * (q[1 + m] * ir);
    qs[4] = fac * fmad(q[4], ir, (Ss - u) * fmad(p * dS, rr, Ss));
    for (int k = 0; k < NC; ++k) F[k] = fmad(S, qs[k] - q[k], f[k]);
}
template <typename T>
__device__ __forceinline__ T vanleer(T dm, T dp) {
    const T pr = dm * dp;
    return pr > T(0) ? T(2) * pr / (dm + dp) : T(0);
}
// gamma and lam / 2 in the type T
template <typename T> __device__ __forceinline__ T gam(const Desc &D);
template <> __device__ __forceinline__ double gam<double>(const Desc &D) { return D.gamma; }
template <> __device__ __forceinline__ float gam<float>(const Desc &D) { return D.gammaf; }
template <typename T> __device__ __forceinline__ T halflam(const Desc &D);
template <> __device__ __forceinline__ double halflam<double>(const Desc &D) { return 0.5 * D.lam; }
template <> __device__ __forceinline__ float halflam<float>(const Desc &D) { return D.hlamf; }
// the state and evolved-state arrays of the type T
template <typename T> __device__ __forceinline__ const T *qsrc(const Desc &D);
template <> __device__ __forceinline__ const double *qsrc<double>(const Desc &D) { return D.Q; }
template <> __device__ __forceinline__ const float *qsrc<float>(const Desc &D) { return D.Qf; }
template <typename T> __device__ __forceinline__ T *esrc(const Desc &D);
template <> __device__ __forceinline__ double *esrc<double>(const Desc &D) { return D.E; }
template <> __device__ __forceinline__ float *esrc<float>(const Desc &D) { return reinterpret_cast<float *>(D.E); }

// the cell at position m along d of the line through (i, j, k) (the
// coordinate along d replaced), with the boundary conditions' ghosts:
// returns its cell index, *flip for a reflective mirror
__device__ __forceinline__ int line_cell(const Desc &D, int d, const int *base, int m, int nal, bool *flip, int *pos) {
    const int bc = D.bc[m < 0 ? 2 * d : 2 * d + 1];
    int mm = m;
    *flip = false;
    if (m < 0 || m >= nal) {
        if (bc == MB_BC_PERIODIC) { mm %= nal; if (mm < 0) mm += nal; }
        else { mm = m < 0 ? -1 - m : 2 * nal - 1 - m; *flip = bc == MB_BC_REFLECTIVE; }
    }
    int ijk[3] = {base[0], base[1], base[2]};
    ijk[d] = mm;
    pos[0] = ijk[0]; pos[1] = ijk[1]; pos[2] = ijk[2];
    return cidx(D, ijk[0], ijk[1], ijk[2]);
}

// MUSCL-Hancock evolved boundary states QL, QR of the cell at position m
// along the line (conserved variables, van Leer, zero slope next to a solid
// cell, first order where an evolved state is not physical)
template <typename T>
__device__ __forceinline__ void evolve5(const Desc &D, int d, const int *base, int m, int nal, T *QL, T *QR) {
    const T *Q = qsrc<T>(D);
    T q[3][NC];
    bool fl[3];
    for (int s = 0; s < 3; ++s) {
        bool flip;
        int pos[3];
        const int c = line_cell(D, d, base, m - 1 + s, nal, &flip, pos);
        fl[s] = fluid_a(D, pos[0], pos[1], pos[2]);
        for (int k = 0; k < NC; ++k) q[s][k] = Q[(size_t)k * D.n + c];
        if (flip) q[s][1 + d] = -q[s][1 + d];
    }
    const bool lim = fl[0] && fl[2];
    const T g = gam<T>(D), hl = halflam<T>(D);
    T qL[NC], qR[NC], fL[NC], fR[NC];
    for (int k = 0; k < NC; ++k) {
        const T sl = lim ? vanleer(q[1][k] - q[0][k], q[2][k] - q[1][k]) : T(0);
        qL[k] = fmad(T(-0.5), sl, q[1][k]);
        qR[k] = fmad(T(0.5), sl, q[1][k]);
    }
    const T rr2 = T(1) / (qL[0] * qR[0]);   // 1/rho of both extrapolated states
    flux5(g, d, qL, qR[0] * rr2, fL);
    flux5(g, d, qR, qL[0] * rr2, fR);
    for (int k = 0; k < NC; ++k) {
        const T df = fL[k] - fR[k];
        QL[k] = fmad(hl, df, qL[k]);
        QR[k] = fmad(hl, df, qR[k]);
    }
    // physical: rho > 0 and p > 0, i.e. 2 rho E > |m|^2
    const bool okL = QL[0] > T(0) && T(2) * QL[0] * QL[4] > QL[1] * QL[1] + QL[2] * QL[2] + QL[3] * QL[3];
    const bool okR = QR[0] > T(0) && T(2) * QR[0] * QR[4] > QR[1] * QR[1] + QR[2] * QR[2] + QR[3] * QR[3];
    if (!okL || !okR)
        for (int k = 0; k < NC; ++k) { QL[k] = q[1][k]; QR[k] = q[1][k]; }
}

// the d-faces form a grid like the cells' with nfl faces along d (x
// fastest): the index of the face at (i, j, k), the low d-face of cell
// (i, j, k) (its d-index may be nal: the high face of the last cell)
__device__ __forceinline__ int fidx(const Desc &D, int nfl, int i, int j, int k) {
    const int m0 = D.d == 0 ? nfl : D.nx, m1 = D.d == 1 ? nfl : D.ny;
    return (k * m1 + j) * m0 + i;
}

// (the kernels of the sweep's line work take the direction d as a template
// argument, so that the per-direction indexing is static)
// the evolved boundary states of every fluid cell along d, once per cell:
// E holds QL in planes 0..NC-1 and QR in planes NC..2NC-1
template <int d, typename T>
__global__ void k3_evolve(Desc D, int nal) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n) return;
    const int base[3] = {c % D.nx, (c / D.nx) % D.ny, c / (D.nx * D.ny)};
    if (!fluid_a(D, base[0], base[1], base[2])) return;
    T QL[NC], QR[NC];
    evolve5(D, d, base, base[d], nal, QL, QR);
    T *E = esrc<T>(D);
    for (int q = 0; q < NC; ++q) {
        E[(size_t)q * D.n + c] = QL[q];
        E[(size_t)(NC + q) * D.n + c] = QR[q];
    }
}

// the stabilised flux bf F2D of every d-face (eqs. Klein2DtotalfluxaMethod2,
// Klein2shieldedFluxMethod2, with the two-sided shielded parts) into the
// NC planes of F, face m of a line between its cells m-1 and m; the
// evolved states of the cells come from E, those of a boundary's ghost
// cells (a periodic ghost is the cell it wraps to) are evolved here
template <int d, typename T>
__global__ void k3_flux(Desc D, int nal, int nfl, int nlines) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int faces = nfl * nlines;
    if (t >= faces) return;
    const int m0 = d == 0 ? nfl : D.nx, m1 = d == 1 ? nfl : D.ny;
    const int base[3] = {(int)(t % m0), (int)((t / m0) % m1), (int)(t / ((long long)m0 * m1))};
    const int m = base[d];
    const bool periodic = D.bc[2 * d] == MB_BC_PERIODIC;
    double out[NC] = {0, 0, 0, 0, 0};
    bool flipL, flipR;
    int pL[3], pR[3];
    const int cL = line_cell(D, d, base, m - 1, nal, &flipL, pL);
    const int cR = line_cell(D, d, base, m, nal, &flipR, pR);
    // face m's time-averaged aperture (the low face of cell m; m = nal: the
    // high face of the last cell): 1 outside R
    const bool fin = in_rf(D, d, base[0], base[1], base[2]);
    const double bf = fin ? D.bt[rfidx(D, d, base[0], base[1], base[2])] : 1.0;
    if (fluid_a(D, pL[0], pL[1], pL[2]) && fluid_a(D, pR[0], pR[1], pR[2]) && (!fin || bf > 0.0)) {
        const T *E = esrc<T>(D);
        T QRa[NC], QLb[NC], G[NC], F[NC];
        if (m >= 1 || periodic) for (int q = 0; q < NC; ++q) QRa[q] = E[(size_t)(NC + q) * D.n + cL];
        else evolve5(D, d, base, m - 1, nal, G, QRa);
        if (m < nal) for (int q = 0; q < NC; ++q) QLb[q] = E[(size_t)q * D.n + cR];
        else evolve5(D, d, base, m, nal, QLb, G);
        hllc5(gam<T>(D), d, QRa, QLb, F);
        const int mR = m < nal ? m : (periodic ? 0 : -1);
        const int mL = m - 1 >= 0 ? m - 1 : (periodic ? nal - 1 : -1);
        double sR = 0.0, sL = 0.0, dR = 0.0, dL = 0.0;
        const double *FBR = nullptr, *FBL = nullptr;
        bool wall = false;   // a neighbour has wall data (else sR = sL = 0, no test needed)
        if (mR >= 0) {
            int c3[3] = {base[0], base[1], base[2]};
            c3[d] = mR;
            int f3[3] = {base[0], base[1], base[2]};
            f3[d] = mR + 1 < nal || !periodic ? mR + 1 : 0;
            if (in_r(D, c3[0], c3[1], c3[2])) {
                const int r = ridx(D, c3[0], c3[1], c3[2]);
                if (D.whas[r]) {
                    wall = true;
                    sR = fmax(0.0, bf - swept(D, f3[0], f3[1], f3[2]));
                    dR = D.wdist[r];
                    FBR = &D.wFB[(size_t)NC * r];
                }
            }
        }
        if (mL >= 0) {
            int c3[3] = {base[0], base[1], base[2]};
            c3[d] = mL;
            if (in_r(D, c3[0], c3[1], c3[2])) {
                const int r = ridx(D, c3[0], c3[1], c3[2]);
                if (D.whas[r]) {
                    wall = true;
                    sL = fmax(0.0, bf - swept(D, c3[0], c3[1], c3[2]));
                    dL = D.wdist[r];
                    FBL = &D.wFB[(size_t)NC * r];
                }
            }
        }
        if (wall && sR + sL > bf) {
            const double sc = bf / (sR + sL);
            sR *= sc;
            sL *= sc;
        }
        if (wall && (sR > 0.0 || sL > 0.0)) {   // the shielded parts, in FP64
            for (int q = 0; q < NC; ++q) {
                const double Fq = F[q];
                double v = (bf - sL - sR) * Fq;
                if (sR > 0.0) v += sR * (FBR[q] + dR * (Fq - FBR[q]));
                if (sL > 0.0) v += sL * (FBL[q] + dL * (Fq - FBL[q]));
                out[q] = v;
            }
        } else {                                // (bf - 0 - 0) F
            const T b = fin ? T(bf) : T(1);
            for (int q = 0; q < NC; ++q) out[q] = widen(b * F[q]);
        }
    }
    // fluxes are stored in FP64 either way, so that the update's
    // differences F_lo - F_hi telescope as in the FP64 path
    for (int q = 0; q < NC; ++q) D.F[(size_t)q * faces + t] = out[q];
}

// alpha_B Q' = alpha_A Q + lam (F_lo - F_hi) + lam (beta_hi - beta_lo)(F^B -
// w_d Q^B) (eqs. Klein2DcompleteMovingMethod2a-c) into Cn (and C in R)
template <int d>
__global__ void k3_update(Desc D, int nal, int nfl) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n) return;
    const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
    const bool periodic = D.bc[2 * d] == MB_BC_PERIODIC;
    double v[NC] = {0, 0, 0, 0, 0};
    unsigned char u = 0;
    if (fluid_a(D, i, j, k)) {
        const int ijk[3] = {i, j, k};
        const int m = ijk[d];
        const int faces = nfl * (D.n / nal);
        int hi3[3] = {i, j, k};
        hi3[d] = m + 1 < nal || !periodic ? m + 1 : 0;
        const int flo = fidx(D, nfl, i, j, k), fhi = fidx(D, nfl, hi3[0], hi3[1], hi3[2]);
        const double blo = swept(D, i, j, k), bhi = swept(D, hi3[0], hi3[1], hi3[2]);
        const bool cin = in_r(D, i, j, k);
        const double aA = cin ? D.aA[ridx(D, i, j, k)] : 1.0;
        const bool w = cin && D.whas[ridx(D, i, j, k)] && blo != bhi;
        const int r = w ? ridx(D, i, j, k) : 0;
        for (int q = 0; q < NC; ++q) {
            const double Qq = D.Q[(size_t)q * D.n + c];   // alpha_A Q, which is Q outside R
            double x = (cin ? aA * Qq : Qq) + D.lam * (D.F[(size_t)q * faces + flo] - D.F[(size_t)q * faces + fhi]);
            if (w) {
                const double wt = D.lam * (bhi - blo) * (D.wFB[(size_t)NC * r + q] - D.U[d] * D.wQB[(size_t)NC * r + q]);
                x += wt;
                atomicAdd(&D.wall[q], wt);
            }
            v[q] = x;
        }
        u = 1;
    }
    // C keeps the content for the events, which read it in R only (event
    // cells are cut at pose A or B, their neighbours within R)
    const bool inr = in_r(D, i, j, k);
    for (int q = 0; q < NC; ++q) {
        if (inr) D.C[(size_t)q * D.n + c] = v[q];
        D.Cn[(size_t)q * D.n + c] = v[q];
    }
    D.upd[c] = u;
    // a safeguard seed outside R (alpha_A = alpha_B = 1 there, no event
    // changes the content): a non-physical content
    if (u && !inr && content_bad(v)) add_seed(D, c);
}

// covering / uncovering (Sec. II.C.5): each event cell of R finds its
// neighbour set, the face neighbours, else those sharing an edge, else a
// vertex (recipients: alpha_B > 0, and in donor mode alpha_A > 0), and the
// sum of their alpha_B
__global__ void k3_evprep(Desc D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.rn[0] * D.rn[1] * D.rn[2]) return;
    int i, j, k;
    r_cell(D, t, &i, &j, &k);
    const double aA = D.aA[t], aB = D.aB[t];
    const bool covered = aA > 0.0 && aB == 0.0;
    const bool unc = !D.gcl && aA == 0.0 && aB > 0.0;
    D.evt[t] = 0;
    if (!covered && !unc) return;
    unsigned mask = 0u;
    double asum = 0.0;
    for (int pass = 0; pass < 3 && mask == 0u; ++pass)
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int nzc = (di != 0) + (dj != 0) + (dk != 0);
                    if (nzc == 0 || nzc > pass + 1) continue;
                    int ii, jj, kk;
                    if (nbr(D, i, j, k, di, dj, dk, &ii, &jj, &kk) < 0) continue;
                    const double b = alphaB(D, ii, jj, kk);
                    if (!(b > 0.0)) continue;
                    if (!D.gcl && alphaA(D, ii, jj, kk) == 0.0) continue;
                    mask |= 1u << ((dk + 1) * 9 + (dj + 1) * 3 + (di + 1));
                    asum += b;
                }
    if (mask == 0u) {
        const bool open = (D.bc[0] == MB_BC_TRANSMISSIVE && i == 0) || (D.bc[1] == MB_BC_TRANSMISSIVE && i == D.nx - 1) ||
                          (D.bc[2] == MB_BC_TRANSMISSIVE && j == 0) || (D.bc[3] == MB_BC_TRANSMISSIVE && j == D.ny - 1) ||
                          (D.bc[4] == MB_BC_TRANSMISSIVE && k == 0) || (D.bc[5] == MB_BC_TRANSMISSIVE && k == D.nz - 1);
        if (covered && open) D.evt[t] = 3;
        else atomicOr(D.err, E_NONBR);
        return;
    }
    D.evt[t] = covered ? 1 : 2;
    D.emask[t] = mask;
    D.easum[t] = asum;
}

// the events applied simultaneously, each cell of R gathering the changes
// to its own content in increasing order of the event cells (the order of
// the one-pass definition)
__global__ void k3_events(Desc D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.rn[0] * D.rn[1] * D.rn[2]) return;
    int i, j, k;
    r_cell(D, t, &i, &j, &k);
    const int c = cidx(D, i, j, k);
    const unsigned char e = D.evt[t];
    if (e == 1 || e == 3) {   // covered: its content leaves it
        for (int q = 0; q < NC; ++q) D.Cn[(size_t)q * D.n + c] = 0.0;
        return;
    }
    if (e == 2) {             // uncovered (donor mode): sigma times its donors' contents
        const double sigma = D.aB[t] / (D.aB[t] + D.easum[t]);
        const unsigned mask = D.emask[t];
        for (int q = 0; q < NC; ++q) {
            double tot = 0.0;
            for (int o = 0; o < 27; ++o) {
                if (!((mask >> o) & 1u)) continue;
                int ii, jj, kk;
                const int cc = nbr(D, i, j, k, o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1, &ii, &jj, &kk);
                tot += D.C[(size_t)q * D.n + cc];
            }
            D.Cn[(size_t)q * D.n + c] = sigma * tot;
        }
        D.upd[c] = 1;
        return;
    }
    // a recipient or donor: the event cells among the 26 neighbours that
    // name this cell, in increasing cell index
    int ev[26], ecell[26], ne = 0;
    for (int o = 0; o < 27; ++o) {
        if (o == 13) continue;
        int ii, jj, kk;
        const int cc = nbr(D, i, j, k, o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1, &ii, &jj, &kk);
        if (cc < 0 || !in_r(D, ii, jj, kk)) continue;
        const int r = ridx(D, ii, jj, kk);
        const unsigned char et = D.evt[r];
        if (et != 1 && et != 2) continue;
        // this cell seen from the event cell: the opposite offset
        const int ob = 26 - o;
        if (!((D.emask[r] >> ob) & 1u)) continue;
        int z = ne++;
        while (z > 0 && ecell[z - 1] > cc) { ecell[z] = ecell[z - 1]; ev[z] = ev[z - 1]; --z; }
        ecell[z] = cc;
        ev[z] = r;
    }
    if (ne == 0) return;
    const double aBc = alphaB(D, i, j, k);
    for (int q = 0; q < NC; ++q) {
        double x = D.Cn[(size_t)q * D.n + c];
        for (int m = 0; m < ne; ++m) {
            const int r = ev[m];
            if (D.evt[r] == 1) x += aBc / D.easum[r] * D.C[(size_t)q * D.n + ecell[m]];
            else x -= D.aB[r] / (D.aB[r] + D.easum[r]) * D.C[(size_t)q * D.n + c];
        }
        D.Cn[(size_t)q * D.n + c] = x;
    }
}

// safeguard seeds: non-physical new contents, and cells keeping less than
// COLLAPSE of their volume over the sweep, in the list (cell indices)
// (cells outside R are tested by k3_update, whose contents no later step
// before the safeguard changes; this kernel runs over R, after the events)
__global__ void k3_bad(Desc D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.rn[0] * D.rn[1] * D.rn[2]) return;
    int i, j, k;
    r_cell(D, t, &i, &j, &k);
    const int c = cidx(D, i, j, k);
    if (!D.upd[c]) return;
    const double aB = D.aB[t];
    if (!(aB > 0.0)) return;
    double q[NC];
    for (int m = 0; m < NC; ++m) q[m] = D.Cn[(size_t)m * D.n + c];
    if (content_bad(q) || aB < COLLAPSE * D.aA[t]) add_seed(D, c);
}

// the merges (one thread): each cluster of seeds and their fluid, updated
// face neighbours shares its content in proportion to alpha_B; sums in cell
// order; cells still non-physical seed the next merge
__device__ bool physical5(const Desc &D, int c) {
    const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
    const double aB = alphaB(D, i, j, k);
    double q[NC];
    for (int m = 0; m < NC; ++m) {
        q[m] = D.Cn[(size_t)m * D.n + c] / aB;
        if (!isfinite(q[m])) return false;
    }
    return q[0] > 0.0 && pressure5(D.gamma, q) > 0.0;
}
// (one thread, over global lists: the form for clusters too large for the
// shared-memory form in k3_mix; it continues from layer layer0 with the ns
// seeds in D.seeds and the mixed count so far)
__device__ void mix_serial(const Desc &D, int ns, int layer0, int mixed) {
    int *seed = D.seeds;
    for (int layer = layer0; layer < MIX_LAYERS && ns > 0; ++layer) {
        // seeds in cell order
        for (int x = 1; x < ns; ++x) {
            const int v = seed[x];
            int z = x;
            while (z > 0 && seed[z - 1] > v) { seed[z] = seed[z - 1]; --z; }
            seed[z] = v;
        }
        int nn = 0;
        bool over = false;
        auto add = [&](int c) -> int {
            if (D.lab[c] >= 0) return D.lab[c];
            if (nn >= NODECAP) { over = true; return -1; }
            D.lab[c] = nn;
            D.nodes[nn] = c;
            D.par_[nn] = nn;
            return nn++;
        };
        auto root = [&](int a) { while (D.par_[a] != a) a = D.par_[a]; return a; };
        for (int s = 0; s < ns && !over; ++s) {
            const int c = seed[s];
            const int a = add(c);
            if (a < 0) break;
            const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
            const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
            for (int m = 0; m < 6; ++m) {
                int ii, jj, kk;
                const int cc = nbr(D, i, j, k, off[m][0], off[m][1], off[m][2], &ii, &jj, &kk);
                if (cc < 0 || !(alphaB(D, ii, jj, kk) > 0.0) || !D.upd[cc]) continue;
                const int b = add(cc);
                if (b < 0) break;
                const int ra = root(a), rb = root(b);
                // the root is the smaller cell index
                if (ra != rb) { if (D.nodes[ra] < D.nodes[rb]) D.par_[rb] = ra; else D.par_[ra] = rb; }
            }
        }
        if (over) {
            *D.err |= E_NODECAP;
            for (int m = 0; m < nn; ++m) D.lab[D.nodes[m]] = -1;
            return;
        }
        // every node's root cell (by insertion index), then the nodes in
        // cell order with their root cells
        int *rootcell = D.seeds + SEEDCAP;     // scratch after the seeds
        for (int x = 0; x < nn; ++x) rootcell[x] = D.nodes[root(x)];
        for (int x = 1; x < nn; ++x) {
            const int v = D.nodes[x], rv = rootcell[x];
            int z = x;
            while (z > 0 && D.nodes[z - 1] > v) { D.nodes[z] = D.nodes[z - 1]; rootcell[z] = rootcell[z - 1]; --z; }
            D.nodes[z] = v;
            rootcell[z] = rv;
        }
        // each cluster's sums at the slot of its root cell (its position
        // among the sorted nodes), members added in cell order
        for (int x = 0; x < nn; ++x) for (int q = 0; q <= NC; ++q) D.ntot[(NC + 1) * x + q] = 0.0;
        auto slot = [&](int cell) {
            int lo = 0, hi = nn - 1;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (D.nodes[mid] < cell) lo = mid + 1; else hi = mid; }
            return lo;
        };
        for (int x = 0; x < nn; ++x) {
            const int c = D.nodes[x];
            const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
            const int sr = slot(rootcell[x]);
            D.ntot[(NC + 1) * sr + NC] += alphaB(D, i, j, k);
            for (int q = 0; q < NC; ++q) D.ntot[(NC + 1) * sr + q] += D.Cn[(size_t)q * D.n + c];
        }
        for (int x = 0; x < nn; ++x) {
            const int c = D.nodes[x];
            const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
            const int sr = slot(rootcell[x]);
            const double aB = alphaB(D, i, j, k);
            for (int q = 0; q < NC; ++q)
                D.Cn[(size_t)q * D.n + c] = aB * (D.ntot[(NC + 1) * sr + q] / D.ntot[(NC + 1) * sr + NC]);
        }
        mixed += nn;
        // cells still non-physical, in cell order
        int nb = 0;
        for (int x = 0; x < nn; ++x) {
            const int c = D.nodes[x];
            if (!physical5(D, c)) seed[nb++] = c;
        }
        for (int x = 0; x < nn; ++x) D.lab[D.nodes[x]] = -1;
        ns = nb;
    }
    if (ns > 0) atomicOr(D.err, E_UNSTABLE);   // cells left non-physical after the last merge
    *D.mixed = mixed;
}

// The merges in one 256-thread block over shared memory, while a layer's
// seeds and nodes fit (MIXS_SEEDS seeds, MIXS_NODES nodes); else the
// remaining layers in mix_serial.  The same clusters, sums and write-back
// as mix_serial: the candidate cells (the seeds and their fluid, updated
// face neighbours) are sorted and made unique (the nodes, in cell order);
// the clusters are the connected components of the seed-neighbour edges,
// labelled by their smallest node (repeated minimum over the edges until
// no label changes); each cluster's smallest node's thread sums its
// members in node order, i.e. in cell order.
constexpr int MIXS_THREADS = 256, MIXS_SORT = 1024, MIXS_SEEDS = MIXS_SORT / 7, MIXS_NODES = 320;
__device__ __forceinline__ int node_of(const int *nodes, int nn, int c) {
    int lo = 0, hi = nn - 1;
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (nodes[mid] < c) lo = mid + 1; else hi = mid; }
    return lo;
}
__global__ void __launch_bounds__(MIXS_THREADS) k3_mix(Desc D) {
    __shared__ int cand[MIXS_SORT];
    __shared__ int enode[MIXS_SEEDS * 6];   // per (seed, direction): the neighbour's cell, then its node; -1 none
    __shared__ int snode[MIXS_SEEDS];       // the seed's node
    __shared__ int nodes[MIXS_NODES], lbl[MIXS_NODES];
    __shared__ double cache[MIXS_NODES][NC + 1], sums[MIXS_NODES][NC + 1];
    __shared__ int s_wsum[MIXS_THREADS / 32], s_nn, s_changed, s_nb;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int ns = *D.nseed;
    if (ns > SEEDCAP) {
        if (tid == 0) atomicOr(D.err, E_SEEDCAP);
        ns = SEEDCAP;
    }
    int mixed = 0, layer = 0;
    for (; layer < MIX_LAYERS && ns > 0; ++layer) {
        if (ns > MIXS_SEEDS) break;
        int P = 2;
        while (P < 7 * ns) P <<= 1;
        // candidates: seed s at 7s, its neighbours after it
        for (int x = tid; x < P; x += MIXS_THREADS) cand[x] = INT_MAX;
        __syncthreads();
        for (int s = tid; s < ns; s += MIXS_THREADS) {
            const int c = D.seeds[s];
            const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
            cand[7 * s] = c;
            const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
            for (int m = 0; m < 6; ++m) {
                int ii, jj, kk;
                const int cc = nbr(D, i, j, k, off[m][0], off[m][1], off[m][2], &ii, &jj, &kk);
                const bool ok = cc >= 0 && alphaB(D, ii, jj, kk) > 0.0 && D.upd[cc];
                cand[7 * s + 1 + m] = ok ? cc : INT_MAX;
                enode[6 * s + m] = ok ? cc : -1;
            }
        }
        __syncthreads();
        // bitonic sort of cand[0, P)
        for (int k2 = 2; k2 <= P; k2 <<= 1)
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                for (int x = tid; x < P; x += MIXS_THREADS) {
                    const int y = x ^ j2;
                    if (y > x) {
                        const int a = cand[x], b = cand[y];
                        if ((a > b) == ((x & k2) == 0)) { cand[x] = b; cand[y] = a; }
                    }
                }
                __syncthreads();
            }
        // the distinct cells, in order: a contiguous chunk per thread and a
        // block-wide exclusive scan of the chunks' counts
        const int per = (P + MIXS_THREADS - 1) / MIXS_THREADS, x0 = min(P, tid * per), x1 = min(P, x0 + per);
        int cnt = 0;
        for (int x = x0; x < x1; ++x) cnt += cand[x] != INT_MAX && (x == 0 || cand[x - 1] != cand[x]);
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_wsum[wid] = inc;
        __syncthreads();
        int pos = inc - cnt, tot = 0;
        for (int w = 0; w < MIXS_THREADS / 32; ++w) {
            if (w < wid) pos += s_wsum[w];
            tot += s_wsum[w];
        }
        for (int x = x0; x < x1; ++x)
            if (cand[x] != INT_MAX && (x == 0 || cand[x - 1] != cand[x])) {
                if (pos < MIXS_NODES) nodes[pos] = cand[x];
                ++pos;
            }
        __syncthreads();
        const int nn = tot;
        if (nn > MIXS_NODES) break;
        // edges as node pairs, labels, the nodes' contents and alpha_B
        for (int x = tid; x < 6 * ns; x += MIXS_THREADS)
            if (enode[x] >= 0) enode[x] = node_of(nodes, nn, enode[x]);
        for (int s = tid; s < ns; s += MIXS_THREADS) snode[s] = node_of(nodes, nn, D.seeds[s]);
        for (int x = tid; x < nn; x += MIXS_THREADS) {
            const int c = nodes[x];
            const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
            lbl[x] = x;
            for (int q = 0; q < NC; ++q) cache[x][q] = D.Cn[(size_t)q * D.n + c];
            cache[x][NC] = alphaB(D, i, j, k);
        }
        for (;;) {
            __syncthreads();
            if (tid == 0) s_changed = 0;
            __syncthreads();
            for (int x = tid; x < 6 * ns; x += MIXS_THREADS) {
                const int b = enode[x];
                if (b < 0) continue;
                const int a = snode[x / 6];
                const int la = lbl[a], lb = lbl[b];
                if (la != lb) {
                    const int mn = min(la, lb);
                    atomicMin(&lbl[a], mn);
                    atomicMin(&lbl[b], mn);
                    s_changed = 1;
                }
            }
            __syncthreads();
            const int ch = s_changed;
            if (!ch) break;
        }
        // each cluster's sums (alpha_B and contents) in node order
        for (int r = tid; r < nn; r += MIXS_THREADS) {
            if (lbl[r] != r) continue;
            double acc[NC + 1] = {0, 0, 0, 0, 0, 0};
            for (int x = r; x < nn; ++x) {
                if (lbl[x] != r) continue;
                acc[NC] += cache[x][NC];
                for (int q = 0; q < NC; ++q) acc[q] += cache[x][q];
            }
            for (int q = 0; q <= NC; ++q) sums[r][q] = acc[q];
        }
        if (tid == 0) s_nb = 0;
        __syncthreads();
        // shares in proportion to alpha_B; cells still non-physical seed
        // the next layer (its candidates are sorted, so order is free)
        for (int x = tid; x < nn; x += MIXS_THREADS) {
            const int c = nodes[x], r = lbl[x];
            const double aB = cache[x][NC];
            for (int q = 0; q < NC; ++q) D.Cn[(size_t)q * D.n + c] = aB * (sums[r][q] / sums[r][NC]);
            if (!physical5(D, c)) D.seeds[atomicAdd(&s_nb, 1)] = c;
        }
        mixed += nn;
        __syncthreads();
        ns = s_nb;
        __syncthreads();
    }
    if (layer < MIX_LAYERS && ns > 0) {   // too large for shared memory: the serial form goes on
        if (tid == 0) mix_serial(D, ns, layer, mixed);
        return;
    }
    if (tid == 0 && ns > 0) atomicOr(D.err, E_UNSTABLE);   // cells left non-physical after the last merge
    if (tid == 0) *D.mixed = mixed;
}

// Q = content / alpha_B (NaN where alpha_B = 0 or the cell was not
// updated), with the checks of the new state
// (outside R alpha_B = 1 and the state is the content: its test was the
// seed test, and the safeguard flags cells it leaves non-physical)
__global__ void k3_final(Desc D) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n) return;
    const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
    if (!in_r(D, i, j, k)) {
        for (int m = 0; m < NC; ++m) {
            const double cn = D.Cn[(size_t)m * D.n + c];
            D.Q[(size_t)m * D.n + c] = cn;
            if (D.f32) D.Qf[(size_t)m * D.n + c] = float(cn);
        }
        return;
    }
    const double aB = alphaB(D, i, j, k);
    const bool ok = aB > 0.0 && D.upd[c];
    const double ia = ok ? (aB == 1.0 ? 1.0 : 1.0 / aB) : 0.0;
    double q[NC];
    for (int m = 0; m < NC; ++m) {
        const double cn = D.Cn[(size_t)m * D.n + c];
        q[m] = ok ? (ia == 1.0 ? cn : cn * ia) : NAN;
        D.Q[(size_t)m * D.n + c] = q[m];
        if (D.f32) D.Qf[(size_t)m * D.n + c] = float(q[m]);
    }
    if (aB > 0.0 && !D.upd[c]) atomicOr(D.err, E_UNSTABLE);
    if (ok) {
        bool bad = !(q[0] > 0.0) || !(2.0 * q[0] * q[4] > q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int m = 0; m < NC; ++m) if (!finite64(q[m])) bad = true;
        if (bad) atomicOr(D.err, E_UNSTABLE);
    }
}

// maxima of |u_d| + c over the fluid cells (positive doubles compare as
// their bit patterns)
// (a grid-stride loop, 256-thread blocks: one atomic per block and axis;
// in the type T of the flow arithmetic)
template <typename T>
__global__ void k3_speeds(Desc D) {
    __shared__ double red[3][8];
    const T *Q = qsrc<T>(D);
    const T g = gam<T>(D);
    T s[3] = {T(0), T(0), T(0)};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < D.n; c += gridDim.x * blockDim.x) {
        if (isnan(Q[c])) continue;
        T q[NC];
        for (int m = 0; m < NC; ++m) q[m] = Q[(size_t)m * D.n + c];
        const T ir = T(1) / q[0];
        const T p = (g - T(1)) * (q[4] - T(0.5) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) * ir);
        const T cs = sqrt(g * p * ir);
        for (int a = 0; a < 3; ++a) s[a] = fmax(s[a], fabs(q[1 + a] * ir) + cs);
    }
    const int w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        double v = double(s[a]);
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) red[a][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int q = 0; q < 8; ++q) v = fmax(v, red[threadIdx.x][q]);
        if (v > 0.0) atomicMax((unsigned long long *)&D.smax[threadIdx.x], (unsigned long long)__double_as_longlong(v));
    }
}

// solid cells (alpha = 0 in R at the current pose) read NaN; alpha of every
// cell into out (optional)
__global__ void k3_classify(Desc D, double *alpha_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n) return;
    const int i = c % D.nx, j = (c / D.nx) % D.ny, k = c / (D.nx * D.ny);
    const double a = alphaA(D, i, j, k);
    if (alpha_out) alpha_out[c] = a;
    else if (!(a > 0.0)) for (int m = 0; m < NC; ++m) D.Q[(size_t)m * D.n + c] = NAN;
}

// the FP32 copy of the state (FP32 flux option)
__global__ void k3_to_f32(Desc D) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D.n) return;
    for (int m = 0; m < NC; ++m) D.Qf[(size_t)m * D.n + c] = float(D.Q[(size_t)m * D.n + c]);
}

}  // namespace mb3

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using mb3::Desc;
using mb3::NC;

struct mb3_sim {
    Desc D{};
    int nplane = 0;
    double pn[3 * MB3_MAX_PLANES] = {}, pc[MB3_MAX_PLANES] = {}, bb[6] = {};
    double t = 0.0, T[3] = {0.0, 0.0, 0.0};
    long step = 0;
    int sidx = 0;
    double dt_step = 0.0, cfl = 0.5;
    cudaStream_t st = nullptr;
    cudaStream_t gs[2] = {nullptr, nullptr};      // face apertures and swept apertures beside k3_cells
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    std::string err;
    size_t rcap = 0, rfcap = 0;
    bool prev_ok = false;        // aB / tB hold the current pose over the region q0, qn
    int q0[3] = {0, 0, 0}, qn[3] = {0, 0, 0};
    double wall_host[NC] = {0, 0, 0, 0, 0};
    int merged = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the last sweep's k3_flux
    float flux_ms = 0.0f;
    std::vector<void *> owned;
};

static mb_status fail3(mb3_sim *s, mb_status r, const std::string &m) {
    if (s) s->err = m;
    return r;
}
static mb_status cuda3(mb3_sim *s, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MB_OK;
    return fail3(s, e == cudaErrorMemoryAllocation ? MB_E_NOMEM : MB_E_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
template <class X>
static cudaError_t dalloc(mb3_sim *s, X **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(X));
    if (e == cudaSuccess) s->owned.push_back(q);
    *p = (X *)q;
    return e;
}
static void dfree(mb3_sim *s, void *p) {
    if (!p) return;
    cudaFree(p);
    s->owned.erase(std::remove(s->owned.begin(), s->owned.end(), p), s->owned.end());
}

// the body posed at translation T
static mb3::Body3 posed(const mb3_sim *s, const double *T) {
    mb3::Body3 B;
    memset(&B, 0, sizeof(B));
    B.np = s->nplane;
    for (int f = 0; f < s->nplane; ++f) {
        for (int a = 0; a < 3; ++a) B.n[3 * f + a] = s->pn[3 * f + a];
        B.c[f] = s->pc[f] + (s->pn[3 * f] * T[0] + s->pn[3 * f + 1] * T[1] + s->pn[3 * f + 2] * T[2]);
    }
    return B;
}

// region R: the cells meeting the body's bounding box at translations TA and
// TB, widened by two cells, inside the grid (rn = 0: no body in the grid)
static void region(mb3_sim *s, const double *TA, const double *TB, int *r0, int *rn) {
    const int nn[3] = {s->D.nx, s->D.ny, s->D.nz};
    for (int a = 0; a < 3; ++a) {
        r0[a] = 0;
        rn[a] = 0;
    }
    if (s->nplane == 0) return;
    for (int a = 0; a < 3; ++a) {
        const double u0 = std::min(s->bb[2 * a] + TA[a], s->bb[2 * a] + TB[a]);
        const double u1 = std::max(s->bb[2 * a + 1] + TA[a], s->bb[2 * a + 1] + TB[a]);
        long lo = (long)std::floor((u0 - s->D.lo[a]) / s->D.h[a]) - 2;
        long hi = (long)std::floor((u1 - s->D.lo[a]) / s->D.h[a]) + 2;
        lo = std::max(lo, 0L);
        hi = std::min(hi, (long)nn[a] - 1);
        if (hi < lo) { for (int q = 0; q < 3; ++q) rn[q] = 0; return; }
        r0[a] = (int)lo;
        rn[a] = (int)(hi - lo + 1);
    }
}

// R's buffers for at least rc cells and rf faces per axis
static cudaError_t ensure_r(mb3_sim *s, size_t rc, size_t rf) {
    cudaError_t e = cudaSuccess;
    Desc &D = s->D;
    if (rc > s->rcap) {
        cudaStreamSynchronize(s->st);
        dfree(s, D.aA); dfree(s, D.aM); dfree(s, D.aB); dfree(s, D.tA); dfree(s, D.tB); dfree(s, D.whas);
        dfree(s, D.aP); dfree(s, D.tP);
        s->prev_ok = false;
        dfree(s, D.wdist); dfree(s, D.wFB); dfree(s, D.wQB); dfree(s, D.evt); dfree(s, D.emask); dfree(s, D.easum);
        const size_t c = rc + rc / 4;
        if (e == cudaSuccess) e = dalloc(s, &D.aA, c);
        if (e == cudaSuccess) e = dalloc(s, &D.aM, c);
        if (e == cudaSuccess) e = dalloc(s, &D.aB, c);
        if (e == cudaSuccess) e = dalloc(s, &D.tA, c);
        if (e == cudaSuccess) e = dalloc(s, &D.tB, c);
        if (e == cudaSuccess) e = dalloc(s, &D.aP, c);
        if (e == cudaSuccess) e = dalloc(s, &D.tP, c);
        if (e == cudaSuccess) e = dalloc(s, &D.whas, c);
        if (e == cudaSuccess) e = dalloc(s, &D.wdist, c);
        if (e == cudaSuccess) e = dalloc(s, &D.wFB, NC * c);
        if (e == cudaSuccess) e = dalloc(s, &D.wQB, NC * c);
        if (e == cudaSuccess) e = dalloc(s, &D.evt, c);
        if (e == cudaSuccess) e = dalloc(s, &D.emask, c);
        if (e == cudaSuccess) e = dalloc(s, &D.easum, c);
        s->rcap = e == cudaSuccess ? c : 0;
    }
    if (e == cudaSuccess && rf > s->rfcap) {
        cudaStreamSynchronize(s->st);
        for (int a = 0; a < 3; ++a) dfree(s, D.bM[a]);
        dfree(s, D.bt);
        const size_t c = rf + rf / 4;
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = dalloc(s, &D.bM[a], c);
        if (e == cudaSuccess) e = dalloc(s, &D.bt, c);
        s->rfcap = e == cudaSuccess ? c : 0;
    }
    return e;
}

static unsigned nblk(long long n, int b = 256) { return (unsigned)std::max<long long>(1, (n + b - 1) / b); }

// alpha at translation T over R(T) (into D.aA) and the classification
static cudaError_t pose_alpha(mb3_sim *s, const double *T, Desc &D) {
    region(s, T, T, D.r0, D.rn);
    const size_t rc = (size_t)D.rn[0] * D.rn[1] * D.rn[2];
    const size_t rf = (size_t)(D.rn[0] + 1) * (D.rn[1] + 1) * (D.rn[2] + 1);
    cudaError_t e = ensure_r(s, rc, rf);
    if (e != cudaSuccess) return e;
    D = s->D, region(s, T, T, D.r0, D.rn);
    if (rc > 0) {
        const mb3::Body3 B = posed(s, T);
        mb3::k3_cells<<<nblk(32LL * (long long)rc), 256, 0, s->st>>>(D, B, B, B, mb3::CELLS_ONE);   // one pose
    }
    e = cudaGetLastError();
    s->prev_ok = e == cudaSuccess;
    for (int a = 0; a < 3; ++a) { s->q0[a] = D.r0[a]; s->qn[a] = D.rn[a]; }
    return e;
}

extern "C" {

mb_status mb3_create(const mb3_grid *g, double gamma, double cfl, const mb3_body *b, int uncover_mode,
                     mb3_sim **out) {
    if (!out) return MB_E_INVAL;
    *out = nullptr;
    if (!g || !b) return MB_E_INVAL;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || (long long)g->nx * g->ny * g->nz > (1LL << 30)) return MB_E_INVAL;
    for (int a = 0; a < 3; ++a) if (!(g->hi[a] > g->lo[a])) return MB_E_INVAL;
    for (int q = 0; q < 6; ++q) if (g->bc[q] < 0 || g->bc[q] > 2) return MB_E_INVAL;
    for (int a = 0; a < 3; ++a) if ((g->bc[2 * a] == MB_BC_PERIODIC) != (g->bc[2 * a + 1] == MB_BC_PERIODIC)) return MB_E_INVAL;
    // the stencil's two ghost cells mirror two cells of a non-periodic axis
    const int nax[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) if (nax[a] < 2 && g->bc[2 * a] != MB_BC_PERIODIC) return MB_E_INVAL;
    if (!(gamma > 1.0) || !(cfl > 0.0 && cfl <= 1.0)) return MB_E_INVAL;
    if (uncover_mode != MB_UNCOVER_DONOR && uncover_mode != MB_UNCOVER_FLUX_GCL) return MB_E_INVAL;
    if (b->nplane < 0 || b->nplane > MB3_MAX_PLANES || (b->nplane > 0 && (!b->normals || !b->offsets))) return MB_E_INVAL;
    mb3_sim *s = new mb3_sim();
    Desc &D = s->D;
    D.nx = g->nx; D.ny = g->ny; D.nz = g->nz;
    D.n = g->nx * g->ny * g->nz;
    const int nn[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        D.lo[a] = g->lo[a];
        D.h[a] = (g->hi[a] - g->lo[a]) / nn[a];
        D.U[a] = b->U[a];
    }
    for (int q = 0; q < 6; ++q) D.bc[q] = g->bc[q];
    D.gamma = gamma;
    D.gammaf = (float)gamma;
    D.gcl = uncover_mode == MB_UNCOVER_FLUX_GCL;
    s->cfl = cfl;
    s->nplane = b->nplane;
    for (int f = 0; f < b->nplane; ++f) {
        for (int a = 0; a < 3; ++a) s->pn[3 * f + a] = b->normals[3 * f + a];
        s->pc[f] = b->offsets[f];
    }
    for (int q = 0; q < 6; ++q) s->bb[q] = b->bbox[q];
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&s->gs[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
    const size_t n = D.n;
    size_t fmax_ = 0;
    for (int a = 0; a < 3; ++a) fmax_ = std::max(fmax_, (size_t)(nn[a] + 1) * (n / nn[a]));
    if (e == cudaSuccess) e = dalloc(s, &D.Q, NC * n);
    if (e == cudaSuccess) e = dalloc(s, &D.Qn, NC * n);
    if (e == cudaSuccess) e = dalloc(s, &D.C, NC * n);
    if (e == cudaSuccess) e = dalloc(s, &D.Cn, NC * n);
    if (e == cudaSuccess) e = dalloc(s, &D.F, NC * fmax_);
    if (e == cudaSuccess) e = dalloc(s, &D.E, 2 * NC * n);
    if (e == cudaSuccess) e = dalloc(s, &D.upd, n);
    if (e == cudaSuccess) e = dalloc(s, &D.err, 1);
    if (e == cudaSuccess) e = dalloc(s, &D.wall, NC);
    if (e == cudaSuccess) e = dalloc(s, &D.seeds, mb3::SEEDCAP + mb3::NODECAP);
    if (e == cudaSuccess) e = dalloc(s, &D.nseed, 1);
    if (e == cudaSuccess) e = dalloc(s, &D.lab, n);
    if (e == cudaSuccess) e = dalloc(s, &D.par_, mb3::NODECAP);
    if (e == cudaSuccess) e = dalloc(s, &D.nodes, mb3::NODECAP);
    if (e == cudaSuccess) e = dalloc(s, &D.ntot, (NC + 1) * (size_t)mb3::NODECAP);
    if (e == cudaSuccess) e = dalloc(s, &D.mixed, 1);
    if (e == cudaSuccess) e = dalloc(s, &D.smax, 3);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.lab, 0xff, n * sizeof(int), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.err, 0, sizeof(int), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.Q, 0, NC * n * sizeof(double), s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        const mb_status r = e == cudaErrorMemoryAllocation ? MB_E_NOMEM : MB_E_CUDA;
        mb3_destroy(s);
        return r;
    }
    *out = s;
    return MB_OK;
}

void mb3_destroy(mb3_sim *s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    for (int q = 0; q < 2; ++q) if (s->gs[q]) cudaStreamSynchronize(s->gs[q]);
    for (void *p : s->owned) cudaFree(p);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->fork) cudaEventDestroy(s->fork);
    for (int q = 0; q < 2; ++q) {
        if (s->join[q]) cudaEventDestroy(s->join[q]);
        if (s->gs[q]) cudaStreamDestroy(s->gs[q]);
    }
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

const char *mb3_last_error(const mb3_sim *s) { return s ? s->err.c_str() : "NULL simulation"; }

static mb_status err_status(mb3_sim *s, int w) {
    if (w & (mb3::E_SEEDCAP | mb3::E_NODECAP))
        return fail3(s, MB_E_CAPACITY, "positivity safeguard: more cells than its lists hold");
    if (w & mb3::E_NONBR) return fail3(s, MB_E_UNSTABLE, "covered/uncovered cell without a fluid neighbour");
    if (w & mb3::E_UNSTABLE) return fail3(s, MB_E_UNSTABLE, "non-physical state after the safeguard");
    return MB_OK;
}

mb_status mb3_write_state(mb3_sim *s, const double *Q, double t, const double *T) {
    if (!s || !Q || !T) return MB_E_INVAL;
    cudaError_t e = cudaMemcpyAsync(s->D.Q, Q, NC * (size_t)s->D.n * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->D.err, 0, sizeof(int), s->st);
    Desc D = s->D;
    if (e == cudaSuccess) e = pose_alpha(s, T, D);
    if (e == cudaSuccess) mb3::k3_classify<<<nblk(s->D.n), 256, 0, s->st>>>(D, nullptr);
    if (e == cudaSuccess && D.f32) mb3::k3_to_f32<<<nblk(s->D.n), 256, 0, s->st>>>(D);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_write_state");
    s->t = t;
    for (int a = 0; a < 3; ++a) s->T[a] = T[a];
    s->step = 0;
    s->sidx = 0;
    return MB_OK;
}

mb_status mb3_read_state(mb3_sim *s, double *Q, double *alpha, double *clock) {
    if (!s) return MB_E_INVAL;
    cudaError_t e = cudaSuccess;
    if (Q) e = cudaMemcpyAsync(Q, s->D.Q, NC * (size_t)s->D.n * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (alpha && e == cudaSuccess) {
        Desc D = s->D;
        e = pose_alpha(s, s->T, D);
        if (e == cudaSuccess) mb3::k3_classify<<<nblk(s->D.n), 256, 0, s->st>>>(D, s->D.C);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(alpha, s->D.C, (size_t)s->D.n * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    }
    int w = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w, s->D.err, sizeof(int), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_read_state");
    if (clock) {
        clock[0] = s->t;
        for (int a = 0; a < 3; ++a) clock[1 + a] = s->T[a];
        clock[4] = (double)s->step;
    }
    return err_status(s, w);
}

mb_status mb3_sweep(mb3_sim *s, int d, double dt) {
    if (!s || d < 0 || d > 2 || !(dt > 0.0)) return MB_E_INVAL;
    if (s->sidx > 0 && dt != s->dt_step) return fail3(s, MB_E_STATE, "the sweeps of a step must share dt");
    cudaError_t e = cudaSuccess;
    if (s->sidx == 0) {
        s->dt_step = dt;
        e = cudaMemcpyAsync(s->D.Qn, s->D.Q, NC * (size_t)s->D.n * sizeof(double), cudaMemcpyDeviceToDevice, s->st);
    }
    const double delta = s->D.U[d] * dt;
    double TA[3] = {s->T[0], s->T[1], s->T[2]}, TM[3] = {TA[0], TA[1], TA[2]}, TB[3] = {TA[0], TA[1], TA[2]};
    TB[d] += delta;
    TM[d] += 0.5 * delta;
    int r0[3], rn[3];
    region(s, TA, TB, r0, rn);
    const size_t rc = (size_t)rn[0] * rn[1] * rn[2];
    const size_t rf = (size_t)(rn[0] + 1) * (rn[1] + 1) * (rn[2] + 1);
    if (e == cudaSuccess) e = ensure_r(s, rc, rf);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_sweep buffers");
    // pose A is the last pose computed (the previous sweep's B, or the pose
    // of the last state write or read): its fractions move to aP
    const bool reuse = s->prev_ok;
    if (reuse) {
        std::swap(s->D.aB, s->D.aP);
        std::swap(s->D.tB, s->D.tP);
        for (int a = 0; a < 3; ++a) { s->D.p0[a] = s->q0[a]; s->D.pn[a] = s->qn[a]; }
    }
    s->prev_ok = false;
    Desc D = s->D;
    for (int a = 0; a < 3; ++a) { D.r0[a] = r0[a]; D.rn[a] = rn[a]; }
    D.d = d;
    D.lam = dt / D.h[d];
    D.hlamf = 0.5f * (float)D.lam;
    const int nn[3] = {D.nx, D.ny, D.nz};
    const int nal = nn[d], nlines = D.n / nal;
    const bool periodic = D.bc[2 * d] == MB_BC_PERIODIC;
    const int nfl = periodic ? nal : nal + 1;
    if (e == cudaSuccess) e = cudaMemsetAsync(D.wall, 0, NC * sizeof(double), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.nseed, 0, sizeof(int), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.mixed, 0, sizeof(int), s->st);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_sweep");
    const mb3::Body3 BA = posed(s, TA), BM = posed(s, TM), BB = posed(s, TB);
    if (rc > 0) {
        // the three geometry kernels are independent (each writes its own
        // arrays); the cut cells near a body's corners make each of them a
        // long tail on few SMs, so they run side by side on three streams
        cudaEventRecord(s->fork, s->st);
        cudaStreamWaitEvent(s->gs[0], s->fork, 0);
        cudaStreamWaitEvent(s->gs[1], s->fork, 0);
        mb3::k3_cells<<<nblk(32LL * (reuse ? 2 : 3) * (long long)rc), 256, 0, s->st>>>(
            D, BA, BM, BB, reuse ? mb3::CELLS_REUSE_A : mb3::CELLS_ALL);
        long long nfaces = 0;
        for (int a = 0; a < 4; ++a) {
            const int ax = a < 3 ? a : d;
            nfaces += (long long)(rn[0] + (ax == 0)) * (rn[1] + (ax == 1)) * (rn[2] + (ax == 2));
        }
        mb3::k3_faces<<<nblk(nfaces), 256, 0, s->gs[0]>>>(D, BM, BA, delta);
        if (delta != 0.0) {
            const long long nsw = (long long)(rn[0] + (d == 0)) * (rn[1] + (d == 1)) * (rn[2] + (d == 2));
            mb3::k3_swept<<<nblk(32LL * nsw), 256, 0, s->gs[1]>>>(D, BA, delta);
        }
        for (int q = 0; q < 2; ++q) {
            cudaEventRecord(s->join[q], s->gs[q]);
            cudaStreamWaitEvent(s->st, s->join[q], 0);
        }
        mb3::k3_wall<<<nblk((long long)rc), 256, 0, s->st>>>(D);
    }
    const bool f = D.f32;
    const auto evolve = d == 0 ? (f ? mb3::k3_evolve<0, float> : mb3::k3_evolve<0, double>)
                      : d == 1 ? (f ? mb3::k3_evolve<1, float> : mb3::k3_evolve<1, double>)
                               : (f ? mb3::k3_evolve<2, float> : mb3::k3_evolve<2, double>);
    const auto flux = d == 0 ? (f ? mb3::k3_flux<0, float> : mb3::k3_flux<0, double>)
                    : d == 1 ? (f ? mb3::k3_flux<1, float> : mb3::k3_flux<1, double>)
                             : (f ? mb3::k3_flux<2, float> : mb3::k3_flux<2, double>);
    const auto update = d == 0 ? mb3::k3_update<0> : d == 1 ? mb3::k3_update<1> : mb3::k3_update<2>;
    evolve<<<nblk(D.n), 256, 0, s->st>>>(D, nal);
    cudaEventRecord(s->ev0, s->st);
    flux<<<nblk((long long)nfl * nlines), 256, 0, s->st>>>(D, nal, nfl, nlines);
    cudaEventRecord(s->ev1, s->st);
    update<<<nblk(D.n), 256, 0, s->st>>>(D, nal, nfl);
    if (rc > 0) {
        mb3::k3_evprep<<<nblk((long long)rc), 256, 0, s->st>>>(D);
        mb3::k3_events<<<nblk((long long)rc), 256, 0, s->st>>>(D);
    }
    if (rc > 0) mb3::k3_bad<<<nblk((long long)rc), 256, 0, s->st>>>(D);
    mb3::k3_mix<<<1, mb3::MIXS_THREADS, 0, s->st>>>(D);
    mb3::k3_final<<<nblk(D.n), 256, 0, s->st>>>(D);
    int w = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->wall_host, D.wall, NC * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s->merged, D.mixed, sizeof(int), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w, D.err, sizeof(int), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_sweep");
    s->prev_ok = true;
    for (int a = 0; a < 3; ++a) { s->q0[a] = r0[a]; s->qn[a] = rn[a]; }
    cudaEventElapsedTime(&s->flux_ms, s->ev0, s->ev1);
    s->T[d] = TB[d];
    if (++s->sidx == 3) {
        s->sidx = 0;
        s->t += dt;
        s->step++;
    }
    return err_status(s, w);
}

mb_status mb3_cfl_dt(mb3_sim *s, double *dt) {
    if (!s || !dt) return MB_E_INVAL;
    double sm[3] = {0, 0, 0};
    cudaError_t e = cudaMemsetAsync(s->D.smax, 0, 3 * sizeof(double), s->st);
    const unsigned nb = std::min(nblk(s->D.n), 152u * 8u);
    if (e == cudaSuccess && s->D.f32) mb3::k3_speeds<float><<<nb, 256, 0, s->st>>>(s->D);
    else if (e == cudaSuccess) mb3::k3_speeds<double><<<nb, 256, 0, s->st>>>(s->D);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(sm, s->D.smax, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_cfl_dt");
    double r = 1e300;
    for (int a = 0; a < 3; ++a) {
        double S = sm[a];
        if (s->nplane > 0) S = std::max(S, std::fabs(s->D.U[a]));
        if (S <= 0.0) S = 1e-300;
        r = std::min(r, s->D.h[a] / S);
    }
    *dt = s->cfl * r;
    return MB_OK;
}

mb_status mb3_step(mb3_sim *s, double dt, double *dt_used) {
    if (!s) return MB_E_INVAL;
    if (s->sidx != 0) return fail3(s, MB_E_STATE, "mb3_step in the middle of a step");
    if (!(dt > 0.0)) {
        const mb_status r = mb3_cfl_dt(s, &dt);
        if (r != MB_OK) return r;
    }
    if (dt_used) *dt_used = dt;
    const bool odd = s->step & 1;
    mb_status first = MB_OK;
    for (int m = 0; m < 3; ++m) {
        const mb_status r = mb3_sweep(s, odd ? 2 - m : m, dt);
        if (r != MB_OK && first == MB_OK) first = r;
        if (r == MB_E_CUDA || r == MB_E_NOMEM || r == MB_E_INVAL || r == MB_E_STATE) return r;
    }
    return first;
}

mb_status mb3_last_sweep(mb3_sim *s, double *wall, int *merged) {
    if (!s) return MB_E_INVAL;
    if (wall) for (int q = 0; q < NC; ++q) wall[q] = s->wall_host[q];
    if (merged) *merged = s->merged;
    return MB_OK;
}

mb_status mb3_set_precision(mb3_sim *s, int precision) {
    if (!s || (precision != MB_FP64 && precision != MB_FP32)) return MB_E_INVAL;
    if (s->sidx != 0) return fail3(s, MB_E_STATE, "mb3_set_precision in the middle of a step");
    cudaError_t e = cudaSuccess;
    if (precision == MB_FP32 && !s->D.Qf) e = dalloc(s, &s->D.Qf, NC * (size_t)s->D.n);
    if (e != cudaSuccess) return cuda3(s, e, "mb3_set_precision");
    s->D.f32 = precision == MB_FP32;
    if (s->D.f32) mb3::k3_to_f32<<<nblk(s->D.n), 256, 0, s->st>>>(s->D);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    return cuda3(s, e, "mb3_set_precision");
}

mb_status mb3_flux_time(mb3_sim *s, double *ms) {
    if (!s || !ms) return MB_E_INVAL;
    *ms = s->flux_ms;
    return MB_OK;
}

}  // extern "C"
