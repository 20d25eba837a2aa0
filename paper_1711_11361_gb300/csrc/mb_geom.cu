// mb_geom.cu -- per-sweep cut-cell geometry of the moving body
// (arXiv 1711.11361, Sec. II.A volume fractions, Sec. II.B apertures and
// shielded distance, Sec. II.C.4 time-averaged apertures, normal and
// distance).  Compiled without FMA contraction so that node coordinates,
// posed vertices and the touch predicate are bit-reproducible.
//
// Layout: one warp per grid column of the body's bounding box.  The warp
// gathers the polygon edges overlapping its column into shared memory and
// evaluates every rectangle area with Green's theorem,
//   area(R ∩ body) = Σ_edges ∫_{e∩R} (x - x_o) dy + |x_s - x_o| · L(x_s),
// where x_s is the side of R on a grid line, x_o the opposite side and L the
// solid length of the segment on x_s (a sum over the few edges crossing that
// line).  Only edges meeting R enter, so no far-away edge is ever integrated.
#include "mb_internal.cuh"

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace mb {

constexpr int GEOM_WARPS = 4;
constexpr int EMAX = 192;           // edges per column and pose
constexpr int LMAX = 32;            // crossings per grid line of a column
constexpr int MAXROWWORDS = 256;    // ny <= 8192

// edges of one column at one pose, in polygon order
struct GeoBuf {
    double xa[EMAX], ya[EMAX], xb[EMAX], yb[EMAX];
    double ovl[EMAX];                 // x-overlap with the column
    short jlo[EMAX], jhi[EMAX];       // rows the edge may meet (widened x-range)
    unsigned char mov[EMAX];
    double lyc[2][LMAX];              // crossings of the grid lines x_l (0) and x_r (1)
    signed char ls[2][LMAX];          // +1 edge runs to +x (body above), -1 otherwise
    unsigned char lf[2][LMAX];        // bit0: crossing from the left, bit1: from the right
    int lcnt[2];
    int cnt;
};

struct GeoWarp {
    GeoBuf G;
    unsigned bA[MAXROWWORDS], bB[MAXROWWORDS], bM[MAXROWWORDS];
    int wpre[MAXROWWORDS + 1];
};

// Comparisons of finite doubles on integer keys.  On GB300 every FP64
// instruction, compares, min/max and selects included, takes the SM's narrow
// FP64 pipe; the geometry's decisions run on the integer pipes instead, with
// the same results (-0 and +0 compare equal, as in IEEE comparisons).  The
// key of -0 is that of +0; other doubles keep their bits, negative ones with
// the magnitude bits inverted, so that signed 64-bit order is double order.
__device__ __forceinline__ long long dk(double v) {
    long long b = __double_as_longlong(v);
    b = (b == (long long)0x8000000000000000ull) ? 0ll : b;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ bool dlt(double a, double b) { return dk(a) < dk(b); }
__device__ __forceinline__ bool dle(double a, double b) { return dk(a) <= dk(b); }
__device__ __forceinline__ bool deq(double a, double b) { return dk(a) == dk(b); }
__device__ __forceinline__ bool dneg(double a) { return dk(a) < 0; }       // a < 0
__device__ __forceinline__ bool dpos(double a) { return dk(a) > 0; }       // a > 0
__device__ __forceinline__ bool dzero(double a) { return (__double_as_longlong(a) << 1) == 0; }   // a == 0
__device__ __forceinline__ double dmin(double a, double b) { return dlt(a, b) ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return dlt(b, a) ? a : b; }
__device__ __forceinline__ double clamp01(double a) { return dneg(a) ? 0.0 : (dlt(1.0, a) ? 1.0 : a); }

// ---------------------------------------------------------------------------
// K0: time step, poses of the sweep, posed vertices, conservative FP32 x
// bounds of every edge, column and row range of the body.  POSE_PARTS CTAs
// per instance share its vertices; each computes the time step and poses
// (the same arithmetic), CTA 0 stores them, and the last CTA to finish turns
// the merged extent into the column and row ranges.
// ---------------------------------------------------------------------------
constexpr int POSE_PARTS = 8;

// order-preserving 64-bit key of a double (and back)
__device__ __forceinline__ unsigned long long dkey(double v) {
    const long long b = __double_as_longlong(v);
    return (unsigned long long)(b ^ ((b >> 63) & 0x7fffffffffffffffLL)) ^ 0x8000000000000000ull;
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    const unsigned long long u = k ^ 0x8000000000000000ull;
    return __longlong_as_double((long long)(u ^ (((long long)u >> 63) & 0x7fffffffffffffffLL)));
}

__global__ void k_pose(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, const double *__restrict__ vx,
                       const double *__restrict__ vy, const unsigned char *__restrict__ vmov,
                       const int *__restrict__ vnext, double *__restrict__ px, double *__restrict__ py,
                       float *__restrict__ ebox, int total_v, int dir, int sidx, double dt_host,
                       int *__restrict__ defer_count) {
    const int inst = blockIdx.x / POSE_PARTS, part = blockIdx.x % POSE_PARTS;
    // the sweep's list of deferred bulk cell pairs starts empty (its readers
    // of the sweep before have finished; its writers of this sweep follow)
    if (blockIdx.x == 0 && threadIdx.x == 0 && defer_count) *defer_count = 0;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    __shared__ double sh[16];
    __shared__ int last_cta;
    if (threadIdx.x == 0) {
        double dt;
        if (sidx == 0) {
            if (dt_host > 0.0) {
                dt = dt_host;
            } else {
                double Sx = __longlong_as_double((long long)y.S[0]);
                double Sy = __longlong_as_double((long long)y.S[1]);
                Sx = fmax(Sx, I.wall_bound[0]);
                Sy = fmax(Sy, I.wall_bound[1]);
                if (Sx <= 0.0) Sx = 1e-300;
                if (Sy <= 0.0) Sy = 1e-300;
                dt = I.cfl * fmin(I.dx / Sx, I.dy / Sy);
            }
        } else {
            dt = y.dt;
        }
        const double tA = y.t + (sidx == 0 ? 0.0 : 0.5 * dt);
        const double tB = y.t + (sidx == 0 ? 0.5 * dt : dt);
        const double tM = y.t + (sidx == 0 ? 0.25 * dt : 0.75 * dt);
        double thA = 0.0, thB = 0.0, thM = 0.0, Om = 0.0;
        if (I.rotating) {
            thA = I.a0 + I.a1 * sin(I.omega * tA);
            thB = I.a0 + I.a1 * sin(I.omega * tB);
            thM = I.a0 + I.a1 * sin(I.omega * tM);
            Om = I.a1 * I.omega * cos(I.omega * tM);
        }
        const double delta = I.U[dir] * dt;
        double cA = 1.0, sA = 0.0, cB = 1.0, sB = 0.0, cM = 1.0, sM = 0.0;   // identity for a translating body
        if (I.rotating) {
            sincos(thA, &sA, &cA);
            sincos(thB, &sB, &cB);
            sincos(thM, &sM, &cM);
        }
        const double XA = y.X, YA = y.Y;
        const double XB = dir == 0 ? y.X + delta : y.X, YB = dir == 1 ? y.Y + delta : y.Y;
        const double XM = dir == 0 ? y.X + 0.5 * delta : y.X, YM = dir == 1 ? y.Y + 0.5 * delta : y.Y;
        if (part == 0) {
            if (sidx == 0) {
                y.dt = dt;
            } else {
                if (dt_host > 0.0 && dt_host != dt) y.err |= ERR_STATE;
                // the last sweep of the step gathers the wave speeds of the next step's dt
                y.S[0] = 0ull;
                y.S[1] = 0ull;
            }
            y.lam = dt / (dir == 0 ? I.dx : I.dy);
            y.lamf = (float)y.lam;
            y.delta = delta;
            // the concurrent bulk pass may update a cell before this sweep's
            // geometry is known only when the body moves by less than a cell
            // along the sweep and does not rotate (its band then lies within one
            // cell, along the sweep, of the cells touched at the start pose)
            y.defer_all = (I.serial_bulk || I.rotating || fabs(delta) >= 0.9 * (dir == 0 ? I.dx : I.dy)) ? 1 : 0;
            y.XA = XA; y.YA = YA; y.XB = XB; y.YB = YB; y.XM = XM; y.YM = YM;
            y.thA = thA; y.thB = thB; y.thM = thM;
            y.cA = cA; y.sA = sA; y.cB = cB; y.sB = sB; y.cM = cM; y.sM = sM;
            y.Om = Om;
            y.band_count = 0;
            y.nbad = 0;
            y.nbadlist = 0;
            y.nbulk = 0;
            y.mixed = 0;
            for (int q = 0; q < MAXC; ++q) y.wall_sum[q] = 0.0;
        }
        sh[0] = XA; sh[1] = YA; sh[2] = XM; sh[3] = YM; sh[4] = XB; sh[5] = YB;
        sh[6] = cA; sh[7] = sA; sh[8] = cM; sh[9] = sM; sh[10] = cB; sh[11] = sB;
    }
    __syncthreads();
    // posed position of vertex a at pose P (0: A, 1: M, 2: B)
    auto posed = [&](int a, int P, double &xo, double &yo) {
        const double x0 = vx[a], y0 = vy[a];
        const double X = sh[2 * P], Yy = sh[2 * P + 1], c = sh[6 + 2 * P], s = sh[7 + 2 * P];
        if (!vmov[a]) {
            xo = x0; yo = y0;
        } else if (I.rotating) {
            double ddx = x0 - I.pivot[0], ddy = y0 - I.pivot[1];
            double rx = c * ddx - s * ddy;
            double ry = s * ddx + c * ddy;
            xo = (I.pivot[0] + rx) + X;
            yo = (I.pivot[1] + ry) + Yy;
        } else {
            xo = x0 + X;
            yo = y0 + Yy;
        }
    };
    // extent as order-preserving integer keys (minima complemented): integer
    // compares and shuffles instead of FP64 ones
    unsigned long long kx0 = 0ull, kx1 = 0ull, ky0 = 0ull, ky1 = 0ull;
    for (int k = part * blockDim.x + threadIdx.x; k < I.nv; k += POSE_PARTS * blockDim.x) {
        const int a = I.voff + k, b = vnext[a];
        for (int P = 0; P < 3; ++P) {
            double xo, yo, xb, yb;
            posed(a, P, xo, yo);
            posed(b, P, xb, yb);
            px[(size_t)P * total_v + a] = xo;
            py[(size_t)P * total_v + a] = yo;
            const unsigned long long kxa = dkey(xo), kya = dkey(yo), kxb = dkey(xb);
            kx0 = max(kx0, ~kxa); kx1 = max(kx1, kxa);
            ky0 = max(ky0, ~kya); ky1 = max(ky1, kya);
            // conservative FP32 x-range of edge a -> b (rounded outward)
            const bool alo = kxa <= kxb;
            ebox[((size_t)P * total_v + a) * 2] = __double2float_rd(alo ? xo : xb);
            ebox[((size_t)P * total_v + a) * 2 + 1] = __double2float_ru(alo ? xb : xo);
        }
    }
    __shared__ unsigned long long kred[4][32];
    for (int o = 16; o > 0; o >>= 1) {
        kx0 = max(kx0, __shfl_xor_sync(0xffffffffu, kx0, o));
        kx1 = max(kx1, __shfl_xor_sync(0xffffffffu, kx1, o));
        ky0 = max(ky0, __shfl_xor_sync(0xffffffffu, ky0, o));
        ky1 = max(ky1, __shfl_xor_sync(0xffffffffu, ky1, o));
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { kred[0][w] = kx0; kred[1][w] = kx1; kred[2][w] = ky0; kred[3][w] = ky1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            kx0 = max(kx0, kred[0][k]); kx1 = max(kx1, kred[1][k]);
            ky0 = max(ky0, kred[2][k]); ky1 = max(ky1, kred[3][k]);
        }
        if (kx1) {   // this CTA posed vertices
            atomicMax(&y.bbkey[0], kx0);
            atomicMax(&y.bbkey[1], kx1);
            atomicMax(&y.bbkey[2], ky0);
            atomicMax(&y.bbkey[3], ky1);
        }
        __threadfence();
        last_cta = atomicAdd(&y.pose_done, 1) == POSE_PARTS - 1;
    }
    __syncthreads();
    if (last_cta && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long k0 = atomicExch(&y.bbkey[0], 0ull), k1 = atomicExch(&y.bbkey[1], 0ull);
        const unsigned long long k2 = atomicExch(&y.bbkey[2], 0ull), k3 = atomicExch(&y.bbkey[3], 0ull);
        y.pose_done = 0;
        const double xmin = dkey_inv(~k0), xmax = dkey_inv(k1);
        const double ymin = dkey_inv(~k2), ymax = dkey_inv(k3);
        int c0 = (int)floor(fmax((xmin - I.x0) / I.dx, -4.0)) - 1;
        int c1 = (int)floor(fmin((xmax - I.x0) / I.dx, (double)I.nx + 4.0)) + 1;
        int r0 = (int)floor(fmax((ymin - I.y0) / I.dy, -4.0)) - 1;
        int r1 = (int)floor(fmin((ymax - I.y0) / I.dy, (double)I.ny + 4.0)) + 1;
        if (I.nv == 0) { c0 = 1; c1 = 0; r0 = 1; r1 = 0; }
        if (c0 < 0) c0 = 0;
        if (c1 > I.nx - 1) c1 = I.nx - 1;
        if (r0 < 0) r0 = 0;
        if (r1 > I.ny - 1) r1 = I.ny - 1;
        if (c1 - c0 + 1 > I.gcol_max) { c1 = c0 + I.gcol_max - 1; atomicOr(&y.err, ERR_EDGE_CAP); }
        y.col0 = c0;
        y.col1 = c1;
        y.row0 = r0;
        y.row1 = r1;
    }
}

// ---------------------------------------------------------------------------
// rows of an edge inside the x-range [X0, X1]
// ---------------------------------------------------------------------------
// y-extent of an edge inside the closed x-range [xl, xr]; false if disjoint
__device__ __forceinline__ bool edge_yrange(double xa, double ya, double xb, double yb, double xl, double xr,
                                            double *elo, double *ehi) {
    double lo = dmin(xa, xb), hi = dmax(xa, xb);
    if (hi < xl || lo > xr) return false;
    double e0, e1;
    if (xa == xb) {
        e0 = ya; e1 = yb;
    } else {
        double xc0 = lo > xl ? lo : xl;
        double xc1 = hi < xr ? hi : xr;
        double slope = (yb - ya) / (xb - xa);
        e0 = (xc0 == xa) ? ya : ((xc0 == xb) ? yb : ya + (xc0 - xa) * slope);
        e1 = (xc1 == xa) ? ya : ((xc1 == xb) ? yb : ya + (xc1 - xa) * slope);
    }
    *elo = dmin(e0, e1);
    *ehi = dmax(e0, e1);
    return true;
}

__device__ __forceinline__ int row_floor(const InstDesc &I, double yv) {
    double f = (yv - I.y0) * I.rdy;
    f = fmin(fmax(f, -4.0), (double)I.ny + 4.0);
    return (int)floor(f);
}

// ---------------------------------------------------------------------------
// warp-cooperative gather of the edges overlapping [gxl, gxr] at pose P; marks
// the rows whose closed cell of column [xl, xr] an edge meets (touch bits)
// ---------------------------------------------------------------------------
__device__ void gather(GeoBuf &G, const InstDesc &I, const double *__restrict__ px, const double *__restrict__ py,
                       const float *__restrict__ ebox, const int *__restrict__ vnext,
                       const unsigned char *__restrict__ vmov, int P, int total_v, double xl, double xr, double gxl,
                       double gxr, unsigned *touch, int lane, int *err) {
    const double *PX = px + (size_t)P * total_v, *PY = py + (size_t)P * total_v;
    const float *EB = ebox + (size_t)P * total_v * 2;
    const float fl = __double2float_rd(gxl), fr = __double2float_ru(gxr);
    int cnt = 0, lc0 = 0, lc1 = 0;
    for (int base = 0; base < I.nv; base += 32) {
        const int k = base + lane;
        const int a = I.voff + k;
        bool take = false;
        if (k < I.nv) take = EB[2 * a + 1] >= fl && EB[2 * a] <= fr;
        const unsigned m = __ballot_sync(0xffffffffu, take);
        double xa = 0, ya = 0, xb = 0, yb = 0;
        bool c0 = false, c1 = false;
        if (take) {
            const int b = vnext[a];
            xa = PX[a]; ya = PY[a]; xb = PX[b]; yb = PY[b];
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            const double lo = dmin(xa, xb), hi = dmax(xa, xb);
            if (pos < EMAX) {
                G.xa[pos] = xa; G.ya[pos] = ya; G.xb[pos] = xb; G.yb[pos] = yb;
                G.mov[pos] = vmov[a];
                G.ovl[pos] = dmax(0.0, dmin(xr, hi) - dmax(xl, lo));
                double elo, ehi;
                if (edge_yrange(xa, ya, xb, yb, gxl, gxr, &elo, &ehi)) {
                    G.jlo[pos] = (short)(row_floor(I, elo) - 1);
                    G.jhi[pos] = (short)(row_floor(I, ehi) + 1);
                } else {
                    G.jlo[pos] = 1;
                    G.jhi[pos] = 0;
                }
            }
            if (touch) {
                double elo, ehi;
                if (edge_yrange(xa, ya, xb, yb, xl, xr, &elo, &ehi)) {
                    int jl = row_floor(I, elo) - 1, jh = row_floor(I, ehi) + 1;
                    if (jl < 0) jl = 0;
                    if (jh > I.ny - 1) jh = I.ny - 1;
                    for (int j = jl; j <= jh; ++j) {
                        double ybj = node_coord(I.y0, j, I.dy), ytj = node_coord(I.y0, j + 1, I.dy);
                        if (ehi >= ybj && elo <= ytj) atomicOr(&touch[j >> 5], 1u << (j & 31));
                    }
                }
            }
            c0 = xa != xb && lo <= xl && xl <= hi;
            c1 = xa != xb && lo <= xr && xr <= hi;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, c0), m1 = __ballot_sync(0xffffffffu, c1);
        for (int L = 0; L < 2; ++L) {
            const bool c = L == 0 ? c0 : c1;
            const unsigned mm = L == 0 ? m0 : m1;
            int &lc = L == 0 ? lc0 : lc1;
            if (c) {
                const int p = lc + __popc(mm & ((1u << lane) - 1u));
                if (p < LMAX) {
                    const double xs = L == 0 ? xl : xr;
                    const double lo = dmin(xa, xb), hi = dmax(xa, xb);
                    G.lyc[L][p] = ya + (xs - xa) * (yb - ya) / (xb - xa);
                    G.ls[L][p] = xa < xb ? 1 : -1;
                    G.lf[L][p] = (unsigned char)((lo < xs ? 1 : 0) | (xs < hi ? 2 : 0));
                }
            }
            lc += __popc(mm);
        }
        cnt += __popc(m);
    }
    if (cnt > EMAX || lc0 > LMAX || lc1 > LMAX) {
        if (lane == 0) *err |= ERR_EDGE_CAP;
    }
    if (lane == 0) {
        G.cnt = cnt < EMAX ? cnt : EMAX;
        G.lcnt[0] = lc0 < LMAX ? lc0 : LMAX;
        G.lcnt[1] = lc1 < LMAX ? lc1 : LMAX;
    }
    __syncwarp();
}

// solid length of {x_L} x [y0r, y1r] (L = 0: x_l, 1: x_r); left_limit takes
// crossings as seen from the left of the line (min < x <= max)
__device__ __forceinline__ double line_solid_v(const GeoBuf &G, int L, double y0r, double y1r, bool left_limit) {
    double s = 0.0;
    const unsigned char want = left_limit ? 1 : 2;
    for (int e = 0; e < G.lcnt[L]; ++e) {
        if (!(G.lf[L][e] & want)) continue;
        double yc = G.lyc[L][e];
        double cl = yc < y0r ? y0r : (yc > y1r ? y1r : yc);
        s += (double)G.ls[L][e] * (y1r - cl);
    }
    return s;
}

// solid length of [x_l, x_r] x {y_f} (y_f = y_jf): edges below the row
// band contribute their whole overlap, the others the part below y_f
__device__ double line_solid_h(const GeoBuf &G, double xl, double xr, double yf, int jf) {
    double L = 0.0;
    for (int e = 0; e < G.cnt; ++e) {
        const double s = G.xa[e] < G.xb[e] ? 1.0 : -1.0;
        if (G.jhi[e] < jf - 1) { L += s * G.ovl[e]; continue; }
        if (G.jlo[e] > jf) continue;
        const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e], yb = G.yb[e];
        const double p = dmax(xl, dmin(xa, xb)), q = dmin(xr, dmax(xa, xb));
        if (!(q > p)) continue;
        const double k = (yb - ya) / (xb - xa);
        const double yp = ya + (p - xa) * k, yq = ya + (q - xa) * k;
        double m;
        if (yp < yf && yq < yf) m = q - p;
        else if (!(yp < yf) && !(yq < yf)) m = 0.0;
        else {
            double xs = p + (q - p) * ((yf - yp) / (yq - yp));
            xs = xs < p ? p : (xs > q ? q : xs);
            m = yp < yf ? xs - p : q - xs;
        }
        L += s * m;
    }
    return L;
}

// sum over the edges meeting [rx0,rx1]x[ry0,ry1] (candidates: rows ja..jb) of
// the integral of (x - xo) dy along the clipped edge; vertical edges on the
// grid side xs are skipped.  Optionally accumulates the wall normal times
// length (into the body: (-dy, dx) of the clipped pieces) and whether a
// moving edge meets the closed rectangle.
__device__ double rect_edges(const GeoBuf &G, int ja, int jb, double rx0, double rx1, double ry0, double ry1,
                             double xo, double xs, double *nlx, double *nly, bool *mov) {
    const double lx0 = rx0 - xo, lx1 = rx1 - xo, ly1 = ry1 - ry0;
    double A = 0.0;
    for (int e = 0; e < G.cnt; ++e) {
        if (G.jhi[e] < ja || G.jlo[e] > jb) continue;
        const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e], yb = G.yb[e];
        if (dmax(ya, yb) < ry0 || dmin(ya, yb) > ry1 || dmax(xa, xb) < rx0 || dmin(xa, xb) > rx1) continue;
        const double ax = xa - xo, ay = ya - ry0, bx = xb - xo, by = yb - ry0;
        const double ddx = bx - ax, ddy = by - ay;
        double t0 = 0.0, t1 = 1.0;
        bool ok = true;
        const double pp[4] = {-ddx, ddx, -ddy, ddy};
        const double qq[4] = {ax - lx0, lx1 - ax, ay, ly1 - ay};
        for (int k = 0; k < 4; ++k) {
            if (pp[k] == 0.0) {
                if (qq[k] < 0.0) ok = false;
                continue;
            }
            const double r = qq[k] / pp[k];
            if (pp[k] < 0.0) t0 = dmax(t0, r);
            else t1 = dmin(t1, r);
        }
        if (!ok || t1 < t0) continue;
        if (mov && G.mov[e]) *mov = true;
        if (xa == xb && xa == xs) continue;   // vertical edge on the grid side
        if (!(t1 > t0)) continue;
        const double xc0 = ax + t0 * ddx, xc1 = ax + t1 * ddx;
        A += ddy * (t1 - t0) * (0.5 * (xc0 + xc1));
        if (nlx) {
            *nlx -= ddy * (t1 - t0);
            *nly += ddx * (t1 - t0);
        }
    }
    return A;
}

__device__ __forceinline__ double cell_alpha(const GeoBuf &G, const InstDesc &I, int j, double xl, double xr,
                                             double yb, double yt, double *nlx, double *nly, bool *mov) {
    double A = rect_edges(G, j, j, xl, xr, yb, yt, xl, xr, nlx, nly, mov) + (xr - xl) * line_solid_v(G, 1, yb, yt, true);
    double a = clamp01(1.0 - A / (I.dx * I.dy));
    return a < ALPHA_MIN ? 0.0 : a;
}

// fluid fraction of the strip between a grid line and its copy displaced by
// w (>0: to the right / up); `line` is 0 (x_l) or 1 (x_r) for vertical strips
__device__ double strip_beta_x(const GeoBuf &G, const InstDesc &I, int j, int line, double xs, double w, double yb,
                               double yt) {
    if (w > 0.0) {   // [xs, xs + w]: grid side on the left, crossings seen from the right
        double x1 = xs + w;
        double A = rect_edges(G, j, j, xs, x1, yb, yt, x1, xs, nullptr, nullptr, nullptr) +
                   (x1 - xs) * line_solid_v(G, line, yb, yt, false);
        return clamp01(1.0 - A / ((x1 - xs) * I.dy));
    }
    double x0 = xs + w;   // [xs - |w|, xs]: grid side on the right
    double A = rect_edges(G, j, j, x0, xs, yb, yt, x0, xs, nullptr, nullptr, nullptr) +
               (xs - x0) * line_solid_v(G, line, yb, yt, true);
    return clamp01(1.0 - A / ((xs - x0) * I.dy));
}

__device__ double strip_beta_y(const GeoBuf &G, const InstDesc &I, int j, double xl, double xr, double ys, double w) {
    double y0 = w > 0.0 ? ys : ys + w, y1 = w > 0.0 ? ys + w : ys;
    int ja = w > 0.0 ? j : j - 1, jb = w > 0.0 ? j + 1 : j;
    double A = rect_edges(G, ja, jb, xl, xr, y0, y1, xl, xr, nullptr, nullptr, nullptr) +
               (xr - xl) * line_solid_v(G, 1, y0, y1, true);
    return clamp01(1.0 - A / ((y1 - y0) * I.dx));
}

// instantaneous aperture of a face of cell (i, j) along dir: hi != 0 -> the
// high face (x_r or y_t), else the low face
__device__ __forceinline__ double face_ap(const GeoBuf &G, const InstDesc &I, int dir, bool hi, int j, double xl,
                                          double xr, double yb, double yt) {
    if (dir == 0) return clamp01(1.0 - line_solid_v(G, hi ? 1 : 0, yb, yt, true) / I.dy);
    return clamp01(1.0 - line_solid_h(G, xl, xr, hi ? yt : yb, hi ? j + 1 : j) / I.dx);
}

// time-averaged aperture (translation: exact swept strip, evaluated with the
// body at the end pose B, where the strip of the start pose appears shifted
// by the translation) of the face owned by the cell (own_hi: high face) or of
// its domain-boundary face (boundary: the face it does not own)
__device__ double swept_face_B(const GeoBuf &G, const InstDesc &I, int dir, double delta, bool hi, int j, double xl,
                               double xr, double yb, double yt) {
    if (delta == 0.0) return face_ap(G, I, dir, hi, j, xl, xr, yb, yt);
    if (dir == 0) return strip_beta_x(G, I, j, hi ? 1 : 0, hi ? xr : xl, delta, yb, yt);
    return strip_beta_y(G, I, j, xl, xr, hi ? yt : yb, delta);
}

// ---------------------------------------------------------------------------
// K1: band records (cells touched by the body at the start or end pose, or
// the middle pose when rotating) with their geometry.  One CTA per group of
// GC adjacent columns: warp 0 gathers the edges near the group, every band
// cell of the group gets a thread, and each column keeps a bit list of the
// edges that can meet its cells.
// ---------------------------------------------------------------------------
constexpr int GC = GEO_GC;          // columns per group
constexpr int EMAXG = 384;          // edges per group and pose
constexpr int LMAXG = 32;           // crossings per grid line
constexpr int NWB = 64;             // bitmap words per column (2048 rows of the body's extent)
constexpr int GEOMG_THREADS = 256;  // one CTA per group; its warps share the group's edges
constexpr int EWORDS = EMAXG / 32;  // words of a column's edge bit list

struct GeoBufG {
    double xa[EMAXG], ya[EMAXG], xb[EMAXG], yb[EMAXG];
    double slope[EMAXG];            // (yb - ya) / (xb - xa)
    double idx[EMAXG], idy[EMAXG];  // 1 / (xb - xa), 1 / (yb - ya) (0 if the difference is 0)
    float fx0[EMAXG], fx1[EMAXG], fy0[EMAXG], fy1[EMAXG];   // bounding box rounded outward
    short jlo[EMAXG], jhi[EMAXG];   // rows the edge may meet
    short ilo[EMAXG], ihi[EMAXG];   // columns whose widened range the edge may meet
    unsigned char mov[EMAXG];
    unsigned char pc0[EMAXG];       // first group column the edge's x-range may meet
    int pp[EMAXG + 1];              // prefix over edges of their (edge, column) pairs
    int npair;
    unsigned chm[GEOMG_THREADS / 4];      // gather: take masks of a batch of vertex chunks
    int chp[GEOMG_THREADS / 4 + 1];       // gather: their exclusive prefix
    unsigned cm[GC][EWORDS];        // per column: edges whose candidate columns contain it
    unsigned lm[GC + 1][EWORDS];    // per grid line: edges crossing it
    double xln[GC + 1];             // x of the grid lines x_{i0} .. x_{i0+GC}
    double lyc[GC + 1][LMAXG];      // crossings of those grid lines
    signed char ls[GC + 1][LMAXG];
    unsigned char lf[GC + 1][LMAXG];
    int lcnt[GC + 1];
    int cnt;
};

struct GeoWarpG {
    GeoBufG G;
    unsigned bA[GC][NWB], bB[GC][NWB], bM[GC][NWB];
    int wpre[GC * NWB + 1];
};

__device__ __forceinline__ bool edge_yrange_s(double xa, double ya, double xb, double yb, double slope, double xl,
                                              double xr, double *elo, double *ehi) {
    const long long kxa = dk(xa), kxb = dk(xb), kxl = dk(xl), kxr = dk(xr);
    const bool alo = kxa < kxb;
    const double lo = alo ? xa : xb, hi = alo ? xb : xa;
    const long long klo = alo ? kxa : kxb, khi = alo ? kxb : kxa;
    if (khi < kxl || klo > kxr) return false;
    double e0, e1;
    if (kxa == kxb) {
        e0 = ya; e1 = yb;
    } else {
        const bool c0l = klo > kxl, c1h = khi < kxr;
        const double xc0 = c0l ? lo : xl;
        const double xc1 = c1h ? hi : xr;
        const long long kc0 = c0l ? klo : kxl, kc1 = c1h ? khi : kxr;
        e0 = (kc0 == kxa) ? ya : ((kc0 == kxb) ? yb : ya + (xc0 - xa) * slope);
        e1 = (kc1 == kxa) ? ya : ((kc1 == kxb) ? yb : ya + (xc1 - xa) * slope);
    }
    *elo = dmin(e0, e1);
    *ehi = dmax(e0, e1);
    return true;
}

// FP32 floors for candidate ranges (superset tests with a one-cell margin):
// the FP64 offset rounded to FP32 and scaled is within 0.01 cell of the exact
// position for grids up to 16384 cells
__device__ __forceinline__ int row_floor_f(const InstDesc &I, double yv) {
    float f = __double2float_rn(yv - I.y0) * I.rdyf;
    f = fminf(fmaxf(f, -4.0f), (float)I.ny + 4.0f);
    return (int)floorf(f);
}
__device__ __forceinline__ int col_floor_f(const InstDesc &I, double xv) {
    float f = __double2float_rn(xv - I.x0) * I.rdxf;
    f = fminf(fmaxf(f, -4.0f), (float)I.nx + 4.0f);
    return (int)floorf(f);
}

__device__ __forceinline__ int col_floor(const InstDesc &I, double xv) {
    double f = (xv - I.x0) * I.rdx;
    f = fmin(fmax(f, -4.0), (double)I.nx + 4.0);
    return (int)floor(f);
}

// all threads: the edges whose x-range meets the group's widened x-range at
// pose P, compacted into G in vertex order with their per-edge data.  The
// warps test batches of 32-vertex chunks against the FP32 x-bounds together;
// a prefix over the chunks' counts keeps the vertex order.
constexpr int GNW = GEOMG_THREADS / 32;     // warps per CTA
constexpr int GCPW = 8;                     // chunks per warp and batch
constexpr int GNCH = GNW * GCPW;            // chunks per batch
static_assert(GNCH == GEOMG_THREADS / 4, "chunk batch arrays of GeoBufG");
__device__ void gather_g(GeoBufG &G, const InstDesc &I, const double *__restrict__ px, const double *__restrict__ py,
                         const float *__restrict__ ebox, const int *__restrict__ vnext,
                         const unsigned char *__restrict__ vmov, int P, int total_v, int i0, int ncol, double ad,
                         int tid, int *err) {
    const int lane = tid & 31, warp = tid >> 5;
    const double *PX = px + (size_t)P * total_v, *PY = py + (size_t)P * total_v;
    const float2 *EB = (const float2 *)(ebox + (size_t)P * total_v * 2) + I.voff;
    if (tid <= ncol) G.xln[tid] = I.xn[i0 + tid];
    __syncthreads();
    const double gxl = G.xln[0] - ad, gxr = G.xln[ncol] + ad;
    const float fl = __double2float_rd(gxl), fr = __double2float_ru(gxr);
    int cnt = 0;
    for (int b0 = 0; b0 < I.nv; b0 += 32 * GNCH) {
        float2 eb[GCPW];
#pragma unroll
        for (int u = 0; u < GCPW; ++u) {
            const int k = b0 + (warp + u * GNW) * 32 + lane;
            eb[u] = k < I.nv ? EB[k] : make_float2(1.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < GCPW; ++u) {
            const int k = b0 + (warp + u * GNW) * 32 + lane;
            const bool take = k < I.nv && eb[u].y >= fl && eb[u].x <= fr;
            const unsigned m = __ballot_sync(0xffffffffu, take);
            if (lane == 0) G.chm[warp + u * GNW] = m;
        }
        __syncthreads();
        if (warp == 0) {   // exclusive prefix of the chunks' counts
            int run = 0;
            for (int q0 = 0; q0 < GNCH; q0 += 32) {
                const int c = __popc(G.chm[q0 + lane]);
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                G.chp[q0 + lane] = run + incl - c;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) G.chp[GNCH] = run;
        }
        __syncthreads();
        for (int u = 0; u < GCPW; ++u) {
            const int q = warp + u * GNW;
            const unsigned m = G.chm[q];
            if (!((m >> lane) & 1u)) continue;
            const int k = b0 + q * 32 + lane;
            const int a = I.voff + k;
            const int pos = cnt + G.chp[q] + __popc(m & ((1u << lane) - 1u));
            if (pos >= EMAXG) continue;
            const int b = vnext[a];
            const double xa = PX[a], ya = PY[a], xb = PX[b], yb = PY[b];
            const double rx = xa != xb ? 1.0 / (xb - xa) : 0.0;
            const double sl = (yb - ya) * rx;
            const double lo = dmin(xa, xb), hi = dmax(xa, xb);
            G.xa[pos] = xa; G.ya[pos] = ya; G.xb[pos] = xb; G.yb[pos] = yb;
            G.slope[pos] = sl;
            G.idx[pos] = rx;
            G.idy[pos] = ya != yb ? 1.0 / (yb - ya) : 0.0;
            G.fx0[pos] = __double2float_rd(lo);
            G.fx1[pos] = __double2float_ru(hi);
            G.fy0[pos] = __double2float_rd(dmin(ya, yb));
            G.fy1[pos] = __double2float_ru(dmax(ya, yb));
            G.mov[pos] = vmov[a];
            double elo, ehi;
            if (edge_yrange_s(xa, ya, xb, yb, sl, gxl, gxr, &elo, &ehi)) {
                G.jlo[pos] = (short)(row_floor_f(I, elo) - 1);
                G.jhi[pos] = (short)(row_floor_f(I, ehi) + 1);
            } else {
                G.jlo[pos] = 1;
                G.jhi[pos] = 0;
            }
            G.ilo[pos] = (short)(col_floor_f(I, lo - ad) - 1);
            G.ihi[pos] = (short)(col_floor_f(I, hi + ad) + 1);
            // group columns whose closed x-range the edge may meet
            const int c0 = col_floor_f(I, lo) - 1 - i0, c1 = col_floor_f(I, hi) + 1 - i0;
            const int ca = c0 < 0 ? 0 : c0, cb = c1 > ncol - 1 ? ncol - 1 : c1;
            const int np = cb >= ca ? cb - ca + 1 : 0;
            G.pc0[pos] = (unsigned char)(np ? ca : 0);
            G.pp[pos] = np;
        }
        cnt += G.chp[GNCH];
        __syncthreads();
    }
    const int n = cnt < EMAXG ? cnt : EMAXG;
    if (warp == 0) {   // pair counts -> exclusive prefix over the edges
        int run = 0;
        for (int e0 = 0; e0 < n; e0 += 32) {
            const int e = e0 + lane;
            const int c = e < n ? G.pp[e] : 0;
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (e < n) G.pp[e] = run + incl - c;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            G.pp[n] = run;
            G.npair = run;
            G.cnt = n;
            if (cnt > EMAXG) *err |= ERR_EDGE_CAP;
        }
    }
    __syncthreads();
}

// all threads, after gather_g: per column the bit list of the edges whose
// candidate columns contain it, per grid line x_{i0+L} the bit list of the
// edges crossing it, and (bits != nullptr) the rows of each column whose
// closed cell an edge meets (exact predicate)
__device__ void index_g(GeoBufG &G, const InstDesc &I, int i0, int ncol, int row0, int nwb, unsigned (*bits)[NWB],
                        int tid) {
    const int n = G.cnt, nwd = (n + 31) >> 5;
    for (int p = tid; p < (2 * ncol + 1) * nwd; p += GEOMG_THREADS) {
        const int r = p / nwd, w = p - r * nwd;
        unsigned msk = 0u;
        if (r < ncol) {
            const int i = i0 + r;
            for (int b = 0; b < 32; ++b) {
                const int e = w * 32 + b;
                if (e < n && G.ilo[e] <= i && i <= G.ihi[e]) msk |= 1u << b;
            }
            G.cm[r][w] = msk;
        } else {
            const int L = r - ncol;
            const double xs = G.xln[L];
            const float fxs = (float)xs;
            unsigned cand = 0u;
            for (int b = 0; b < 32; ++b) {
                const int e = w * 32 + b;
                if (e < n && G.fx1[e] >= fxs && G.fx0[e] <= fxs) cand |= 1u << b;
            }
            for (; cand; cand &= cand - 1u) {
                const int b = __ffs(cand) - 1, e = w * 32 + b;
                const double xa = G.xa[e], xb = G.xb[e];
                const long long ka = dk(xa), kb = dk(xb), ks = dk(xs);
                if (ka != kb && (ka < kb ? (ka <= ks && ks <= kb) : (kb <= ks && ks <= ka))) msk |= 1u << b;
            }
            G.lm[L][w] = msk;
        }
    }
    if (!bits) return;
    // (edge, column) pairs whose x-ranges may meet, enumerated densely
    const int npair = G.npair;
    for (int p = tid; p < npair; p += GEOMG_THREADS) {
        int a = 0, b = n - 1;
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (G.pp[mid] <= p) a = mid; else b = mid - 1;
        }
        const int e = a, c = G.pc0[e] + (p - G.pp[e]);
        const double xl = G.xln[c], xr = G.xln[c + 1];
        double elo, ehi;
        if (!edge_yrange_s(G.xa[e], G.ya[e], G.xb[e], G.yb[e], G.slope[e], xl, xr, &elo, &ehi)) continue;
        const int jf0 = row_floor_f(I, elo), jf1 = row_floor_f(I, ehi);
        int jl = jf0 - 1, jh = jf1 + 1;
        if (jl < row0) jl = row0;
        if (jh > I.ny - 1) jh = I.ny - 1;
        if (jh > row0 + 32 * nwb - 1) jh = row0 + 32 * nwb - 1;
        for (int j = jl; j <= jh; ++j) {
            // rows jf0+1 .. jf1-1 lie strictly inside [elo, ehi] whatever the
            // rounding of the floors; the exact predicate decides the rest
            bool hit = j > jf0 && j < jf1;
            if (!hit) hit = dle(I.yn[j], ehi) && dle(elo, I.yn[j + 1]);
            if (hit) atomicOr(&bits[c][(j - row0) >> 5], 1u << ((j - row0) & 31));
        }
    }
}

// lanes 0..ncol of one warp, after index_g: the crossing lists of the grid
// lines in edge order (crossing y, direction, which side of the line the
// edge extends to)
__device__ void compact_lines_g(GeoBufG &G, int ncol, int lane, int *err) {
    if (lane <= GC) {
        int k = 0;
        if (lane <= ncol) {
            const int L = lane;
            const double xs = G.xln[L];
            const int nwd = (G.cnt + 31) >> 5;
            for (int w = 0; w < nwd; ++w)
                for (unsigned m = G.lm[L][w]; m; m &= m - 1u) {
                    const int e = w * 32 + __ffs(m) - 1;
                    if (k < LMAXG) {
                        const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e];
                        const double lo = dmin(xa, xb), hi = dmax(xa, xb);
                        G.lyc[L][k] = ya + (xs - xa) * G.slope[e];
                        G.ls[L][k] = xa < xb ? 1 : -1;
                        G.lf[L][k] = (unsigned char)((lo < xs ? 1 : 0) | (xs < hi ? 2 : 0));
                    }
                    ++k;
                }
            if (k > LMAXG) *err |= ERR_EDGE_CAP;
        }
        G.lcnt[lane] = k < LMAXG ? k : LMAXG;
    }
}

// loop over the edges on column c's bit list, in gather order; `continue` in
// the body moves to the next edge
#define FOR_COL_EDGES(G, c, e)                                                              \
    for (int e##_w = 0, e##_n = ((G).cnt + 31) >> 5; e##_w < e##_n; ++e##_w)                 \
        for (unsigned e##_m = (G).cm[c][e##_w]; e##_m; e##_m &= e##_m - 1u)                  \
            if (const int e = e##_w * 32 + __ffs(e##_m) - 1; true)

// resumable walk over column c's edge bit list.  The geometry queries first
// collect a lane's candidate edges with integer / FP32 tests (divergent but
// cheap), then run the FP64 arithmetic over the collected edges, so that the
// lanes of a warp execute the FP64 block together instead of once per edge
// any lane needs.
constexpr int SVN = 8;              // candidate edges collected per round
struct ColIter {
    int w, n;
    unsigned m;
};
__device__ __forceinline__ void col_iter_init(const GeoBufG &G, int c, ColIter &it) {
    it.n = (G.cnt + 31) >> 5;
    it.w = 0;
    it.m = it.n ? G.cm[c][0] : 0u;
}
__device__ __forceinline__ int col_iter_next(const GeoBufG &G, int c, ColIter &it) {
    while (it.m == 0u) {
        if (++it.w >= it.n) return -1;
        it.m = G.cm[c][it.w];
    }
    const int e = it.w * 32 + __ffs(it.m) - 1;
    it.m &= it.m - 1u;
    return e;
}

__device__ __forceinline__ double line_solid_vg(const GeoBufG &G, int L, double y0r, double y1r, bool left_limit) {
    double s = 0.0;
    const unsigned char want = left_limit ? 1 : 2;
    const long long k0 = dk(y0r), k1 = dk(y1r);
    for (int e = 0; e < G.lcnt[L]; ++e) {
        if (!(G.lf[L][e] & want)) continue;
        const double yc = G.lyc[L][e];
        const long long kc = dk(yc);
        const double cl = kc < k0 ? y0r : (kc > k1 ? y1r : yc);
        // crossing direction +-1: add or subtract the length (exact, as the product)
        if (G.ls[L][e] > 0) s += y1r - cl;
        else s -= y1r - cl;
    }
    return s;
}

// solid length of [x_l, x_r] x {y_f} (column c of the group, y_f = y_jf): the
// winding number just right of x_l from the crossings of that grid line,
// then the crossings of y_f inside the column, in order along x
__device__ double line_solid_hg(const GeoBufG &G, int c, int i, double xl, double xr, double yf, int jf) {
    int w = 0;
    const long long kyf = dk(yf), kxl = dk(xl), kxr = dk(xr);
    for (int e = 0; e < G.lcnt[c]; ++e)
        if ((G.lf[c][e] & 2) && dk(G.lyc[c][e]) < kyf) w += G.ls[c][e];
    double ex[8];
    int ed[8], ne = 0;
    bool overflow = false;
    const float fyf = (float)yf;
    ColIter it;
    col_iter_init(G, c, it);
    for (;;) {
        int sv[SVN], ns = 0, en;
        while (ns < SVN && (en = col_iter_next(G, c, it)) >= 0) {
            if (G.jhi[en] < jf - 1 || G.jlo[en] > jf) continue;
            if (G.fy1[en] < fyf || G.fy0[en] > fyf) continue;
            sv[ns++] = en;
        }
        for (int q = 0; q < ns; ++q) {
            const int e = sv[q];
            const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e], yb = G.yb[e];
            const long long kya = dk(ya), kyb = dk(yb);
            if (kya == kyb) continue;
            if ((kya < kyf) == (kyb < kyf)) continue;
            const double xs = deq(xa, xb) ? xa : xa + (yf - ya) * (xb - xa) * G.idy[e];
            const long long kxs = dk(xs);
            if (!(kxs > kxl && kxs < kxr)) continue;
            // crossing the boundary left to right: the interior of a
            // counter-clockwise polygon lies left of its edges
            const int dw = kyb > kya ? -1 : 1;
            if (ne < 8) {
                int p = ne++;
                while (p > 0 && dlt(xs, ex[p - 1])) { ex[p] = ex[p - 1]; ed[p] = ed[p - 1]; --p; }
                ex[p] = xs;
                ed[p] = dw;
            } else {
                overflow = true;
            }
        }
        if (ns < SVN) break;
    }
    if (overflow) {   // many crossings inside one column: integrate edge by edge
        double L = 0.0;
        FOR_COL_EDGES(G, c, e) {
            const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e];
            const double p = dmax(xl, dmin(xa, xb)), q = dmin(xr, dmax(xa, xb));
            if (!(q > p)) continue;
            const double s = xa < xb ? 1.0 : -1.0;
            const double k = G.slope[e];
            const double yp = ya + (p - xa) * k, yq = ya + (q - xa) * k;
            double m;
            if (yp < yf && yq < yf) m = q - p;
            else if (!(yp < yf) && !(yq < yf)) m = 0.0;
            else {
                double xs = p + (q - p) * ((yf - yp) / (yq - yp));
                xs = xs < p ? p : (xs > q ? q : xs);
                m = yp < yf ? xs - p : q - xs;
            }
            L += s * m;
        }
        return L;
    }
    double L = 0.0, pos = xl;
    for (int k = 0; k < ne; ++k) {
        if (w > 0) L += ex[k] - pos;
        pos = ex[k];
        w += ed[k];
    }
    if (w > 0) L += xr - pos;
    return L;
}

__device__ double rect_edges_g(const GeoBufG &G, int c, int ja, int jb, double rx0, double rx1, double ry0,
                               double ry1, double xo, double xs, double *nlx, double *nly, bool *mov) {
    const double lx0 = rx0 - xo, lx1 = rx1 - xo, ly1 = ry1 - ry0;
    const long long krx0 = dk(rx0), krx1 = dk(rx1), kry0 = dk(ry0), kry1 = dk(ry1);
    const long long klx0 = dk(lx0), klx1 = dk(lx1), kly1 = dk(ly1), kxs = dk(xs);
    const float frx0 = __double2float_rd(rx0), frx1 = __double2float_ru(rx1);
    const float fry0 = __double2float_rd(ry0), fry1 = __double2float_ru(ry1);
    double A = 0.0;
    ColIter it;
    col_iter_init(G, c, it);
    for (;;) {
        int sv[SVN], ns = 0, en;
        while (ns < SVN && (en = col_iter_next(G, c, it)) >= 0) {
            if (G.jhi[en] < ja || G.jlo[en] > jb) continue;
            if (G.fy1[en] < fry0 || G.fy0[en] > fry1 || G.fx1[en] < frx0 || G.fx0[en] > frx1) continue;
            sv[ns++] = en;
        }
        for (int k = 0; k < ns; ++k) {
            const int e = sv[k];
            const double xa = G.xa[e], xb = G.xb[e], ya = G.ya[e], yb = G.yb[e];
            const long long kxa = dk(xa), kxb = dk(xb), kya = dk(ya), kyb = dk(yb);
            if ((kya < kry0 && kyb < kry0) || (kya > kry1 && kyb > kry1) || (kxa < krx0 && kxb < krx0) ||
                (kxa > krx1 && kxb > krx1))
                continue;
            const double ax = xa - xo, ay = ya - ry0, bx = xb - xo, by = yb - ry0;
            const double ddx = bx - ax, ddy = by - ay;
            double t0 = 0.0, t1 = 1.0;
            bool ok = true;
            if (dzero(ddx)) {
                const long long kax = dk(ax);
                if (kax < klx0 || kax > klx1) ok = false;
            } else {
                const double inv = G.idx[e];
                const double ra = (lx0 - ax) * inv, rb = (lx1 - ax) * inv;
                t0 = dmax(t0, dmin(ra, rb));
                t1 = dmin(t1, dmax(ra, rb));
            }
            if (dzero(ddy)) {
                const long long kay = dk(ay);
                if (kay < 0 || kay > kly1) ok = false;
            } else {
                const double inv = G.idy[e];
                const double ra = (0.0 - ay) * inv, rb = (ly1 - ay) * inv;
                t0 = dmax(t0, dmin(ra, rb));
                t1 = dmin(t1, dmax(ra, rb));
            }
            if (!ok || dlt(t1, t0)) continue;
            if (mov && G.mov[e]) *mov = true;
            if (kxa == kxb && kxa == kxs) continue;   // vertical edge on the grid side
            if (!dlt(t0, t1)) continue;
            const double xc0 = ax + t0 * ddx, xc1 = ax + t1 * ddx;
            A += ddy * (t1 - t0) * (0.5 * (xc0 + xc1));
            if (nlx) {
                *nlx -= ddy * (t1 - t0);
                *nly += ddx * (t1 - t0);
            }
        }
        if (ns < SVN) break;
    }
    return A;
}

__device__ __forceinline__ double cell_alpha_g(const GeoBufG &G, const InstDesc &I, int c, int i, int j, double xl,
                                               double xr, double yb, double yt, double *nlx, double *nly, bool *mov) {
    double A = rect_edges_g(G, c, j, j, xl, xr, yb, yt, xl, xr, nlx, nly, mov) +
               (xr - xl) * line_solid_vg(G, c + 1, yb, yt, true);
    double a = clamp01(1.0 - A / (I.dx * I.dy));
    return a < ALPHA_MIN ? 0.0 : a;
}

__device__ double face_ap_g(const GeoBufG &G, const InstDesc &I, int dir, bool hi, int c, int i, int j, double xl,
                            double xr, double yb, double yt) {
    if (dir == 0) return clamp01(1.0 - line_solid_vg(G, hi ? c + 1 : c, yb, yt, true) / I.dy);
    return clamp01(1.0 - line_solid_hg(G, c, i, xl, xr, hi ? yt : yb, hi ? j + 1 : j) / I.dx);
}

__device__ double swept_face_Bg(const GeoBufG &G, const InstDesc &I, int dir, double delta, bool hi, int c, int i,
                                int j, double xl, double xr, double yb, double yt) {
    if (delta == 0.0) return face_ap_g(G, I, dir, hi, c, i, j, xl, xr, yb, yt);
    if (dir == 0) {
        const int line = hi ? c + 1 : c;
        const double xs = hi ? xr : xl;
        if (delta > 0.0) {
            const double x1 = xs + delta;
            const double A = rect_edges_g(G, c, j, j, xs, x1, yb, yt, x1, xs, nullptr, nullptr, nullptr) +
                             (x1 - xs) * line_solid_vg(G, line, yb, yt, false);
            return clamp01(1.0 - A / ((x1 - xs) * I.dy));
        }
        const double x0 = xs + delta;
        const double A = rect_edges_g(G, c, j, j, x0, xs, yb, yt, x0, xs, nullptr, nullptr, nullptr) +
                         (xs - x0) * line_solid_vg(G, line, yb, yt, true);
        return clamp01(1.0 - A / ((xs - x0) * I.dy));
    }
    const double ys = hi ? yt : yb;
    const double y0 = delta > 0.0 ? ys : ys + delta, y1 = delta > 0.0 ? ys + delta : ys;
    const int ja = delta > 0.0 ? j : j - 1, jb = delta > 0.0 ? j + 1 : j;
    const double A = rect_edges_g(G, c, ja, jb, xl, xr, y0, y1, xl, xr, nullptr, nullptr, nullptr) +
                     (xr - xl) * line_solid_vg(G, c + 1, y0, y1, true);
    return clamp01(1.0 - A / ((y1 - y0) * I.dx));
}

// the band cells of geometry group gw (one CTA)
__device__ __forceinline__ void geom_group(int gw, const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                           const int *__restrict__ ginst, const double *__restrict__ px,
                                           const double *__restrict__ py, const float *__restrict__ ebox,
                                           const int *__restrict__ vnext, const unsigned char *__restrict__ vmov,
                                           int total_v, int n_inst, int total_groups, int dir,
                                           BandRec *__restrict__ R, double *__restrict__ bnd, int &sh_base) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    GeoWarpG &W = *(GeoWarpG *)gsm;
    GeoBufG &G = W.G;
    if (gw >= total_groups) return;
    const int lo = ginst[gw];
    const InstDesc &I = D[lo];
    InstDyn &y = Y[lo];
    const int i0 = y.col0 + GC * (gw - I.gcol_off);
    if (i0 > y.col1 || i0 >= I.nx || I.nv == 0) return;
    const int ncol = min(GC, min(y.col1, I.nx - 1) - i0 + 1);
    const double delta = y.delta;
    const bool own_hi = I.rotating || delta >= 0.0;
    const double ad = fabs(delta);
    const int row0 = y.row0;
    const int nwb = (y.row1 - y.row0) / 32 + 1;
    int err = 0;
    if (y.row1 < y.row0) return;
    if (nwb > NWB) {
        if (tid == 0) atomicOr(&y.err, ERR_BAND_CAP);
        return;
    }
    for (int w = tid; w < GC * NWB; w += GEOMG_THREADS) {
        (&W.bA[0][0])[w] = 0u;
        (&W.bB[0][0])[w] = 0u;
        (&W.bM[0][0])[w] = 0u;
    }
    __syncthreads();
    // touched at the start pose: class bytes kept from the previous sweep
    const int nrow = y.row1 - row0 + 1;
    for (int p = tid; p < nrow * ncol; p += GEOMG_THREADS) {
        const int jr = p / ncol, c = p - jr * ncol;
        if (I.cls[(row0 + jr) * I.pitch + i0 + c] & CLS_TOUCH) atomicOr(&W.bA[c][jr >> 5], 1u << (jr & 31));
    }
    if (I.rotating) {   // touched at the middle pose
        gather_g(G, I, px, py, ebox, vnext, vmov, 1, total_v, i0, ncol, ad, tid, &err);
        index_g(G, I, i0, ncol, row0, nwb, W.bM, tid);
        __syncthreads();
    }
    gather_g(G, I, px, py, ebox, vnext, vmov, 2, total_v, i0, ncol, ad, tid, &err);
    index_g(G, I, i0, ncol, row0, nwb, W.bB, tid);
    __syncthreads();
    if (warp == 1) compact_lines_g(G, ncol, lane, &err);
    // band cells in (column, row) order: prefix counts over the words
    const int nw = ncol * nwb;
    if (warp == 0) {
        int running = 0;
        for (int w0 = 0; w0 < nw; w0 += 32) {
            const int w = w0 + lane;
            const int c = w / nwb, k = w % nwb;
            int cnt = w < nw ? __popc(W.bA[c][k] | W.bB[c][k] | W.bM[c][k]) : 0;
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (w < nw) W.wpre[w] = running + incl - cnt;
            running += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            W.wpre[GC * NWB] = running;
            int b = running ? atomicAdd(&y.band_count, running) : 0;
            if (b + running > I.rec_cap) { err |= ERR_BAND_CAP; b = -1; }
            sh_base = b;
        }
    }
    __syncthreads();
    const int T = W.wpre[GC * NWB];
    const int base = sh_base;
    if (base < 0 || T == 0) {
        if (err) atomicOr(&y.err, err);
        return;
    }
    auto locate = [&](int t, int *c, int *j, int *k, int *bit) {
        int a = 0, b = nw - 1;
        while (a < b) {
            int m = (a + b + 1) >> 1;
            if (W.wpre[m] <= t) a = m; else b = m - 1;
        }
        *c = a / nwb;
        *k = a % nwb;
        const unsigned mask = W.bA[*c][*k] | W.bB[*c][*k] | W.bM[*c][*k];
        *bit = __fns(mask, 0, t - W.wpre[a] + 1);
        *j = row0 + (*k) * 32 + *bit;
    };
    const double wsimp_B = 1.0 / 6.0, wsimp_M = 4.0 / 6.0, wsimp_A = 1.0 / 6.0;
    // Each band cell's geometric queries run on separate threads (two in
    // pass B, three in pass M), so that the CTA's threads share the FP64
    // clipping work evenly; the pass-M partial results wait in the record
    // (aM, nx, ny, d, wx, pad) for the per-cell step that combines them.
    // pass B (edges of the end pose are in G): 0: alpha_B and flags, 1: the
    // owned face's time-averaged aperture
    for (int u = tid; u < 2 * T; u += GEOMG_THREADS) {
        const int part = u >= T ? 1 : 0, t = u - part * T;   // parts in contiguous blocks: warps stay uniform
        int c, j, k, bit;
        locate(t, &c, &j, &k, &bit);
        const int i = i0 + c;
        BandRec &r = R[I.rec_base + base + t];
        const double xl = G.xln[c], xr = G.xln[c + 1];
        const double yb = I.yn[j], yt = I.yn[j + 1];
        const int cell = j * I.pitch + i;
        if (part == 0) {
            const bool tA = (W.bA[c][k] >> bit) & 1u, tB = (W.bB[c][k] >> bit) & 1u, tM = (W.bM[c][k] >> bit) & 1u;
            r.cell = cell;
            r.i = i;
            r.j = j;
            bool mov = false;
            r.aB = cell_alpha_g(G, I, c, i, j, xl, xr, yb, yt, nullptr, nullptr, &mov);
            r.aA = I.alpha[cell];
            const bool movA = (I.cls[cell] & CLS_MOVT) != 0;
            r.flags = (tA ? RF_TOUCH_A : 0) | (tB ? RF_TOUCH_B : 0) | (tM ? RF_TOUCH_M : 0) |
                      ((mov || movA) ? RF_MOVING : 0) | (mov ? RF_MOV_B : 0);
        } else {
            const bool need_bnd =
                dir == 0 ? ((own_hi && i == 0 && I.bc[0] != 2) || (!own_hi && i == I.nx - 1 && I.bc[1] != 2))
                         : ((own_hi && j == 0 && I.bc[2] != 2) || (!own_hi && j == I.ny - 1 && I.bc[3] != 2));
            double bo, bb = 0.0;
            if (I.rotating) {
                bo = wsimp_B * face_ap_g(G, I, dir, true, c, i, j, xl, xr, yb, yt);
                if (need_bnd) bb = wsimp_B * face_ap_g(G, I, dir, false, c, i, j, xl, xr, yb, yt);
            } else {
                bo = swept_face_Bg(G, I, dir, delta, own_hi, c, i, j, xl, xr, yb, yt);
                if (need_bnd) bb = swept_face_Bg(G, I, dir, delta, !own_hi, c, i, j, xl, xr, yb, yt);
            }
            r.bown = bo;
            bnd[I.rec_base + base + t] = bb;
        }
    }
    // pass M: 0: alpha_M, the aperture-closure normal and the moving flag,
    // 1: low face aperture (and the rotating body's Simpson term), 2: high
    // face aperture
    __syncthreads();
    gather_g(G, I, px, py, ebox, vnext, vmov, 1, total_v, i0, ncol, ad, tid, &err);
    index_g(G, I, i0, ncol, row0, nwb, nullptr, tid);
    __syncthreads();
    if (warp == 1) compact_lines_g(G, ncol, lane, &err);
    __syncthreads();
    for (int u = tid; u < 3 * T; u += GEOMG_THREADS) {
        const int part = u / T, t = u - part * T;
        int c, j, k, bit;
        locate(t, &c, &j, &k, &bit);
        const int i = i0 + c;
        const int ri = I.rec_base + base + t;
        BandRec &r = R[ri];
        const double xl = G.xln[c], xr = G.xln[c + 1];
        const double yb = I.yn[j], yt = I.yn[j + 1];
        if (part == 0) {
            bool mov = false;
            double nlx = 0.0, nly = 0.0;
            r.aM = cell_alpha_g(G, I, c, i, j, xl, xr, yb, yt, &nlx, &nly, &mov);
            r.nx = nlx;
            r.ny = nly;
            r.aux = mov ? 1 : 0;
        } else if (part == 1) {
            if (I.rotating) {
                r.bown += wsimp_M * face_ap_g(G, I, dir, true, c, i, j, xl, xr, yb, yt);
                const bool need_bnd = dir == 0 ? (i == 0 && I.bc[0] != 2) : (j == 0 && I.bc[2] != 2);
                if (need_bnd) bnd[ri] += wsimp_M * face_ap_g(G, I, dir, false, c, i, j, xl, xr, yb, yt);
            }
            r.d = face_ap_g(G, I, dir, false, c, i, j, xl, xr, yb, yt);
        } else {
            r.wx = face_ap_g(G, I, dir, true, c, i, j, xl, xr, yb, yt);
        }
    }
    __syncthreads();
    for (int t = tid; t < T; t += GEOMG_THREADS) {
        int c, j, k, bit;
        locate(t, &c, &j, &k, &bit);
        const int i = i0 + c;
        const int ri = I.rec_base + base + t;
        BandRec &r = R[ri];
        const double aM = r.aM, blo = r.d, bhi = r.wx, nlx = r.nx, nly = r.ny;
        int fl = r.flags | (r.aux ? RF_MOVING : 0);
        r.aux = 0;
        const double db = fabs(blo - bhi);
        const double ahat = aM - dmin(blo, bhi);
        // equally open faces (|delta beta| <= 1e-12, where both terms are
        // round-off): d = 1
        r.d = db > 1e-12 ? clamp01(ahat / db) : 1.0;
        // Where two bodies touch along an edge (a piston sliding in a tube),
        // their edges cancel in this sum and no fluid boundary is left; the
        // sum keeps a rounding residual of about eps x the edge length, which
        // must not be normalised into a unit normal.  A wall in a cell with
        // alpha >= ALPHA_MIN is at least ~1e-5 of the cell size long.
        const double L = sqrt(nlx * nlx + nly * nly);
        const bool wall = L > 1e-9 * fmax(I.dx, I.dy);
        r.nx = wall ? nlx / L : 0.0;
        r.ny = wall ? nly / L : 0.0;
        double wx = 0.0, wy = 0.0;
        if (fl & RF_MOVING) {
            const double xc = I.x0 + ((double)i + 0.5) * I.dx, yc = I.y0 + ((double)j + 0.5) * I.dy;
            const double pcx = I.pivot[0] + y.XM, pcy = I.pivot[1] + y.YM;
            wx = I.U[0] - y.Om * (yc - pcy);
            wy = I.U[1] + y.Om * (xc - pcx);
        }
        r.wx = wx;
        r.wy = wy;
        const bool unc = r.aA == 0.0 && r.aB > 0.0;
        const bool cov = r.aA > 0.0 && r.aB == 0.0;
        if (unc) fl |= RF_UNCOV;
        if (cov) fl |= RF_COVER;
        if (r.aA > 0.0 || (unc && I.ucov == 1)) fl |= RF_FLUID_A;
        if (r.aB > 0.0) fl |= RF_FLUID_B;
        r.flags = fl;
        r.mix = -1;
        I.rec[r.cell] = ri;
        I.cls[r.cell] |= CLS_BAND;
    }
    if (I.rotating) {
        __syncthreads();
        gather_g(G, I, px, py, ebox, vnext, vmov, 0, total_v, i0, ncol, ad, tid, &err);
        index_g(G, I, i0, ncol, row0, nwb, nullptr, tid);
        __syncthreads();
        if (warp == 1) compact_lines_g(G, ncol, lane, &err);
        __syncthreads();
        for (int t = tid; t < T; t += GEOMG_THREADS) {
            int c, j, k, bit;
            locate(t, &c, &j, &k, &bit);
            const int i = i0 + c;
            const int ri = I.rec_base + base + t;
            const double xl = G.xln[c], xr = G.xln[c + 1];
            const double yb = I.yn[j], yt = I.yn[j + 1];
            R[ri].bown += wsimp_A * face_ap_g(G, I, dir, true, c, i, j, xl, xr, yb, yt);
            const bool need_bnd = dir == 0 ? (i == 0 && I.bc[0] != 2) : (j == 0 && I.bc[2] != 2);
            if (need_bnd) bnd[ri] += wsimp_A * face_ap_g(G, I, dir, false, c, i, j, xl, xr, yb, yt);
        }
    }
    if (err) atomicOr(&y.err, err);
}

// One CTA per geometry group (a grid capped below the group count, looping
// over the groups so that bulk CTAs find room beside it, measured slower).
__global__ void __launch_bounds__(GEOMG_THREADS, 3) k_geom(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                            const int *__restrict__ ginst,
                                                            const double *__restrict__ px, const double *__restrict__ py,
                                                            const float *__restrict__ ebox,
                                                            const int *__restrict__ vnext,
                                                            const unsigned char *__restrict__ vmov, int total_v,
                                                            int n_inst, int total_groups, int dir,
                                                            BandRec *__restrict__ R, double *__restrict__ bnd) {
    __shared__ int sh_base;
    geom_group(blockIdx.x, D, Y, ginst, px, py, ebox, vnext, vmov, total_v, n_inst, total_groups, dir, R, bnd,
               sh_base);
}

// ---------------------------------------------------------------------------
// full classification at the pose in slot 0 (create / write_state / alpha)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GEOM_WARPS * 32) k_classify(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                            const double *__restrict__ px,
                                                            const double *__restrict__ py,
                                                            const float *__restrict__ ebox,
                                                            const int *__restrict__ vnext,
                                                            const unsigned char *__restrict__ vmov, int total_v,
                                                            int inst0, double *__restrict__ alpha_out) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    GeoWarp &W = ((GeoWarp *)gsm)[wib];
    GeoBuf &G = W.G;
    const int inst = inst0 + blockIdx.y;
    const InstDesc &I = D[inst];
    const int i = blockIdx.x * GEOM_WARPS + wib;
    if (i >= I.nx) return;
    const double xl = node_coord(I.x0, i, I.dx), xr = node_coord(I.x0, i + 1, I.dx);
    const int nwords = (I.ny + 31) >> 5;
    int err = 0;
    for (int w = lane; w < nwords; w += 32) W.bB[w] = W.bA[w] = 0u;
    __syncwarp();
    if (I.nv) gather(G, I, px, py, ebox, vnext, vmov, 0, total_v, xl, xr, xl, xr, W.bB, lane, &err);
    else if (lane == 0) { G.cnt = 0; G.lcnt[0] = G.lcnt[1] = 0; }
    __syncwarp();
    // rows that rect_edges examines an edge for (jlo <= j <= jhi)
    for (int e = lane; e < G.cnt; e += 32) {
        const int a = max((int)G.jlo[e], 0), z = min((int)G.jhi[e], I.ny - 1);
        for (int w = a >> 5; w <= (z >> 5) && a <= z; ++w) {
            const int lo = max(a - 32 * w, 0), hi = min(z - 32 * w, 31);
            const unsigned m = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
            atomicOr(&W.bA[w], m);
        }
    }
    __syncwarp();
    for (int j = lane; j < I.ny; j += 32) {
        const double yb = I.yn[j], yt = I.yn[j + 1];
        const bool touched = (W.bB[j >> 5] >> (j & 31)) & 1u;
        bool mov = false;
        // A cell that no edge meets and whose rows rect_edges examines no edge
        // for, with no crossing of x_r within [yb, yt]: rect_edges is 0 and
        // x_r is solid over the whole cell or over none of it, S times its
        // height (S: the signed crossings below the cell).  The same value as
        // cell_alpha, without its FP64 work in the common case S = 0.
        bool fast = !touched && !((W.bA[j >> 5] >> (j & 31)) & 1u);
        int S = 0;
        if (fast) {
            const long long kb = dk(yb), kt = dk(yt);
            for (int e = 0; e < G.lcnt[1]; ++e) {
                if (!(G.lf[1][e] & 1)) continue;
                const long long kc = dk(G.lyc[1][e]);
                if (kc < kb) S += G.ls[1][e];
                else if (kc <= kt) fast = false;
            }
        }
        double a;
        if (!fast) {
            a = cell_alpha(G, I, j, xl, xr, yb, yt, nullptr, nullptr, &mov);
        } else if (S == 0) {
            a = 1.0;
        } else {
            const double A = (xr - xl) * ((double)S * (yt - yb));
            a = clamp01(1.0 - A / (I.dx * I.dy));
            if (a < ALPHA_MIN) a = 0.0;
        }
        uint8_t c = touched ? CLS_TOUCH : 0;
        if (mov) c |= CLS_MOVT;
        if (a == 0.0) c |= CLS_SOLID;
        else if (touched) c |= CLS_CUT;
        const int cell = j * I.pitch + i;
        I.cls[cell] = c;
        I.rec[cell] = -1;
        I.alpha[cell] = a;
        if (alpha_out) alpha_out[(size_t)j * I.nx + i] = a;
    }
    if (lane == 0 && err) atomicOr(&Y[inst].err, err);
}

// pose of instance `inst` at its current (t, X, Y) into slot 0, with the
// FP32 x-bounds of its edges
__global__ void k_pose_current(const InstDesc *__restrict__ D, const InstDyn *__restrict__ Y,
                               const double *__restrict__ vx, const double *__restrict__ vy,
                               const unsigned char *__restrict__ vmov, const int *__restrict__ vnext,
                               double *__restrict__ px, double *__restrict__ py, float *__restrict__ ebox,
                               int inst0) {
    const int inst = inst0 + blockIdx.x;
    const InstDesc &I = D[inst];
    const InstDyn &y = Y[inst];
    double th = I.rotating ? y.th : 0.0;
    double c = cos(th), s = sin(th);
    for (int k = threadIdx.x; k < I.nv; k += blockDim.x) {
        int a = I.voff + k;
        double x0 = vx[a], y0 = vy[a], xo, yo;
        if (!vmov[a]) {
            xo = x0; yo = y0;
        } else if (I.rotating) {
            double ddx = x0 - I.pivot[0], ddy = y0 - I.pivot[1];
            double rx = c * ddx - s * ddy;
            double ry = s * ddx + c * ddy;
            xo = (I.pivot[0] + rx) + y.X;
            yo = (I.pivot[1] + ry) + y.Y;
        } else {
            xo = x0 + y.X;
            yo = y0 + y.Y;
        }
        px[a] = xo;
        py[a] = yo;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < I.nv; k += blockDim.x) {
        int a = I.voff + k, b = vnext[a];
        ebox[2 * a] = __double2float_rd(dmin(px[a], px[b]));
        ebox[2 * a + 1] = __double2float_ru(dmax(px[a], px[b]));
    }
}

// grid-line coordinates of every instance (one block per instance)
__global__ void k_nodes(const InstDesc *__restrict__ D) {
    const InstDesc &I = D[blockIdx.x];
    double *xn = const_cast<double *>(I.xn), *yn = const_cast<double *>(I.yn);
    for (int i = threadIdx.x; i <= I.nx; i += blockDim.x) xn[i] = node_coord(I.x0, i, I.dx);
    for (int j = threadIdx.x; j <= I.ny; j += blockDim.x) yn[j] = node_coord(I.y0, j, I.dy);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t geom_smem() { return sizeof(GeoWarp) * GEOM_WARPS; }
static size_t geomg_smem() { return sizeof(GeoWarpG); }

void geom_init() {
    cudaFuncSetAttribute(k_geom, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geomg_smem());
    cudaFuncSetAttribute(k_classify, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geom_smem());
}

void launch_nodes(const InstDesc *D, int n_inst, cudaStream_t st) {
    if (n_inst > 0) k_nodes<<<n_inst, 256, 0, st>>>(D);
}

void launch_pose(const InstDesc *D, InstDyn *Y, const double *vx, const double *vy, const unsigned char *vmov,
                 const int *vnext, double *px, double *py, float *ebox, int total_v, int n_inst, int dir, int sidx,
                 double dt, int *defer_count, cudaStream_t st) {
    k_pose<<<n_inst * POSE_PARTS, 256, 0, st>>>(D, Y, vx, vy, vmov, vnext, px, py, ebox, total_v, dir, sidx, dt,
                                                 defer_count);
}

void launch_geom(const InstDesc *D, InstDyn *Y, const int *ginst, const double *px, const double *py, const float *ebox,
                 const int *vnext, const unsigned char *vmov, int total_v, int n_inst, int total_groups, int dir,
                 BandRec *R, double *bnd, cudaStream_t st) {
    const int blocks = total_groups;
    if (blocks > 0)
        k_geom<<<blocks, GEOMG_THREADS, geomg_smem(), st>>>(D, Y, ginst, px, py, ebox, vnext, vmov, total_v, n_inst,
                                                             total_groups, dir, R, bnd);
}

void launch_classify(const InstDesc *D, InstDyn *Y, const double *vx, const double *vy, const unsigned char *vmov,
                     double *px, double *py, float *ebox, const int *vnext, int total_v, int inst0, int ninst,
                     int max_nx, double *alpha_out, cudaStream_t st) {
    if (ninst <= 0 || max_nx <= 0) return;
    k_pose_current<<<ninst, 256, 0, st>>>(D, Y, vx, vy, vmov, vnext, px, py, ebox, inst0);
    const dim3 grid((max_nx + GEOM_WARPS - 1) / GEOM_WARPS, ninst);
    k_classify<<<grid, GEOM_WARPS * 32, geom_smem(), st>>>(D, Y, px, py, ebox, vnext, vmov, total_v, inst0,
                                                         ninst == 1 ? alpha_out : nullptr);
}

}  // namespace mb

// ---------------------------------------------------------------------------
// Allocation-free cut-cell classification.
//
// For callers that cannot allocate device memory themselves (code that runs
// while an application forbids cudaMalloc: inside real-time or latency-
// critical loops, in plugins whose host framework owns every allocation, or
// in processes near their memory limit), this entry point computes the volume
// fractions and classes of a posed body with no allocation at all.  Its
// working memory -- the instance descriptor, the copied vertices, the posed
// vertices and their FP32 x-bounds -- lives in one file-scope device array
// of fixed size that every GPU loading this library holds until the process
// exits.  All calls share that array: calls that overlap on the GPU (e.g. on
// two streams) race and must be serialised by the caller.
// ---------------------------------------------------------------------------
#include "../../include/mb.h"

namespace mb {

constexpr int NA_MAX_V = 16384;             // polygon vertices per call
constexpr int NA_MAX_N = 8192;              // nx and ny per call
constexpr size_t NA_OFF_DESC = 0;
constexpr size_t NA_OFF_DYN = 1024;
constexpr size_t NA_OFF_VX = 2048;
constexpr size_t NA_OFF_VY = NA_OFF_VX + 8 * (size_t)NA_MAX_V;
constexpr size_t NA_OFF_PX = NA_OFF_VY + 8 * (size_t)NA_MAX_V;
constexpr size_t NA_OFF_PY = NA_OFF_PX + 8 * (size_t)NA_MAX_V;
constexpr size_t NA_OFF_EBOX = NA_OFF_PY + 8 * (size_t)NA_MAX_V;
constexpr size_t NA_OFF_NEXT = NA_OFF_EBOX + 8 * (size_t)NA_MAX_V;
constexpr size_t NA_OFF_MOV = NA_OFF_NEXT + 4 * (size_t)NA_MAX_V;
constexpr size_t NA_BYTES = NA_OFF_MOV + (size_t)NA_MAX_V;   // about 0.7 MB

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

// host-side stand-in `g_na_scratch` is not a device address: kernels get the
// address that cudaGetSymbolAddress returns for the current device, looked up
// once per device (std::call_once, so concurrent first calls from several
// host threads are safe)
constexpr int NA_MAX_DEV = 64;
static void *g_na_addr[NA_MAX_DEV];
static cudaError_t g_na_setup_err[NA_MAX_DEV];
static std::once_flag g_na_once[NA_MAX_DEV];

// variant of k_classify writing unpitched outputs and no record map
__global__ void __launch_bounds__(GEOM_WARPS * 32) k_classify_na(const InstDesc *__restrict__ D,
                                                               InstDyn *__restrict__ Y,
                                                               const double *__restrict__ px,
                                                               const double *__restrict__ py,
                                                               const float *__restrict__ ebox,
                                                               const int *__restrict__ vnext,
                                                               const unsigned char *__restrict__ vmov, int total_v,
                                                               double *__restrict__ alpha_out,
                                                               unsigned char *__restrict__ cls_out) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    GeoWarp &W = ((GeoWarp *)gsm)[wib];
    GeoBuf &G = W.G;
    const InstDesc &I = D[0];
    const int i = blockIdx.x * GEOM_WARPS + wib;
    if (i >= I.nx) return;
    const double xl = node_coord(I.x0, i, I.dx), xr = node_coord(I.x0, i + 1, I.dx);
    const int nwords = (I.ny + 31) >> 5;
    int err = 0;
    for (int w = lane; w < nwords; w += 32) W.bB[w] = 0u;
    __syncwarp();
    if (I.nv) gather(G, I, px, py, ebox, vnext, vmov, 0, total_v, xl, xr, xl, xr, W.bB, lane, &err);
    else if (lane == 0) { G.cnt = 0; G.lcnt[0] = G.lcnt[1] = 0; }
    __syncwarp();
    for (int j = lane; j < I.ny; j += 32) {
        const double yb = node_coord(I.y0, j, I.dy), yt = node_coord(I.y0, j + 1, I.dy);
        const bool touched = (W.bB[j >> 5] >> (j & 31)) & 1u;
        bool mov = false;
        const double a = cell_alpha(G, I, j, xl, xr, yb, yt, nullptr, nullptr, &mov);
        uint8_t c = touched ? CLS_TOUCH : 0;
        if (mov) c |= CLS_MOVT;
        if (a == 0.0) c |= CLS_SOLID;
        else if (touched) c |= CLS_CUT;
        alpha_out[(size_t)j * I.nx + i] = a;
        cls_out[(size_t)j * I.nx + i] = c;
    }
    if (lane == 0 && err) atomicOr(&Y[0].err, err);
}

}  // namespace mb

// per host thread, like the scratch vectors of the call below
static thread_local std::string g_na_error;

extern "C" mb_status mb_cut_cells_noalloc(const mb_grid *grid, const mb_body *body, const mb_motion *motion,
                                          double X, double Y, double theta, double *alpha_dev,
                                          unsigned char *class_dev, void *stream) {
    using namespace mb;
    // every argument check comes before the first CUDA call
    if (!grid || !body || !motion || !alpha_dev || !class_dev) {
        g_na_error = "mb_cut_cells_noalloc: NULL argument";
        return MB_E_INVAL;
    }
    if (body->npoly < 0 || (body->npoly > 0 && (!body->poly_start || !body->poly_moving || !body->vx || !body->vy))) {
        g_na_error = "mb_cut_cells_noalloc: body arrays missing";
        return MB_E_INVAL;
    }
    const int nv = body->npoly > 0 ? body->poly_start[body->npoly] : 0;
    if (grid->nx < 1 || grid->ny < 1 || grid->nx > NA_MAX_N || grid->ny > NA_MAX_N) {
        g_na_error = "mb_cut_cells_noalloc: nx and ny must lie in [1, 8192]";
        return MB_E_INVAL;
    }
    if (nv > NA_MAX_V) {
        g_na_error = "mb_cut_cells_noalloc: more than 16384 polygon vertices (the fixed scratch limit)";
        return MB_E_INVAL;
    }
    if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0)) {
        g_na_error = "mb_cut_cells_noalloc: empty domain";
        return MB_E_INVAL;
    }
    if (body->npoly > 0 && body->poly_start[0] != 0) {
        g_na_error = "mb_cut_cells_noalloc: poly_start[0] must be 0";
        return MB_E_INVAL;
    }
    for (int p = 0; p < body->npoly; ++p) {
        if (body->poly_start[p + 1] - body->poly_start[p] < 3) {
            g_na_error = "mb_cut_cells_noalloc: polygon with fewer than 3 vertices";
            return MB_E_INVAL;
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) {
        g_na_error = std::string("mb_cut_cells_noalloc: no current device: ") + cudaGetErrorString(e);
        return MB_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // one-time set-up on this device (the first call per device does it, and
    // should therefore come before any stream capture)
    std::call_once(g_na_once[dev], [dev]() {
        void *p = nullptr;
        cudaError_t r = cudaGetSymbolAddress(&p, g_na_scratch);
        if (r == cudaSuccess && !p) r = cudaErrorInvalidSymbol;
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_classify_na, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geom_smem());
        g_na_addr[dev] = r == cudaSuccess ? p : nullptr;
        g_na_setup_err[dev] = r;
    });
    if (g_na_setup_err[dev] != cudaSuccess) {
        g_na_error = std::string("mb_cut_cells_noalloc: set-up of the scratch array failed: ") +
                     cudaGetErrorString(g_na_setup_err[dev]);
        return MB_E_CUDA;
    }
    unsigned char *base = (unsigned char *)g_na_addr[dev];
    // descriptor of a one-instance, unpitched grid
    InstDesc I;
    memset(&I, 0, sizeof(I));
    I.nx = grid->nx; I.ny = grid->ny; I.pitch = grid->nx;
    I.nc = grid->equation == MB_EULER ? 4 : 1;
    I.x0 = grid->x0; I.y0 = grid->y0;
    I.dx = (grid->x1 - grid->x0) / (double)grid->nx;
    I.dy = (grid->y1 - grid->y0) / (double)grid->ny;
    I.rdx = 1.0 / I.dx;
    I.rdy = 1.0 / I.dy;
    for (int q = 0; q < 4; ++q) I.bc[q] = grid->bc[q];
    I.nv = nv;
    I.voff = 0;
    I.rotating = (theta != 0.0 || motion->a0 != 0.0 || motion->a1 != 0.0) ? 1 : 0;
    I.pivot[0] = motion->pivot[0]; I.pivot[1] = motion->pivot[1];
    InstDyn y;
    memset(&y, 0, sizeof(y));   // clears the error word of this call
    y.X = X; y.Y = Y; y.th = theta;
    static thread_local std::vector<int> hnext;
    static thread_local std::vector<unsigned char> hmov;
    hnext.assign(nv > 0 ? nv : 1, 0);
    hmov.assign(nv > 0 ? nv : 1, 0);
    for (int p = 0; p < body->npoly; ++p) {
        const int a = body->poly_start[p], z = body->poly_start[p + 1];
        for (int v = a; v < z; ++v) {
            hnext[v] = v + 1 < z ? v + 1 : a;
            hmov[v] = body->poly_moving[p] ? 1 : 0;
        }
    }
    e = cudaMemcpyAsync(base + NA_OFF_DESC, &I, sizeof(I), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + NA_OFF_DYN, &y, sizeof(y), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(base + NA_OFF_VX, body->vx, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(base + NA_OFF_VY, body->vy, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(base + NA_OFF_NEXT, hnext.data(), 4 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(base + NA_OFF_MOV, hmov.data(), (size_t)nv, cudaMemcpyHostToDevice, st);
    // the host vectors above are reused by the next call: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_na_error = std::string("mb_cut_cells_noalloc: copy to scratch failed: ") + cudaGetErrorString(e);
        return MB_E_CUDA;
    }
    const InstDesc *D = (const InstDesc *)(base + NA_OFF_DESC);
    InstDyn *Yd = (InstDyn *)(base + NA_OFF_DYN);
    double *px = (double *)(base + NA_OFF_PX), *py = (double *)(base + NA_OFF_PY);
    float *ebox = (float *)(base + NA_OFF_EBOX);
    const int *vnext = (const int *)(base + NA_OFF_NEXT);
    const unsigned char *vmov = (const unsigned char *)(base + NA_OFF_MOV);
    const double *vx = (const double *)(base + NA_OFF_VX), *vy = (const double *)(base + NA_OFF_VY);
    k_pose_current<<<1, 256, 0, st>>>(D, Yd, vx, vy, vmov, vnext, px, py, ebox, 0);
    const int blocks = (grid->nx + GEOM_WARPS - 1) / GEOM_WARPS;
    k_classify_na<<<blocks, GEOM_WARPS * 32, geom_smem(), st>>>(D, Yd, px, py, ebox, vnext, vmov, nv > 0 ? nv : 1,
                                                                 alpha_dev, class_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_na_error = std::string("mb_cut_cells_noalloc: launch failed: ") + cudaGetErrorString(e);
        return MB_E_CUDA;
    }
    // the kernels' error word (a column whose edge or crossing lists would
    // exceed their fixed capacity clips them and sets it): read back into
    // host memory, so that truncated lists never pass as a result
    int herr = 0;
    e = cudaMemcpyAsync(&herr, &Yd->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        g_na_error = std::string("mb_cut_cells_noalloc: ") + cudaGetErrorString(e);
        return MB_E_CUDA;
    }
    if (herr & ERR_EDGE_CAP) {
        g_na_error = "mb_cut_cells_noalloc: a grid column meets more than 192 polygon edges, or one of its grid "
                     "lines more than 32 edges; the outputs are not valid (use a finer grid or fewer vertices)";
        return MB_E_CAPACITY;
    }
    if (herr) {
        g_na_error = "mb_cut_cells_noalloc: device error word " + std::to_string(herr);
        return MB_E_CUDA;
    }
    return MB_OK;
}

extern "C" const char *mb_noalloc_last_error(void) { return g_na_error.c_str(); }
