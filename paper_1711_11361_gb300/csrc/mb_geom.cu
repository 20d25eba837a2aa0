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

namespace mb {

constexpr int GEOM_WARPS = 4;
constexpr int EMAX = 256;           // edges per column and pose
constexpr int MAXROWWORDS = 256;    // ny <= 8192

struct EdgeBuf {
    double xa[EMAX], ya[EMAX], xb[EMAX], yb[EMAX];
    unsigned char mov[EMAX];
};

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }
__device__ __forceinline__ double clamp01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }

// ---------------------------------------------------------------------------
// K0: time step, poses of the sweep, posed vertices, column range
// ---------------------------------------------------------------------------
__global__ void k_pose(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, const double *__restrict__ vx,
                       const double *__restrict__ vy, const unsigned char *__restrict__ vmov, double *__restrict__ px,
                       double *__restrict__ py, int total_v, int dir, int sidx, double dt_host) {
    const int inst = blockIdx.x;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    __shared__ double sh[16];
    __shared__ double red[4][32];
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
            y.dt = dt;
            y.S[0] = 0ull;
            y.S[1] = 0ull;
        } else {
            dt = y.dt;
            if (dt_host > 0.0 && dt_host != dt) y.err |= ERR_STATE;
        }
        double tA = y.t + (sidx == 0 ? 0.0 : 0.5 * dt);
        double tB = y.t + (sidx == 0 ? 0.5 * dt : dt);
        double tM = y.t + (sidx == 0 ? 0.25 * dt : 0.75 * dt);
        double thA = 0.0, thB = 0.0, thM = 0.0, Om = 0.0;
        if (I.rotating) {
            thA = I.a0 + I.a1 * sin(I.omega * tA);
            thB = I.a0 + I.a1 * sin(I.omega * tB);
            thM = I.a0 + I.a1 * sin(I.omega * tM);
            Om = I.a1 * I.omega * cos(I.omega * tM);
        }
        double delta = I.U[dir] * dt;
        y.delta = delta;
        y.XA = y.X; y.YA = y.Y;
        y.XB = dir == 0 ? y.X + delta : y.X;
        y.YB = dir == 1 ? y.Y + delta : y.Y;
        y.XM = dir == 0 ? y.X + 0.5 * delta : y.X;
        y.YM = dir == 1 ? y.Y + 0.5 * delta : y.Y;
        y.thA = thA; y.thB = thB; y.thM = thM;
        y.cA = cos(thA); y.sA = sin(thA);
        y.cB = cos(thB); y.sB = sin(thB);
        y.cM = cos(thM); y.sM = sin(thM);
        y.Om = Om;
        y.band_count = 0;
        y.nbad = 0;
        y.mixed = 0;
        for (int q = 0; q < MAXC; ++q) y.wall_sum[q] = 0.0;
        sh[0] = y.XA; sh[1] = y.YA; sh[2] = y.XM; sh[3] = y.YM; sh[4] = y.XB; sh[5] = y.YB;
        sh[6] = y.cA; sh[7] = y.sA; sh[8] = y.cM; sh[9] = y.sM; sh[10] = y.cB; sh[11] = y.sB;
    }
    __syncthreads();
    double xmin = 1e300, xmax = -1e300;
    for (int k = threadIdx.x; k < I.nv; k += blockDim.x) {
        int a = I.voff + k;
        double x0 = vx[a], y0 = vy[a];
        for (int P = 0; P < 3; ++P) {   // 0: A, 1: M, 2: B
            double X = sh[2 * P], Yy = sh[2 * P + 1], c = sh[6 + 2 * P], s = sh[7 + 2 * P];
            double xo, yo;
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
            px[(size_t)P * total_v + a] = xo;
            py[(size_t)P * total_v + a] = yo;
            xmin = dmin(xmin, xo);
            xmax = dmax(xmax, xo);
        }
    }
    // block reduction of the x extent
    for (int o = 16; o > 0; o >>= 1) {
        xmin = dmin(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = dmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = xmin; red[1][w] = xmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { xmin = dmin(xmin, red[0][k]); xmax = dmax(xmax, red[1][k]); }
        int c0 = (int)floor((xmin - I.x0) / I.dx) - 1;
        int c1 = (int)floor((xmax - I.x0) / I.dx) + 1;
        if (I.nv == 0) { c0 = 1; c1 = 0; }
        if (c0 < 0) c0 = 0;
        if (c1 > I.nx - 1) c1 = I.nx - 1;
        if (c1 - c0 + 1 > I.gcol_max) { c1 = c0 + I.gcol_max - 1; y.err |= ERR_EDGE_CAP; }
        y.col0 = c0;
        y.col1 = c1;
    }
}

// ---------------------------------------------------------------------------
// warp-cooperative edge gather for one column and pose
// ---------------------------------------------------------------------------
__device__ int gather_edges(EdgeBuf &E, const InstDesc &I, const double *px, const double *py, const int *vnext,
                            const unsigned char *vmov, int P, int total_v, double gxl, double gxr, int lane,
                            int *err) {
    int cnt = 0;
    const double *PX = px + (size_t)P * total_v, *PY = py + (size_t)P * total_v;
    for (int base = 0; base < I.nv; base += 32) {
        int k = base + lane;
        bool take = false;
        double xa = 0, ya = 0, xb = 0, yb = 0;
        int a = I.voff + k;
        if (k < I.nv) {
            int b = vnext[a];
            xa = PX[a]; xb = PX[b];
            take = dmax(xa, xb) >= gxl && dmin(xa, xb) <= gxr;
            if (take) { ya = PY[a]; yb = PY[b]; }
        }
        unsigned m = __ballot_sync(0xffffffffu, take);
        if (take) {
            int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (pos < EMAX) {
                E.xa[pos] = xa; E.ya[pos] = ya; E.xb[pos] = xb; E.yb[pos] = yb;
                E.mov[pos] = vmov[a];
            }
        }
        cnt += __popc(m);
    }
    __syncwarp();
    if (cnt > EMAX) {
        if (lane == 0) *err |= ERR_EDGE_CAP;
        cnt = EMAX;
    }
    return cnt;
}

// y-extent of an edge inside the closed column [xl, xr]; false if disjoint
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

// mark rows j whose closed cell [xl,xr]x[y_j,y_j+1] meets an edge
__device__ void mark_rows(const EdgeBuf &E, int cnt, const InstDesc &I, double xl, double xr, unsigned *bits,
                          int lane) {
    for (int e = lane; e < cnt; e += 32) {
        double elo, ehi;
        if (!edge_yrange(E.xa[e], E.ya[e], E.xb[e], E.yb[e], xl, xr, &elo, &ehi)) continue;
        double flo = (elo - I.y0) / I.dy, fhi = (ehi - I.y0) / I.dy;
        flo = fmin(fmax(flo, -4.0), (double)I.ny + 4.0);
        fhi = fmin(fmax(fhi, -4.0), (double)I.ny + 4.0);
        int jlo = (int)floor(flo) - 1, jhi = (int)floor(fhi) + 1;
        if (jlo < 0) jlo = 0;
        if (jhi > I.ny - 1) jhi = I.ny - 1;
        for (int j = jlo; j <= jhi; ++j) {
            double yb = node_coord(I.y0, j, I.dy), yt = node_coord(I.y0, j + 1, I.dy);
            if (ehi >= yb && elo <= yt) atomicOr(&bits[j >> 5], 1u << (j & 31));
        }
    }
}

// solid length of the vertical segment {xs} x [y0r, y1r]; left_limit selects
// the crossing convention min < xs <= max (limit from the left), otherwise
// min <= xs < max
__device__ double line_solid_v(const EdgeBuf &E, int cnt, double xs, double y0r, double y1r, bool left_limit) {
    double L = 0.0;
    for (int e = 0; e < cnt; ++e) {
        double xa = E.xa[e], xb = E.xb[e];
        double lo = dmin(xa, xb), hi = dmax(xa, xb);
        bool cr = left_limit ? (lo < xs && xs <= hi) : (lo <= xs && xs < hi);
        if (!cr) continue;
        double ya = E.ya[e], yb = E.yb[e];
        double yc = ya + (xs - xa) * (yb - ya) / (xb - xa);
        double s = xa < xb ? 1.0 : -1.0;
        double cl = yc < y0r ? y0r : (yc > y1r ? y1r : yc);
        L += s * (y1r - cl);
    }
    return L;
}

// solid length of the horizontal segment [xl, xr] x {yf} inside the column:
// each edge contributes the x-measure over which it lies below yf
__device__ double line_solid_h(const EdgeBuf &E, int cnt, double xl, double xr, double yf) {
    double L = 0.0;
    for (int e = 0; e < cnt; ++e) {
        double xa = E.xa[e], xb = E.xb[e], ya = E.ya[e], yb = E.yb[e];
        double p = dmax(xl, dmin(xa, xb)), q = dmin(xr, dmax(xa, xb));
        if (!(q > p)) continue;
        double s = xa < xb ? 1.0 : -1.0;
        double k = (yb - ya) / (xb - xa);
        double yp = ya + (p - xa) * k, yq = ya + (q - xa) * k;
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

// area of body ∩ [rx0,rx1] x [ry0,ry1]; grid side on the right (x_s = rx1,
// crossings taken from the left) or on the left (x_s = rx0, from the right)
__device__ double solid_area(const EdgeBuf &E, int cnt, double rx0, double rx1, double ry0, double ry1,
                             bool grid_right) {
    double xo = grid_right ? rx0 : rx1;
    double xs = grid_right ? rx1 : rx0;
    double lx0 = rx0 - xo, lx1 = rx1 - xo, ly1 = ry1 - ry0;
    double A = 0.0;
    for (int e = 0; e < cnt; ++e) {
        double xa = E.xa[e], xb = E.xb[e], ya = E.ya[e], yb = E.yb[e];
        if (dmax(ya, yb) < ry0 || dmin(ya, yb) > ry1 || dmax(xa, xb) < rx0 || dmin(xa, xb) > rx1) continue;
        if (xa == xb && xa == xs) continue;   // vertical edge on the grid side
        double ax = xa - xo, ay = ya - ry0, bx = xb - xo, by = yb - ry0;
        double ddx = bx - ax, ddy = by - ay;
        double t0 = 0.0, t1 = 1.0;
        bool ok = true;
        double pp[4] = {-ddx, ddx, -ddy, ddy};
        double qq[4] = {ax - lx0, lx1 - ax, ay, ly1 - ay};
        for (int k = 0; k < 4; ++k) {
            if (pp[k] == 0.0) {
                if (qq[k] < 0.0) ok = false;
                continue;
            }
            double r = qq[k] / pp[k];
            if (pp[k] < 0.0) t0 = dmax(t0, r);
            else t1 = dmin(t1, r);
        }
        if (!ok || !(t1 > t0)) continue;
        double xc0 = ax + t0 * ddx, xc1 = ax + t1 * ddx;
        A += ddy * (t1 - t0) * (0.5 * (xc0 + xc1));
    }
    A += (rx1 - rx0) * line_solid_v(E, cnt, xs, ry0, ry1, grid_right);
    return A;
}

// touched-by-moving-edge test of a closed cell
__device__ bool cell_moving(const EdgeBuf &E, int cnt, double xl, double xr, double yb, double yt) {
    for (int e = 0; e < cnt; ++e) {
        if (!E.mov[e]) continue;
        double elo, ehi;
        if (edge_yrange(E.xa[e], E.ya[e], E.xb[e], E.yb[e], xl, xr, &elo, &ehi) && ehi >= yb && elo <= yt)
            return true;
    }
    return false;
}

__device__ __forceinline__ double cell_alpha(const EdgeBuf &E, int cnt, const InstDesc &I, double xl, double xr,
                                             double yb, double yt) {
    double A = solid_area(E, cnt, xl, xr, yb, yt, true);
    double a = clamp01(1.0 - A / (I.dx * I.dy));
    return a < ALPHA_MIN ? 0.0 : a;
}

// time-averaged aperture of the face owned by cell (i,j) along dir at pose P
// (P = 0 start, 1 middle, 2 end).  Translating sweeps use the exact swept strip
// at the start pose; rotating sweeps Simpson's rule over the three poses; a
// static direction the start-pose aperture.  Owner rule: delta >= 0 -> the
// high face, delta < 0 -> the low face.
__device__ double owned_face_part(const EdgeBuf &E, int cnt, const InstDesc &I, int dir, double delta, int P,
                                  double xl, double xr, double yb, double yt) {
    if (I.rotating) {
        double w = P == 1 ? 4.0 / 6.0 : 1.0 / 6.0;
        double ap = dir == 0 ? 1.0 - line_solid_v(E, cnt, xr, yb, yt, true) / I.dy
                             : 1.0 - line_solid_h(E, cnt, xl, xr, yt) / I.dx;
        return w * clamp01(ap);
    }
    if (P != 0) return 0.0;
    if (delta == 0.0) {
        double ap = dir == 0 ? 1.0 - line_solid_v(E, cnt, xr, yb, yt, true) / I.dy
                             : 1.0 - line_solid_h(E, cnt, xl, xr, yt) / I.dx;
        return clamp01(ap);
    }
    if (dir == 0) {
        double sl = delta > 0 ? xr - delta : xl, sr = delta > 0 ? xr : xl - delta;
        double A = solid_area(E, cnt, sl, sr, yb, yt, delta > 0);
        return clamp01(1.0 - A / ((sr - sl) * I.dy));
    }
    double sl = delta > 0 ? yt - delta : yb, sr = delta > 0 ? yt : yb - delta;
    double A = solid_area(E, cnt, xl, xr, sl, sr, true);
    return clamp01(1.0 - A / ((sr - sl) * I.dx));
}

// time-averaged aperture of the domain-boundary face that a boundary cell does
// not own (x-low face when delta >= 0, x-high face when delta < 0, same for y)
__device__ double boundary_face_part(const EdgeBuf &E, int cnt, const InstDesc &I, int dir, double delta, int P,
                                     double xl, double xr, double yb, double yt) {
    if (I.rotating) {
        double w = P == 1 ? 4.0 / 6.0 : 1.0 / 6.0;
        double ap = dir == 0 ? 1.0 - line_solid_v(E, cnt, xl, yb, yt, true) / I.dy
                             : 1.0 - line_solid_h(E, cnt, xl, xr, yb) / I.dx;
        return w * clamp01(ap);
    }
    if (P != 0) return 0.0;
    if (delta == 0.0) {
        double ap = dir == 0 ? 1.0 - line_solid_v(E, cnt, xl, yb, yt, true) / I.dy
                             : 1.0 - line_solid_h(E, cnt, xl, xr, yb) / I.dx;
        return clamp01(ap);
    }
    if (dir == 0) {
        // delta > 0: strip left of the x-low face; delta < 0: right of the x-high face
        double sl = delta > 0 ? xl - delta : xr, sr = delta > 0 ? xl : xr - delta;
        double A = solid_area(E, cnt, sl, sr, yb, yt, delta > 0);
        return clamp01(1.0 - A / ((sr - sl) * I.dy));
    }
    double sl = delta > 0 ? yb - delta : yt, sr = delta > 0 ? yb : yt - delta;
    double A = solid_area(E, cnt, xl, xr, sl, sr, true);
    return clamp01(1.0 - A / ((sr - sl) * I.dx));
}

// ---------------------------------------------------------------------------
// K1: band records (cells touched by the body at the start or end pose, or
// the middle pose when rotating) with their geometry
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GEOM_WARPS * 32) k_geom(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                        const double *__restrict__ px, const double *__restrict__ py,
                                                        const int *__restrict__ vnext,
                                                        const unsigned char *__restrict__ vmov, int total_v,
                                                        int n_inst, int total_cols, int dir, BandRec *__restrict__ R,
                                                        double *__restrict__ bnd) {
    __shared__ EdgeBuf Es[GEOM_WARPS];
    __shared__ unsigned bitsA[GEOM_WARPS][MAXROWWORDS], bitsB[GEOM_WARPS][MAXROWWORDS];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * GEOM_WARPS + wib;
    if (gw >= total_cols) return;
    // instance of this geometry column
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].gcol_off <= gw) lo = mid; else hi = mid - 1;
    }
    const int inst = lo;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    const int i = y.col0 + (gw - I.gcol_off);
    if (i > y.col1 || i >= I.nx || I.nv == 0) return;
    EdgeBuf &E = Es[wib];
    unsigned *bA = bitsA[wib], *bB = bitsB[wib];
    const double xl = node_coord(I.x0, i, I.dx), xr = node_coord(I.x0, i + 1, I.dx);
    const double delta = y.delta;
    const bool own_hi = I.rotating || delta >= 0.0;   // owner rule of the sweep-direction faces
    const bool xbnd_lo = dir == 0 && I.bc[0] != 2 && i == 0;
    const bool xbnd_hi = dir == 0 && I.bc[1] != 2 && i == I.nx - 1;
    // gather range: the column, widened by |delta| at a non-periodic x boundary
    double gxl = xl, gxr = xr;
    if (xbnd_lo) gxl = xl - fabs(delta);
    if (xbnd_hi) gxr = xr + fabs(delta);
    const int nwords = (I.ny + 31) >> 5;
    int err = 0;
    for (int w = lane; w < nwords; w += 32) { bA[w] = 0u; bB[w] = 0u; }
    __syncwarp();
    // pass 1: touched rows at A, B (and M when rotating)
    const int poses[3] = {0, 2, 1};
    for (int pi = 0; pi < (I.rotating ? 3 : 2); ++pi) {
        int P = poses[pi];
        int cnt = gather_edges(E, I, px, py, vnext, vmov, P, total_v, gxl, gxr, lane, &err);
        mark_rows(E, cnt, I, xl, xr, pi == 1 ? bB : bA, lane);   // M (rotating) is or-ed into the A map
        __syncwarp();
    }
    __syncwarp();
    // count band rows and reserve records (rows in increasing order)
    int base = 0;
    if (lane == 0) {
        int tot = 0;
        for (int w = 0; w < nwords; ++w) tot += __popc(bA[w] | bB[w]);
        base = tot ? atomicAdd(&y.band_count, tot) : 0;
        if (base + tot > I.rec_cap) { err |= ERR_BAND_CAP; base = -1; }
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base < 0) { if (lane == 0) atomicOr(&y.err, err); return; }
    // pass 2: per pose quantities for each band row
    for (int pi = 0; pi < 3; ++pi) {
        const int P = pi == 0 ? 0 : (pi == 1 ? 2 : 1);   // A, B, M
        int cnt = gather_edges(E, I, px, py, vnext, vmov, P, total_v, gxl, gxr, lane, &err);
        int running = 0;
        for (int w0 = 0; w0 < nwords; w0 += 32) {
            int w = w0 + lane;
            unsigned m = w < nwords ? (bA[w] | bB[w]) : 0u;
            int c = __popc(m);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int idx = base + running + incl - c;
            running += __shfl_sync(0xffffffffu, incl, 31);
            while (m) {
                int b = __ffs(m) - 1;
                m &= m - 1;
                const int j = w * 32 + b;
                BandRec &r = R[I.rec_base + idx];
                ++idx;
                const double yb = node_coord(I.y0, j, I.dy), yt = node_coord(I.y0, j + 1, I.dy);
                const bool tA = (bA[w] >> b) & 1u, tB = (bB[w] >> b) & 1u;
                // the domain-boundary face this boundary cell does not own
                const bool need_bnd =
                    dir == 0 ? ((own_hi && i == 0 && I.bc[0] != 2) || (!own_hi && i == I.nx - 1 && I.bc[1] != 2))
                             : ((own_hi && j == 0 && I.bc[2] != 2) || (!own_hi && j == I.ny - 1 && I.bc[3] != 2));
                if (P == 0) {
                    r.cell = j * I.pitch + i;
                    r.i = i;
                    r.j = j;
                    r.aA = cell_alpha(E, cnt, I, xl, xr, yb, yt);
                    r.bown = owned_face_part(E, cnt, I, dir, delta, 0, xl, xr, yb, yt);
                    bnd[I.rec_base + idx - 1] =
                        need_bnd ? boundary_face_part(E, cnt, I, dir, delta, 0, xl, xr, yb, yt) : 0.0;
                    int fl = (tA ? RF_TOUCH_A : 0) | (tB ? RF_TOUCH_B : 0);
                    if (cell_moving(E, cnt, xl, xr, yb, yt)) fl |= RF_MOVING;
                    r.flags = fl;
                } else if (P == 2) {
                    r.aB = cell_alpha(E, cnt, I, xl, xr, yb, yt);
                    if (I.rotating) {
                        r.bown += owned_face_part(E, cnt, I, dir, delta, 2, xl, xr, yb, yt);
                        if (need_bnd) bnd[I.rec_base + idx - 1] += boundary_face_part(E, cnt, I, dir, delta, 2, xl, xr, yb, yt);
                    }
                    if (cell_moving(E, cnt, xl, xr, yb, yt)) r.flags |= RF_MOVING;
                } else {
                    const double aM = cell_alpha(E, cnt, I, xl, xr, yb, yt);
                    r.aM = aM;
                    if (I.rotating) {
                        r.bown += owned_face_part(E, cnt, I, dir, delta, 1, xl, xr, yb, yt);
                        if (need_bnd) bnd[I.rec_base + idx - 1] += boundary_face_part(E, cnt, I, dir, delta, 1, xl, xr, yb, yt);
                    }
                    int fl = r.flags;
                    if (cell_moving(E, cnt, xl, xr, yb, yt)) fl |= RF_MOVING;
                    // instantaneous apertures at the mid pose
                    const double bW = clamp01(1.0 - line_solid_v(E, cnt, xl, yb, yt, true) / I.dy);
                    const double bE = clamp01(1.0 - line_solid_v(E, cnt, xr, yb, yt, true) / I.dy);
                    const double bS = clamp01(1.0 - line_solid_h(E, cnt, xl, xr, yb) / I.dx);
                    const double bN = clamp01(1.0 - line_solid_h(E, cnt, xl, xr, yt) / I.dx);
                    // shielded distance d = alpha_hat / |delta beta| (eq. Klein2DalphaHat)
                    const double blo = dir == 0 ? bW : bS, bhi = dir == 0 ? bE : bN;
                    const double db = fabs(blo - bhi);
                    const double ahat = aM - dmin(blo, bhi);
                    r.d = db > 0.0 ? clamp01(ahat / db) : 1.0;
                    // wall normal from aperture closure, into the body
                    const double nLx = (bW - bE) * I.dy, nLy = (bS - bN) * I.dx;
                    const double L = sqrt(nLx * nLx + nLy * nLy);
                    r.nx = L > 0.0 ? nLx / L : 0.0;
                    r.ny = L > 0.0 ? nLy / L : 0.0;
                    // wall velocity at the cell centre
                    double wx = 0.0, wy = 0.0;
                    if (fl & RF_MOVING) {
                        const double xc = I.x0 + ((double)i + 0.5) * I.dx, yc = I.y0 + ((double)j + 0.5) * I.dy;
                        const double pcx = I.pivot[0] + y.XM, pcy = I.pivot[1] + y.YM;
                        wx = I.U[0] - y.Om * (yc - pcy);
                        wy = I.U[1] + y.Om * (xc - pcx);
                    }
                    r.wx = wx;
                    r.wy = wy;
                    // classes
                    const bool unc = r.aA == 0.0 && r.aB > 0.0;
                    const bool cov = r.aA > 0.0 && r.aB == 0.0;
                    if (unc) fl |= RF_UNCOV;
                    if (cov) fl |= RF_COVER;
                    if (r.aA > 0.0 || (unc && I.ucov == 1)) fl |= RF_FLUID_A;
                    if (r.aB > 0.0) fl |= RF_FLUID_B;
                    r.flags = fl;
                    r.mix = -1;
                    // publish: class byte and record index of this cell
                    I.rec[r.cell] = I.rec_base + idx - 1;
                    I.cls[r.cell] |= CLS_BAND;
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0 && err) atomicOr(&y.err, err);
}

// ---------------------------------------------------------------------------
// full classification at the current pose (create / write_state / alpha read)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GEOM_WARPS * 32) k_classify(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                            const double *__restrict__ px,
                                                            const double *__restrict__ py,
                                                            const int *__restrict__ vnext,
                                                            const unsigned char *__restrict__ vmov, int total_v,
                                                            int inst, double *__restrict__ alpha_out) {
    __shared__ EdgeBuf Es[GEOM_WARPS];
    __shared__ unsigned bits[GEOM_WARPS][MAXROWWORDS];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const InstDesc &I = D[inst];
    const int i = blockIdx.x * GEOM_WARPS + wib;
    if (i >= I.nx) return;
    EdgeBuf &E = Es[wib];
    unsigned *bt = bits[wib];
    const double xl = node_coord(I.x0, i, I.dx), xr = node_coord(I.x0, i + 1, I.dx);
    const int nwords = (I.ny + 31) >> 5;
    int err = 0;
    for (int w = lane; w < nwords; w += 32) bt[w] = 0u;
    __syncwarp();
    int cnt = I.nv ? gather_edges(E, I, px, py, vnext, vmov, 0, total_v, xl, xr, lane, &err) : 0;
    mark_rows(E, cnt, I, xl, xr, bt, lane);
    __syncwarp();
    for (int j = lane; j < I.ny; j += 32) {
        const double yb = node_coord(I.y0, j, I.dy), yt = node_coord(I.y0, j + 1, I.dy);
        const bool touched = (bt[j >> 5] >> (j & 31)) & 1u;
        double a = cnt ? cell_alpha(E, cnt, I, xl, xr, yb, yt) : 1.0;
        uint8_t c = 0;
        if (a == 0.0) c = CLS_SOLID;
        else if (touched) c = CLS_CUT;
        I.cls[j * I.pitch + i] = c;
        I.rec[j * I.pitch + i] = -1;
        if (alpha_out) alpha_out[(size_t)j * I.nx + i] = a;
    }
    if (lane == 0 && err) atomicOr(&Y[inst].err, err);
}

// pose of instance `inst` at its current (t, X, Y) into pose slot 0
__global__ void k_pose_current(const InstDesc *__restrict__ D, const InstDyn *__restrict__ Y,
                               const double *__restrict__ vx, const double *__restrict__ vy,
                               const unsigned char *__restrict__ vmov, double *__restrict__ px,
                               double *__restrict__ py, int inst) {
    const InstDesc &I = D[inst];
    const InstDyn &y = Y[inst];
    double th = I.rotating ? I.a0 + I.a1 * sin(I.omega * y.t) : 0.0;
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
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_pose(const InstDesc *D, InstDyn *Y, const double *vx, const double *vy, const unsigned char *vmov,
                 double *px, double *py, int total_v, int n_inst, int dir, int sidx, double dt, cudaStream_t st) {
    k_pose<<<n_inst, 256, 0, st>>>(D, Y, vx, vy, vmov, px, py, total_v, dir, sidx, dt);
}

void launch_geom(const InstDesc *D, InstDyn *Y, const double *px, const double *py, const int *vnext,
                 const unsigned char *vmov, int total_v, int n_inst, int total_cols, int dir, BandRec *R,
                 double *bnd, cudaStream_t st) {
    int blocks = (total_cols + GEOM_WARPS - 1) / GEOM_WARPS;
    if (blocks > 0)
        k_geom<<<blocks, GEOM_WARPS * 32, 0, st>>>(D, Y, px, py, vnext, vmov, total_v, n_inst, total_cols, dir, R, bnd);
}

void launch_classify(const InstDesc *D, InstDyn *Y, const double *vx, const double *vy, const unsigned char *vmov,
                     double *px, double *py, const int *vnext, int total_v, int inst, int nx, double *alpha_out,
                     cudaStream_t st) {
    k_pose_current<<<1, 256, 0, st>>>(D, Y, vx, vy, vmov, px, py, inst);
    int blocks = (nx + GEOM_WARPS - 1) / GEOM_WARPS;
    k_classify<<<blocks, GEOM_WARPS * 32, 0, st>>>(D, Y, px, py, vnext, vmov, total_v, inst, alpha_out);
}

}  // namespace mb
