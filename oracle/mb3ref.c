/* Three-dimensional oracle: a plain, slow, FP64 CPU implementation of the
 * dimensionally split moving-boundary cut-cell method in three dimensions
 * (Sec. II.C.4, eqs. Klein2DcompleteMovingMethod2a-c: x, y and z sweeps,
 * each with the time-averaged boundary movement of its own direction).
 * Test infrastructure only: the tests, the smoke check and the bench's CPU
 * legs use it; the CUDA path never does.
 *
 * Readings (the same as the two-dimensional oracle's unless stated):
 *   - the body is one convex polyhedron, the half-spaces n_f . x <= c_f in
 *     body coordinates (the paper's cone as a pyramid on a regular polygon),
 *     translating at the constant velocity U (the paper's 3-D test moves a
 *     cone through a stationary shock); no rotation;
 *   - a sweep along d moves the body by U_d dt along d (pose A to pose B);
 *     the step runs x, y, z on even steps and z, y, x on odd steps;
 *   - volume fraction alpha = fluid volume / cell volume, from clipping the
 *     cell box by the body's planes; alpha < 1e-10 counts as solid;
 *   - face aperture = fluid fraction of the face rectangle; the time-averaged
 *     aperture of a d-face under translation = the fluid fraction of the box
 *     the face sweeps (the exact time average of eq. timeAveragedBeta);
 *   - shielded distance d = (alpha_M - min(beta_lo, beta_hi)) / |beta_lo -
 *     beta_hi| from the mid pose's apertures of the two d-faces, clamped to
 *     [0, 1], and 1 when they differ by 1e-12 or less (round-off: both
 *     terms vanish); wall normal from aperture closure at the mid pose (into the
 *     body); wall velocity U;
 *   - wall state: the exact wall Riemann problem of eq. riemann_wallvel
 *     with the three-dimensional normal; advective part from the step-start
 *     state, the momentum pressure from the sweep-start state;
 *   - MUSCL-Hancock in conserved variables, harmonic van Leer, zero slope
 *     next to a solid cell, first order where an evolved state is not
 *     physical; HLLC with Davis wave speeds;
 *   - two-sided stabilised face flux as the two-dimensional stab_face;
 *   - covering / uncovering (Sec. II.C.5) simultaneously, over the six face
 *     neighbours, else the cells sharing an edge (the 18-neighbourhood), else
 *     those sharing a vertex (26), as two dimensions take the face
 *     neighbours, else the 8-neighbourhood; a covered cell on a
 *     transmissive side with no neighbour passes its content out; uncovered
 *     cells by the donor equations (the paper's) or, in flux-GCL mode, from
 *     a provisional state (the neighbours' alpha-weighted average at the
 *     sweep start) carried through the sweep's fluxes;
 *   - positivity safeguard over the six face neighbours, seeded also by
 *     cells that keep less than 1% of their volume over the sweep;
 *   - dt = CFL min_d(h_d / S_d), S_d = max over fluid cells of |u_d| + c,
 *     raised to |U_d|.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add anywhere). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define O3_NC 5
#define O3_ALPHA_MIN 1e-10
#define O3_MIX_LAYERS 8
#define O3_COLLAPSE 0.01
#define O3_MAXP 32          /* body planes */
#define O3_BC_TRANSMISSIVE 0
#define O3_BC_REFLECTIVE 1
#define O3_BC_PERIODIC 2
#define O3_UNCOVER_DONOR 0
#define O3_UNCOVER_FLUX_GCL 1
#define O3_OK 0
#define O3_E_INVAL -1
#define O3_E_UNSTABLE -4
#define O3_E_STATE -6

typedef struct {
    int nx, ny, nz;
    double x0, y0, z0, x1, y1, z1;
    double gamma, cfl;
    int bc[6];              /* x-low, x-high, y-low, y-high, z-low, z-high */
    int nplane;
    double pn[3 * O3_MAXP]; /* outward unit normals */
    double pc[O3_MAXP];     /* n . x <= c inside, body coordinates */
    double U[3];
    int uncover_mode;
} o3_config;

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double clamp01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }
static int wrapi(int k, int n) { k %= n; return k < 0 ? k + n : k; }

/* ------------------------------------------------------------------------ */
/* convex clipping                                                          */
/* ------------------------------------------------------------------------ */
#define O3_MAXF (6 + O3_MAXP)   /* faces of a clipped box */
#define O3_MAXV 40              /* vertices of one face */

typedef struct { double p[O3_MAXV][3]; int n; } face_t;
typedef struct { face_t f[O3_MAXF]; int nf; } poly3_t;

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* the box [lo, hi] as six faces, each counter-clockwise seen from outside */
static void box_poly(const double *lo, const double *hi, poly3_t *P) {
    double v[8][3];
    for (int k = 0; k < 8; ++k) {
        v[k][0] = (k & 1) ? hi[0] : lo[0];
        v[k][1] = (k & 2) ? hi[1] : lo[1];
        v[k][2] = (k & 4) ? hi[2] : lo[2];
    }
    static const int F[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    P->nf = 6;
    for (int f = 0; f < 6; ++f) {
        P->f[f].n = 4;
        for (int k = 0; k < 4; ++k) memcpy(P->f[f].p[k], v[F[f][k]], sizeof(double) * 3);
    }
}

/* the part of P with n . x <= c into Q; the cut closes with a cap polygon
 * on the plane (its points sorted by angle about their centroid) */
static void clip_poly(const poly3_t *P, poly3_t *Q, const double *n, double c) {
    double cut[O3_MAXF * 2][3];
    int ncut = 0;
    Q->nf = 0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        face_t *G = &Q->f[Q->nf];
        G->n = 0;
        for (int k = 0; k < F->n; ++k) {
            const double *a = F->p[k], *b = F->p[(k + 1) % F->n];
            double sa = dot3(n, a) - c, sb = dot3(n, b) - c;
            int ina = sa <= 0.0, inb = sb <= 0.0;
            if (ina && G->n < O3_MAXV) memcpy(G->p[G->n++], a, sizeof(double) * 3);
            if (ina != inb) {
                double t = sa / (sa - sb), x[3];
                for (int m = 0; m < 3; ++m) x[m] = a[m] + t * (b[m] - a[m]);
                if (G->n < O3_MAXV) memcpy(G->p[G->n++], x, sizeof(double) * 3);
                if (ncut < O3_MAXF * 2) memcpy(cut[ncut++], x, sizeof(double) * 3);
            }
        }
        if (G->n >= 3 && Q->nf < O3_MAXF - 1) Q->nf++;
    }
    if (ncut >= 3 && Q->nf > 0) {
        /* cap: in-plane basis (e1, e2) with e1 x e2 = n, points by angle */
        double cen[3] = {0, 0, 0}, e1[3], e2[3], a[3] = {1, 0, 0};
        for (int k = 0; k < ncut; ++k) for (int m = 0; m < 3; ++m) cen[m] += cut[k][m] / ncut;
        if (fabs(n[0]) > 0.9) { a[0] = 0; a[1] = 1; }
        cross3(n, a, e1);
        double l = sqrt(dot3(e1, e1));
        for (int m = 0; m < 3; ++m) e1[m] /= l;
        cross3(n, e1, e2);
        double ang[O3_MAXF * 2];
        int idx[O3_MAXF * 2];
        for (int k = 0; k < ncut; ++k) {
            double r[3] = {cut[k][0] - cen[0], cut[k][1] - cen[1], cut[k][2] - cen[2]};
            ang[k] = atan2(dot3(r, e2), dot3(r, e1));
            idx[k] = k;
        }
        for (int x = 1; x < ncut; ++x) {   /* insertion sort by angle */
            int t = idx[x], z = x;
            while (z > 0 && ang[idx[z - 1]] > ang[t]) { idx[z] = idx[z - 1]; --z; }
            idx[z] = t;
        }
        face_t *C = &Q->f[Q->nf++];
        C->n = 0;
        for (int k = 0; k < ncut && C->n < O3_MAXV; ++k) memcpy(C->p[C->n++], cut[idx[k]], sizeof(double) * 3);
    }
}

/* volume of a closed polytope whose faces are counter-clockwise seen from
 * outside (divergence theorem, fan triangles about each face's first point) */
static double poly_volume(const poly3_t *P) {
    double V = 0.0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t *F = &P->f[f];
        for (int k = 1; k + 1 < F->n; ++k) {
            double c[3];
            cross3(F->p[k], F->p[k + 1], c);
            V += dot3(F->p[0], c);
        }
    }
    return V / 6.0;
}

/* planes of the body posed at translation T: n . x <= c + n . T */
static void posed_planes(const o3_config *cf, const double *T, double *cpos) {
    for (int f = 0; f < cf->nplane; ++f) cpos[f] = cf->pc[f] + dot3(&cf->pn[3 * f], T);
}

/* volume of box [lo, hi] inside the body; *touch: the box meets the body
 * boundary (part of it inside, part outside).  Only the planes that cut the
 * box clip it, in coordinates relative to lo (plane offsets c - n . lo). */
static double solid_volume(const o3_config *cf, const double *cpos, const double *lo, const double *hi, int *touch) {
    static poly3_t buf[2];
    const double h[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]}, z[3] = {0.0, 0.0, 0.0};
    const double vol = h[0] * h[1] * h[2];
    int cutting[O3_MAXP], ncp = 0;
    double cl[O3_MAXP];
    for (int f = 0; f < cf->nplane; ++f) {
        cl[f] = cpos[f] - dot3(&cf->pn[3 * f], lo);
        int nin = 0;
        for (int k = 0; k < 8; ++k) {
            double v[3] = {(k & 1) ? h[0] : 0.0, (k & 2) ? h[1] : 0.0, (k & 4) ? h[2] : 0.0};
            if (dot3(&cf->pn[3 * f], v) <= cl[f]) ++nin;
        }
        if (nin == 0) { if (touch) *touch = 0; return 0.0; }   /* the box lies outside this plane */
        if (nin < 8) cutting[ncp++] = f;
    }
    if (ncp == 0) { if (touch) *touch = 0; return vol; }
    box_poly(z, h, &buf[0]);
    int cur = 0;
    for (int m = 0; m < ncp && buf[cur].nf > 0; ++m) {
        const int f = cutting[m];
        clip_poly(&buf[cur], &buf[1 - cur], &cf->pn[3 * f], cl[f]);
        cur = 1 - cur;
    }
    if (touch) *touch = buf[cur].nf > 0;
    return buf[cur].nf > 0 ? dmin(vol, dmax(0.0, poly_volume(&buf[cur]))) : 0.0;
}

/* solid area of the rectangle {x_a = v} x [lo_b, hi_b] x [lo_c, hi_c] (a, b,
 * c a cyclic permutation of the axes): the rectangle clipped by the planes'
 * traces (a two-dimensional Sutherland-Hodgman), shoelace area */
static double solid_area(const o3_config *cf, const double *cpos, int a, double v, double lob, double hib, double loc,
                         double hic) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    double px[2 * O3_MAXP + 8], py[2 * O3_MAXP + 8], qx[2 * O3_MAXP + 8], qy[2 * O3_MAXP + 8];
    int n = 4;
    const double wb = hib - lob, wc = hic - loc;   /* coordinates relative to (lob, loc) */
    px[0] = 0.0; py[0] = 0.0; px[1] = wb; py[1] = 0.0; px[2] = wb; py[2] = wc; px[3] = 0.0; py[3] = wc;
    for (int f = 0; f < cf->nplane && n > 0; ++f) {
        const double *nn = &cf->pn[3 * f];
        const double cc = cpos[f] - nn[a] * v - nn[b] * lob - nn[c] * loc;   /* nn[b] y + nn[c] z <= cc */
        int m = 0;
        for (int k = 0; k < n; ++k) {
            double ax = px[k], ay = py[k], bx = px[(k + 1) % n], by = py[(k + 1) % n];
            double sa = nn[b] * ax + nn[c] * ay - cc, sb = nn[b] * bx + nn[c] * by - cc;
            int ina = sa <= 0.0, inb = sb <= 0.0;
            if (ina) { qx[m] = ax; qy[m] = ay; ++m; }
            if (ina != inb) {
                double t = sa / (sa - sb);
                qx[m] = ax + t * (bx - ax);
                qy[m] = ay + t * (by - ay);
                ++m;
            }
        }
        n = m;
        memcpy(px, qx, sizeof(double) * n);
        memcpy(py, qy, sizeof(double) * n);
    }
    if (n < 3) return 0.0;
    double A = 0.0;
    for (int k = 0; k < n; ++k) A += px[k] * py[(k + 1) % n] - px[(k + 1) % n] * py[k];
    return dmin(wb * wc, dmax(0.0, 0.5 * A));
}

/* ------------------------------------------------------------------------ */
/* simulation state and per-pose geometry                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    o3_config c;
    double bb[6];           /* body bounding box in body coordinates */
    double h[3];            /* dx, dy, dz */
    int n;                  /* cells */
    double *Q, *Qn;         /* O3_NC planes of n cells, NaN in solids; step-start state */
    double t, T[3];
    long step;
    int sweep_in_step;
    double dt_step;
    int status;
    double wall_last[O3_NC];
    int mixed_last;
    double *wall_cell;      /* last sweep, per cell: has, d, n_x, n_y, n_z */
} o3_sim;

typedef struct {
    double *alpha;
    unsigned char *touched;
    double *b[3];           /* apertures of the x-, y- and z-faces */
} o3_geom;

static int nfaces(const o3_sim *s, int a) {
    const int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    return a == 0 ? (nx + 1) * ny * nz : (a == 1 ? nx * (ny + 1) * nz : nx * ny * (nz + 1));
}
/* cell (i, j, k) and the low face along a of cell (i, j, k) */
static int cidx(const o3_sim *s, int i, int j, int k) { return (k * s->c.ny + j) * s->c.nx + i; }
static int fidx(const o3_sim *s, int a, int i, int j, int k) {
    const int nx = s->c.nx, ny = s->c.ny;
    return a == 0 ? (k * ny + j) * (nx + 1) + i : (a == 1 ? (k * (ny + 1) + j) * nx + i : (k * ny + j) * nx + i);
}
static double node(const o3_sim *s, int a, int i) {
    const double o = a == 0 ? s->c.x0 : (a == 1 ? s->c.y0 : s->c.z0);
    return o + (double)i * s->h[a];
}

static void geom_alloc(const o3_sim *s, o3_geom *g) {
    g->alpha = (double *)malloc(sizeof(double) * s->n);
    g->touched = (unsigned char *)malloc((size_t)s->n);
    for (int a = 0; a < 3; ++a) g->b[a] = (double *)malloc(sizeof(double) * nfaces(s, a));
}
static void geom_free(o3_geom *g) {
    free(g->alpha); free(g->touched);
    for (int a = 0; a < 3; ++a) free(g->b[a]);
}

/* cell range [lo, hi] along a whose cells meet the interval [u0, u1] widened
 * by a cell */
static void cell_range(const o3_sim *s, int a, double u0, double u1, int *lo, int *hi) {
    const int na = a == 0 ? s->c.nx : (a == 1 ? s->c.ny : s->c.nz);
    const double o = a == 0 ? s->c.x0 : (a == 1 ? s->c.y0 : s->c.z0);
    int l = (int)floor((u0 - o) / s->h[a]) - 1, r = (int)floor((u1 - o) / s->h[a]) + 1;
    *lo = l < 0 ? 0 : l;
    *hi = r > na - 1 ? na - 1 : r;
}

/* volume fractions, touch flags and apertures of every cell and face with
 * the body at translation T (Sec. II.A, II.B) */
static void compute_geometry(const o3_sim *s, const double *T, o3_geom *g) {
    const int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    for (int c = 0; c < s->n; ++c) { g->alpha[c] = 1.0; g->touched[c] = 0; }
    for (int a = 0; a < 3; ++a) for (int f = 0; f < nfaces(s, a); ++f) g->b[a][f] = 1.0;
    if (s->c.nplane == 0) return;
    double cpos[O3_MAXP];
    posed_planes(&s->c, T, cpos);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) cell_range(s, a, s->bb[2 * a] + T[a], s->bb[2 * a + 1] + T[a], &lo[a], &hi[a]);
    const double cv = s->h[0] * s->h[1] * s->h[2];
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const double bl[3] = {node(s, 0, i), node(s, 1, j), node(s, 2, k)};
                const double bh[3] = {node(s, 0, i + 1), node(s, 1, j + 1), node(s, 2, k + 1)};
                int touch = 0;
                const double V = solid_volume(&s->c, cpos, bl, bh, &touch);
                const double al = clamp01(1.0 - V / cv);
                const int c = cidx(s, i, j, k);
                g->alpha[c] = al < O3_ALPHA_MIN ? 0.0 : al;
                g->touched[c] = (unsigned char)touch;
            }
    /* faces normal to a: position node(a, .), the other two axes cyclic */
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c2 = (a + 2) % 3;
        int l2[3] = {lo[0], lo[1], lo[2]}, h2[3] = {hi[0], hi[1], hi[2]};
        h2[a] += 1;
        const double area = s->h[b] * s->h[c2];
        for (int k = l2[2]; k <= h2[2]; ++k)
            for (int j = l2[1]; j <= h2[1]; ++j)
                for (int i = l2[0]; i <= h2[0]; ++i) {
                    const int ijk[3] = {i, j, k};
                    const double v = node(s, a, ijk[a]);
                    const double A = solid_area(&s->c, cpos, a, v, node(s, b, ijk[b]), node(s, b, ijk[b] + 1),
                                                node(s, c2, ijk[c2]), node(s, c2, ijk[c2] + 1));
                    g->b[a][fidx(s, a, i, j, k)] = clamp01(1.0 - A / area);
                }
    }
}

/* time-averaged apertures of the d-faces while the body at translation T
 * moves by delta along d: fluid fraction of the box the face sweeps through
 * the body in the body's frame, [x_f - delta, x_f] at pose A (the solid that
 * crosses the face during the move), divided by its realised width (as the
 * two-dimensional oracle) */
static void compute_swept(const o3_sim *s, int d, const double *T, double delta, double *out) {
    const int nf = nfaces(s, d);
    for (int f = 0; f < nf; ++f) out[f] = 1.0;
    if (s->c.nplane == 0) return;
    double cpos[O3_MAXP];
    posed_planes(&s->c, T, cpos);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        double u0 = s->bb[2 * a] + T[a], u1 = s->bb[2 * a + 1] + T[a];
        if (a == d) { u0 = dmin(u0, u0 + delta); u1 = dmax(u1, u1 + delta); }
        cell_range(s, a, u0, u1, &lo[a], &hi[a]);
    }
    hi[d] += 1;
    const int b = (d + 1) % 3, c2 = (d + 2) % 3;
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const int ijk[3] = {i, j, k};
                double bl[3], bh[3];
                for (int a = 0; a < 3; ++a) { bl[a] = node(s, a, ijk[a]); bh[a] = node(s, a, ijk[a] + 1); }
                const double xf = node(s, d, ijk[d]);
                bl[d] = delta > 0.0 ? xf - delta : xf;
                bh[d] = delta > 0.0 ? xf : xf - delta;
                const double V = solid_volume(&s->c, cpos, bl, bh, NULL);
                out[fidx(s, d, i, j, k)] = clamp01(1.0 - V / ((bh[d] - bl[d]) * s->h[b] * s->h[c2]));
            }
}

/* ------------------------------------------------------------------------ */
/* Euler fluxes (5 components: rho, rho u, rho v, rho w, E)                 */
/* ------------------------------------------------------------------------ */
static double pressure3(double g, const double *q) {
    return (g - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}

static void euler_flux3(double g, int d, const double *q, double *f) {
    const double rho = q[0], un = q[1 + d] / rho, p = pressure3(g, q);
    f[0] = rho * un;
    for (int m = 0; m < 3; ++m) f[1 + m] = q[1 + m] * un + (m == d ? p : 0.0);
    f[4] = un * (q[4] + p);
}

/* HLLC with Davis wave speeds (Toro, Riemann Solvers ch. 10), along d */
void o3_hllc(double g, int d, const double *qL, const double *qR, double *F) {
    const int in = 1 + d;
    const double rL = qL[0], rR = qR[0];
    const double uL = qL[in] / rL, uR = qR[in] / rR;
    const double pL = pressure3(g, qL), pR = pressure3(g, qR);
    const double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    const double SL = dmin(uL - cL, uR - cR), SR = dmax(uL + cL, uR + cR);
    if (SL >= 0.0) { euler_flux3(g, d, qL, F); return; }
    if (SR <= 0.0) { euler_flux3(g, d, qR, F); return; }
    const double num = pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR);
    const double den = rL * (SL - uL) - rR * (SR - uR);
    const double Ss = num / den;
    const int left = Ss >= 0.0;
    const double *q = left ? qL : qR;
    const double r = left ? rL : rR, u = left ? uL : uR, p = left ? pL : pR, S = left ? SL : SR;
    double f[O3_NC], qs[O3_NC];
    euler_flux3(g, d, q, f);
    const double fac = r * (S - u) / (S - Ss);
    qs[0] = fac;
    for (int m = 0; m < 3; ++m) qs[1 + m] = m == d ? fac * Ss : fac * (q[1 + m] / r);
    qs[4] = fac * (q[4] / r + (Ss - u) * (Ss + p / (r * (S - u))));
    for (int k = 0; k < O3_NC; ++k) F[k] = f[k] + S * (qs[k] - q[k]);
}

static double vanleer(double dm, double dp) {
    const double pr = dm * dp;
    return pr > 0.0 ? 2.0 * pr / (dm + dp) : 0.0;
}

/* exact wall Riemann problem (eq. riemann_wallvel) with normal n (into the
 * body) and wall velocity w: rho*, p*, u* (tangential part kept) */
void o3_wall_state(double g, const double *q, const double *n, const double *w, double *rs, double *ps, double *us) {
    const double rho = q[0], p = pressure3(g, q);
    const double u[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
    const double du = (u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) - (w[0] * n[0] + w[1] * n[1] + w[2] * n[2]);
    const double mu = (g - 1.0) / (g + 1.0);
    double pst, rst;
    if (du > 0.0) {
        const double A = 2.0 / ((g + 1.0) * rho), B = mu * p;
        pst = p + du / (2.0 * A) * (du + sqrt(du * du + 4.0 * A * (p + B)));
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

/* ------------------------------------------------------------------------ */
/* covering / uncovering and the positivity safeguard                       */
/* ------------------------------------------------------------------------ */
/* neighbour (i+di, j+dj, k+dk) of cell (i, j, k) under the periodic sides;
 * -1 outside the grid */
static int nbr(const o3_sim *s, int i, int j, int k, int di, int dj, int dk) {
    int ii = i + di, jj = j + dj, kk = k + dk;
    if (s->c.bc[0] == O3_BC_PERIODIC) ii = wrapi(ii, s->c.nx);
    if (s->c.bc[2] == O3_BC_PERIODIC) jj = wrapi(jj, s->c.ny);
    if (s->c.bc[4] == O3_BC_PERIODIC) kk = wrapi(kk, s->c.nz);
    if (ii < 0 || ii >= s->c.nx || jj < 0 || jj >= s->c.ny || kk < 0 || kk >= s->c.nz) return -1;
    return cidx(s, ii, jj, kk);
}

/* Sec. II.C.5 in three dimensions (donor mode), applied simultaneously (as
 * in two dimensions): a covered cell's residual content goes to its fluid
 * neighbours at B in proportion to their volume fractions; an uncovered
 * cell takes sigma times its donors' contents, sigma = alphaB / (alphaB +
 * sum of the donors' alphaB), each donor losing sigma times its own; the
 * neighbours are the six face neighbours, else the 18 sharing an edge or a
 * face, else all 26; a
 * covered cell on a transmissive side with no neighbour passes its content
 * out of the domain */
static int cover_uncover3(const o3_sim *s, const double *alphaA, const double *alphaB, const double *C, double *Cn,
                          unsigned char *updated) {
    const int n = s->n, nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    int err = O3_OK;
    memcpy(Cn, C, sizeof(double) * O3_NC * n);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = cidx(s, i, j, k);
                const int covered = alphaA[c] > 0.0 && alphaB[c] == 0.0;
                const int unc = s->c.uncover_mode == O3_UNCOVER_DONOR && alphaA[c] == 0.0 && alphaB[c] > 0.0;
                if (!covered && !unc) continue;
                int nb[26], nnb = 0;
                double asum = 0.0;
                for (int pass = 0; pass < 3 && nnb == 0; ++pass)
                    for (int dk = -1; dk <= 1; ++dk)
                        for (int dj = -1; dj <= 1; ++dj)
                            for (int di = -1; di <= 1; ++di) {
                                const int nz_ = (di != 0) + (dj != 0) + (dk != 0);
                                if (nz_ == 0 || nz_ > pass + 1) continue;
                                const int cc = nbr(s, i, j, k, di, dj, dk);
                                if (cc < 0 || !(alphaB[cc] > 0.0)) continue;
                                if (s->c.uncover_mode == O3_UNCOVER_DONOR && alphaA[cc] == 0.0) continue;
                                nb[nnb++] = cc;
                                asum += alphaB[cc];
                            }
                if (nnb == 0) {
                    const int open = (s->c.bc[0] == O3_BC_TRANSMISSIVE && i == 0) ||
                                     (s->c.bc[1] == O3_BC_TRANSMISSIVE && i == nx - 1) ||
                                     (s->c.bc[2] == O3_BC_TRANSMISSIVE && j == 0) ||
                                     (s->c.bc[3] == O3_BC_TRANSMISSIVE && j == ny - 1) ||
                                     (s->c.bc[4] == O3_BC_TRANSMISSIVE && k == 0) ||
                                     (s->c.bc[5] == O3_BC_TRANSMISSIVE && k == nz - 1);
                    if (covered && open) for (int q = 0; q < O3_NC; ++q) Cn[q * n + c] = 0.0;
                    else err = O3_E_UNSTABLE;
                    continue;
                }
                if (covered) {
                    for (int m = 0; m < nnb; ++m)
                        for (int q = 0; q < O3_NC; ++q) Cn[q * n + nb[m]] += alphaB[nb[m]] / asum * C[q * n + c];
                    for (int q = 0; q < O3_NC; ++q) Cn[q * n + c] = 0.0;
                } else {
                    const double sigma = alphaB[c] / (alphaB[c] + asum);
                    for (int q = 0; q < O3_NC; ++q) {
                        double tot = 0.0;
                        for (int m = 0; m < nnb; ++m) tot += C[q * n + nb[m]];
                        Cn[q * n + c] = sigma * tot;
                        for (int m = 0; m < nnb; ++m) Cn[q * n + nb[m]] -= sigma * C[q * n + nb[m]];
                    }
                    updated[c] = 1;
                }
            }
    return err;
}

/* positivity safeguard (the two-dimensional reading, six face neighbours):
 * non-physical cells, and in the first merge cells with 0 < alphaB <
 * O3_COLLAPSE alphaA, merge with their fluid updated face neighbours; each
 * cluster shares its content in proportion to alphaB; up to O3_MIX_LAYERS
 * merges; returns the cells merged */
static int safeguard3(const o3_sim *s, double g, const double *alphaA, const double *alphaB,
                      const unsigned char *updated, double *Cn) {
    const int n = s->n, nx = s->c.nx, ny = s->c.ny;
    int mixed = 0;
    static const int D6[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int layer = 0; layer < O3_MIX_LAYERS; ++layer) {
        int *lab = (int *)malloc(sizeof(int) * n);
        unsigned char *bad = (unsigned char *)calloc((size_t)n, 1);
        int nbad = 0;
        for (int c = 0; c < n; ++c) {
            lab[c] = -1;
            const double aB = alphaB[c];
            if (!(aB > 0.0) || !updated[c]) continue;
            double q[O3_NC];
            for (int m = 0; m < O3_NC; ++m) q[m] = Cn[m * n + c] / aB;
            int b = !(q[0] > 0.0) || !(pressure3(g, q) > 0.0);
            for (int m = 0; m < O3_NC; ++m) if (!isfinite(q[m])) b = 1;
            if (layer == 0 && alphaA && aB < O3_COLLAPSE * alphaA[c]) b = 1;
            if (b) { bad[c] = 1; nbad++; }
        }
        if (nbad) {
            int *par = (int *)malloc(sizeof(int) * n);
            for (int c = 0; c < n; ++c) par[c] = c;
            for (int c = 0; c < n; ++c) {
                if (!bad[c]) continue;
                const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
                lab[c] = c;
                for (int m = 0; m < 6; ++m) {
                    const int cc = nbr(s, i, j, k, D6[m][0], D6[m][1], D6[m][2]);
                    if (cc < 0 || !(alphaB[cc] > 0.0) || !updated[cc]) continue;
                    lab[cc] = cc;
                    int ra = c, rb = cc;
                    while (par[ra] != ra) ra = par[ra];
                    while (par[rb] != rb) rb = par[rb];
                    if (ra != rb) { if (ra < rb) par[rb] = ra; else par[ra] = rb; }
                }
            }
            double *tot = (double *)calloc((size_t)n * (O3_NC + 1), sizeof(double));
            for (int c = 0; c < n; ++c) {
                if (lab[c] < 0) continue;
                int r = c; while (par[r] != r) r = par[r];
                lab[c] = r;
                tot[(O3_NC + 1) * r + O3_NC] += alphaB[c];
                for (int q = 0; q < O3_NC; ++q) tot[(O3_NC + 1) * r + q] += Cn[q * n + c];
            }
            for (int c = 0; c < n; ++c) {
                if (lab[c] < 0) continue;
                mixed++;
                const int r = lab[c];
                for (int q = 0; q < O3_NC; ++q)
                    Cn[q * n + c] = alphaB[c] * (tot[(O3_NC + 1) * r + q] / tot[(O3_NC + 1) * r + O3_NC]);
            }
            free(tot); free(par);
        }
        free(lab); free(bad);
        if (!nbad) break;
    }
    return mixed;
}

/* ------------------------------------------------------------------------ */
/* one directional sweep (eqs. Klein2DcompleteMovingMethod2a-c)             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int has;
    double d;               /* shielded distance (mid pose) */
    double FB[O3_NC];       /* boundary flux along the sweep direction */
    double QB[O3_NC];       /* boundary state */
    double wd;              /* wall velocity along the sweep */
    double n[3];            /* wall normal (mid pose), for diagnostics */
} wall3_t;

/* as the two-dimensional stab_face (eqs. Klein2DtotalfluxaMethod2,
 * Klein2shieldedFluxMethod2): bf F2D = (bf - sL - sR) F + sR [FB_R + d_R (F -
 * FB_R)] + sL [FB_L + d_L (F - FB_L)], s = max(0, bf - bfar), both scaled
 * by bf / (sL + sR) when their sum exceeds bf */
static void stab_face3(double bf, const double *F, const wall3_t *wL, double bfarL, const wall3_t *wR, double bfarR,
                       double *out) {
    double sR = 0.0, sL = 0.0;
    if (wR) sR = dmax(0.0, bf - bfarR);
    if (wL) sL = dmax(0.0, bf - bfarL);
    if (sR + sL > bf) { const double sc = bf / (sR + sL); sR *= sc; sL *= sc; }
    for (int q = 0; q < O3_NC; ++q) {
        double v = (bf - sL - sR) * F[q];
        if (sR > 0.0) v += sR * (wR->FB[q] + wR->d * (F[q] - wR->FB[q]));
        if (sL > 0.0) v += sL * (wL->FB[q] + wL->d * (F[q] - wL->FB[q]));
        out[q] = v;
    }
}

/* cell at position m along d of line l, and the d-face below it */
static void line_map(const o3_sim *s, int d, int l, int *a, int *b) {
    const int nx = s->c.nx, ny = s->c.ny;
    if (d == 0) { *a = l % ny; *b = l / ny; }
    else if (d == 1) { *a = l % nx; *b = l / nx; }
    else { *a = l % nx; *b = l / nx; }
}
static int lcell(const o3_sim *s, int d, int a, int b, int m) {
    return d == 0 ? cidx(s, m, a, b) : (d == 1 ? cidx(s, a, m, b) : cidx(s, a, b, m));
}
static int lface(const o3_sim *s, int d, int a, int b, int m) {
    return d == 0 ? fidx(s, 0, m, a, b) : (d == 1 ? fidx(s, 1, a, m, b) : fidx(s, 2, a, b, m));
}

int o3_sweep(o3_sim *s, int d, double dt) {
    if (d < 0 || d > 2) return O3_E_INVAL;
    const int n = s->n, nc = O3_NC;
    const double g = s->c.gamma;
    const int sidx = s->sweep_in_step;
    if (sidx > 0 && dt != s->dt_step) return O3_E_STATE;
    if (sidx == 0) {
        s->dt_step = dt;
        memcpy(s->Qn, s->Q, sizeof(double) * nc * n);
    }
    const double delta = s->c.U[d] * dt;
    double TA[3] = {s->T[0], s->T[1], s->T[2]}, TB[3], TM[3];
    memcpy(TB, TA, sizeof(TB));
    memcpy(TM, TA, sizeof(TM));
    TB[d] += delta;
    TM[d] += 0.5 * delta;
    o3_geom gA, gB, gM;
    geom_alloc(s, &gA); geom_alloc(s, &gB); geom_alloc(s, &gM);
    compute_geometry(s, TA, &gA);
    compute_geometry(s, TB, &gB);
    compute_geometry(s, TM, &gM);
    const int nf = nfaces(s, d);
    double *bt = (double *)malloc(sizeof(double) * nf);
    if (delta != 0.0) compute_swept(s, d, TA, delta, bt);
    else memcpy(bt, gA.b[d], sizeof(double) * nf);

    const int nal = d == 0 ? s->c.nx : (d == 1 ? s->c.ny : s->c.nz);
    const int nln = n / nal;
    const double lam = dt / s->h[d];
    const int periodic = s->c.bc[2 * d] == O3_BC_PERIODIC;

    const int gcl = s->c.uncover_mode == O3_UNCOVER_FLUX_GCL;
    unsigned char *fluidA = (unsigned char *)malloc((size_t)n), *band = (unsigned char *)malloc((size_t)n);
    for (int c = 0; c < n; ++c) {
        const int unc = gA.alpha[c] == 0.0 && gB.alpha[c] > 0.0;
        fluidA[c] = gA.alpha[c] > 0.0 || (gcl && unc);
        band[c] = gA.touched[c] || gB.touched[c];
    }
    /* sweep-start state; in flux-GCL mode an uncovered cell's provisional
     * state is the alpha_A-weighted average of its fluid face neighbours,
     * else of its 26-neighbourhood */
    double *Qs = (double *)malloc(sizeof(double) * O3_NC * n);
    memcpy(Qs, s->Q, sizeof(double) * O3_NC * n);
    int err0 = O3_OK;
    if (gcl) {
        for (int k = 0; k < s->c.nz; ++k)
            for (int j = 0; j < s->c.ny; ++j)
                for (int i = 0; i < s->c.nx; ++i) {
                    const int c = cidx(s, i, j, k);
                    if (!(gA.alpha[c] == 0.0 && gB.alpha[c] > 0.0)) continue;
                    double acc[O3_NC] = {0, 0, 0, 0, 0}, wsum = 0.0;
                    for (int pass = 0; pass < 3 && wsum == 0.0; ++pass)
                        for (int dk = -1; dk <= 1; ++dk)
                            for (int dj = -1; dj <= 1; ++dj)
                                for (int di = -1; di <= 1; ++di) {
                                    const int nzc = (di != 0) + (dj != 0) + (dk != 0);
                                    if (nzc == 0 || nzc > pass + 1) continue;
                                    const int cc = nbr(s, i, j, k, di, dj, dk);
                                    if (cc < 0 || !(gA.alpha[cc] > 0.0)) continue;
                                    wsum += gA.alpha[cc];
                                    for (int q = 0; q < O3_NC; ++q) acc[q] += gA.alpha[cc] * s->Q[q * n + cc];
                                }
                    if (wsum == 0.0) { err0 = O3_E_UNSTABLE; continue; }
                    for (int q = 0; q < O3_NC; ++q) Qs[q * n + c] = acc[q] / wsum;
                }
    }
    /* wall data per band cell (Sec. II.B, II.C.3, II.C.4) */
    wall3_t *W = (wall3_t *)calloc((size_t)n, sizeof(wall3_t));
    memset(s->wall_cell, 0, sizeof(double) * 5 * n);
    const int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int c = cidx(s, i, j, k);
                if (!band[c] || !fluidA[c]) continue;
                wall3_t *w = &W[c];
                w->has = 1;
                const int ijk[3] = {i, j, k};
                int hi3[3] = {i, j, k};
                hi3[d] += 1;
                const double blo = gM.b[d][fidx(s, d, i, j, k)], bhi = gM.b[d][fidx(s, d, hi3[0], hi3[1], hi3[2])];
                const double db = fabs(blo - bhi);
                const double ahat = gM.alpha[c] - dmin(blo, bhi);
                w->d = db > 1e-12 ? clamp01(ahat / db) : 1.0;   /* below: round-off, equally open faces */
                /* normal from aperture closure at the mid pose, into the body */
                double nL[3];
                for (int a = 0; a < 3; ++a) {
                    int up[3] = {ijk[0], ijk[1], ijk[2]};
                    up[a] += 1;
                    const double bl = gM.b[a][fidx(s, a, i, j, k)], bu = gM.b[a][fidx(s, a, up[0], up[1], up[2])];
                    nL[a] = (bl - bu) * s->h[(a + 1) % 3] * s->h[(a + 2) % 3];
                }
                const double L = sqrt(nL[0] * nL[0] + nL[1] * nL[1] + nL[2] * nL[2]);
                for (int a = 0; a < 3; ++a) w->n[a] = L > 0.0 ? nL[a] / L : 0.0;
                w->wd = s->c.U[d];
                {
                    double *wc = &s->wall_cell[5 * c];
                    wc[0] = 1.0; wc[1] = w->d; wc[2] = w->n[0]; wc[3] = w->n[1]; wc[4] = w->n[2];
                }
                double qn[O3_NC], qc[O3_NC];
                const int fresh = s->Qn[c] != s->Qn[c];
                for (int q = 0; q < nc; ++q) { qc[q] = Qs[q * n + c]; qn[q] = fresh ? qc[q] : s->Qn[q * n + c]; }
                double rs, ps_step, us[3], rs2, ps_sw, us2[3];
                o3_wall_state(g, qn, w->n, s->c.U, &rs, &ps_step, us);
                o3_wall_state(g, qc, w->n, s->c.U, &rs2, &ps_sw, us2);
                const double Eadv = ps_step / (g - 1.0) + 0.5 * rs * (us[0] * us[0] + us[1] * us[1] + us[2] * us[2]);
                const double ud = us[d];
                w->QB[0] = rs;
                for (int m = 0; m < 3; ++m) w->QB[1 + m] = rs * us[m];
                w->QB[4] = Eadv;
                w->FB[0] = rs * ud;
                for (int m = 0; m < 3; ++m) w->FB[1 + m] = rs * ud * us[m] + (m == d ? ps_sw : 0.0);
                w->FB[4] = ud * (Eadv + ps_step);
            }

    double *C = (double *)calloc((size_t)nc * n, sizeof(double));
    unsigned char *updated = (unsigned char *)calloc((size_t)n, 1);
    for (int q = 0; q < nc; ++q) s->wall_last[q] = 0.0;
    const int len = nal + 4;
    double *Ql = (double *)malloc(sizeof(double) * nc * len);
    double *QLb = (double *)malloc(sizeof(double) * nc * len), *QRb = (double *)malloc(sizeof(double) * nc * len);
    unsigned char *fl = (unsigned char *)malloc((size_t)len);
    double *F2 = (double *)malloc(sizeof(double) * nc * (nal + 1));
    const int in = 1 + d;
    for (int l = 0; l < nln; ++l) {
        int la, lb;
        line_map(s, d, l, &la, &lb);
        for (int kk = -2; kk < nal + 2; ++kk) {
            int m = kk, flip = 0;
            if (kk < 0 || kk >= nal) {
                const int bc = s->c.bc[kk < 0 ? 2 * d : 2 * d + 1];
                if (bc == O3_BC_PERIODIC) m = wrapi(kk, nal);
                else { m = kk < 0 ? -1 - kk : 2 * nal - 1 - kk; flip = bc == O3_BC_REFLECTIVE; }
            }
            const int c = lcell(s, d, la, lb, m);
            fl[kk + 2] = fluidA[c];
            for (int q = 0; q < nc; ++q) Ql[q * len + kk + 2] = Qs[q * n + c];
            if (flip) Ql[in * len + kk + 2] = -Ql[in * len + kk + 2];
        }
        /* MUSCL-Hancock */
        for (int kk = -1; kk <= nal; ++kk) {
            const int a = kk + 2;
            if (!fl[a]) continue;
            const int lim = fl[a - 1] && fl[a + 1];
            double qL[O3_NC], qR[O3_NC], fLv[O3_NC], fRv[O3_NC];
            for (int q = 0; q < nc; ++q) {
                const double sl = lim ? vanleer(Ql[q * len + a] - Ql[q * len + a - 1], Ql[q * len + a + 1] - Ql[q * len + a]) : 0.0;
                qL[q] = Ql[q * len + a] - 0.5 * sl;
                qR[q] = Ql[q * len + a] + 0.5 * sl;
            }
            euler_flux3(g, d, qL, fLv);
            euler_flux3(g, d, qR, fRv);
            for (int q = 0; q < nc; ++q) {
                const double dfl = 0.5 * lam * (fLv[q] - fRv[q]);
                QLb[q * len + a] = qL[q] + dfl;
                QRb[q * len + a] = qR[q] + dfl;
            }
            double eL[O3_NC], eR[O3_NC];
            for (int q = 0; q < nc; ++q) { eL[q] = QLb[q * len + a]; eR[q] = QRb[q * len + a]; }
            if (!(eL[0] > 0.0) || !(eR[0] > 0.0) || !(pressure3(g, eL) > 0.0) || !(pressure3(g, eR) > 0.0))
                for (int q = 0; q < nc; ++q) { QLb[q * len + a] = Ql[q * len + a]; QRb[q * len + a] = Ql[q * len + a]; }
        }
        /* faces m = 0..nal (face m between cells m-1 and m) */
        const int nfl = periodic ? nal : nal + 1;
        for (int m = 0; m < nfl; ++m) {
            const int a = m + 2;
            const double bf = bt[lface(s, d, la, lb, m)];
            for (int q = 0; q < nc; ++q) F2[nc * m + q] = 0.0;
            if (!(fl[a - 1] && fl[a] && bf > 0.0)) continue;
            double qL[O3_NC], qR[O3_NC], F[O3_NC];
            for (int q = 0; q < nc; ++q) { qL[q] = QRb[q * len + a - 1]; qR[q] = QLb[q * len + a]; }
            o3_hllc(g, d, qL, qR, F);
            const int mR = m < nal ? m : (periodic ? 0 : -1);
            const int mL = m - 1 >= 0 ? m - 1 : (periodic ? nal - 1 : -1);
            const wall3_t *wR = NULL, *wL = NULL;
            double bfarR = 0.0, bfarL = 0.0;
            if (mR >= 0) {
                const int cR = lcell(s, d, la, lb, mR);
                bfarR = bt[lface(s, d, la, lb, mR + 1 < nal || !periodic ? mR + 1 : 0)];
                if (W[cR].has) wR = &W[cR];
            }
            if (mL >= 0) {
                const int cL = lcell(s, d, la, lb, mL);
                bfarL = bt[lface(s, d, la, lb, mL)];
                if (W[cL].has) wL = &W[cL];
            }
            stab_face3(bf, F, wL, bfarL, wR, bfarR, &F2[nc * m]);
        }
        if (periodic) for (int q = 0; q < nc; ++q) F2[nc * nal + q] = F2[q];
        /* conservative update in alpha Q form */
        for (int m = 0; m < nal; ++m) {
            const int c = lcell(s, d, la, lb, m);
            if (!fluidA[c]) continue;
            const double blo = bt[lface(s, d, la, lb, m)];
            const double bhi = bt[lface(s, d, la, lb, m + 1 < nal || !periodic ? m + 1 : 0)];
            const double aA = gA.alpha[c];
            for (int q = 0; q < nc; ++q) {
                double v = aA * Qs[q * n + c] + lam * (F2[nc * m + q] - F2[nc * (m + 1) + q]);
                if (blo != bhi && W[c].has) {
                    const double wt = lam * (bhi - blo) * (W[c].FB[q] - W[c].wd * W[c].QB[q]);
                    v += wt;
                    s->wall_last[q] += wt;
                }
                C[q * n + c] = v;
            }
            updated[c] = 1;
        }
    }
    free(Ql); free(QLb); free(QRb); free(fl); free(F2);

    double *Cn = (double *)malloc(sizeof(double) * nc * n);
    int err = cover_uncover3(s, gA.alpha, gB.alpha, C, Cn, updated);
    if (err0 != O3_OK) err = err0;
    s->mixed_last = safeguard3(s, g, gA.alpha, gB.alpha, updated, Cn);
    for (int c = 0; c < n; ++c) {
        const double aB = gB.alpha[c];
        for (int q = 0; q < nc; ++q) s->Q[q * n + c] = (aB > 0.0 && updated[c]) ? Cn[q * n + c] / aB : NAN;
        if (aB > 0.0 && !updated[c]) err = O3_E_UNSTABLE;
        if (aB > 0.0 && updated[c]) {
            double q5[O3_NC];
            for (int q = 0; q < nc; ++q) q5[q] = s->Q[q * n + c];
            int bad = !(q5[0] > 0.0) || !(pressure3(g, q5) > 0.0);
            for (int q = 0; q < nc; ++q) if (!isfinite(q5[q])) bad = 1;
            if (bad) err = O3_E_UNSTABLE;
        }
    }
    free(Cn); free(C); free(updated); free(W); free(fluidA); free(band); free(bt); free(Qs);
    geom_free(&gA); geom_free(&gB); geom_free(&gM);
    s->T[d] = TB[d];
    if (++s->sweep_in_step == 3) {
        s->sweep_in_step = 0;
        s->t += dt;
        s->step++;
    }
    if (err != O3_OK) s->status = err;
    return err;
}

/* one step: x, y, z on even steps, z, y, x on odd steps */
int o3_step(o3_sim *s, double dt) {
    if (s->sweep_in_step != 0) return O3_E_STATE;
    const int odd = (int)(s->step & 1);
    int err = O3_OK;
    for (int m = 0; m < 3; ++m) {
        const int r = o3_sweep(s, odd ? 2 - m : m, dt);
        if (r != O3_OK && err == O3_OK) err = r;
    }
    return err;
}

double o3_cfl_dt(const o3_sim *s) {
    const int n = s->n;
    double S[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < n; ++c) {
        if (s->Q[c] != s->Q[c]) continue;
        double q[O3_NC];
        for (int m = 0; m < O3_NC; ++m) q[m] = s->Q[m * n + c];
        const double cs = sqrt(s->c.gamma * pressure3(s->c.gamma, q) / q[0]);
        for (int a = 0; a < 3; ++a) S[a] = dmax(S[a], fabs(q[1 + a] / q[0]) + cs);
    }
    double r = 1e300;
    for (int a = 0; a < 3; ++a) {
        if (s->c.nplane > 0) S[a] = dmax(S[a], fabs(s->c.U[a]));
        if (S[a] <= 0.0) S[a] = 1e-300;
        r = dmin(r, s->h[a] / S[a]);
    }
    return s->c.cfl * r;
}

/* ------------------------------------------------------------------------ */
/* interface                                                                */
/* ------------------------------------------------------------------------ */
o3_sim *o3_create(const o3_config *cfg, const double *bb) {
    if (!cfg || cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nplane < 0 || cfg->nplane > O3_MAXP) return NULL;
    /* the stencil's two ghost cells mirror two cells of a non-periodic axis */
    const int nax[3] = {cfg->nx, cfg->ny, cfg->nz};
    for (int a = 0; a < 3; ++a) if (nax[a] < 2 && cfg->bc[2 * a] != O3_BC_PERIODIC) return NULL;
    o3_sim *s = (o3_sim *)calloc(1, sizeof(o3_sim));
    s->c = *cfg;
    memcpy(s->bb, bb, sizeof(s->bb));
    s->h[0] = (cfg->x1 - cfg->x0) / cfg->nx;
    s->h[1] = (cfg->y1 - cfg->y0) / cfg->ny;
    s->h[2] = (cfg->z1 - cfg->z0) / cfg->nz;
    s->n = cfg->nx * cfg->ny * cfg->nz;
    s->Q = (double *)calloc((size_t)O3_NC * s->n, sizeof(double));
    s->Qn = (double *)calloc((size_t)O3_NC * s->n, sizeof(double));
    s->wall_cell = (double *)calloc((size_t)5 * s->n, sizeof(double));
    return s;
}

void o3_destroy(o3_sim *s) {
    if (!s) return;
    free(s->Q); free(s->Qn); free(s->wall_cell); free(s);
}

/* state Q (O3_NC planes of nx*ny*nz, x fastest) at time t with the body at
 * translation T; solid cells become NaN */
int o3_set_state(o3_sim *s, const double *Q, double t, const double *T, long step) {
    s->t = t;
    memcpy(s->T, T, sizeof(s->T));
    s->step = step;
    s->sweep_in_step = 0;
    s->status = O3_OK;
    o3_geom g;
    geom_alloc(s, &g);
    compute_geometry(s, s->T, &g);
    for (int c = 0; c < s->n; ++c)
        for (int q = 0; q < O3_NC; ++q) s->Q[q * s->n + c] = g.alpha[c] > 0.0 ? Q[q * s->n + c] : NAN;
    geom_free(&g);
    return O3_OK;
}

/* state, volume fractions at the current pose, clock {t, X, Y, Z, step} */
int o3_get_state(o3_sim *s, double *Q, double *alpha, double *clock) {
    if (Q) memcpy(Q, s->Q, sizeof(double) * O3_NC * s->n);
    if (alpha) {
        o3_geom g;
        geom_alloc(s, &g);
        compute_geometry(s, s->T, &g);
        memcpy(alpha, g.alpha, sizeof(double) * s->n);
        geom_free(&g);
    }
    if (clock) {
        clock[0] = s->t;
        for (int a = 0; a < 3; ++a) clock[1 + a] = s->T[a];
        clock[4] = (double)s->step;
    }
    return s->status;
}

/* geometry at translation T: alpha (n), touched (n), apertures of the x-,
 * y- and z-faces (any may be NULL) */
int o3_geometry(o3_sim *s, const double *T, double *alpha, unsigned char *touched, double *bx, double *by,
                double *bz) {
    o3_geom g;
    geom_alloc(s, &g);
    compute_geometry(s, T, &g);
    if (alpha) memcpy(alpha, g.alpha, sizeof(double) * s->n);
    if (touched) memcpy(touched, g.touched, (size_t)s->n);
    if (bx) memcpy(bx, g.b[0], sizeof(double) * nfaces(s, 0));
    if (by) memcpy(by, g.b[1], sizeof(double) * nfaces(s, 1));
    if (bz) memcpy(bz, g.b[2], sizeof(double) * nfaces(s, 2));
    geom_free(&g);
    return O3_OK;
}

/* time-averaged apertures of the d-faces for a move by delta from T */
int o3_swept(o3_sim *s, int d, const double *T, double delta, double *out) {
    if (d < 0 || d > 2) return O3_E_INVAL;
    if (delta == 0.0) {
        o3_geom g;
        geom_alloc(s, &g);
        compute_geometry(s, T, &g);
        memcpy(out, g.b[d], sizeof(double) * nfaces(s, d));
        geom_free(&g);
        return O3_OK;
    }
    compute_swept(s, d, T, delta, out);
    return O3_OK;
}

/* the last sweep's wall data per cell (5 n doubles: has, d, n_x, n_y, n_z) */
void o3_last_wall(const o3_sim *s, double *out) { memcpy(out, s->wall_cell, sizeof(double) * 5 * s->n); }

/* the covering / uncovering step alone on given fields (alpha at poses A
 * and B, the contents C after the flux update; Cn and the updated flags out),
 * for tests of its neighbour passes and shares */
int o3_cover_uncover(o3_sim *s, const double *alphaA, const double *alphaB, const double *C, double *Cn,
                     unsigned char *updated) {
    return cover_uncover3(s, alphaA, alphaB, C, Cn, updated);
}

/* the positivity safeguard alone on given fields (Cn in place), for tests
 * of its clusters and shares; returns the cells merged */
int o3_safeguard(o3_sim *s, const double *alphaA, const double *alphaB, const unsigned char *updated, double *Cn) {
    return safeguard3(s, s->c.gamma, alphaA, alphaB, updated, Cn);
}

/* the last sweep's summed wall terms (O3_NC) and cells merged */
int o3_last_sweep(const o3_sim *s, double *wall) {
    if (wall) memcpy(wall, s->wall_last, sizeof(double) * O3_NC);
    return s->mixed_last;
}

/* volume of the body inside the box [lo, hi] with the body at T (for pins) */
double o3_solid_volume(const o3_sim *s, const double *T, const double *lo, const double *hi) {
    double cpos[O3_MAXP];
    posed_planes(&s->c, T, cpos);
    return solid_volume(&s->c, cpos, lo, hi, NULL);
}
