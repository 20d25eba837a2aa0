/*
 * mbref.c -- plain, slow FP64 CPU oracle for one directional sweep of the
 * moving-boundary, flux-stabilised Cartesian cut-cell method of Bennett,
 * Nikiforakis & Klein (arXiv 1711.11361).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * Every step follows the paper in its own order, written out over whole
 * arrays with no fusion or blocking:
 *   Sec. II.A  finite-volume update (eq. EulerDiscreteRegular / EulerDiscreteCutCell)
 *   Sec. II.B  static flux stabilisation (eqs. Klein2Dtotalfluxa, Klein2Dunshieldeda,
 *              Klein2shieldedFlux, Klein2DalphaHat, KleinAdvectivePressureSplitA)
 *   Sec. II.C.3 moving-wall ghost state (eq. riemann_wallvel) and the resultant
 *              wall contribution (eq. Klein2DMovingResultantFluxes)
 *   Sec. II.C.4 time-averaged apertures / distance (eqs. timeAveragedBeta,
 *              timeAveragedAlpha, Klein2shieldedFluxMethod2,
 *              ModifiedBoundaryFluxMethod2, Klein2DtotalfluxaMethod2,
 *              Klein2DcompleteMovingMethod2a-b)
 *   Sec. II.C.5 covering / uncovering (eqs. volumeWeighting,
 *              cutCellInitialisation, cutCellInitialisationDonorCellUpdate,
 *              massDeficitEquation, cutCellCoverDonation)
 *   Sec. II.C.5 (last paragraph) standard fluxes: MUSCL-Hancock + HLLC + van Leer.
 *
 * Geometry is the plain definition: the body is a union of polygons with
 * disjoint interiors (two may touch along an edge, as a piston rod sliding in
 * its tube; areas and solid lengths add over the polygons, and the wall
 * normal from aperture closure is zero where only such a contact is left in
 * a cell); cell volume fractions are areas from Sutherland-Hodgman clipping,
 * face apertures are lengths from sorted line/polygon crossings, and the
 * swept (time-averaged) aperture of a face under translation is the fluid
 * fraction of the strip the face sweeps through the body, which is the exact
 * value of the time average in eq. timeAveragedBeta.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add anywhere).
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MIX_LAYERS 8   /* merges of the positivity safeguard per sweep */
#define OR_COLLAPSE 0.01  /* a cell keeping less of its volume over a sweep seeds a merge */
#define OR_EULER 0
#define OR_ADVECTION 1
#define OR_BC_TRANSMISSIVE 0
#define OR_BC_REFLECTIVE 1
#define OR_BC_PERIODIC 2
#define OR_UNCOVER_DONOR 0
#define OR_UNCOVER_FLUX_GCL 1

#define OR_OK 0
#define OR_E_INVAL -1
#define OR_E_NOMEM -2
#define OR_E_UNSTABLE -4
#define OR_E_STATE -6

typedef struct {
    int nx, ny;
    double x0, y0, x1, y1;
    int bc[4];              /* x-low, x-high, y-low, y-high */
    int equation;           /* OR_EULER (4 components) or OR_ADVECTION (1) */
    double adv[2];          /* advection velocity (OR_ADVECTION only) */
    double gamma;
    double cfl;
    int uncover_mode;       /* OR_UNCOVER_DONOR (paper) or OR_UNCOVER_FLUX_GCL */
    int npoly;
    const int *poly_start;  /* npoly+1 offsets into vx/vy; each polygon CCW */
    const int *poly_moving; /* 1: moves with the body motion, 0: fixed */
    const double *vx, *vy;  /* vertices at t = 0 */
    double U[2];            /* translation velocity */
    double pivot[2];        /* rotation centre at t = 0 */
    double a0, a1, omega;   /* theta(t) = a0 + a1 sin(omega t) */
    int axisym;             /* Euler in axisymmetric form: y is the radius from the axis y = y0 */
} or_config;

typedef struct {
    double *alpha;          /* nx*ny volume fraction */
    unsigned char *touched; /* nx*ny: a polygon edge meets the closed cell */
    unsigned char *moving;  /* nx*ny: a moving polygon's edge meets the closed cell */
    double *bx;             /* (nx+1)*ny aperture of x-face i in row j: [j*(nx+1)+i] */
    double *by;             /* nx*(ny+1) aperture of y-face j in column i: [j*nx+i] */
} or_geom;

typedef struct {
    or_config c;
    int *pstart, *pmoving;
    double *vx, *vy;
    int nv;
    double dx, dy;
    int nc;
    double *Q, *Qn;
    double t, X, Y;
    long step;
    int sweep_in_step;
    double dt_step;
    int status;
    double rmax;            /* largest distance of a moving vertex from the pivot */
    double *px, *py;        /* posed vertices (scratch) */
    double wall_last[4];    /* sum over cells of the last sweep's wall terms (content units) */
    int mixed_last;         /* cells merged by the positivity safeguard in the last sweep */
    /* last sweep, kept for diagnostics: direction, time-averaged apertures
     * of its faces, and per cell the wall data (has, d, n_x, n_y, w_x, w_y) */
    int last_dir;
    double *bt_last;
    double *wall_cell;
} or_sim;

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double clamp01(double a) { return a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a); }
/* Volume fractions below this are treated as solid: their content would be
 * round-off of neighbouring contents (a reading; the paper sets no floor). */
#define OR_ALPHA_MIN 1e-10

static double node_x(const or_sim *s, int i) { return s->c.x0 + (double)i * s->dx; }
static double node_y(const or_sim *s, int j) { return s->c.y0 + (double)j * s->dy; }

static int rotating(const or_sim *s) { return s->c.a0 != 0.0 || s->c.a1 != 0.0; }
static double theta_at(const or_sim *s, double tau) { return s->c.a0 + s->c.a1 * sin(s->c.omega * tau); }
static double thetadot_at(const or_sim *s, double tau) { return s->c.a1 * s->c.omega * cos(s->c.omega * tau); }

/* Pose of the body: moving polygons are rotated by theta about the pivot and
 * translated by (X, Y); fixed polygons stay where they are. */
static void pose_vertices(or_sim *s, double X, double Y, double th, int rot) {
    double c = cos(th), sn = sin(th);
    for (int p = 0; p < s->c.npoly; ++p) {
        for (int k = s->pstart[p]; k < s->pstart[p + 1]; ++k) {
            if (!s->pmoving[p]) { s->px[k] = s->vx[k]; s->py[k] = s->vy[k]; continue; }
            if (rot) {
                double ddx = s->vx[k] - s->c.pivot[0];
                double ddy = s->vy[k] - s->c.pivot[1];
                double rx = c * ddx - sn * ddy;
                double ry = sn * ddx + c * ddy;
                s->px[k] = (s->c.pivot[0] + rx) + X;
                s->py[k] = (s->c.pivot[1] + ry) + Y;
            } else {
                s->px[k] = s->vx[k] + X;
                s->py[k] = s->vy[k] + Y;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* geometry: Sutherland-Hodgman clipping and line crossings                 */
/* ------------------------------------------------------------------------ */
typedef struct { double *x, *y; int n, cap; } poly_t;

static void poly_reserve(poly_t *p, int n) {
    if (n <= p->cap) return;
    int cap = n * 2 + 16;
    p->x = (double *)realloc(p->x, sizeof(double) * cap);
    p->y = (double *)realloc(p->y, sizeof(double) * cap);
    p->cap = cap;
}
static void poly_free(poly_t *p) { free(p->x); free(p->y); p->x = p->y = NULL; p->n = p->cap = 0; }

/* Clip `in` against one axis-aligned half-plane: axis 0 -> x, 1 -> y;
 * keep_ge != 0 keeps coord >= v, else coord <= v.  Textbook Sutherland-Hodgman. */
static void sh_clip(const poly_t *in, poly_t *out, int axis, double v, int keep_ge) {
    out->n = 0;
    poly_reserve(out, 2 * in->n + 2);
    for (int k = 0; k < in->n; ++k) {
        int k1 = (k + 1) % in->n;
        double ax = in->x[k], ay = in->y[k], bx = in->x[k1], by = in->y[k1];
        double ca = axis == 0 ? ax : ay, cb = axis == 0 ? bx : by;
        int ina = keep_ge ? (ca >= v) : (ca <= v);
        int inb = keep_ge ? (cb >= v) : (cb <= v);
        if (ina && inb) {
            out->x[out->n] = bx; out->y[out->n] = by; out->n++;
        } else if (ina != inb) {
            double tt = (v - ca) / (cb - ca);
            double ix, iy;
            if (axis == 0) { ix = v; iy = ay + tt * (by - ay); }
            else { iy = v; ix = ax + tt * (bx - ax); }
            out->x[out->n] = ix; out->y[out->n] = iy; out->n++;
            if (inb) { out->x[out->n] = bx; out->y[out->n] = by; out->n++; }
        }
    }
}

/* Shoelace area of a polygon, coordinates taken relative to (ox, oy). */
static double shoelace(const poly_t *p, double ox, double oy) {
    double a = 0.0;
    for (int k = 0; k < p->n; ++k) {
        int k1 = (k + 1) % p->n;
        double xa = p->x[k] - ox, ya = p->y[k] - oy, xb = p->x[k1] - ox, yb = p->y[k1] - oy;
        a += xa * yb - xb * ya;
    }
    return 0.5 * a;
}

/* Touch predicate: does edge a->b meet the closed cell [xl,xr]x[yb,yt]?  The
 * edge is clipped to the closed column and its y-extent there compared with
 * the row. */
static int edge_touches(double xa, double ya, double xb, double yb_, double xl, double xr, double ylo_c, double yhi_c) {
    double lo = dmin(xa, xb), hi = dmax(xa, xb);
    if (hi < xl || lo > xr) return 0;
    double e0, e1;
    if (xa == xb) {
        e0 = ya; e1 = yb_;
    } else {
        double xc0 = lo > xl ? lo : xl;
        double xc1 = hi < xr ? hi : xr;
        double slope = (yb_ - ya) / (xb - xa);
        e0 = (xc0 == xa) ? ya : ((xc0 == xb) ? yb_ : ya + (xc0 - xa) * slope);
        e1 = (xc1 == xa) ? ya : ((xc1 == xb) ? yb_ : ya + (xc1 - xa) * slope);
    }
    double elo = dmin(e0, e1), ehi = dmax(e0, e1);
    return ehi >= ylo_c && elo <= yhi_c;
}

/* Even-odd point-in-body test (horizontal ray). */
static int point_inside(const or_sim *s, double x, double y) {
    int in = 0;
    for (int p = 0; p < s->c.npoly; ++p) {
        int a0 = s->pstart[p], n = s->pstart[p + 1] - a0;
        for (int k = 0; k < n; ++k) {
            double xa = s->px[a0 + k], ya = s->py[a0 + k];
            double xb = s->px[a0 + (k + 1) % n], yb = s->py[a0 + (k + 1) % n];
            if ((ya > y) != (yb > y)) {
                double xi = xa + (y - ya) * (xb - xa) / (yb - ya);
                if (x < xi) in = !in;
            }
        }
    }
    return in;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Solid length of the segment {v} x [lo,hi] (axis = 0: vertical line x = v)
 * or [lo,hi] x {v} (axis = 1: horizontal line y = v): crossings of the line
 * with each polygon, sorted, paired into inside intervals. */
static double solid_length(const or_sim *s, int axis, double v, double lo, double hi, double *buf) {
    double L = 0.0;
    for (int p = 0; p < s->c.npoly; ++p) {
        int a0 = s->pstart[p], n = s->pstart[p + 1] - a0, m = 0;
        for (int k = 0; k < n; ++k) {
            double xa = s->px[a0 + k], ya = s->py[a0 + k];
            double xb = s->px[a0 + (k + 1) % n], yb = s->py[a0 + (k + 1) % n];
            double ca = axis == 0 ? xa : ya, cb = axis == 0 ? xb : yb;
            if ((ca < v) != (cb < v)) {
                double oa = axis == 0 ? ya : xa, ob = axis == 0 ? yb : xb;
                buf[m++] = oa + (v - ca) * (ob - oa) / (cb - ca);
            }
        }
        qsort(buf, (size_t)m, sizeof(double), cmp_double);
        for (int k = 0; k + 1 < m; k += 2) {
            double a = dmax(buf[k], lo), b = dmin(buf[k + 1], hi);
            if (b > a) L += b - a;
        }
    }
    return L;
}

/* Clip every polygon to the horizontal strip [ylo, yhi]; the pieces are
 * appended as separate polygons into `rows` (up to npoly entries). */
static void clip_to_row(const or_sim *s, double ylo, double yhi, poly_t *rows, poly_t *tmp) {
    for (int p = 0; p < s->c.npoly; ++p) {
        int a0 = s->pstart[p], n = s->pstart[p + 1] - a0;
        poly_reserve(tmp, n);
        tmp->n = n;
        memcpy(tmp->x, s->px + a0, sizeof(double) * n);
        memcpy(tmp->y, s->py + a0, sizeof(double) * n);
        poly_t mid = {0};
        sh_clip(tmp, &mid, 1, ylo, 1);
        sh_clip(&mid, &rows[p], 1, yhi, 0);
        poly_free(&mid);
    }
}

/* Solid area of [xl,xr] x (row already clipped) from the row pieces. */
static double solid_area_in_row(const or_sim *s, const poly_t *rows, double xl, double xr, double ox, double oy) {
    double A = 0.0;
    poly_t a = {0}, b = {0};
    for (int p = 0; p < s->c.npoly; ++p) {
        if (rows[p].n < 3) continue;
        sh_clip(&rows[p], &a, 0, xl, 1);
        if (a.n < 3) continue;
        sh_clip(&a, &b, 0, xr, 0);
        if (b.n < 3) continue;
        A += shoelace(&b, ox, oy);
    }
    poly_free(&a); poly_free(&b);
    return A;
}

static void bbox_posed(const or_sim *s, double *bb) {
    bb[0] = bb[2] = 1e300; bb[1] = bb[3] = -1e300;
    for (int k = 0; k < s->nv; ++k) {
        bb[0] = dmin(bb[0], s->px[k]); bb[1] = dmax(bb[1], s->px[k]);
        bb[2] = dmin(bb[2], s->py[k]); bb[3] = dmax(bb[3], s->py[k]);
    }
}

static void geom_alloc(const or_sim *s, or_geom *g) {
    int nx = s->c.nx, ny = s->c.ny;
    g->alpha = (double *)malloc(sizeof(double) * nx * ny);
    g->touched = (unsigned char *)malloc((size_t)nx * ny);
    g->moving = (unsigned char *)malloc((size_t)nx * ny);
    g->bx = (double *)malloc(sizeof(double) * (nx + 1) * ny);
    g->by = (double *)malloc(sizeof(double) * nx * (ny + 1));
}
static void geom_free(or_geom *g) { free(g->alpha); free(g->touched); free(g->moving); free(g->bx); free(g->by); }

/* Volume fractions, touch flags and instantaneous apertures of every cell and
 * face at the pose currently held in px/py (Sec. II.A: alpha = fluid volume /
 * cell volume; Sec. II.B: beta = fluid fraction of a face). */
static void compute_geometry(const or_sim *s, or_geom *g) {
    int nx = s->c.nx, ny = s->c.ny;
    double bb[4];
    bbox_posed(s, bb);
    for (int k = 0; k < nx * ny; ++k) { g->alpha[k] = 1.0; g->touched[k] = 0; g->moving[k] = 0; }
    for (int k = 0; k < (nx + 1) * ny; ++k) g->bx[k] = 1.0;
    for (int k = 0; k < nx * (ny + 1); ++k) g->by[k] = 1.0;
    if (s->nv == 0) return;
    double *buf = (double *)malloc(sizeof(double) * (s->nv + 4));
    poly_t *rows = (poly_t *)calloc((size_t)s->c.npoly, sizeof(poly_t));
    poly_t tmp = {0};
    for (int j = 0; j < ny; ++j) {
        double yl = node_y(s, j), yh = node_y(s, j + 1);
        if (yh < bb[2] || yl > bb[3]) continue;
        clip_to_row(s, yl, yh, rows, &tmp);
        for (int i = 0; i < nx; ++i) {
            double xl = node_x(s, i), xr = node_x(s, i + 1);
            if (xr < bb[0] || xl > bb[1]) continue;
            int touched = 0, mov = 0;
            for (int p = 0; p < s->c.npoly; ++p) {
                int a0 = s->pstart[p], n = s->pstart[p + 1] - a0;
                for (int k = 0; k < n; ++k) {
                    int kb = a0 + (k + 1) % n;
                    if (edge_touches(s->px[a0 + k], s->py[a0 + k], s->px[kb], s->py[kb], xl, xr, yl, yh)) {
                        touched = 1;
                        if (s->pmoving[p]) mov = 1;
                    }
                }
            }
            int c = j * nx + i;
            g->touched[c] = (unsigned char)touched;
            g->moving[c] = (unsigned char)mov;
            if (touched) {
                double A = solid_area_in_row(s, rows, xl, xr, xl, yl);
                double a = clamp01(1.0 - A / (s->dx * s->dy));
                g->alpha[c] = a < OR_ALPHA_MIN ? 0.0 : a;
            } else {
                double xc = s->c.x0 + ((double)i + 0.5) * s->dx;
                double yc = s->c.y0 + ((double)j + 0.5) * s->dy;
                g->alpha[c] = point_inside(s, xc, yc) ? 0.0 : 1.0;
            }
        }
    }
    /* vertical faces: line x = x_i */
    for (int i = 0; i <= nx; ++i) {
        double xf = node_x(s, i);
        if (xf < bb[0] || xf > bb[1]) continue;
        for (int j = 0; j < ny; ++j) {
            double yl = node_y(s, j), yh = node_y(s, j + 1);
            if (yh < bb[2] || yl > bb[3]) continue;
            g->bx[j * (nx + 1) + i] = clamp01(1.0 - solid_length(s, 0, xf, yl, yh, buf) / s->dy);
        }
    }
    /* horizontal faces: line y = y_j */
    for (int j = 0; j <= ny; ++j) {
        double yf = node_y(s, j);
        if (yf < bb[2] || yf > bb[3]) continue;
        for (int i = 0; i < nx; ++i) {
            double xl = node_x(s, i), xr = node_x(s, i + 1);
            if (xr < bb[0] || xl > bb[1]) continue;
            g->by[j * nx + i] = clamp01(1.0 - solid_length(s, 1, yf, xl, xr, buf) / s->dx);
        }
    }
    for (int p = 0; p < s->c.npoly; ++p) poly_free(&rows[p]);
    free(rows); poly_free(&tmp); free(buf);
}

/* Swept aperture of every d-face under a translation by `delta` (world units)
 * along d during the sweep (eq. timeAveragedBeta evaluated exactly): with the
 * body at its start pose, the fraction of the face covered at time t equals
 * the covered fraction of the segment displaced by -(t/dt)*delta, so the
 * time average is the fluid area fraction of the strip between the face and
 * its displaced copy. */
static void compute_swept(const or_sim *s, int d, double delta, double *out) {
    int nx = s->c.nx, ny = s->c.ny;
    double bb[4];
    bbox_posed(s, bb);
    int nf = d == 0 ? (nx + 1) * ny : nx * (ny + 1);
    for (int k = 0; k < nf; ++k) out[k] = 1.0;
    if (s->nv == 0) return;
    /* each strip's area is divided by its realised width (sr - sl), not by
     * |delta|, so that rounding of x_f - delta does not bias thin strips */
    poly_t *rows = (poly_t *)calloc((size_t)s->c.npoly, sizeof(poly_t));
    poly_t tmp = {0};
    if (d == 0) {
        for (int j = 0; j < ny; ++j) {
            double yl = node_y(s, j), yh = node_y(s, j + 1);
            if (yh < bb[2] || yl > bb[3]) continue;
            clip_to_row(s, yl, yh, rows, &tmp);
            for (int i = 0; i <= nx; ++i) {
                double xf = node_x(s, i);
                double sl = delta > 0 ? xf - delta : xf, sr = delta > 0 ? xf : xf - delta;
                if (sr < bb[0] || sl > bb[1]) continue;
                double A = solid_area_in_row(s, rows, sl, sr, xf, yl);
                out[j * (nx + 1) + i] = clamp01(1.0 - A / ((sr - sl) * s->dy));
            }
        }
    } else {
        /* horizontal strips: clip to the strip's rows, then to the column */
        for (int j = 0; j <= ny; ++j) {
            double yf = node_y(s, j);
            double sl = delta > 0 ? yf - delta : yf, sr = delta > 0 ? yf : yf - delta;
            if (sr < bb[2] || sl > bb[3]) continue;
            clip_to_row(s, sl, sr, rows, &tmp);
            for (int i = 0; i < nx; ++i) {
                double xl = node_x(s, i), xr = node_x(s, i + 1);
                if (xr < bb[0] || xl > bb[1]) continue;
                double A = solid_area_in_row(s, rows, xl, xr, xl, yf);
                out[j * nx + i] = clamp01(1.0 - A / ((sr - sl) * s->dx));
            }
        }
    }
    for (int p = 0; p < s->c.npoly; ++p) poly_free(&rows[p]);
    free(rows); poly_free(&tmp);
}

/* ------------------------------------------------------------------------ */
/* physics: Euler flux, HLLC, van Leer, MUSCL-Hancock (Sec. II.C.5)         */
/* ------------------------------------------------------------------------ */
/* Conserved Q = [rho, rho u, rho v, E]; e = p/(rho (gamma-1)) (Sec. II.A). */
static double pressure(double g, const double *q) {
    return (g - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

/* Physical flux along direction d (0: x, 1: y). */
static void euler_flux(double g, int d, const double *q, double *f) {
    double rho = q[0], u = q[1] / rho, v = q[2] / rho, p = pressure(g, q);
    double un = d == 0 ? u : v;
    f[0] = rho * un;
    f[1] = q[1] * un + (d == 0 ? p : 0.0);
    f[2] = q[2] * un + (d == 1 ? p : 0.0);
    f[3] = un * (q[3] + p);
}

/* HLLC with Davis wave-speed estimates (Toro, Riemann Solvers ch. 10). */
void or_hllc(double g, int d, const double *qL, const double *qR, double *F) {
    int in = d == 0 ? 1 : 2;
    double rL = qL[0], rR = qR[0];
    double uL = qL[in] / rL, uR = qR[in] / rR;
    double pL = pressure(g, qL), pR = pressure(g, qR);
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double SL = dmin(uL - cL, uR - cR), SR = dmax(uL + cL, uR + cR);
    double fL[4], fR[4];
    if (SL >= 0.0) { euler_flux(g, d, qL, F); return; }
    if (SR <= 0.0) { euler_flux(g, d, qR, F); return; }
    double num = pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR);
    double den = rL * (SL - uL) - rR * (SR - uR);
    double Ss = num / den;
    if (Ss >= 0.0) {
        euler_flux(g, d, qL, fL);
        double fac = rL * (SL - uL) / (SL - Ss);
        double qs[4];
        qs[0] = fac;
        qs[in] = fac * Ss;
        qs[3 - in] = fac * (qL[3 - in] / rL);
        qs[3] = fac * (qL[3] / rL + (Ss - uL) * (Ss + pL / (rL * (SL - uL))));
        for (int k = 0; k < 4; ++k) F[k] = fL[k] + SL * (qs[k] - qL[k]);
    } else {
        euler_flux(g, d, qR, fR);
        double fac = rR * (SR - uR) / (SR - Ss);
        double qs[4];
        qs[0] = fac;
        qs[in] = fac * Ss;
        qs[3 - in] = fac * (qR[3 - in] / rR);
        qs[3] = fac * (qR[3] / rR + (Ss - uR) * (Ss + pR / (rR * (SR - uR))));
        for (int k = 0; k < 4; ++k) F[k] = fR[k] + SR * (qs[k] - qR[k]);
    }
}

static double vanleer(double dm, double dp) {
    double pr = dm * dp;
    return pr > 0.0 ? 2.0 * pr / (dm + dp) : 0.0;
}

static void phys_flux(const or_sim *s, int d, const double *q, double *f) {
    if (s->c.equation == OR_EULER) euler_flux(s->c.gamma, d, q, f);
    else f[0] = s->c.adv[d] * q[0];
}

static void riemann_flux(const or_sim *s, int d, const double *qL, const double *qR, double *F) {
    if (s->c.equation == OR_EULER) or_hllc(s->c.gamma, d, qL, qR, F);
    else F[0] = s->c.adv[d] > 0.0 ? s->c.adv[d] * qL[0] : s->c.adv[d] * qR[0];
}

/* ------------------------------------------------------------------------ */
/* moving-wall boundary state (Sec. II.B, Sec. II.C.3)                      */
/* ------------------------------------------------------------------------ */
/* Exact solution of the wall Riemann problem whose ghost state has
 * u_g = u - 2(u.n)n + 2(w.n)n, rho_g = rho, p_g = p (eq. riemann_wallvel).
 * By symmetry the contact moves with the wall, u*.n = w.n; with
 * du = u.n - w.n the fluid side is a shock when du > 0 (wall advancing into
 * the fluid; closed-form root of the Rankine-Hugoniot pressure relation) and
 * a rarefaction when du < 0 (isentropic relation; vacuum when the wall
 * outruns the escape speed).  Outputs rho*, p*, u* (slip: tangential part
 * kept). */
void or_wall_state(double g, const double *q, double nx, double ny, double wx, double wy,
                   double *rs, double *ps, double *usx, double *usy) {
    double rho = q[0], u = q[1] / rho, v = q[2] / rho, p = pressure(g, q);
    double un = u * nx + v * ny, wn = wx * nx + wy * ny;
    double du = un - wn;
    double mu = (g - 1.0) / (g + 1.0);
    double pst, rst;
    if (du > 0.0) {
        double A = 2.0 / ((g + 1.0) * rho), B = mu * p;
        pst = p + du / (2.0 * A) * (du + sqrt(du * du + 4.0 * A * (p + B)));
        double pr = pst / p;
        rst = rho * (pr + mu) / (mu * pr + 1.0);
    } else {
        double c = sqrt(g * p / rho);
        double x = 1.0 + 0.5 * (g - 1.0) * du / c;
        if (x > 0.0) {
            pst = p * pow(x, 2.0 * g / (g - 1.0));
            rst = rho * pow(pst / p, 1.0 / g);
        } else {
            pst = 0.0;
            rst = 0.0;
        }
    }
    double floor_ = 1e-12 * p;
    *ps = pst > floor_ ? pst : floor_;
    *rs = rst > 1e-12 * rho ? rst : 1e-12 * rho;
    *usx = u - du * nx;
    *usy = v - du * ny;
}

/* ------------------------------------------------------------------------ */
/* simulation object                                                        */
/* ------------------------------------------------------------------------ */
or_sim *or_create(const or_config *cfg) {
    if (!cfg || cfg->nx < 4 || cfg->ny < 4) return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->c = *cfg;
    int np = cfg->npoly;
    s->pstart = (int *)malloc(sizeof(int) * (np + 1));
    s->pmoving = (int *)malloc(sizeof(int) * (np > 0 ? np : 1));
    s->pstart[0] = 0;
    for (int p = 0; p < np; ++p) { s->pstart[p + 1] = cfg->poly_start[p + 1]; s->pmoving[p] = cfg->poly_moving[p]; }
    s->nv = np > 0 ? cfg->poly_start[np] : 0;
    s->vx = (double *)malloc(sizeof(double) * (s->nv + 1));
    s->vy = (double *)malloc(sizeof(double) * (s->nv + 1));
    s->px = (double *)malloc(sizeof(double) * (s->nv + 1));
    s->py = (double *)malloc(sizeof(double) * (s->nv + 1));
    if (s->nv) { memcpy(s->vx, cfg->vx, sizeof(double) * s->nv); memcpy(s->vy, cfg->vy, sizeof(double) * s->nv); }
    s->c.poly_start = s->pstart; s->c.poly_moving = s->pmoving; s->c.vx = s->vx; s->c.vy = s->vy;
    s->dx = (cfg->x1 - cfg->x0) / (double)cfg->nx;
    s->dy = (cfg->y1 - cfg->y0) / (double)cfg->ny;
    s->nc = cfg->equation == OR_EULER ? 4 : 1;
    s->Q = (double *)malloc(sizeof(double) * s->nc * cfg->nx * cfg->ny);
    s->Qn = (double *)malloc(sizeof(double) * s->nc * cfg->nx * cfg->ny);
    for (int k = 0; k < s->nc * cfg->nx * cfg->ny; ++k) s->Q[k] = s->Qn[k] = NAN;
    {
        int nfmax = (cfg->nx + 1) * cfg->ny > cfg->nx * (cfg->ny + 1) ? (cfg->nx + 1) * cfg->ny : cfg->nx * (cfg->ny + 1);
        s->bt_last = (double *)calloc((size_t)nfmax, sizeof(double));
        s->wall_cell = (double *)calloc((size_t)6 * cfg->nx * cfg->ny, sizeof(double));
        s->last_dir = -1;
    }
    s->rmax = 0.0;
    for (int p = 0; p < np; ++p) {
        if (!s->pmoving[p]) continue;
        for (int k = s->pstart[p]; k < s->pstart[p + 1]; ++k) {
            double r = hypot(s->vx[k] - cfg->pivot[0], s->vy[k] - cfg->pivot[1]);
            s->rmax = dmax(s->rmax, r);
        }
    }
    return s;
}

void or_destroy(or_sim *s) {
    if (!s) return;
    free(s->pstart); free(s->pmoving); free(s->vx); free(s->vy); free(s->px); free(s->py);
    free(s->Q); free(s->Qn); free(s->bt_last); free(s->wall_cell); free(s);
}

int or_num_components(const or_sim *s) { return s->nc; }

/* Pose the body at (X, Y, theta) and return the full geometry arrays. */
int or_geometry(or_sim *s, double X, double Y, double theta, double *alpha, unsigned char *touched,
                double *bx, double *by) {
    pose_vertices(s, X, Y, theta, rotating(s) || theta != 0.0);
    or_geom g;
    geom_alloc(s, &g);
    compute_geometry(s, &g);
    int nx = s->c.nx, ny = s->c.ny;
    if (alpha) memcpy(alpha, g.alpha, sizeof(double) * nx * ny);
    if (touched) memcpy(touched, g.touched, (size_t)nx * ny);
    if (bx) memcpy(bx, g.bx, sizeof(double) * (nx + 1) * ny);
    if (by) memcpy(by, g.by, sizeof(double) * nx * (ny + 1));
    geom_free(&g);
    return OR_OK;
}

/* Swept aperture of the d-faces for a translation by delta from (X, Y, theta). */
int or_swept(or_sim *s, int d, double X, double Y, double theta, double delta, double *out) {
    pose_vertices(s, X, Y, theta, rotating(s) || theta != 0.0);
    compute_swept(s, d, delta, out);
    return OR_OK;
}

/* Current alpha (at the present pose: after the first sweep of a step the
 * body has turned through half of the step's rotation). */
static void current_alpha(or_sim *s, double *alpha) {
    double tp = s->t + (s->sweep_in_step == 1 ? 0.5 * s->dt_step : 0.0);
    double th = rotating(s) ? theta_at(s, tp) : 0.0;
    pose_vertices(s, s->X, s->Y, th, rotating(s));
    or_geom g;
    geom_alloc(s, &g);
    compute_geometry(s, &g);
    memcpy(alpha, g.alpha, sizeof(double) * s->c.nx * s->c.ny);
    geom_free(&g);
}

/* Write the state (SoA, nc planes of nx*ny).  Solid cells are set to NaN. */
int or_set_state(or_sim *s, const double *Q, double t, double X, double Y, long step) {
    int n = s->c.nx * s->c.ny;
    s->t = t; s->X = X; s->Y = Y; s->step = step; s->sweep_in_step = 0; s->status = OR_OK;
    double *alpha = (double *)malloc(sizeof(double) * n);
    current_alpha(s, alpha);
    for (int c = 0; c < s->nc; ++c)
        for (int k = 0; k < n; ++k) s->Q[c * n + k] = alpha[k] > 0.0 ? Q[c * n + k] : NAN;
    free(alpha);
    return OR_OK;
}

int or_get_state(or_sim *s, double *Q, double *alpha, double *tXY) {
    int n = s->c.nx * s->c.ny;
    if (Q) memcpy(Q, s->Q, sizeof(double) * s->nc * n);
    if (alpha) current_alpha(s, alpha);
    if (tXY) { tXY[0] = s->t; tXY[1] = s->X; tXY[2] = s->Y; tXY[3] = (double)s->step; }
    return s->status;
}

/* ------------------------------------------------------------------------ */
/* CFL time step (Sec. III: CFL number on regular-cell size)                */
/* ------------------------------------------------------------------------ */
/* dt = CFL * min(dx / S_x, dy / S_y), S_d = max over fluid cells of |u_d| + c
 * (|a_d| for advection), raised to the body's largest wall speed along d. */
double or_cfl_dt(const or_sim *s) {
    int n = s->c.nx * s->c.ny;
    double S[2] = {0.0, 0.0};
    for (int k = 0; k < n; ++k) {
        if (s->Q[k] != s->Q[k]) continue; /* solid */
        if (s->c.equation == OR_EULER) {
            double q[4] = {s->Q[k], s->Q[n + k], s->Q[2 * n + k], s->Q[3 * n + k]};
            double rho = q[0], u = q[1] / rho, v = q[2] / rho, p = pressure(s->c.gamma, q);
            double c = sqrt(s->c.gamma * p / rho);
            S[0] = dmax(S[0], fabs(u) + c);
            S[1] = dmax(S[1], fabs(v) + c);
        } else {
            S[0] = dmax(S[0], fabs(s->c.adv[0]));
            S[1] = dmax(S[1], fabs(s->c.adv[1]));
        }
    }
    double wr = fabs(s->c.a1 * s->c.omega) * s->rmax;
    S[0] = dmax(S[0], fabs(s->c.U[0]) + wr);
    S[1] = dmax(S[1], fabs(s->c.U[1]) + wr);
    if (S[0] <= 0.0) S[0] = 1e-300;
    if (S[1] <= 0.0) S[1] = 1e-300;
    return s->c.cfl * dmin(s->dx / S[0], s->dy / S[1]);
}

/* ------------------------------------------------------------------------ */
/* one directional sweep                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int has;             /* wall data computed */
    double d;            /* average shielded distance (mid pose) */
    double FB[4];        /* boundary flux along the sweep direction */
    double QB[4];        /* boundary state */
    double wd;           /* wall velocity component along the sweep */
} wall_t;

static int wrapi(int k, int n) { k %= n; return k < 0 ? k + n : k; }

/* Stabilised flux of one face (eqs. Klein2DtotalfluxaMethod2,
 * Klein2shieldedFluxMethod2), times its time-averaged aperture bf:
 *   bf F2D = (bf - sL - sR) F + sR [FB_R + d_R (F - FB_R)] + sL [FB_L + d_L (F - FB_L)],
 * where the shielded part attached to the face by a neighbour with wall data
 * is s = max(0, bf - bfar), bfar the aperture of that neighbour's far face.
 * When both neighbours shield the face and sL + sR > bf, both parts are
 * scaled by bf / (sL + sR) (a reading: the paper treats one side only).
 * wL / wR are NULL when that neighbour has no wall data. */
static void stab_face(int nc, double bf, const double *F, const wall_t *wL, double bfarL, const wall_t *wR,
                      double bfarR, double *out) {
    double sR = 0.0, sLv = 0.0;
    if (wR) sR = dmax(0.0, bf - bfarR);
    if (wL) sLv = dmax(0.0, bf - bfarL);
    if (sR + sLv > bf) { double sc = bf / (sR + sLv); sR *= sc; sLv *= sc; }
    for (int q = 0; q < nc; ++q) {
        double v = (bf - sLv - sR) * F[q];
        if (sR > 0.0) v += sR * (wR->FB[q] + wR->d * (F[q] - wR->FB[q]));
        if (sLv > 0.0) v += sLv * (wL->FB[q] + wL->d * (F[q] - wL->FB[q]));
        out[q] = v;
    }
}

/* stab_face with plain arguments (has* = 0: that neighbour has no wall data) */
void or_stab_face(int nc, double bf, const double *F, int hasL, double bfarL, double dL, const double *FBL,
                  int hasR, double bfarR, double dR, const double *FBR, double *out) {
    wall_t wl, wr;
    memset(&wl, 0, sizeof(wl));
    memset(&wr, 0, sizeof(wr));
    wl.d = dL; wr.d = dR;
    for (int q = 0; q < nc; ++q) { wl.FB[q] = hasL ? FBL[q] : 0.0; wr.FB[q] = hasR ? FBR[q] : 0.0; }
    stab_face(nc, bf, F, hasL ? &wl : NULL, bfarL, hasR ? &wr : NULL, bfarR, out);
}

/* Covering / uncovering (Sec. II.C.5), applied simultaneously to all cells
 * (Jacobi: every event reads the contents C from before any event, a
 * reading; the paper is silent on simultaneous events).  C holds the new
 * contents alpha^B Q' of the update; Cn receives the contents after the
 * events.  A cell is covered when alphaA > 0 and alphaB = 0: its residual
 * content (eq. massDeficitEquation: what the update left in it) goes to the
 * fluid face neighbours at B in proportion to their volume fractions (eq.
 * cutCellCoverDonation).  A cell is uncovered when alphaA = 0 and
 * alphaB > 0; in donor mode it takes sigma * (sum of the donors' contents),
 * sigma = alphaB / (alphaB + sum of the donors' alphaB) (eqs.
 * volumeWeighting, cutCellInitialisation), and each donor loses sigma times
 * its own content (eq. cutCellInitialisationDonorCellUpdate); donors are the
 * fluid face neighbours at B that are not themselves uncovered.  With no
 * such face neighbour the 8-neighbourhood is used (a reading).  A covered
 * cell on a transmissive side of the domain (open_sides: bit 0 x-low, 1
 * x-high, 2 y-low, 3 y-high) with no fluid neighbour at all passes its
 * residual out of the domain (a reading: a body leaving the domain).
 * updated[c] is set for donor-initialised cells.  Returns OR_E_UNSTABLE when
 * any other cell has no neighbour to exchange with. */
static int cover_uncover(int nx, int ny, int perx, int pery, int open_sides, int nc, int mode, const double *alphaA,
                         const double *alphaB, const double *C, double *Cn, unsigned char *updated) {
    const int n = nx * ny;
    int err = OR_OK;
    memcpy(Cn, C, sizeof(double) * nc * n);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            int covered = alphaA[c] > 0.0 && alphaB[c] == 0.0;
            int donor_unc = mode == OR_UNCOVER_DONOR && alphaA[c] == 0.0 && alphaB[c] > 0.0;
            if (!covered && !donor_unc) continue;
            /* neighbour sets: face neighbours first, then the 8-neighbourhood */
            int nb[8], nnb = 0;
            double asum = 0.0;
            for (int pass = 0; pass < 2 && nnb == 0; ++pass) {
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        if (di == 0 && dj == 0) continue;
                        if (pass == 0 && di != 0 && dj != 0) continue;
                        int ii = i + di, jj = j + dj;
                        if (perx) ii = wrapi(ii, nx);
                        if (pery) jj = wrapi(jj, ny);
                        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
                        int cc = jj * nx + ii;
                        if (!(alphaB[cc] > 0.0)) continue;
                        if (mode == OR_UNCOVER_DONOR && alphaA[cc] == 0.0) continue; /* no content yet */
                        nb[nnb++] = cc;
                        asum += alphaB[cc];
                    }
            }
            if (nnb == 0) {
                const int open = ((open_sides & 1) && i == 0) || ((open_sides & 2) && i == nx - 1) ||
                                 ((open_sides & 4) && j == 0) || ((open_sides & 8) && j == ny - 1);
                if (covered && open) {
                    for (int q = 0; q < nc; ++q) Cn[q * n + c] = 0.0;   /* leaves the domain */
                } else {
                    err = OR_E_UNSTABLE;
                }
                continue;
            }
            if (covered) {
                for (int m = 0; m < nnb; ++m)
                    for (int q = 0; q < nc; ++q) Cn[q * n + nb[m]] += alphaB[nb[m]] / asum * C[q * n + c];
                for (int q = 0; q < nc; ++q) Cn[q * n + c] = 0.0;
            } else {
                double sigma = alphaB[c] / (alphaB[c] + asum);
                for (int q = 0; q < nc; ++q) {
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

/* cover_uncover on caller arrays (updated may be NULL) */
int or_cover_uncover(int nx, int ny, int perx, int pery, int open_sides, int nc, int mode, const double *alphaA,
                     const double *alphaB, const double *C, double *Cn, unsigned char *updated) {
    unsigned char *u = updated ? updated : (unsigned char *)calloc((size_t)nx * ny, 1);
    int r = cover_uncover(nx, ny, perx, pery, open_sides, nc, mode, alphaA, alphaB, C, Cn, u);
    if (!updated) free(u);
    return r;
}

/* Positivity safeguard (a reading; the paper gives none): a cell whose
 * content is non-physical (rho <= 0, p <= 0 or non-finite, Euler only) is
 * merged with its fluid, updated face neighbours; every connected cluster of
 * such cells and their neighbours shares its total content in proportion to
 * the volume fractions alphaB.  Cells still non-physical after a merge seed
 * the next one, which reaches one layer of neighbours further, up to
 * OR_MIX_LAYERS merges.  The first merge is also seeded by every cell that
 * kept less than OR_COLLAPSE of its volume over the sweep (0 < alphaB <
 * OR_COLLAPSE alphaA; alphaA may be NULL): the stabilised update leaves such
 * a cell a content of the order of its shielded volume at the mid pose
 * (Sec. II.C.4), so its state, content / alphaB, is amplified by up to
 * alphaA / alphaB -- the growth of the state as the volume fraction
 * vanishes that Sec. II.C.1 describes -- and can be physical but far out
 * of range.  Exactly conservative.  Cn is updated in place; returns the
 * number of cells merged (summed over the merges). */
static int safeguard(int nx, int ny, int perx, int pery, double g, const double *alphaA, const double *alphaB,
                     const unsigned char *updated, double *Cn) {
    const int n = nx * ny;
    int mixed = 0;
    for (int layer = 0; layer < OR_MIX_LAYERS; ++layer) {
        int *lab = (int *)malloc(sizeof(int) * n);
        unsigned char *bad = (unsigned char *)calloc((size_t)n, 1);
        int nbad = 0;
        for (int c = 0; c < n; ++c) {
            lab[c] = -1;
            double aB = alphaB[c];
            if (!(aB > 0.0) || !updated[c]) continue;
            double q[4] = {Cn[c] / aB, Cn[n + c] / aB, Cn[2 * n + c] / aB, Cn[3 * n + c] / aB};
            int b = !(q[0] > 0.0) || !(pressure(g, q) > 0.0);
            for (int k = 0; k < 4; ++k) if (!isfinite(q[k])) b = 1;
            if (layer == 0 && alphaA && aB < OR_COLLAPSE * alphaA[c]) b = 1;
            if (b) { bad[c] = 1; nbad++; }
        }
        if (nbad) {
            /* union-find over bad cells and their fluid face neighbours */
            int *par = (int *)malloc(sizeof(int) * n);
            for (int c = 0; c < n; ++c) par[c] = c;
            for (int c = 0; c < n; ++c) {
                if (!bad[c]) continue;
                int i = c % nx, j = c / nx;
                lab[c] = c;
                int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
                for (int m = 0; m < 4; ++m) {
                    int ii = i + dd[m][0], jj = j + dd[m][1];
                    if (perx) ii = wrapi(ii, nx);
                    if (pery) jj = wrapi(jj, ny);
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
                    int cc = jj * nx + ii;
                    if (!(alphaB[cc] > 0.0) || !updated[cc]) continue;
                    lab[cc] = cc;
                    int ra = c, rb = cc;
                    while (par[ra] != ra) ra = par[ra];
                    while (par[rb] != rb) rb = par[rb];
                    if (ra != rb) { if (ra < rb) par[rb] = ra; else par[ra] = rb; }
                }
            }
            double *tot = (double *)calloc((size_t)n * 5, sizeof(double));
            for (int c = 0; c < n; ++c) {
                if (lab[c] < 0) continue;
                int r = c; while (par[r] != r) r = par[r];
                lab[c] = r;
                tot[5 * r + 4] += alphaB[c];
                for (int q = 0; q < 4; ++q) tot[5 * r + q] += Cn[q * n + c];
            }
            for (int c = 0; c < n; ++c) {
                if (lab[c] < 0) continue;
                mixed++;
                int r = lab[c];
                for (int q = 0; q < 4; ++q) Cn[q * n + c] = alphaB[c] * (tot[5 * r + q] / tot[5 * r + 4]);
            }
            free(tot); free(par);
        }
        free(lab); free(bad);
        if (!nbad) break;
    }
    return mixed;
}

/* safeguard on caller arrays (Euler contents, 4 planes of nx*ny) */
int or_safeguard(int nx, int ny, int perx, int pery, double g, const double *alphaA, const double *alphaB,
                 const unsigned char *updated, double *Cn) {
    return safeguard(nx, ny, perx, pery, g, alphaA, alphaB, updated, Cn);
}

/* Geometric source of the axisymmetric Euler equations (a reading: the
 * paper models its open-ended tube, Sec. III.E, in axisymmetric form without
 * stating how the source is integrated).  With x axial and y the radius r
 * measured from the axis y = y0, the planar fluxes of the sweeps miss the
 * term -(1/r) [rho v, rho u v, rho v^2, v (E + p)].  It is applied as a step
 * of its own after every radial (y) sweep, explicitly over the sweep's dt,
 * to the state of every fluid cell, r taken at the cell centre
 * (j + 1/2) dy.  Returns OR_E_UNSTABLE when a state turns non-physical. */
static int axisym_source(or_sim *s, double dt) {
    const int nx = s->c.nx, ny = s->c.ny, n = nx * ny;
    const double g = s->c.gamma;
    int err = OR_OK;
    for (int j = 0; j < ny; ++j) {
        const double r = ((double)j + 0.5) * s->dy;
        for (int i = 0; i < nx; ++i) {
            const int c = j * nx + i;
            if (s->Q[c] != s->Q[c]) continue;   /* solid */
            double q[4] = {s->Q[c], s->Q[n + c], s->Q[2 * n + c], s->Q[3 * n + c]};
            const double v = q[2] / q[0], p = pressure(g, q);
            const double f = dt * v / r;
            s->Q[c] = q[0] - f * q[0];
            s->Q[n + c] = q[1] - f * q[1];
            s->Q[2 * n + c] = q[2] - f * q[2];
            s->Q[3 * n + c] = q[3] - f * (q[3] + p);
            double qn[4] = {s->Q[c], s->Q[n + c], s->Q[2 * n + c], s->Q[3 * n + c]};
            if (!(qn[0] > 0.0) || !(pressure(g, qn) > 0.0)) err = OR_E_UNSTABLE;
        }
    }
    return err;
}

/* Sweep `d` with time step dt.  The body moves by U_d*dt along d (and by half
 * of the step's rotation) between the start pose A and the end pose B. */
int or_sweep(or_sim *s, int d, double dt) {
    if (d != 0 && d != 1) return OR_E_INVAL;
    const int nx = s->c.nx, ny = s->c.ny, n = nx * ny, nc = s->nc;
    const double g = s->c.gamma;
    const int rot = rotating(s);
    const int sidx = s->sweep_in_step;
    if (sidx == 1 && dt != s->dt_step) return OR_E_STATE;
    if (sidx == 0) {
        s->dt_step = dt;
        memcpy(s->Qn, s->Q, sizeof(double) * nc * n); /* step-start state, NaN in solids */
    }
    /* poses */
    double tA = s->t + (sidx == 0 ? 0.0 : 0.5 * dt);
    double tB = s->t + (sidx == 0 ? 0.5 * dt : dt);
    double tM = s->t + (sidx == 0 ? 0.25 * dt : 0.75 * dt);
    double thA = rot ? theta_at(s, tA) : 0.0, thB = rot ? theta_at(s, tB) : 0.0, thM = rot ? theta_at(s, tM) : 0.0;
    double delta = s->c.U[d] * dt;
    double XA = s->X, YA = s->Y;
    double XB = d == 0 ? XA + delta : XA, YB = d == 1 ? YA + delta : YA;
    double XM = d == 0 ? XA + 0.5 * delta : XA, YM = d == 1 ? YA + 0.5 * delta : YA;

    or_geom gA, gB, gM;
    geom_alloc(s, &gA); geom_alloc(s, &gB); geom_alloc(s, &gM);
    pose_vertices(s, XA, YA, thA, rot); compute_geometry(s, &gA);
    int nf = d == 0 ? (nx + 1) * ny : nx * (ny + 1);
    double *bt = (double *)malloc(sizeof(double) * nf);
    /* time-averaged apertures of the d-faces (eq. timeAveragedBeta) */
    if (!rot && delta != 0.0) {
        compute_swept(s, d, delta, bt);                /* exact swept strip at pose A */
    }
    pose_vertices(s, XB, YB, thB, rot); compute_geometry(s, &gB);
    pose_vertices(s, XM, YM, thM, rot); compute_geometry(s, &gM);
    const double *bA = d == 0 ? gA.bx : gA.by, *bB = d == 0 ? gB.bx : gB.by, *bM = d == 0 ? gM.bx : gM.by;
    if (rot) {
        for (int k = 0; k < nf; ++k) bt[k] = (bA[k] + 4.0 * bM[k] + bB[k]) / 6.0; /* Simpson */
    } else if (delta == 0.0) {
        memcpy(bt, bA, sizeof(double) * nf);
    }

    const int nal = d == 0 ? nx : ny;     /* cells along the sweep */
    const int nln = d == 0 ? ny : nx;     /* lines */
    const double h = d == 0 ? s->dx : s->dy;
    const double lam = dt / h;
    const int periodic = s->c.bc[2 * d] == OR_BC_PERIODIC;
    const int ucov = s->c.uncover_mode;
#define CELL(l, k) ((d) == 0 ? (l) * nx + (k) : (k) * nx + (l))
#define FACE(l, k) ((d) == 0 ? (l) * (nx + 1) + (k) : (k) * nx + (l))

    /* classes */
    unsigned char *fluidA = (unsigned char *)malloc((size_t)n), *uncov = (unsigned char *)malloc((size_t)n);
    unsigned char *band = (unsigned char *)malloc((size_t)n);
    for (int k = 0; k < n; ++k) {
        uncov[k] = gA.alpha[k] == 0.0 && gB.alpha[k] > 0.0;
        fluidA[k] = gA.alpha[k] > 0.0 || (ucov == OR_UNCOVER_FLUX_GCL && uncov[k]);
        band[k] = gA.touched[k] || gB.touched[k] || (rot && gM.touched[k]);
    }
    /* sweep-start state with provisional states for flux-GCL uncovered cells */
    double *Qs = (double *)malloc(sizeof(double) * nc * n);
    memcpy(Qs, s->Q, sizeof(double) * nc * n);
    int err = OR_OK;
    if (ucov == OR_UNCOVER_FLUX_GCL) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c = j * nx + i;
                if (!uncov[c]) continue;
                double acc[4] = {0, 0, 0, 0}, wsum = 0.0;
                for (int pass = 0; pass < 2 && wsum == 0.0; ++pass) {
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            if (di == 0 && dj == 0) continue;
                            if (pass == 0 && di != 0 && dj != 0) continue;
                            int ii = i + di, jj = j + dj;
                            if (s->c.bc[0] == OR_BC_PERIODIC) ii = wrapi(ii, nx);
                            if (s->c.bc[2] == OR_BC_PERIODIC) jj = wrapi(jj, ny);
                            if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
                            int cc = jj * nx + ii;
                            if (!(gA.alpha[cc] > 0.0)) continue;
                            wsum += gA.alpha[cc];
                            for (int q = 0; q < nc; ++q) acc[q] += gA.alpha[cc] * s->Q[q * n + cc];
                        }
                }
                if (wsum == 0.0) { err = OR_E_UNSTABLE; continue; }
                for (int q = 0; q < nc; ++q) Qs[q * n + c] = acc[q] / wsum;
            }
    }

    /* kept for diagnostics */
    s->last_dir = d;
    memcpy(s->bt_last, bt, sizeof(double) * nf);
    memset(s->wall_cell, 0, sizeof(double) * 6 * n);

    /* wall data per band cell (Sec. II.B, II.C.3, II.C.4) */
    wall_t *W = (wall_t *)calloc((size_t)n, sizeof(wall_t));
    double Om = rot ? thetadot_at(s, tM) : 0.0;
    double pcx = s->c.pivot[0] + XM, pcy = s->c.pivot[1] + YM;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = j * nx + i;
            if (!band[c] || !fluidA[c]) continue;
            wall_t *w = &W[c];
            w->has = 1;
            /* shielded distance at the mid pose: alpha_hat = alpha - min(beta),
             * d = alpha_hat / |delta beta| (eqs. Klein2DalphaHat, timeAveragedAlpha);
             * d = 1 when the two apertures differ by 1e-12 or less, where
             * both alpha_hat and |delta beta| are round-off and their ratio
             * means nothing (the limit of equally open faces) */
            double blo = d == 0 ? gM.bx[j * (nx + 1) + i] : gM.by[j * nx + i];
            double bhi = d == 0 ? gM.bx[j * (nx + 1) + i + 1] : gM.by[(j + 1) * nx + i];
            double db = fabs(blo - bhi);
            double ahat = gM.alpha[c] - dmin(blo, bhi);
            w->d = db > 1e-12 ? clamp01(ahat / db) : 1.0;
            /* wall normal from aperture closure at the mid pose, pointing into the body */
            double bW = gM.bx[j * (nx + 1) + i], bE = gM.bx[j * (nx + 1) + i + 1];
            double bS = gM.by[j * nx + i], bN = gM.by[(j + 1) * nx + i];
            double nLx = (bW - bE) * s->dy, nLy = (bS - bN) * s->dx;
            double L = sqrt(nLx * nLx + nLy * nLy);
            double nxv = L > 0.0 ? nLx / L : 0.0, nyv = L > 0.0 ? nLy / L : 0.0;
            /* wall velocity at the cell centre */
            double wx = 0.0, wy = 0.0;
            if (gA.moving[c] || gB.moving[c] || gM.moving[c]) {
                double xc = s->c.x0 + ((double)i + 0.5) * s->dx, yc = s->c.y0 + ((double)j + 0.5) * s->dy;
                wx = s->c.U[0] - Om * (yc - pcy);
                wy = s->c.U[1] + Om * (xc - pcx);
            }
            w->wd = d == 0 ? wx : wy;
            {
                double *wc = &s->wall_cell[6 * c];
                wc[0] = 1.0; wc[1] = w->d; wc[2] = nxv; wc[3] = nyv; wc[4] = wx; wc[5] = wy;
            }
            /* advective state from the step-start state (common to both sweeps),
             * pressure per sweep (eq. KleinAdvectivePressureSplitA and text after it) */
            double qn[4], qc[4];
            int fresh = s->Qn[c] != s->Qn[c];
            for (int q = 0; q < nc; ++q) { qc[q] = Qs[q * n + c]; qn[q] = fresh ? qc[q] : s->Qn[q * n + c]; }
            if (s->c.equation == OR_EULER) {
                double rs, ps_step, usx, usy, rs2, ps_sw, u2x, u2y;
                or_wall_state(g, qn, nxv, nyv, wx, wy, &rs, &ps_step, &usx, &usy);
                or_wall_state(g, qc, nxv, nyv, wx, wy, &rs2, &ps_sw, &u2x, &u2y);
                double Eadv = ps_step / (g - 1.0) + 0.5 * rs * (usx * usx + usy * usy);
                double ud = d == 0 ? usx : usy;
                w->QB[0] = rs; w->QB[1] = rs * usx; w->QB[2] = rs * usy; w->QB[3] = Eadv;
                w->FB[0] = rs * ud;
                w->FB[1] = rs * ud * usx + (d == 0 ? ps_sw : 0.0);
                w->FB[2] = rs * ud * usy + (d == 1 ? ps_sw : 0.0);
                w->FB[3] = ud * (Eadv + ps_step);
            } else {
                w->QB[0] = qn[0];
                w->FB[0] = s->c.adv[d] * qn[0];
            }
        }

    /* new contents alpha^B Q' (before cover/uncover redistribution) */
    double *C = (double *)malloc(sizeof(double) * nc * n);
    for (int k = 0; k < nc * n; ++k) C[k] = 0.0;
    unsigned char *updated = (unsigned char *)calloc((size_t)n, 1);

    for (int q = 0; q < 4; ++q) s->wall_last[q] = 0.0;
    s->mixed_last = 0;
    /* per-line work arrays, ghost cells -2..nal+1 */
    int len = nal + 4;
    double *Ql = (double *)malloc(sizeof(double) * 4 * len);
    double *QLb = (double *)malloc(sizeof(double) * 4 * len), *QRb = (double *)malloc(sizeof(double) * 4 * len);
    unsigned char *fl = (unsigned char *)malloc((size_t)len);
    double *Fst = (double *)malloc(sizeof(double) * 4 * (nal + 1));
    unsigned char *hasF = (unsigned char *)malloc((size_t)(nal + 1));
    double *F2 = (double *)malloc(sizeof(double) * 4 * (nal + 1));
    int in = d == 0 ? 1 : 2;

    for (int l = 0; l < nln; ++l) {
        /* gather line with ghosts */
        for (int kk = -2; kk < nal + 2; ++kk) {
            int k = kk, flip = 0;
            if (kk < 0 || kk >= nal) {
                int side = kk < 0 ? 2 * d : 2 * d + 1;
                int bc = s->c.bc[side];
                if (bc == OR_BC_PERIODIC) k = wrapi(kk, nal);
                else { k = kk < 0 ? -1 - kk : 2 * nal - 1 - kk; flip = bc == OR_BC_REFLECTIVE; }
            }
            int c = CELL(l, k);
            fl[kk + 2] = fluidA[c];
            for (int q = 0; q < nc; ++q) Ql[q * len + kk + 2] = Qs[q * n + c];
            if (flip && nc == 4) Ql[in * len + kk + 2] = -Ql[in * len + kk + 2];
        }
        /* MUSCL-Hancock: limited slopes, boundary extrapolation, half-step evolution */
        for (int kk = -1; kk <= nal; ++kk) {
            int a = kk + 2;
            if (!fl[a]) continue;
            int lim = fl[a - 1] && fl[a + 1];
            double qL[4], qR[4], fLv[4], fRv[4];
            for (int q = 0; q < nc; ++q) {
                double sl = lim ? vanleer(Ql[q * len + a] - Ql[q * len + a - 1], Ql[q * len + a + 1] - Ql[q * len + a]) : 0.0;
                qL[q] = Ql[q * len + a] - 0.5 * sl;
                qR[q] = Ql[q * len + a] + 0.5 * sl;
            }
            phys_flux(s, d, qL, fLv);
            phys_flux(s, d, qR, fRv);
            for (int q = 0; q < nc; ++q) {
                double dfl = 0.5 * lam * (fLv[q] - fRv[q]);
                QLb[q * len + a] = qL[q] + dfl;
                QRb[q * len + a] = qR[q] + dfl;
            }
            /* first-order fallback when an evolved boundary state is not
             * physical (a reading: rho > 0 and p > 0 are required by HLLC) */
            if (nc == 4) {
                double eL[4], eR[4];
                for (int q = 0; q < 4; ++q) { eL[q] = QLb[q * len + a]; eR[q] = QRb[q * len + a]; }
                if (!(eL[0] > 0.0) || !(eR[0] > 0.0) || !(pressure(g, eL) > 0.0) || !(pressure(g, eR) > 0.0))
                    for (int q = 0; q < 4; ++q) { QLb[q * len + a] = Ql[q * len + a]; QRb[q * len + a] = Ql[q * len + a]; }
            }
        }
        /* faces k = 0..nal: face k lies between cells k-1 and k */
        int nfl = periodic ? nal : nal + 1;
        for (int k = 0; k < nfl; ++k) {
            int a = k + 2;
            double bf = bt[FACE(l, k)];
            hasF[k] = fl[a - 1] && fl[a] && bf > 0.0;
            for (int q = 0; q < 4; ++q) { Fst[4 * k + q] = 0.0; F2[4 * k + q] = 0.0; }
            if (!hasF[k]) continue;
            double qL[4], qR[4];
            for (int q = 0; q < nc; ++q) { qL[q] = QRb[q * len + a - 1]; qR[q] = QLb[q * len + a]; }
            riemann_flux(s, d, qL, qR, &Fst[4 * k]);
            /* stabilised face flux (eqs. Klein2DtotalfluxaMethod2, Klein2shieldedFluxMethod2) */
            int kR = k < nal ? k : (periodic ? 0 : -1);
            int kL = k - 1 >= 0 ? k - 1 : (periodic ? nal - 1 : -1);
            const wall_t *wR = NULL, *wL = NULL;
            double bfarR = 0.0, bfarL = 0.0;
            if (kR >= 0) {
                int cR = CELL(l, kR);
                bfarR = bt[FACE(l, kR + 1 < nal || !periodic ? kR + 1 : 0)];
                if (W[cR].has) wR = &W[cR];
            }
            if (kL >= 0) {
                int cL = CELL(l, kL);
                bfarL = bt[FACE(l, kL)];
                if (W[cL].has) wL = &W[cL];
            }
            stab_face(nc, bf, &Fst[4 * k], wL, bfarL, wR, bfarR, &F2[4 * k]);
        }
        /* conservative update in alpha Q form (eqs. Klein2DcompleteMovingMethod2a-b) */
        for (int k = 0; k < nal; ++k) {
            int c = CELL(l, k);
            if (!fluidA[c]) continue;
            int klo = k, khi = (k + 1 < nal || !periodic) ? k + 1 : 0;
            double blo = bt[FACE(l, k)], bhi = bt[FACE(l, k + 1 < nal || !periodic ? k + 1 : 0)];
            double aA = gA.alpha[c];
            for (int q = 0; q < nc; ++q) {
                double v = aA * Qs[q * n + c] + lam * (F2[4 * klo + q] - F2[4 * khi + q]);
                if (blo != bhi && W[c].has) {
                    double wt = lam * (bhi - blo) * (W[c].FB[q] - W[c].wd * W[c].QB[q]);
                    v += wt;
                    s->wall_last[q] += wt;
                }
                C[q * n + c] = v;
            }
            updated[c] = 1;
        }
    }

    /* covering / uncovering (Sec. II.C.5), applied simultaneously */
    double *Cn = (double *)malloc(sizeof(double) * nc * n);
    const int perx = s->c.bc[0] == OR_BC_PERIODIC, pery = s->c.bc[2] == OR_BC_PERIODIC;
    int open_sides = 0;
    for (int side = 0; side < 4; ++side)
        if (s->c.bc[side] == OR_BC_TRANSMISSIVE) open_sides |= 1 << side;
    if (cover_uncover(nx, ny, perx, pery, open_sides, nc, ucov, gA.alpha, gB.alpha, C, Cn, updated) != OR_OK)
        err = OR_E_UNSTABLE;

    /* positivity safeguard */
    if (s->c.equation == OR_EULER) s->mixed_last = safeguard(nx, ny, perx, pery, g, gA.alpha, gB.alpha, updated, Cn);

    /* new state Q' = content / alpha^B */
    for (int c = 0; c < n; ++c) {
        double aB = gB.alpha[c];
        for (int q = 0; q < nc; ++q) s->Q[q * n + c] = (aB > 0.0 && updated[c]) ? Cn[q * n + c] / aB : NAN;
        if (aB > 0.0 && !updated[c]) err = OR_E_UNSTABLE;
        if (aB > 0.0 && updated[c]) {
            if (nc == 4) {
                double q[4] = {s->Q[c], s->Q[n + c], s->Q[2 * n + c], s->Q[3 * n + c]};
                int bad = !(q[0] > 0.0) || !(pressure(g, q) > 0.0);
                for (int k = 0; k < 4; ++k) if (!isfinite(q[k])) bad = 1;
                if (bad) err = OR_E_UNSTABLE;
            } else if (!isfinite(s->Q[c])) err = OR_E_UNSTABLE;
        }
    }

    /* geometric source of the axisymmetric form after the radial sweep */
    if (s->c.axisym && d == 1 && s->c.equation == OR_EULER && axisym_source(s, dt) != OR_OK) err = OR_E_UNSTABLE;

    /* advance pose / time */
    s->X = XB; s->Y = YB;
    if (sidx == 1) { s->t += dt; s->step += 1; s->sweep_in_step = 0; }
    else s->sweep_in_step = 1;
    if (err != OR_OK) s->status = err;

    free(Ql); free(QLb); free(QRb); free(fl); free(Fst); free(hasF); free(F2);
    free(C); free(Cn); free(updated); free(W); free(Qs); free(fluidA); free(uncov); free(band); free(bt);
    geom_free(&gA); geom_free(&gB); geom_free(&gM);
#undef CELL
#undef FACE
    return err;
}

/* One time step: two sweeps, x then y on even steps and y then x on odd
 * steps (Sec. II.A, Strang-type alternation).  dt <= 0 selects the CFL step. */
int or_step(or_sim *s, double dt, double *dt_used) {
    if (s->sweep_in_step != 0) return OR_E_STATE;
    if (dt <= 0.0) dt = or_cfl_dt(s);
    if (dt_used) *dt_used = dt;
    int d1 = (s->step % 2 == 0) ? 0 : 1;
    int r1 = or_sweep(s, d1, dt);
    int r2 = or_sweep(s, 1 - d1, dt);
    return r1 != OR_OK ? r1 : r2;
}

int or_status(const or_sim *s) { return s->status; }

/* Diagnostics of the last sweep: sum of wall terms (per unit cell area, one
 * entry per component) and the number of cells the safeguard merged. */
int or_last_sweep(const or_sim *s, double *wall) {
    if (wall) for (int q = 0; q < 4; ++q) wall[q] = s->wall_last[q];
    return s->mixed_last;
}

/* Time-averaged apertures of the last sweep's faces (the layout of or_swept
 * for its direction); returns that direction (-1 before the first sweep). */
int or_last_faces(const or_sim *s, double *bt) {
    if (s->last_dir < 0) return -1;
    int nx = s->c.nx, ny = s->c.ny;
    int nf = s->last_dir == 0 ? (nx + 1) * ny : nx * (ny + 1);
    if (bt) memcpy(bt, s->bt_last, sizeof(double) * nf);
    return s->last_dir;
}

/* Wall data of the last sweep per cell, 6 doubles each: 1 if the cell had
 * wall data, the shielded distance d, the wall normal (n_x, n_y) and the
 * wall velocity (w_x, w_y) at the mid pose; zeros elsewhere. */
void or_last_wall(const or_sim *s, double *out) {
    memcpy(out, s->wall_cell, sizeof(double) * 6 * s->c.nx * s->c.ny);
}
