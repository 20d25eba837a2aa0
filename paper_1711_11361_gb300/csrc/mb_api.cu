// mb_api.cu -- host runtime behind the C ABI in include/mb.h.
//
// A sim is a batch of instances laid out as independent grids in device
// memory.  Every sweep is one fixed sequence of kernel launches over the
// whole batch (pose -> geometry -> band prep -> band faces -> bulk -> events
// -> safeguard -> finalize); mb_run captures a step (two sweeps) as a CUDA
// graph and replays it.  Three state buffers rotate so that the step-start
// state stays readable during the second sweep (the common advective wall
// state of Sec. II.B is taken from it).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mb.h"
#include "mb_internal.cuh"

namespace mb {
void geom_init();
void launch_nodes(const InstDesc *, int, cudaStream_t);
void launch_pose(const InstDesc *, InstDyn *, const double *, const double *, const unsigned char *, const int *,
                 double *, double *, float *, int, int, int, int, double, int *, cudaStream_t);
void launch_geom(const InstDesc *, InstDyn *, const int *, const double *, const double *, const float *, const int *,
                 const unsigned char *, int, int, int, int, BandRec *, double *, cudaStream_t);
void launch_classify(const InstDesc *, InstDyn *, const double *, const double *, const unsigned char *, double *,
                     double *, float *, const int *, int, int, int, int, double *, cudaStream_t);
template <class T>
void launch_band_stage(int, const InstDesc *, InstDyn *, BandRec *, const double *, int *, int, int, int, int,
                       int, int, int, int, cudaStream_t);
template <class T>
void launch_bulk(int, int, const InstDesc *, InstDyn *, const BandRec *, int, int, int, int, int, int, int, DeferList,
                 int, cudaStream_t);
template <class T>
int bulk_blocks_per_sm(int);
double fp64_probe_rate(cudaStream_t st);
template <class T>
void launch_axisym_source(const InstDesc *, InstDyn *, int, int, int, cudaStream_t);
template <class T, class H>
void launch_write_state(const InstDesc *, InstDyn *, const H *const *, const H *, int, int, int, int, cudaStream_t);
template <class T, class H>
void launch_read_state(const InstDesc *, H *const *, H *, int, int, int, int, cudaStream_t);
}  // namespace mb

using namespace mb;

static std::string g_create_error;

// host copy of an instance's body and the device buffers it owns
struct InstHost {
    std::vector<double> vx, vy;
    std::vector<unsigned char> mov;
    std::vector<int> next;        // next vertex of each edge, instance-local
    std::vector<void *> allocs;   // state buffers, classes, record index, alpha, grid lines
};

struct mb_sim {
    int n = 0;
    int prec = MB_FP64;
    int eq = MB_EULER;
    int nsm = 0;
    std::vector<InstDesc> hd;
    std::vector<InstHost> ih;
    // capacities (elements) of the shared arrays below
    size_t cap_vx = 0, cap_vy = 0, cap_mov = 0, cap_next = 0, cap_px = 0, cap_py = 0, cap_ebox = 0;
    size_t cap_rec = 0, cap_bnd = 0, cap_dd = 0, cap_dy = 0, cap_ginst = 0;
    InstDesc *dd = nullptr;
    InstDyn *dy = nullptr;
    double *vx = nullptr, *vy = nullptr, *px = nullptr, *py = nullptr;
    float *ebox = nullptr;        // FP32 x-bounds of every edge at the three poses
    unsigned char *vmov = nullptr;
    int *vnext = nullptr;
    int total_v = 0;
    BandRec *rec = nullptr;
    double *bnd = nullptr;
    int total_rec = 0;
    int *boff = nullptr;          // used band records before each instance (n + 1), per sweep
    size_t cap_boff = 0;
    double *stage = nullptr;      // staging for state I/O (nc * max cells doubles)
    size_t stage_len = 0;
    double *bstage = nullptr;     // batched state I/O: every instance's FP64 state
    size_t cap_bstage = 0;
    const double **iop = nullptr; // batched state I/O: per-instance pointers into bstage
    size_t cap_iop = 0;
    int total_cols = 0;           // geometry groups
    int *ginst = nullptr;         // instance of each geometry group
    int total_tiles[2] = {0, 0};
    int bulk_grid[2] = {0, 0};
    // cell pairs whose bulk update waits for the band fluxes (FP32 Euler)
    int2 *ditem = nullptr;
    int *dcount = nullptr;
    size_t cap_ditem = 0, cap_dcount = 0;
    // the geometry and band-flux kernels of a sweep run on this stream,
    // concurrently with the bulk pass on the sim's stream (FP32 Euler)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_mid = nullptr;   // caller's event recorded between a step's two sweeps (optional)
    int graph_kernels = 0;          // kernel nodes of the step graph captured last
    bool overlap = true;          // mb_set_overlap
    // launch shapes of the bulk kernels (mb_autotune): CTA size, register
    // budget and ring depth per direction of the FP32x2 kernels, rows per
    // thread of the y sweep
    int tune_cta[2] = {64 | SHAPE_MINB4 | SHAPE_RING8, 64 | SHAPE_MINB4};
    int tune_yseg = 64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int cur = 0;          // buffer holding the latest state (between steps)
    int qn = 0;           // buffer holding the step-start state
    int sidx = 0;         // sweep index within the step
    long long nstep = 0;  // steps taken since the last write_state of instance 0
    std::string err;
    std::map<std::tuple<int, int, unsigned long long>, cudaGraphExec_t> graphs;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
    std::vector<cudaEvent_t> free_events;
};

static mb_status fail(mb_sim *s, mb_status st, const std::string &msg) {
    if (s) s->err = msg;
    else g_create_error = msg;
    return st;
}

static mb_status cuda_check(mb_sim *s, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return MB_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(s, e == cudaErrorMemoryAllocation ? MB_E_NOMEM : MB_E_CUDA, m);
}

// device buffer owned by one instance (freed with it)
template <class P>
static cudaError_t ialloc(InstHost &h, P **p, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
    if (e == cudaSuccess) {
        h.allocs.push_back(v);
        *p = (P *)v;
    }
    return e;
}

// shared array: reallocated (contents dropped) when it must grow
template <class P>
static cudaError_t ensure(P **p, size_t &cap, size_t need, size_t elem) {
    if (*p && cap >= need) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    size_t n = std::max<size_t>(need + need / 4, 1);
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, n * elem);
    if (e != cudaSuccess) { cap = 0; return e; }
    *p = (P *)v;
    cap = n;
    return cudaSuccess;
}

static void drop_graphs(mb_sim *s) {
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
}

static void free_all(mb_sim *s) {
    drop_graphs(s);
    for (auto &e : s->evs) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    s->evs.clear();
    for (auto &h : s->ih)
        for (void *p : h.allocs) cudaFree(p);
    s->ih.clear();
    void *shared[] = {s->dd, s->dy, s->vx, s->vy, s->px, s->py, s->ebox, s->vmov, s->vnext,
                      s->rec, s->bnd, s->stage, s->ginst, s->ditem, s->dcount, s->iop, s->bstage, s->boff};
    for (void *p : shared)
        if (p) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    s->stream = nullptr;
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    s->side = nullptr;
    s->ev_fork = s->ev_join = nullptr;
}

static mb_status map_err(mb_sim *s, int e) {
    if (!e) return MB_OK;
    std::string m;
    mb_status st = MB_E_UNSTABLE;
    if (e & ERR_EDGE_CAP) { m += "edge list of a geometry column overflowed; "; st = MB_E_CAPACITY; }
    if (e & ERR_BAND_CAP) { m += "band record capacity overflowed; "; st = MB_E_CAPACITY; }
    if (e & ERR_DEFER_CAP) { m += "list of bulk cells deferred to the band fluxes overflowed; "; st = MB_E_CAPACITY; }
    if (e & ERR_STATE) { m += "second sweep of a step used another dt; "; st = MB_E_STATE; }
    if (e & ERR_NONBR) m += "covered/uncovered cell without a fluid neighbour; ";
    if (e & ERR_UNSTABLE) m += "non-physical state (rho or p <= 0 or non-finite); ";
    if (e & ERR_MIX_CAP) m += "more non-physical cells in one sweep than the positivity safeguard lists; ";
    if (e & ERR_MIX_BULK) m += "a merged cluster is still non-physical; ";
    if (e & ERR_MIX_BAND) m += "a cut cell is still non-physical after the safeguard; ";
    if (e & (ERR_EDGE_CAP | ERR_BAND_CAP | ERR_STATE | ERR_DEFER_CAP)) {
    } else {
        st = MB_E_UNSTABLE;
    }
    s->err = m;
    return st;
}

extern "C" {

const char *mb_last_error(const mb_sim *sim) { return sim ? sim->err.c_str() : g_create_error.c_str(); }

// MB_EULER_AXISYM is MB_EULER plus the geometric source step
static int base_equation(int eq) { return eq == MB_EULER_AXISYM ? MB_EULER : eq; }

// checks of one instance against the batch's precision and equation
static const char *check_instance(const mb_grid &g, const mb_body &b, int prec, int eq) {
    if (g.nx < 8 || g.ny < 8 || g.nx > 16384 || g.ny > 8192) return "grid size out of range";
    if (!(g.x1 > g.x0) || !(g.y1 > g.y0)) return "empty domain";
    if ((g.bc[0] == MB_BC_PERIODIC) != (g.bc[1] == MB_BC_PERIODIC) ||
        (g.bc[2] == MB_BC_PERIODIC) != (g.bc[3] == MB_BC_PERIODIC))
        return "periodic boundaries must come in pairs";
    if (g.equation != MB_EULER && g.equation != MB_ADVECTION && g.equation != MB_EULER_AXISYM)
        return "unknown equation";
    if (g.precision != prec) return "all instances of a batch share one precision";
    if (base_equation(g.equation) != base_equation(eq)) return "all instances of a batch share one equation";
    if (g.equation == MB_EULER_AXISYM && !(g.y0 == 0.0)) return "axisymmetric instances need y0 = 0 (the axis)";
    if (!(g.cfl > 0.0 && g.cfl <= 1.0)) return "cfl must be in (0, 1]";
    if (b.npoly < 0 || (b.npoly > 0 && (!b.poly_start || !b.poly_moving || !b.vx || !b.vy))) return "bad body";
    for (int p = 0; p < b.npoly; ++p)
        if (b.poly_start[p + 1] - b.poly_start[p] < 3) return "polygon with < 3 vertices";
    return nullptr;
}

// descriptor of one instance (device pointers and offsets into the shared
// arrays are set by make_instance and relayout)
static void describe_instance(int prec, int yseg, const mb_grid &g, double gamma, const mb_body &b,
                              const mb_motion &m, InstDesc &I, InstHost &h) {
    memset(&I, 0, sizeof(I));
    I.nx = g.nx; I.ny = g.ny;
    I.pitch = (g.nx + 31) / 32 * 32;
    I.nc = base_equation(g.equation) == MB_EULER ? 4 : 1;
    I.x0 = g.x0; I.y0 = g.y0;
    I.dx = (g.x1 - g.x0) / (double)g.nx;
    I.dy = (g.y1 - g.y0) / (double)g.ny;
    I.rdx = 1.0 / I.dx;
    I.rdy = 1.0 / I.dy;
    I.rdxf = (float)I.rdx;
    I.rdyf = (float)I.rdy;
    for (int q = 0; q < 4; ++q) I.bc[q] = g.bc[q];
    I.eq = base_equation(g.equation);
    I.axisym = g.equation == MB_EULER_AXISYM ? 1 : 0;
    I.ucov = g.uncover_mode;
    I.adv[0] = g.adv[0]; I.adv[1] = g.adv[1];
    I.gamma = gamma;
    I.cfl = g.cfl;
    I.U[0] = m.U[0]; I.U[1] = m.U[1];
    I.pivot[0] = m.pivot[0]; I.pivot[1] = m.pivot[1];
    I.a0 = m.a0; I.a1 = m.a1; I.omega = m.omega;
    I.rotating = (m.a0 != 0.0 || m.a1 != 0.0) ? 1 : 0;
    I.nv = b.npoly > 0 ? b.poly_start[b.npoly] : 0;
    double rmax = 0.0, perim = 0.0, bx0 = 1e300, bx1 = -1e300;
    bool has_static = false;
    for (int p = 0; p < b.npoly; ++p) {
        int a = b.poly_start[p], z = b.poly_start[p + 1];
        if (!b.poly_moving[p]) has_static = true;
        for (int v = a; v < z; ++v) {
            int w = v + 1 < z ? v + 1 : a;
            h.vx.push_back(b.vx[v]);
            h.vy.push_back(b.vy[v]);
            h.mov.push_back(b.poly_moving[p] ? 1 : 0);
            h.next.push_back(w);
            perim += std::hypot(b.vx[w] - b.vx[v], b.vy[w] - b.vy[v]);
            bx0 = std::min(bx0, b.vx[v]);
            bx1 = std::max(bx1, b.vx[v]);
            if (b.poly_moving[p]) rmax = std::max(rmax, std::hypot(b.vx[v] - m.pivot[0], b.vy[v] - m.pivot[1]));
        }
    }
    double wr = std::fabs(m.a1 * m.omega) * rmax;
    I.wall_bound[0] = std::fabs(m.U[0]) + wr;
    I.wall_bound[1] = std::fabs(m.U[1]) + wr;
    double hh = std::min(I.dx, I.dy);
    long long cap = 4LL * (long long)std::ceil(perim / hh) + 2LL * I.nv + 1024;
    if (I.rotating) cap *= 2;
    cap = std::min<long long>(cap, (long long)g.nx * g.ny);
    I.rec_cap = (int)cap;
    int gcols = g.nx;
    if (!has_static && I.nv > 0) {
        double width = I.rotating ? 2.0 * rmax : (bx1 - bx0);
        gcols = std::min(g.nx, (int)std::ceil(width / I.dx) + 8);
    }
    if (I.nv == 0) gcols = 0;
    I.gcol_max = gcols;
    // bulk work items: x sweep one warp per row; y sweep one warp per 32
    // columns (64 for the FP32 Euler kernel that carries two columns per
    // thread) and 64-row segment
    I.tiles_x[0] = 1;
    I.ntiles[0] = g.ny;
    const int ycols = (prec == MB_FP32 && base_equation(g.equation) == MB_EULER) ? 64 : 32;
    I.tiles_x[1] = (g.nx + ycols - 1) / ycols;
    I.yseg = yseg;
    I.ntiles[1] = I.tiles_x[1] * ((g.ny + yseg - 1) / yseg);
}

// descriptor and device buffers of one instance
static cudaError_t make_instance(mb_sim *s, const mb_grid &g, double gamma, const mb_body &b, const mb_motion &m,
                                 InstDesc &I, InstHost &h) {
    describe_instance(s->prec, s->tune_yseg, g, gamma, b, m, I, h);
    I.serial_bulk = s->overlap ? 0 : 1;
    const size_t esz = s->prec == MB_FP32 ? 4 : 8;
    const size_t cells = (size_t)I.pitch * g.ny;
    cudaError_t e = cudaSuccess;
    for (int bb = 0; bb < 3 && e == cudaSuccess; ++bb) e = ialloc(h, &I.Q[bb], cells * I.nc * esz);
    if (e == cudaSuccess) e = ialloc(h, &I.cls, cells);
    if (e == cudaSuccess) e = ialloc(h, &I.rec, cells * sizeof(int));
    if (e == cudaSuccess) e = ialloc(h, &I.alpha, cells * sizeof(double));
    double *xn = nullptr, *yn = nullptr;
    if (e == cudaSuccess) e = ialloc(h, &xn, (g.nx + 1) * sizeof(double));
    if (e == cudaSuccess) e = ialloc(h, &yn, (g.ny + 1) * sizeof(double));
    I.xn = xn;
    I.yn = yn;
    if (e == cudaSuccess) e = cudaMemsetAsync(I.cls, 0, cells, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.rec, 0xff, cells * sizeof(int), s->stream);
    return e;
}

// device bytes an instance holds (its own buffers and its share of the
// shared arrays), for admission by memory budget
static size_t instance_bytes(const InstDesc &I, int prec) {
    const size_t esz = prec == MB_FP32 ? 4 : 8;
    const size_t cells = (size_t)I.pitch * I.ny;
    return 3 * cells * I.nc * esz + cells * (1 + 4 + 8) + (size_t)(I.nx + I.ny + 2) * 8 +
           (size_t)I.rec_cap * (sizeof(BandRec) + 8) + (size_t)I.nv * 100 + sizeof(InstDesc) + sizeof(InstDyn) +
           (size_t)I.nx * I.ny * I.nc * 8;
}

// offsets of every instance in the shared arrays, those arrays, the
// descriptors and the instance of every geometry group; the dynamic state of
// new instance k is the old instance from[k]'s (zero when from[k] < 0).  The
// stream must be idle.
static cudaError_t relayout(mb_sim *s, int old_n, const std::vector<int> &from) {
    const int n = (int)s->hd.size();
    std::vector<InstDyn> old(old_n), dyn(n);
    cudaError_t e = cudaSuccess;
    if (old_n > 0) e = cudaMemcpy(old.data(), s->dy, old_n * sizeof(InstDyn), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < n; ++k) {
        if (from[k] >= 0) dyn[k] = old[from[k]];
        else memset(&dyn[k], 0, sizeof(InstDyn));
    }
    std::vector<double> hvx, hvy;
    std::vector<unsigned char> hmov;
    std::vector<int> hnext;
    int rec_total = 0, tiles0 = 0, tiles1 = 0;
    size_t max_cells = 1;
    for (int k = 0; k < n; ++k) {
        InstDesc &I = s->hd[k];
        const InstHost &h = s->ih[k];
        I.voff = (int)hvx.size();
        hvx.insert(hvx.end(), h.vx.begin(), h.vx.end());
        hvy.insert(hvy.end(), h.vy.begin(), h.vy.end());
        hmov.insert(hmov.end(), h.mov.begin(), h.mov.end());
        for (int w : h.next) hnext.push_back(I.voff + w);
        I.rec_base = rec_total;
        rec_total += I.rec_cap;
        I.tile_off[0] = tiles0;
        I.tile_off[1] = tiles1;
        tiles0 += I.ntiles[0];
        tiles1 += I.ntiles[1];
        max_cells = std::max(max_cells, (size_t)I.nx * I.ny);
    }
    // geometry groups (GEO_GC columns, one CTA each): instances with more
    // polygon vertices first, so that the groups with the most cut cells start
    // in the first wave of CTAs
    std::vector<int> order(n), ginst;
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s->hd[a].nv > s->hd[b].nv; });
    int col_total = 0;
    for (int k : order) {
        InstDesc &I = s->hd[k];
        I.gcol_off = col_total;
        const int ng = (I.gcol_max + GEO_GC - 1) / GEO_GC;
        for (int q = 0; q < ng; ++q) ginst.push_back(k);
        col_total += ng;
    }
    const size_t tv = std::max<size_t>(1, hvx.size());
    if (e == cudaSuccess) e = ensure(&s->vx, s->cap_vx, tv, sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->vy, s->cap_vy, tv, sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->vmov, s->cap_mov, tv, 1);
    if (e == cudaSuccess) e = ensure(&s->vnext, s->cap_next, tv, sizeof(int));
    if (e == cudaSuccess) e = ensure(&s->px, s->cap_px, 3 * tv, sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->py, s->cap_py, 3 * tv, sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->ebox, s->cap_ebox, 3 * tv * 2, sizeof(float));
    if (e == cudaSuccess) e = ensure(&s->rec, s->cap_rec, std::max(1, rec_total), sizeof(BandRec));
    if (e == cudaSuccess) e = ensure(&s->bnd, s->cap_bnd, std::max(1, rec_total), sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->stage, s->stage_len, max_cells * 4, sizeof(double));
    if (e == cudaSuccess) e = ensure(&s->iop, s->cap_iop, std::max(1, n), sizeof(double *));
    if (e == cudaSuccess) e = ensure(&s->boff, s->cap_boff, (size_t)n + 1, sizeof(int));
    if (e == cudaSuccess) e = ensure(&s->dd, s->cap_dd, std::max(1, n), sizeof(InstDesc));
    if (e == cudaSuccess) e = ensure(&s->dy, s->cap_dy, std::max(1, n), sizeof(InstDyn));
    if (e == cudaSuccess) e = ensure(&s->ginst, s->cap_ginst, std::max<size_t>(1, ginst.size()), sizeof(int));
    // a touched cell defers at most 4 cell pairs of its line; the cells
    // touched at a sweep's start pose are band cells of the sweep before
    if (e == cudaSuccess) e = ensure(&s->ditem, s->cap_ditem, 4 * (size_t)rec_total + 4096, sizeof(int2));
    if (e == cudaSuccess) e = ensure(&s->dcount, s->cap_dcount, 1, sizeof(int));
    if (e != cudaSuccess) return e;
    // the posed vertices of pose slot 0 are refreshed by every classification;
    // the other slots by every sweep
    if (!hvx.empty()) {
        e = cudaMemcpy(s->vx, hvx.data(), hvx.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->vy, hvy.data(), hvy.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->vmov, hmov.data(), hmov.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->vnext, hnext.data(), hnext.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && n > 0) e = cudaMemcpy(s->dd, s->hd.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n > 0) e = cudaMemcpy(s->dy, dyn.data(), n * sizeof(InstDyn), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ginst.empty())
        e = cudaMemcpy(s->ginst, ginst.data(), ginst.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    s->n = n;
    s->total_v = (int)hvx.size();
    s->total_rec = rec_total;
    s->total_cols = col_total;
    s->total_tiles[0] = tiles0;
    s->total_tiles[1] = tiles1;
    drop_graphs(s);
    return cudaSuccess;
}

// classes and volume fractions of instances k .. k+cnt-1 at their current
// poses (alpha_out: the volume fractions of a single instance, nx*ny)
static void classify_instances(mb_sim *s, int k, int cnt, double *alpha_out, cudaStream_t st) {
    int max_nx = 0;
    for (int q = k; q < k + cnt; ++q) max_nx = std::max(max_nx, s->hd[q].nx);
    launch_classify(s->dd, s->dy, s->vx, s->vy, s->vmov, s->px, s->py, s->ebox, s->vnext, s->total_v, k, cnt, max_nx,
                    alpha_out, st);
}

mb_status mb_batch_create(int n, const mb_grid *grids, const double *gammas, const mb_body *bodies,
                          const mb_motion *motions, mb_sim **out) {
    if (!out) return fail(nullptr, MB_E_INVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !grids || !bodies || !motions) return fail(nullptr, MB_E_INVAL, "bad batch arguments");
    for (int k = 0; k < n; ++k) {
        const char *msg = check_instance(grids[k], bodies[k], grids[0].precision, grids[0].equation);
        if (msg) return fail(nullptr, MB_E_INVAL, msg);
    }
    mb_sim *s = new mb_sim();
    s->prec = grids[0].precision;
    s->eq = base_equation(grids[0].equation);
#define CK(x)                                                     \
    do {                                                          \
        cudaError_t _e = (x);                                     \
        if (_e != cudaSuccess) {                                  \
            mb_status _st = cuda_check(s, _e, #x);                \
            g_create_error = s->err;                              \
            free_all(s);                                          \
            delete s;                                             \
            return _st;                                           \
        }                                                         \
    } while (0)
    CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
    {
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, hi));
        CK(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
    s->hd.resize(n);
    s->ih.resize(n);
    for (int k = 0; k < n; ++k)
        CK(make_instance(s, grids[k], gammas ? gammas[k] : 1.4, bodies[k], motions[k], s->hd[k], s->ih[k]));
    CK(cudaStreamSynchronize(s->stream));
    geom_init();
    CK(relayout(s, 0, std::vector<int>(n, -1)));
    launch_nodes(s->dd, n, s->stream);
    for (int d = 0; d < 2; ++d) {
        int bps = s->prec == MB_FP32 ? bulk_blocks_per_sm<float>(d) : bulk_blocks_per_sm<double>(d);
        s->bulk_grid[d] = bps * s->nsm;
    }
    // initial classes at t = 0
    classify_instances(s, 0, n, nullptr, s->stream);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
#undef CK
    *out = s;
    return MB_OK;
}

mb_status mb_batch_add(mb_sim *sim, const mb_grid *grid, double gamma, const mb_body *body, const mb_motion *motion,
                       int *inst) {
    if (!sim || !grid || !body || !motion) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_batch_add in the middle of a step");
    const char *msg = check_instance(*grid, *body, sim->prec, sim->eq);
    if (msg) return fail(sim, MB_E_INVAL, msg);
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "batch_add sync");
    const int old_n = sim->n;
    InstDesc I;
    InstHost h;
    e = make_instance(sim, *grid, gamma, *body, *motion, I, h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) {
        for (void *p : h.allocs) cudaFree(p);
        return cuda_check(sim, e, "batch_add buffers");
    }
    sim->hd.push_back(I);
    sim->ih.push_back(std::move(h));
    std::vector<int> from(old_n + 1);
    for (int k = 0; k < old_n; ++k) from[k] = k;
    from[old_n] = -1;
    e = relayout(sim, old_n, from);
    if (e == cudaSuccess) {
        launch_nodes(sim->dd, sim->n, sim->stream);
        classify_instances(sim, old_n, 1, nullptr, sim->stream);
        e = cudaStreamSynchronize(sim->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_check(sim, e, "batch_add");
    if (inst) *inst = old_n;
    return MB_OK;
}

mb_status mb_batch_remove(mb_sim *sim, int inst) {
    if (!sim || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_batch_remove in the middle of a step");
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "batch_remove sync");
    const int old_n = sim->n;
    for (void *p : sim->ih[inst].allocs) cudaFree(p);
    sim->hd.erase(sim->hd.begin() + inst);
    sim->ih.erase(sim->ih.begin() + inst);
    std::vector<int> from(old_n - 1);
    for (int k = 0; k < old_n - 1; ++k) from[k] = k < inst ? k : k + 1;
    e = relayout(sim, old_n, from);
    if (e != cudaSuccess) return cuda_check(sim, e, "batch_remove");
    if (sim->n == 0) sim->nstep = 0;
    return MB_OK;
}

size_t mb_instance_bytes(const mb_sim *sim, int inst) {
    if (!sim || inst < 0 || inst >= sim->n) return 0;
    return instance_bytes(sim->hd[inst], sim->prec);
}

size_t mb_request_bytes(const mb_grid *grid, const mb_body *body, const mb_motion *motion) {
    if (!grid || !body || !motion) return 0;
    if (check_instance(*grid, *body, grid->precision, grid->equation)) return 0;
    InstDesc I;
    InstHost h;
    describe_instance(grid->precision, 64, *grid, 1.4, *body, *motion, I, h);
    return instance_bytes(I, grid->precision);
}

mb_status mb_create(const mb_grid *grid, double gamma, const mb_body *body, const mb_motion *motion, mb_sim **out) {
    if (!grid || !body || !motion) return fail(nullptr, MB_E_INVAL, "NULL argument");
    return mb_batch_create(1, grid, &gamma, body, motion, out);
}

void mb_destroy(mb_sim *sim) {
    if (!sim) return;
    if (sim->stream) cudaStreamSynchronize(sim->stream);
    free_all(sim);
    delete sim;
}

mb_status mb_set_stream(mb_sim *sim, void *stream) {
    if (!sim) return MB_E_INVAL;
    cudaStreamSynchronize(sim->stream);
    for (auto &kv : sim->graphs) cudaGraphExecDestroy(kv.second);
    sim->graphs.clear();
    if (stream) {
        if (sim->own_stream) cudaStreamDestroy(sim->stream);
        sim->own_stream = false;
        sim->stream = (cudaStream_t)stream;
    } else if (!sim->own_stream) {
        cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking);
        sim->own_stream = true;
    }
    return MB_OK;
}

mb_status mb_set_overlap(mb_sim *sim, int enable) {
    if (!sim) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_set_overlap in the middle of a step");
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    sim->overlap = enable != 0;
    drop_graphs(sim);   // captured steps hold the launch sequence of the old setting
    for (auto &I : sim->hd) I.serial_bulk = sim->overlap ? 0 : 1;
    if (e == cudaSuccess && sim->n > 0)
        e = cudaMemcpy(sim->dd, sim->hd.data(), sim->n * sizeof(InstDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(sim, e, "set overlap");
    return MB_OK;
}

static mb_status do_sweep(mb_sim *s, int dir, double dt) {
    int src, dst, qn;
    if (s->sidx == 0) {
        s->qn = s->cur;
        src = s->cur;
        dst = (s->cur + 1) % 3;
    } else {
        src = (s->qn + 1) % 3;
        dst = (s->qn + 2) % 3;
    }
    qn = s->qn;
    const int last = s->sidx == 1;
    cudaStream_t st = s->stream;
    // k_pose also empties the sweep's list of deferred bulk cell pairs
    launch_pose(s->dd, s->dy, s->vx, s->vy, s->vmov, s->vnext, s->px, s->py, s->ebox, s->total_v, s->n, dir, s->sidx,
                dt, s->dcount, st);
    auto band = [&](int stage, cudaStream_t sx) {
        if (s->prec == MB_FP32)
            launch_band_stage<float>(stage, s->dd, s->dy, s->rec, s->bnd, s->boff, s->n, s->total_rec,
                                     dir, src, dst, qn, s->sidx, last, sx);
        else
            launch_band_stage<double>(stage, s->dd, s->dy, s->rec, s->bnd, s->boff, s->n, s->total_rec,
                                      dir, src, dst, qn, s->sidx, last, sx);
    };
    auto geom_band = [&](cudaStream_t sx) {
        launch_geom(s->dd, s->dy, s->ginst, s->px, s->py, s->ebox, s->vnext, s->vmov, s->total_v, s->n, s->total_cols,
                    dir, s->rec, s->bnd, sx);
        band(0, sx);
        band(1, sx);
    };
    const int eq = s->eq;
    // whether an instance may take the deferred pass whole this sweep (a
    // rotating body, a host time step, or a CFL number that lets a body move
    // 0.9 cells per sweep)
    bool any_dall = dt > 0.0;
    for (const auto &I : s->hd) any_dall = any_dall || I.rotating || I.cfl >= 0.9 || I.serial_bulk;
    const DeferList dl{s->ditem, s->dcount, (int)std::min<size_t>(s->cap_ditem, 0x7fffffff)};
    auto bulk = [&](int mode) {

        if (s->prec == MB_FP32)
            launch_bulk<float>(dir, eq, s->dd, s->dy, s->rec, s->n, s->total_tiles[dir], src, dst, last,
                               s->tune_cta[dir], mode, dl, any_dall ? 1 : 0, st);
        else
            launch_bulk<double>(dir, eq, s->dd, s->dy, s->rec, s->n, s->total_tiles[dir], src, dst, last,
                                s->tune_cta[dir], mode, dl, any_dall ? 1 : 0, st);
    };
    const bool two_pass = s->prec == MB_FP32 && eq == MB_EULER;
    if (two_pass && !s->timing) {
        // geometry and band fluxes (FP64 pipe, latency) on the side stream
        // while the bulk pass that needs no band data (FP32 pipe, HBM) runs
        // on the sim's stream; the deferred cells after both
        cudaEventRecord(s->ev_fork, st);
        cudaStreamWaitEvent(s->side, s->ev_fork, 0);
        geom_band(s->side);
        band(2, s->side);   // covering / uncovering: band records only, no bulk cell
        cudaEventRecord(s->ev_join, s->side);
        bulk(0);
        cudaStreamWaitEvent(st, s->ev_join, 0);
        bulk(1);
    } else {
        geom_band(st);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (s->timing) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, st);
        }
        bulk(0);
        bulk(1);
        if (s->timing) {
            cudaEventRecord(e1, st);
            s->evs.push_back({e0, e1});
        }
    }
    if (!(two_pass && !s->timing)) band(2, st);
    band(3, st);
    band(4, st);
    if (dir == 1 && s->eq == MB_EULER) {
        // geometric source of the axisymmetric instances after the radial sweep
        bool axi = false;
        for (const auto &I : s->hd) axi = axi || I.axisym;
        if (axi) {
            if (s->prec == MB_FP32) launch_axisym_source<float>(s->dd, s->dy, s->n, s->total_tiles[0], dst, st);
            else launch_axisym_source<double>(s->dd, s->dy, s->n, s->total_tiles[0], dst, st);
        }
    }
    if (s->sidx == 1) {
        s->cur = dst;
        s->sidx = 0;
        s->nstep++;
    } else {
        s->sidx = 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(s, e, "sweep launch");
    return MB_OK;
}

mb_status mb_sweep(mb_sim *sim, int dir, double dt) {
    if (!sim) return MB_E_INVAL;
    if (sim->n == 0) return MB_OK;
    if (dir != 0 && dir != 1) return fail(sim, MB_E_INVAL, "dir must be 0 or 1");
    if (!(dt > 0.0)) return fail(sim, MB_E_INVAL, "mb_sweep needs dt > 0");
    return do_sweep(sim, dir, dt);
}

static mb_status issue_step(mb_sim *sim, double dt) {
    if (sim->n == 0) return MB_OK;   // an empty batch (all instances removed)
    int d1 = (sim->nstep % 2 == 0) ? 0 : 1;
    mb_status r = do_sweep(sim, d1, dt);
    if (r != MB_OK) return r;
    if (sim->ev_mid) {
        // an external record: inside a stream capture a plain record would
        // become a dependency edge and never time anything
        cudaError_t e = cudaEventRecordWithFlags(sim->ev_mid, sim->stream, cudaEventRecordExternal);
        if (e != cudaSuccess) return cuda_check(sim, e, "sweep event");
    }
    return do_sweep(sim, 1 - d1, dt);
}

mb_status mb_step(mb_sim *sim, double dt, double *dt_used) {
    if (!sim) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_step in the middle of a step");
    mb_status r = issue_step(sim, dt > 0.0 ? dt : 0.0);
    if (r != MB_OK) return r;
    if (dt_used) {
        std::vector<InstDyn> h(sim->n);
        cudaError_t e = cudaMemcpyAsync(h.data(), sim->dy, sim->n * sizeof(InstDyn), cudaMemcpyDeviceToHost, sim->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
        if (e != cudaSuccess) return cuda_check(sim, e, "dt readback");
        for (int k = 0; k < sim->n; ++k) dt_used[k] = h[k].dt;
    }
    return MB_OK;
}

mb_status mb_run(mb_sim *sim, int nsteps, double dt) {
    if (!sim || nsteps < 0) return MB_E_INVAL;
    if (sim->n == 0) return MB_OK;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_run in the middle of a step");
    double dth = dt > 0.0 ? dt : 0.0;
    for (int k = 0; k < nsteps; ++k) {
        if (sim->timing) {
            mb_status r = issue_step(sim, dth);
            if (r != MB_OK) return r;
            continue;
        }
        unsigned long long bits;
        memcpy(&bits, &dth, sizeof(bits));
        auto key = std::make_tuple(sim->cur, (int)(sim->nstep % 2), bits);
        auto it = sim->graphs.find(key);
        if (it == sim->graphs.end()) {
            int cur0 = sim->cur;
            long long ns0 = sim->nstep;
            cudaGraph_t g;
            cudaError_t e = cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_check(sim, e, "begin capture");
            mb_status r = issue_step(sim, dth);
            e = cudaStreamEndCapture(sim->stream, &g);
            if (r != MB_OK) return r;
            if (e != cudaSuccess) return cuda_check(sim, e, "end capture");
            cudaGraphExec_t ex;
            // kernel launches per step, for the caller's accounting
            size_t nn = 0;
            if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess) {
                std::vector<cudaGraphNode_t> nodes(nn);
                int kn = 0;
                if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess) {
                    for (auto nd : nodes) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
                    }
                }
                sim->graph_kernels = kn;
            }
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_check(sim, e, "instantiate");
            it = sim->graphs.emplace(key, ex).first;
            sim->cur = cur0;   // capture did not run the step
            sim->nstep = ns0;
        }
        cudaError_t e = cudaGraphLaunch(it->second, sim->stream);
        if (e != cudaSuccess) return cuda_check(sim, e, "graph launch");
        sim->qn = sim->cur;
        sim->cur = (sim->cur + 2) % 3;
        sim->nstep++;
    }
    return MB_OK;
}

mb_status mb_sync(mb_sim *sim) {
    if (!sim) return MB_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "sync");
    std::vector<InstDyn> h(sim->n);
    e = cudaMemcpy(h.data(), sim->dy, sim->n * sizeof(InstDyn), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(sim, e, "dyn readback");
    int err = 0;
    for (auto &x : h) err |= x.err;
    return map_err(sim, err);
}

// batch staging buffer: the FP64 states of all instances back to back
// (allocated on the first batched state I/O call); off[k]: instance k's offset
static cudaError_t batch_stage(mb_sim *sim, std::vector<size_t> &off) {
    off.resize(sim->n + 1);
    off[0] = 0;
    for (int k = 0; k < sim->n; ++k) {
        const InstDesc &I = sim->hd[k];
        off[k + 1] = off[k] + (size_t)I.nx * I.ny * I.nc;
    }
    return ensure(&sim->bstage, sim->cap_bstage, off[sim->n], sizeof(double));
}

static size_t state_elems(const InstDesc &I) { return (size_t)I.nx * I.ny * I.nc; }

// instances k0 .. k0+cnt-1 from host arrays Q[q] at times t[q].  A single
// instance goes through the one-instance staging buffer; a batch is copied
// whole into the batch staging buffer while its classification runs on the
// side stream, then converted by one launch.
// H: the element type of the host states (FP64 or FP32); the staging buffers
// hold them in that type
extern "C++" {
template <class H>
static mb_status write_states(mb_sim *sim, int k0, int cnt, const H *const *Q, const double *t) {
    if (sim->sidx != 0) {
        // abandon the half-done step: the written state starts a new one
        sim->cur = (sim->qn + 1) % 3;
        sim->sidx = 0;
    }
    cudaStream_t st = sim->stream;
    std::vector<InstDyn> ys(cnt);
    int max_ny = 0;
    for (int q = 0; q < cnt; ++q) {
        const InstDesc &I = sim->hd[k0 + q];
        InstDyn &y = ys[q];
        memset(&y, 0, sizeof(y));
        y.t = t[q];
        y.X = I.U[0] * t[q];
        y.Y = I.U[1] * t[q];
        y.th = I.rotating ? I.a0 + I.a1 * std::sin(I.omega * t[q]) : 0.0;
        max_ny = std::max(max_ny, I.ny);
    }
    cudaError_t e = cudaMemcpyAsync(sim->dy + k0, ys.data(), cnt * sizeof(InstDyn), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_check(sim, e, "write_state copy");
    auto launch = [&](const H *const *ptrs, const H *p1, int i0, int ni, int mny) {
        if (sim->prec == MB_FP32) launch_write_state<float, H>(sim->dd, sim->dy, ptrs, p1, i0, ni, mny, sim->cur, st);
        else launch_write_state<double, H>(sim->dd, sim->dy, ptrs, p1, i0, ni, mny, sim->cur, st);
    };
    H *const stage1 = (H *)sim->stage;   // the batch buffer is taken after batch_stage (it may allocate)
    if (cnt == 1) {
        e = cudaMemcpyAsync(stage1, Q[0], state_elems(sim->hd[k0]) * sizeof(H), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_check(sim, e, "write_state copy");
        classify_instances(sim, k0, 1, nullptr, st);
        launch(nullptr, stage1, k0, 1, max_ny);
    } else {
        std::vector<size_t> off;
        e = batch_stage(sim, off);
        if (e != cudaSuccess) return cuda_check(sim, e, "write_states staging");
        H *const bst = (H *)sim->bstage;
        e = cudaEventRecord(sim->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sim->side, sim->ev_fork, 0);
        if (e != cudaSuccess) return cuda_check(sim, e, "write_states fork");
        classify_instances(sim, k0, cnt, nullptr, sim->side);
        e = cudaEventRecord(sim->ev_join, sim->side);
        std::vector<const H *> ptrs(cnt);
        for (int q = 0; q < cnt && e == cudaSuccess; ++q) {
            ptrs[q] = bst + off[k0 + q];
            e = cudaMemcpyAsync(bst + off[k0 + q], Q[q], state_elems(sim->hd[k0 + q]) * sizeof(H),
                                cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sim->iop, ptrs.data(), cnt * sizeof(H *), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, sim->ev_join, 0);
        if (e != cudaSuccess) return cuda_check(sim, e, "write_states copy");
        launch((const H *const *)sim->iop, nullptr, k0, cnt, max_ny);
    }
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(sim, e, "write_state");
    if (k0 == 0) sim->nstep = 0;
    return MB_OK;
}
}  // extern "C++"

// states of instances k0 .. k0+cnt-1 into host arrays Q[q] (entries may be
// NULL); their dynamic records into ys.  A batch is converted by one launch
// into the batch staging buffer, then copied out.
extern "C++" {
template <class H>
static mb_status read_states(mb_sim *sim, int k0, int cnt, H *const *Q, std::vector<InstDyn> &ys) {
    cudaStream_t st = sim->stream;
    const int buf = sim->sidx == 0 ? sim->cur : (sim->qn + 1) % 3;
    auto launch = [&](H *const *ptrs, H *p1, int i0, int ni, int max_ny) {
        if (sim->prec == MB_FP32) launch_read_state<float, H>(sim->dd, ptrs, p1, i0, ni, max_ny, buf, st);
        else launch_read_state<double, H>(sim->dd, ptrs, p1, i0, ni, max_ny, buf, st);
    };
    H *const stage1 = (H *)sim->stage;   // the batch buffer is taken after batch_stage (it may allocate)
    cudaError_t e = cudaSuccess;
    if (cnt == 1) {
        if (Q[0]) {
            launch(nullptr, stage1, k0, 1, sim->hd[k0].ny);
            e = cudaMemcpyAsync(Q[0], stage1, state_elems(sim->hd[k0]) * sizeof(H), cudaMemcpyDeviceToHost, st);
        }
    } else {
        std::vector<size_t> off;
        e = batch_stage(sim, off);
        if (e != cudaSuccess) return cuda_check(sim, e, "read_states staging");
        H *const bst = (H *)sim->bstage;
        std::vector<H *> ptrs(cnt, nullptr);
        int max_ny = 0;
        for (int q = 0; q < cnt; ++q) {
            if (!Q[q]) continue;
            ptrs[q] = bst + off[k0 + q];
            max_ny = std::max(max_ny, sim->hd[k0 + q].ny);
        }
        e = cudaMemcpyAsync(sim->iop, ptrs.data(), cnt * sizeof(H *), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) launch((H *const *)sim->iop, nullptr, k0, cnt, max_ny);
        for (int q = 0; q < cnt && e == cudaSuccess; ++q)
            if (Q[q])
                e = cudaMemcpyAsync(Q[q], ptrs[q], state_elems(sim->hd[k0 + q]) * sizeof(H), cudaMemcpyDeviceToHost,
                                    st);
    }
    if (e != cudaSuccess) return cuda_check(sim, e, "read_state copy");
    ys.resize(cnt);
    e = cudaMemcpyAsync(ys.data(), sim->dy + k0, cnt * sizeof(InstDyn), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(sim, e, "read_state");
    return MB_OK;
}
}  // extern "C++"

static void clock_of(const InstDyn &y, double *clock) {
    clock[0] = y.t;
    clock[1] = y.X;
    clock[2] = y.Y;
    clock[3] = (double)y.step;
}

mb_status mb_write_state(mb_sim *sim, int inst, const double *Q, double t) {
    if (!sim || !Q || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    return write_states(sim, inst, 1, &Q, &t);
}

extern "C++" {
template <class H>
static mb_status write_all(mb_sim *sim, const H *const *Q, const double *t) {
    if (!sim || !Q) return MB_E_INVAL;
    for (int k = 0; k < sim->n; ++k)
        if (!Q[k]) return fail(sim, MB_E_INVAL, "write_states: NULL state array");
    std::vector<double> tt(sim->n, 0.0);
    if (t) tt.assign(t, t + sim->n);
    return write_states(sim, 0, sim->n, Q, tt.data());
}
}  // extern "C++"

mb_status mb_write_states(mb_sim *sim, const double *const *Q, const double *t) { return write_all(sim, Q, t); }

mb_status mb_write_states_f32(mb_sim *sim, const float *const *Q, const double *t) { return write_all(sim, Q, t); }

mb_status mb_read_state(mb_sim *sim, int inst, double *Q, double *alpha, double *clock) {
    if (!sim || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    const InstDesc &I = sim->hd[inst];
    cudaStream_t st = sim->stream;
    if (alpha) {
        classify_instances(sim, inst, 1, sim->stage, st);
        cudaError_t e = cudaMemcpyAsync(alpha, sim->stage, (size_t)I.nx * I.ny * sizeof(double),
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_check(sim, e, "alpha copy");
    }
    std::vector<InstDyn> ys;
    mb_status r = read_states(sim, inst, 1, &Q, ys);
    if (r != MB_OK) return r;
    if (clock) clock_of(ys[0], clock);
    return map_err(sim, ys[0].err);
}

extern "C++" {
template <class H>
static mb_status read_all(mb_sim *sim, H *const *Q, double *clocks) {
    if (!sim || !Q) return MB_E_INVAL;
    std::vector<InstDyn> ys;
    mb_status r = read_states(sim, 0, sim->n, Q, ys);
    if (r != MB_OK) return r;
    r = MB_OK;
    for (int k = 0; k < sim->n; ++k) {
        if (clocks) clock_of(ys[k], clocks + 4 * k);
        if (r == MB_OK && ys[k].err) r = map_err(sim, ys[k].err);
    }
    return r;
}
}  // extern "C++"

mb_status mb_read_states(mb_sim *sim, double *const *Q, double *clocks) { return read_all(sim, Q, clocks); }

mb_status mb_read_states_f32(mb_sim *sim, float *const *Q, double *clocks) { return read_all(sim, Q, clocks); }

mb_status mb_band_records(mb_sim *sim, int inst, void *out, int max_records, int *count) {
    if (!sim || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    InstDyn y;
    cudaError_t e = cudaMemcpyAsync(&y, sim->dy + inst, sizeof(y), cudaMemcpyDeviceToHost, sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "band records");
    int n = std::min(y.band_count, sim->hd[inst].rec_cap);
    if (count) *count = n;
    if (out && max_records > 0) {
        n = std::min(n, max_records);
        e = cudaMemcpy(out, sim->rec + sim->hd[inst].rec_base, (size_t)n * sizeof(BandRec), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_check(sim, e, "band records copy");
    }
    return MB_OK;
}

int mb_band_record_size(void) { return (int)sizeof(BandRec); }

mb_status mb_info(const mb_sim *sim, int inst, int *n_inst, int *nx, int *ny, int *nc) {
    if (!sim) return MB_E_INVAL;
    if (n_inst) *n_inst = sim->n;
    if (inst >= 0 && inst < sim->n) {
        if (nx) *nx = sim->hd[inst].nx;
        if (ny) *ny = sim->hd[inst].ny;
        if (nc) *nc = sim->hd[inst].nc;
    }
    return MB_OK;
}

mb_status mb_diagnostics(mb_sim *sim, int inst, double *out) {
    if (!sim || !out || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    InstDyn y;
    cudaError_t e = cudaMemcpyAsync(&y, sim->dy + inst, sizeof(y), cudaMemcpyDeviceToHost, sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "diagnostics");
    for (int q = 0; q < 4; ++q) out[q] = y.wall_sum[q];
    out[4] = y.mixed;
    out[5] = y.band_count;
    return MB_OK;
}

mb_status mb_probe(mb_sim *sim, int inst, int n, const int *ij, double *out) {
    if (!sim || inst < 0 || inst >= sim->n || n < 0 || (n > 0 && (!ij || !out))) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_probe in the middle of a step");
    const InstDesc &I = sim->hd[inst];
    const size_t esz = sim->prec == MB_FP32 ? 4 : 8;
    const size_t plane = (size_t)I.pitch * I.ny;
    std::vector<unsigned char> raw((size_t)n * I.nc * 8);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const int i = ij[2 * k], j = ij[2 * k + 1];
        if (i < 0 || i >= I.nx || j < 0 || j >= I.ny) return fail(sim, MB_E_INVAL, "mb_probe: cell outside the grid");
        for (int q = 0; q < I.nc && e == cudaSuccess; ++q) {
            const unsigned char *src = (const unsigned char *)I.Q[sim->cur] + ((size_t)q * plane + (size_t)j * I.pitch + i) * esz;
            e = cudaMemcpyAsync(raw.data() + ((size_t)q * n + k) * 8, src, esz, cudaMemcpyDeviceToHost, sim->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "probe");
    for (size_t m = 0; m < (size_t)n * I.nc; ++m) {
        if (esz == 4) {
            float f;
            memcpy(&f, raw.data() + m * 8, 4);
            out[m] = f;
        } else {
            memcpy(&out[m], raw.data() + m * 8, 8);
        }
    }
    return MB_OK;
}

mb_status mb_merge_count(mb_sim *sim, int inst, long long *cells) {
    if (!sim || !cells || inst < 0 || inst >= sim->n) return MB_E_INVAL;
    InstDyn y;
    cudaError_t e = cudaMemcpyAsync(&y, sim->dy + inst, sizeof(y), cudaMemcpyDeviceToHost, sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "merge count");
    *cells = y.mixed_total;
    return MB_OK;
}

// rows per thread of the y sweep for every instance (tile counts follow)
static cudaError_t set_yseg(mb_sim *s, int yseg) {
    if (yseg == s->tune_yseg) return cudaSuccess;
    s->tune_yseg = yseg;
    for (auto &I : s->hd) {
        I.yseg = yseg;
        I.ntiles[1] = I.tiles_x[1] * ((I.ny + yseg - 1) / yseg);
    }
    std::vector<int> from(s->n);
    for (int k = 0; k < s->n; ++k) from[k] = k;
    return relayout(s, s->n, from);
}

mb_status mb_autotune(mb_sim *sim, double *report) {
    if (!sim) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_autotune in the middle of a step");
    if (sim->n == 0) return MB_OK;
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "autotune sync");
    // the bulk kernels alone, from the current state into a free buffer,
    // outside a step (no band cells are marked then; the last-sweep outputs
    // stay off), so the simulation is not changed
    const int src = sim->cur, dst = (sim->cur + 1) % 3;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_bulk = [&](int dir, int cta) -> double {
        auto go = [&]() {
            const DeferList dl{sim->ditem, sim->dcount, (int)std::min<size_t>(sim->cap_ditem, 0x7fffffff)};
            for (int mode = 0; mode < 2; ++mode) {
                if (mode == 0) cudaMemsetAsync(sim->dcount, 0, sizeof(int), sim->stream);
                if (sim->prec == MB_FP32)
                    launch_bulk<float>(dir, sim->eq, sim->dd, sim->dy, sim->rec, sim->n, sim->total_tiles[dir], src,
                                       dst, 0, cta, mode, dl, 0, sim->stream);
                else
                    launch_bulk<double>(dir, sim->eq, sim->dd, sim->dy, sim->rec, sim->n, sim->total_tiles[dir], src,
                                        dst, 0, cta, mode, dl, 0, sim->stream);
            }
        };
        go();
        cudaEventRecord(e0, sim->stream);
        for (int r = 0; r < 3; ++r) go();
        cudaEventRecord(e1, sim->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.0;
    };
    const bool packed = sim->prec == MB_FP32 && sim->eq == MB_EULER;
    // candidate shapes of the FP32x2 kernels: CTA size x register budget
    // (x: also the ring depth); the other kernels have one shape
    std::vector<int> xs, ys;
    if (packed) {
        for (int cta : {64, 128})
            for (int m4 = 0; m4 < 2; ++m4) {
                ys.push_back(cta | (m4 ? SHAPE_MINB4 : 0));
                for (int r8 = 0; r8 < 2; ++r8) xs.push_back(cta | (m4 ? SHAPE_MINB4 : 0) | (r8 ? SHAPE_RING8 : 0));
            }
    } else {
        xs.push_back(256);
        ys.push_back(256);
    }
    const int ysegs[3] = {32, 64, 128};
    double best_x = 1e30, best_y = 1e30;
    int bx = sim->tune_cta[0], by = sim->tune_cta[1], bs = sim->tune_yseg;
    for (int shape : xs) {
        double t = time_bulk(0, shape);
        if (t < best_x) { best_x = t; bx = shape; }
    }
    for (int ys_ = 0; ys_ < 3; ++ys_) {
        e = set_yseg(sim, ysegs[ys_]);
        if (e != cudaSuccess) break;
        for (int shape : ys) {
            double t = time_bulk(1, shape);
            if (t < best_y) { best_y = t; by = shape; bs = ysegs[ys_]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = set_yseg(sim, bs);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(sim, e, "autotune");
    sim->tune_cta[0] = bx;
    sim->tune_cta[1] = by;
    drop_graphs(sim);
    if (report) {
        report[0] = bx & 1023;
        report[1] = by & 1023;
        report[2] = bs;
        report[3] = best_x;
        report[4] = best_y;
        report[5] = (bx & SHAPE_MINB4) ? 4 : 5;
        report[6] = (by & SHAPE_MINB4) ? 4 : 5;
        report[7] = (bx & SHAPE_RING8) ? 8 : 4;
    }
    return MB_OK;
}

mb_status mb_fp64_rate(void *stream, double *fma_per_s) {
    if (!fma_per_s) return MB_E_INVAL;
    const double r = mb::fp64_probe_rate((cudaStream_t)stream);
    if (!(r > 0.0)) return MB_E_CUDA;
    *fma_per_s = r;
    return MB_OK;
}

mb_status mb_enable_timing(mb_sim *sim, int enable) {
    if (!sim) return MB_E_INVAL;
    cudaStreamSynchronize(sim->stream);
    for (auto &ev : sim->evs) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    sim->evs.clear();
    sim->timing = enable != 0;
    return MB_OK;
}

mb_status mb_graph_kernels(const mb_sim *sim, int *kernels_per_step) {
    if (!sim || !kernels_per_step) return MB_E_INVAL;
    *kernels_per_step = sim->graph_kernels;
    return MB_OK;
}

mb_status mb_set_sweep_event(mb_sim *sim, void *event) {
    if (!sim) return MB_E_INVAL;
    if (sim->sidx != 0) return fail(sim, MB_E_STATE, "mb_set_sweep_event in the middle of a step");
    sim->ev_mid = (cudaEvent_t)event;
    drop_graphs(sim);   // the cached graphs hold the old sequence
    return MB_OK;
}

mb_status mb_kernel_time(mb_sim *sim, double *total_ms, int *launches) {
    if (!sim) return MB_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return cuda_check(sim, e, "kernel_time sync");
    double tot = 0.0;
    for (auto &ev : sim->evs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int)sim->evs.size();
    return MB_OK;
}

}  // extern "C"
