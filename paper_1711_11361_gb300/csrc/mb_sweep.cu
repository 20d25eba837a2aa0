// mb_sweep.cu -- the directional sweep proper (arXiv 1711.11361):
//   k_band_prep   provisional states of flux-GCL uncovered cells, the
//                 moving-wall boundary state (eqs. riemann_wallvel,
//                 KleinAdvectivePressureSplitA, ModifiedBoundaryFluxMethod2)
//                 and the covering / uncovering weights (eqs. volumeWeighting,
//                 cutCellCoverDonation)
//   k_band_sweep  stabilised fluxes of every face touching a band cell
//                 (eqs. Klein2shieldedFluxMethod2, Klein2DtotalfluxaMethod2) and
//                 the band cells' new contents (eq. Klein2DcompleteMovingMethod2a)
//   k_bulk        MUSCL-Hancock + HLLC standard fluxes and the conservative
//                 update of every other cell (eq. EulerDiscreteRegular), SMEM
//                 tiles over a persistent grid, CFL wave-speed reduction fused
//   k_events      covering / uncovering redistribution, gathered per cell
//                 (eqs. massDeficitEquation .. cutCellInitialisationDonorCellUpdate)
//   k_mix         positivity safeguard (clusters share content by volume)
//   k_finalize    Q = content / alpha at the end pose, class byte update
#include "mb_internal.cuh"

namespace mb {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_inst_rec(const InstDesc *D, int n_inst, int r) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].rec_base <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class T>
__device__ __forceinline__ const T *buf(const InstDesc &I, int b) { return (const T *)I.Q[b]; }
template <class T>
__device__ __forceinline__ T *bufw(const InstDesc &I, int b) { return (T *)I.Q[b]; }

// cell at position k along line l, with boundary ghosts; returns the cell
// index, whether the position is a real (or periodically wrapped) cell, and
// whether the normal component flips
__device__ __forceinline__ int line_cell(const InstDesc &I, int dir, int l, int k, bool *real, bool *flip) {
    int n = dir == 0 ? I.nx : I.ny;
    int pos = ghost_map(k, n, I.bc[2 * dir], I.bc[2 * dir + 1], flip);
    *real = (k >= 0 && k < n) || I.bc[k < 0 ? 2 * dir : 2 * dir + 1] == 2;
    return cell_index(I, dir, l, pos);
}

template <class T>
struct CellW {
    T q[MAXC];
    bool fluid;
    int rec;       // band record (real cells only) or -1
};

template <class T>
__device__ __forceinline__ void fetch(const InstDesc &I, const BandRec *R, int dir, int src, int l, int k,
                                      CellW<T> &c) {
    bool real, flip;
    int ci = line_cell(I, dir, l, k, &real, &flip);
    uint8_t cl = I.cls[ci];
    int ri = (cl & CLS_BAND) ? I.rec[ci] : -1;
    c.rec = real ? ri : -1;
    const T *Q = buf<T>(I, src);
    size_t plane = (size_t)I.pitch * I.ny;
    if (ri >= 0) {
        const BandRec &r = R[ri];
        c.fluid = (r.flags & RF_FLUID_A) != 0;
        if (c.fluid && (r.flags & RF_UNCOV)) {
            for (int q = 0; q < I.nc; ++q) c.q[q] = (T)r.Qp[q];
        } else {
            for (int q = 0; q < I.nc; ++q) c.q[q] = Q[q * plane + ci];
        }
    } else {
        c.fluid = !(cl & CLS_SOLID);
        for (int q = 0; q < I.nc; ++q) c.q[q] = Q[q * plane + ci];
    }
    if (flip && I.nc == 4) c.q[1 + dir] = -c.q[1 + dir];
}

// time-averaged aperture of the face between along positions a and a+1
__device__ double face_beta(const InstDesc &I, const BandRec *R, const double *bnd, int dir, int l, int a,
                            bool own_hi) {
    int n = dir == 0 ? I.nx : I.ny;
    int o = own_hi ? a : a + 1;
    bool periodic = I.bc[2 * dir] == 2;
    if (periodic) {
        o %= n;
        if (o < 0) o += n;
    }
    if (o >= 0 && o < n) {
        int ci = cell_index(I, dir, l, o);
        uint8_t cl = I.cls[ci];
        if (cl & CLS_BAND) return R[I.rec[ci]].bown;
        return (cl & CLS_SOLID) ? 0.0 : 1.0;
    }
    // owner is a ghost beyond a non-periodic side: the real boundary cell
    // carries this face's value
    int rpos = o < 0 ? 0 : n - 1;
    int ci = cell_index(I, dir, l, rpos);
    uint8_t cl = I.cls[ci];
    if (cl & CLS_BAND) return bnd[I.rec[ci]];
    return (cl & CLS_SOLID) ? 0.0 : 1.0;
}

// ---------------------------------------------------------------------------
// k_band_prep
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_band_prep(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                            int n_inst, int total_rec, int dir, int src, int qn) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_rec) return;
    int inst = find_inst_rec(D, n_inst, r);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return;
    BandRec &b = R[r];
    const size_t plane = (size_t)I.pitch * I.ny;
    const T *QA = buf<T>(I, src), *QN = buf<T>(I, qn);
    const int i = b.i, j = b.j;
    auto nbr_cell = [&](int di, int dj, int *cell) -> bool {
        int ii = i + di, jj = j + dj;
        if (I.bc[0] == 2) { ii %= I.nx; if (ii < 0) ii += I.nx; }
        if (I.bc[2] == 2) { jj %= I.ny; if (jj < 0) jj += I.ny; }
        if (ii < 0 || ii >= I.nx || jj < 0 || jj >= I.ny) return false;
        *cell = jj * I.pitch + ii;
        return true;
    };
    // provisional state of a flux-GCL uncovered cell: volume-weighted average
    // of its fluid neighbours at the start pose (face neighbours first)
    if ((b.flags & RF_UNCOV) && (b.flags & RF_FLUID_A)) {
        double acc[MAXC] = {0, 0, 0, 0}, ws = 0.0;
        for (int pass = 0; pass < 2 && ws == 0.0; ++pass) {
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    if (di == 0 && dj == 0) continue;
                    if (pass == 0 && di != 0 && dj != 0) continue;
                    int c;
                    if (!nbr_cell(di, dj, &c)) continue;
                    uint8_t cl = I.cls[c];
                    double a = (cl & CLS_BAND) ? R[I.rec[c]].aA : ((cl & CLS_SOLID) ? 0.0 : 1.0);
                    if (!(a > 0.0)) continue;
                    ws += a;
                    for (int q = 0; q < I.nc; ++q) acc[q] += a * (double)QA[q * plane + c];
                }
        }
        if (ws == 0.0) {
            atomicOr(&y.err, ERR_NONBR);
            for (int q = 0; q < I.nc; ++q) b.Qp[q] = 0.0;
            b.flags &= ~RF_FLUID_A;
        } else {
            for (int q = 0; q < I.nc; ++q) b.Qp[q] = acc[q] / ws;
        }
    }
    // moving-wall boundary state: advective part from the step-start state,
    // pressure from the sweep-start state
    if (b.flags & RF_FLUID_A) {
        double qc[MAXC], qs[MAXC];
        bool unc = (b.flags & RF_UNCOV) != 0;
        for (int q = 0; q < I.nc; ++q) qc[q] = unc ? b.Qp[q] : (double)QA[q * plane + b.cell];
        double n0 = (double)QN[b.cell];
        bool fresh = n0 != n0;
        for (int q = 0; q < I.nc; ++q) qs[q] = fresh ? qc[q] : (double)QN[q * plane + b.cell];
        if (I.eq == 0) {
            double g = I.gamma;
            double rs, ps_step, usx, usy, rs2, ps_sw, u2x, u2y;
            wall_state(g, qs, b.nx, b.ny, b.wx, b.wy, &rs, &ps_step, &usx, &usy);
            wall_state(g, qc, b.nx, b.ny, b.wx, b.wy, &rs2, &ps_sw, &u2x, &u2y);
            double Eadv = ps_step / (g - 1.0) + 0.5 * rs * (usx * usx + usy * usy);
            double ud = dir == 0 ? usx : usy;
            b.QB[0] = rs; b.QB[1] = rs * usx; b.QB[2] = rs * usy; b.QB[3] = Eadv;
            b.FB[0] = rs * ud;
            b.FB[1] = rs * ud * usx + (dir == 0 ? ps_sw : 0.0);
            b.FB[2] = rs * ud * usy + (dir == 1 ? ps_sw : 0.0);
            b.FB[3] = ud * (Eadv + ps_step);
        } else {
            b.QB[0] = qs[0];
            b.FB[0] = I.adv[dir] * qs[0];
        }
        b.flags |= RF_WALL;
    }
    // covering / uncovering weights over fluid neighbours at the end pose
    const bool donor_unc = (b.flags & RF_UNCOV) && I.ucov == 0;
    if ((b.flags & RF_COVER) || donor_unc) {
        double den = 0.0;
        int found = 0, use8 = 0;
        for (int pass = 0; pass < 2 && found == 0; ++pass) {
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    if (di == 0 && dj == 0) continue;
                    if (pass == 0 && di != 0 && dj != 0) continue;
                    int c;
                    if (!nbr_cell(di, dj, &c)) continue;
                    if (!(I.cls[c] & CLS_BAND)) continue;
                    const BandRec &nb = R[I.rec[c]];
                    if (!(nb.aB > 0.0)) continue;
                    if (I.ucov == 0 && (nb.flags & RF_UNCOV)) continue;
                    den += nb.aB;
                    ++found;
                }
            if (found) use8 = pass;
        }
        if (!found) {
            b.flags |= RF_NONBR;
            atomicOr(&y.err, ERR_NONBR);
            b.den = 0.0;
        } else {
            if (use8) b.flags |= RF_USE8;
            b.den = (b.flags & RF_COVER) ? den : b.aB + den;
        }
    }
}

// ---------------------------------------------------------------------------
// stabilised flux of one face: aperture times F2D (eqs. Klein2shieldedFluxMethod2
// and Klein2DtotalfluxaMethod2 with the one- or two-sided shielded parts).
// Not inlined, so that a face shared by two band cells gets identical bits.
// ---------------------------------------------------------------------------
struct FaceIn {
    double btL, btF, btR;      // apertures of faces (a-1,a), (a,a+1), (a+1,a+2)
    bool hasL, hasR;           // wall data of cells a and a+1
    double dL, dR;
    double FBL[MAXC], FBR[MAXC];
};

template <class T>
__device__ __noinline__ void face_stab(int eq, T g, int dir, T lamT, T av0, T av1, int nc, const CellW<T> *w,
                                       const FaceIn *in, double *out) {
    for (int q = 0; q < MAXC; ++q) out[q] = 0.0;
    if (!(w[1].fluid && w[2].fluid && in->btF > 0.0)) return;
    T QLa[MAXC], QRa[MAXC], QLb[MAXC], QRb[MAXC], F[MAXC];
    evolve(eq, g, dir, lamT, av0, av1, w[0].q, w[1].q, w[2].q, w[0].fluid && w[2].fluid, QLa, QRa);
    evolve(eq, g, dir, lamT, av0, av1, w[1].q, w[2].q, w[3].q, w[1].fluid && w[3].fluid, QLb, QRb);
    riemann_flux(eq, g, dir, av0, av1, QRa, QLb, F);
    double bf = in->btF;
    double sR = in->hasR ? fmax(0.0, bf - in->btR) : 0.0;
    double sL = in->hasL ? fmax(0.0, bf - in->btL) : 0.0;
    if (sR + sL > bf) {
        double sc = bf / (sR + sL);
        sR *= sc;
        sL *= sc;
    }
    for (int q = 0; q < nc; ++q) {
        double Fq = (double)F[q];
        double v = (bf - sL - sR) * Fq;
        if (sR > 0.0) v += sR * (in->FBR[q] + in->dR * (Fq - in->FBR[q]));
        if (sL > 0.0) v += sL * (in->FBL[q] + in->dL * (Fq - in->FBL[q]));
        out[q] = v;
    }
}

// ---------------------------------------------------------------------------
// k_band_sweep: both sweep-direction faces of each band cell and its content
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_band_sweep(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                             const double *__restrict__ bnd, int n_inst, int total_rec, int dir, int src) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_rec) return;
    int inst = find_inst_rec(D, n_inst, r);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return;
    BandRec &b = R[r];
    const int l = dir == 0 ? b.j : b.i, k = dir == 0 ? b.i : b.j;
    const double lam = y.lam;
    const T g = (T)I.gamma, lamT = (T)lam, av0 = (T)I.adv[0], av1 = (T)I.adv[1];
    const bool own_hi = I.rotating || y.delta >= 0.0;
    CellW<T> w[5];
    for (int m = 0; m < 5; ++m) fetch<T>(I, R, dir, src, l, k - 2 + m, w[m]);
    double bt[4];
    for (int m = 0; m < 4; ++m) bt[m] = face_beta(I, R, bnd, dir, l, k - 2 + m, own_hi);
    auto wall_of = [&](const CellW<T> &c, bool *has, double *d, double *FB) {
        *has = false;
        if (c.rec >= 0 && (R[c.rec].flags & RF_WALL)) {
            const BandRec &o = R[c.rec];
            *has = true;
            *d = o.d;
            for (int q = 0; q < MAXC; ++q) FB[q] = o.FB[q];
        }
    };
    FaceIn fi;
    fi.dL = fi.dR = 0.0;
    // low face: cells k-1 | k
    fi.btL = bt[0]; fi.btF = bt[1]; fi.btR = bt[2];
    wall_of(w[1], &fi.hasL, &fi.dL, fi.FBL);
    wall_of(w[2], &fi.hasR, &fi.dR, fi.FBR);
    double Flo[MAXC], Fhi[MAXC];
    face_stab<T>(I.eq, g, dir, lamT, av0, av1, I.nc, &w[0], &fi, Flo);
    // high face: cells k | k+1
    fi.btL = bt[1]; fi.btF = bt[2]; fi.btR = bt[3];
    wall_of(w[2], &fi.hasL, &fi.dL, fi.FBL);
    wall_of(w[3], &fi.hasR, &fi.dR, fi.FBR);
    face_stab<T>(I.eq, g, dir, lamT, av0, av1, I.nc, &w[1], &fi, Fhi);
    for (int q = 0; q < MAXC; ++q) { b.Flo[q] = Flo[q]; b.Fhi[q] = Fhi[q]; }
    // content alpha_B Q' of this cell
    double C[MAXC] = {0, 0, 0, 0};
    if (b.flags & RF_FLUID_A) {
        const double blo = bt[1], bhi = bt[2];
        const double wd = dir == 0 ? b.wx : b.wy;
        for (int q = 0; q < I.nc; ++q) {
            double v = b.aA * (double)w[2].q[q] + lam * (Flo[q] - Fhi[q]);
            if (blo != bhi && (b.flags & RF_WALL)) {
                double wt = lam * (bhi - blo) * (b.FB[q] - wd * b.QB[q]);
                v += wt;
                atomicAdd(&y.wall_sum[q], wt);
            }
            C[q] = v;
        }
    }
    for (int q = 0; q < MAXC; ++q) b.C[q] = C[q];
}

// ---------------------------------------------------------------------------
// k_bulk: standard update of every non-band cell (SMEM tiles, persistent)
// ---------------------------------------------------------------------------
template <int DIR> struct Tile;
template <> struct Tile<0> { static constexpr int W = 128, NL = 2; };
template <> struct Tile<1> { static constexpr int W = 16, NL = 32; };

template <class T, int DIR>
constexpr size_t bulk_smem() {
    constexpr int W = Tile<DIR>::W, NL = Tile<DIR>::NL;
    return sizeof(T) * MAXC * ((W + 4) * NL + 2 * (W + 2) * NL + (W + 1) * NL) + (W + 4) * NL + 64;
}

template <class T, int DIR>
__global__ void __launch_bounds__(256) k_bulk(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                              const BandRec *__restrict__ R, int n_inst, int total_tiles, int src,
                                              int dst, int last) {
    constexpr int W = Tile<DIR>::W, NL = Tile<DIR>::NL, WH = W + 4;
    extern __shared__ __align__(16) unsigned char smem[];
    T *sq = (T *)smem;                       // [MAXC][WH*NL]
    T *sl = sq + MAXC * WH * NL;             // [MAXC][(W+2)*NL]
    T *sr = sl + MAXC * (W + 2) * NL;        // [MAXC][(W+2)*NL]
    T *sf = sr + MAXC * (W + 2) * NL;        // [MAXC][(W+1)*NL]
    uint8_t *sc = (uint8_t *)(sf + MAXC * (W + 1) * NL);
    __shared__ double red[2][8];
    const int tid = threadIdx.x;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        int lo = 0, hi = n_inst - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (D[mid].tile_off[DIR] <= tile) lo = mid; else hi = mid - 1;
        }
        const InstDesc &I = D[lo];
        const int lt = tile - I.tile_off[DIR];
        const int tx = lt % I.tiles_x[DIR], ty = lt / I.tiles_x[DIR];
        const int nal = DIR == 0 ? I.nx : I.ny, nln = DIR == 0 ? I.ny : I.nx;
        const int a0 = DIR == 0 ? tx * W : ty * W;
        const int l0 = DIR == 0 ? ty * NL : tx * NL;
        const T lam = sizeof(T) == 4 ? (T)Y[lo].lamf : (T)Y[lo].lam;
        const T g = (T)I.gamma, av0 = (T)I.adv[0], av1 = (T)I.adv[1];
        const int nc = I.nc, eq = I.eq;
        const size_t plane = (size_t)I.pitch * I.ny;
        const T *Q = buf<T>(I, src);
        T *Qo = bufw<T>(I, dst);
        auto sidx = [&](int l, int kk) { return DIR == 0 ? l * WH + kk : kk * NL + l; };
        // phase 1: load states and classes (ghosts by boundary condition)
        for (int e = tid; e < WH * NL; e += 256) {
            int l = DIR == 0 ? e / WH : e % NL;
            int kk = DIR == 0 ? e % WH : e / NL;
            int line = l0 + l;
            int s = sidx(l, kk);
            if (line >= nln) { sc[s] = CLS_SOLID; continue; }
            bool flip;
            int pos = ghost_map(a0 + kk - 2, nal, I.bc[2 * DIR], I.bc[2 * DIR + 1], &flip);
            int ci = DIR == 0 ? line * I.pitch + pos : pos * I.pitch + line;
            sc[s] = I.cls[ci];
            for (int q = 0; q < nc; ++q) {
                T v = Q[q * plane + ci];
                if (flip && q == 1 + DIR) v = -v;
                sq[q * WH * NL + s] = v;
            }
        }
        __syncthreads();
        // phase 2: evolved boundary states of cells -1..W
        for (int e = tid; e < (W + 2) * NL; e += 256) {
            int l = DIR == 0 ? e / (W + 2) : e % NL;
            int m = DIR == 0 ? e % (W + 2) : e / NL;
            int kk = m + 1;
            int s0 = sidx(l, kk);
            int so = DIR == 0 ? l * (W + 2) + m : m * NL + l;
            if (sc[s0] & CLS_SOLID) continue;
            T qm[MAXC], q0[MAXC], qp[MAXC], QL[MAXC], QR[MAXC];
            int sm = sidx(l, kk - 1), sp = sidx(l, kk + 1);
            for (int q = 0; q < nc; ++q) {
                qm[q] = sq[q * WH * NL + sm];
                q0[q] = sq[q * WH * NL + s0];
                qp[q] = sq[q * WH * NL + sp];
            }
            bool lim = !(sc[sm] & CLS_SOLID) && !(sc[sp] & CLS_SOLID);
            evolve(eq, g, DIR, lam, av0, av1, qm, q0, qp, lim, QL, QR);
            for (int q = 0; q < nc; ++q) {
                sl[q * (W + 2) * NL + so] = QL[q];
                sr[q * (W + 2) * NL + so] = QR[q];
            }
        }
        __syncthreads();
        // phase 3: face fluxes 0..W (face m between cells m-1 and m);
        // faces touching a band cell take the stabilised value of its record
        for (int e = tid; e < (W + 1) * NL; e += 256) {
            int l = DIR == 0 ? e / (W + 1) : e % NL;
            int m = DIR == 0 ? e % (W + 1) : e / NL;
            int sa = sidx(l, m + 1), sb = sidx(l, m + 2);
            int so = DIR == 0 ? l * (W + 1) + m : m * NL + l;
            uint8_t ca = sc[sa], cb = sc[sb];
            T F[MAXC] = {T(0), T(0), T(0), T(0)};
            if ((ca | cb) & CLS_BAND) {
                int line = l0 + l;
                if (line < nln) {
                    bool fl;
                    int pb = ghost_map(a0 + m, nal, I.bc[2 * DIR], I.bc[2 * DIR + 1], &fl);
                    int pa = ghost_map(a0 + m - 1, nal, I.bc[2 * DIR], I.bc[2 * DIR + 1], &fl);
                    int cib = DIR == 0 ? line * I.pitch + pb : pb * I.pitch + line;
                    int cia = DIR == 0 ? line * I.pitch + pa : pa * I.pitch + line;
                    // a ghost beyond a non-periodic side mirrors a real cell:
                    // take the record of the real cell on the other side
                    const bool b_real = (a0 + m < nal) || I.bc[2 * DIR + 1] == 2;
                    const bool a_real = (a0 + m - 1 >= 0) || I.bc[2 * DIR] == 2;
                    if ((cb & CLS_BAND) && (b_real || !a_real || !(ca & CLS_BAND))) {
                        const BandRec &rb = R[I.rec[cib]];
                        for (int q = 0; q < nc; ++q) F[q] = (T)rb.Flo[q];
                    } else {
                        const BandRec &ra = R[I.rec[cia]];
                        for (int q = 0; q < nc; ++q) F[q] = (T)ra.Fhi[q];
                    }
                }
            } else if (!((ca | cb) & CLS_SOLID)) {
                int ia = DIR == 0 ? l * (W + 2) + m : m * NL + l;
                int ib = DIR == 0 ? l * (W + 2) + m + 1 : (m + 1) * NL + l;
                T QRa[MAXC], QLb[MAXC];
                for (int q = 0; q < nc; ++q) {
                    QRa[q] = sr[q * (W + 2) * NL + ia];
                    QLb[q] = sl[q * (W + 2) * NL + ib];
                }
                riemann_flux(eq, g, DIR, av0, av1, QRa, QLb, F);
            }
            for (int q = 0; q < nc; ++q) sf[q * (W + 1) * NL + so] = F[q];
        }
        __syncthreads();
        // phase 4: update cells 0..W-1 of the tile
        T smax0 = T(0), smax1 = T(0);
        int bad = 0;
        for (int e = tid; e < W * NL; e += 256) {
            int l = DIR == 0 ? e / W : e % NL;
            int m = DIR == 0 ? e % W : e / NL;
            int a = a0 + m, line = l0 + l;
            if (a >= nal || line >= nln) continue;
            int s0 = sidx(l, m + 2);
            uint8_t c0 = sc[s0];
            if (c0 & CLS_BAND) continue;
            int ci = DIR == 0 ? line * I.pitch + a : a * I.pitch + line;
            if (c0 & CLS_SOLID) {
                for (int q = 0; q < nc; ++q) Qo[q * plane + ci] = T(NAN);
                continue;
            }
            int flo = DIR == 0 ? l * (W + 1) + m : m * NL + l;
            int fhi = DIR == 0 ? l * (W + 1) + m + 1 : (m + 1) * NL + l;
            T qn[MAXC];
            for (int q = 0; q < nc; ++q) {
                qn[q] = sq[q * WH * NL + s0] + lam * (sf[q * (W + 1) * NL + flo] - sf[q * (W + 1) * NL + fhi]);
                Qo[q * plane + ci] = qn[q];
            }
            if (eq == 0) {
                T ir = fdiv(T(1), qn[0]);
                T p = (g - T(1)) * (qn[3] - T(0.5) * (qn[1] * qn[1] + qn[2] * qn[2]) * ir);
                if (!(qn[0] > T(0)) || !(p > T(0))) bad = 1;
                if (last) {
                    T c = tsqrt(g * p * ir);
                    smax0 = fmax(smax0, fabs(qn[1] * ir) + c);
                    smax1 = fmax(smax1, fabs(qn[2] * ir) + c);
                }
            } else if (last) {
                smax0 = fabs(av0);
                smax1 = fabs(av1);
            }
        }
        if (bad) atomicOr(&Y[lo].err, ERR_UNSTABLE);
        if (last) {
            for (int o = 16; o > 0; o >>= 1) {
                smax0 = fmax(smax0, __shfl_xor_sync(0xffffffffu, smax0, o));
                smax1 = fmax(smax1, __shfl_xor_sync(0xffffffffu, smax1, o));
            }
            if ((tid & 31) == 0) { red[0][tid >> 5] = (double)smax0; red[1][tid >> 5] = (double)smax1; }
            __syncthreads();
            if (tid == 0) {
                double m0 = red[0][0], m1 = red[1][0];
                for (int k = 1; k < 8; ++k) { m0 = fmax(m0, red[0][k]); m1 = fmax(m1, red[1][k]); }
                atomic_max_pos(&Y[lo].S[0], m0);
                atomic_max_pos(&Y[lo].S[1], m1);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_events: covering / uncovering, gathered by each band cell
// ---------------------------------------------------------------------------
__global__ void k_events(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                         int n_inst, int total_rec) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_rec) return;
    int inst = find_inst_rec(D, n_inst, r);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return;
    BandRec &x = R[r];
    const int nc = I.nc;
    const bool x_donor_unc = (x.flags & RF_UNCOV) && I.ucov == 0;
    const bool x_recv = x.aB > 0.0 && !x_donor_unc;   // may receive / donate
    double C[MAXC];
    for (int q = 0; q < MAXC; ++q) C[q] = x.C[q];
    double unc_sum[MAXC] = {0, 0, 0, 0};
    for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
            if (di == 0 && dj == 0) continue;
            int ii = x.i + di, jj = x.j + dj;
            if (I.bc[0] == 2) { ii %= I.nx; if (ii < 0) ii += I.nx; }
            if (I.bc[2] == 2) { jj %= I.ny; if (jj < 0) jj += I.ny; }
            if (ii < 0 || ii >= I.nx || jj < 0 || jj >= I.ny) continue;
            int c = jj * I.pitch + ii;
            if (!(I.cls[c] & CLS_BAND)) continue;
            const BandRec &n = R[I.rec[c]];
            const bool face = di == 0 || dj == 0;
            const bool n_adj = face || (n.flags & RF_USE8);
            const bool n_donor_unc = (n.flags & RF_UNCOV) && I.ucov == 0;
            // x as recipient of a covered neighbour's residual
            if ((n.flags & RF_COVER) && !(n.flags & RF_NONBR) && x_recv && n_adj) {
                double wgt = x.aB / n.den;
                for (int q = 0; q < nc; ++q) C[q] += wgt * n.C[q];
            }
            // x as donor of an uncovered neighbour
            if (n_donor_unc && !(n.flags & RF_NONBR) && x_recv && n_adj) {
                double sig = n.aB / n.den;
                for (int q = 0; q < nc; ++q) C[q] -= sig * x.C[q];
            }
            // x uncovered: collect its donors' contents
            if (x_donor_unc && !(x.flags & RF_NONBR) && n.aB > 0.0 && !n_donor_unc &&
                (face || (x.flags & RF_USE8)))
                for (int q = 0; q < nc; ++q) unc_sum[q] += n.C[q];
        }
    if (x_donor_unc) {
        double sig = (x.flags & RF_NONBR) ? 0.0 : x.aB / x.den;
        for (int q = 0; q < MAXC; ++q) C[q] = sig * unc_sum[q];
    }
    if (x.flags & RF_COVER) for (int q = 0; q < MAXC; ++q) C[q] = 0.0;
    for (int q = 0; q < MAXC; ++q) x.C2[q] = C[q];
    // positivity check of the new state
    if (I.eq == 0 && x.aB > 0.0) {
        double q0 = C[0] / x.aB, q1 = C[1] / x.aB, q2 = C[2] / x.aB, q3 = C[3] / x.aB;
        double p = (I.gamma - 1.0) * (q3 - 0.5 * (q1 * q1 + q2 * q2) / q0);
        bool ok = q0 > 0.0 && p > 0.0 && isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(q3);
        if (!ok) {
            x.flags |= RF_BAD;
            int k = atomicAdd(&y.nbad, 1);
            if (k < 16) y.badlist[k] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// k_mix: positivity safeguard (a reading; the paper gives none): every cluster
// of non-physical cells and their fluid face neighbours shares its total
// content in proportion to volume.  One thread per instance; runs only when
// the instance flagged a bad cell.  Also advances the instance's clock.
// ---------------------------------------------------------------------------
constexpr int MIXCAP = 1024;

template <class T>
__global__ void k_mix(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                      int *__restrict__ scratch, int n_inst, int dst, int sidx) {
    int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= n_inst) return;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    // advance pose and clock
    y.X = y.XB;
    y.Y = y.YB;
    y.th = y.thB;
    if (sidx == 1) {
        y.t += y.dt;
        y.step += 1;
    }
    if (y.nbad == 0) return;
    int *node = scratch + (size_t)inst * 2 * MIXCAP;     // cell index of node
    int *par = node + MIXCAP;
    int nn = 0;
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Qo = bufw<T>(I, dst);
    auto find_node = [&](int cell) -> int {
        for (int k = 0; k < nn; ++k)
            if (node[k] == cell) return k;
        if (nn >= MIXCAP) return -1;
        node[nn] = cell;
        par[nn] = nn;
        return nn++;
    };
    auto root = [&](int k) { while (par[k] != k) k = par[k]; return k; };
    bool overflow = false;
    const bool listed = y.nbad <= 16;
    const int nscan = listed ? y.nbad : y.band_count;
    for (int s = 0; s < nscan; ++s) {
        const int r = listed ? y.badlist[s] : I.rec_base + s;
        const BandRec &b = R[r];
        if (!(b.flags & RF_BAD)) continue;
        int kb = find_node(b.cell);
        if (kb < 0) { overflow = true; break; }
        const int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        for (int m = 0; m < 4; ++m) {
            int ii = b.i + dd[m][0], jj = b.j + dd[m][1];
            if (I.bc[0] == 2) { ii %= I.nx; if (ii < 0) ii += I.nx; }
            if (I.bc[2] == 2) { jj %= I.ny; if (jj < 0) jj += I.ny; }
            if (ii < 0 || ii >= I.nx || jj < 0 || jj >= I.ny) continue;
            int c = jj * I.pitch + ii;
            uint8_t cl = I.cls[c];
            double aB = (cl & CLS_BAND) ? R[I.rec[c]].aB : ((cl & CLS_SOLID) ? 0.0 : 1.0);
            if (!(aB > 0.0)) continue;
            int kn = find_node(c);
            if (kn < 0) { overflow = true; break; }
            int ra = root(kb), rb = root(kn);
            if (ra != rb) { if (ra < rb) par[rb] = ra; else par[ra] = rb; }
        }
        if (overflow) break;
    }
    if (overflow) { y.err |= ERR_UNSTABLE; return; }
    // cluster sums
    for (int k = 0; k < nn; ++k) {
        int rk = root(k);
        if (rk != k) continue;
        double tot[MAXC] = {0, 0, 0, 0}, vol = 0.0;
        for (int m = 0; m < nn; ++m) {
            if (root(m) != k) continue;
            int c = node[m];
            uint8_t cl = I.cls[c];
            if (cl & CLS_BAND) {
                const BandRec &b = R[I.rec[c]];
                vol += b.aB;
                for (int q = 0; q < I.nc; ++q) tot[q] += b.C2[q];
            } else {
                vol += 1.0;
                for (int q = 0; q < I.nc; ++q) tot[q] += (double)Qo[q * plane + c];
            }
        }
        for (int m = 0; m < nn; ++m) {
            if (root(m) != k) continue;
            int c = node[m];
            uint8_t cl = I.cls[c];
            if (cl & CLS_BAND) {
                BandRec &b = R[I.rec[c]];
                for (int q = 0; q < I.nc; ++q) b.C2[q] = b.aB * (tot[q] / vol);
            } else {
                for (int q = 0; q < I.nc; ++q) Qo[q * plane + c] = (T)(tot[q] / vol);
            }
        }
    }
    y.mixed += nn;
}

// ---------------------------------------------------------------------------
// k_finalize: new state of band cells, class bytes of the end pose
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_finalize(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                           int n_inst, int total_rec, int dst, int last) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total_rec) return;
    int inst = find_inst_rec(D, n_inst, r);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return;
    BandRec &b = R[r];
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Qo = bufw<T>(I, dst);
    if (b.aB > 0.0) {
        double q[MAXC];
        for (int k = 0; k < I.nc; ++k) {
            q[k] = b.C2[k] / b.aB;
            Qo[k * plane + b.cell] = (T)q[k];
        }
        if (I.eq == 0) {
            double p = (I.gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
            bool ok = q[0] > 0.0 && p > 0.0 && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
            if (!ok) atomicOr(&y.err, ERR_UNSTABLE);
            if (last) {
                double c = sqrt(I.gamma * p / q[0]);
                atomic_max_pos(&y.S[0], fabs(q[1] / q[0]) + c);
                atomic_max_pos(&y.S[1], fabs(q[2] / q[0]) + c);
            }
        } else if (last) {
            atomic_max_pos(&y.S[0], fabs(I.adv[0]));
            atomic_max_pos(&y.S[1], fabs(I.adv[1]));
        }
    } else {
        for (int k = 0; k < I.nc; ++k) Qo[k * plane + b.cell] = T(NAN);
    }
    const bool tB = (b.flags & RF_TOUCH_B) != 0;
    I.cls[b.cell] = (uint8_t)((b.aB == 0.0 ? CLS_SOLID : 0) | (tB && b.aB > 0.0 ? CLS_CUT : 0) | (tB ? CLS_TOUCH : 0) |
                              ((b.flags & RF_MOV_B) ? CLS_MOVT : 0));
    I.alpha[b.cell] = b.aB;
    I.rec[b.cell] = -1;
}

// ---------------------------------------------------------------------------
// state initialisation and the CFL wave speeds of a state
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_write_state(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, const double *__restrict__ Qh,
                              int inst, int b) {
    const InstDesc &I = D[inst];
    size_t n = (size_t)I.nx * I.ny;
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Q = bufw<T>(I, b);
    double s0 = 0.0, s1 = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % I.nx), j = (int)(e / I.nx);
        int c = j * I.pitch + i;
        bool solid = I.cls[c] & CLS_SOLID;
        double q[MAXC];
        for (int k = 0; k < I.nc; ++k) {
            q[k] = (double)(T)Qh[k * n + e];
            Q[k * plane + c] = solid ? T(NAN) : (T)Qh[k * n + e];
        }
        if (solid) continue;
        if (I.eq == 0) {
            double p = (I.gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
            double c2 = sqrt(I.gamma * p / q[0]);
            s0 = fmax(s0, fabs(q[1] / q[0]) + c2);
            s1 = fmax(s1, fabs(q[2] / q[0]) + c2);
        } else {
            s0 = fabs(I.adv[0]);
            s1 = fabs(I.adv[1]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
        s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&Y[inst].S[0], s0);
        atomic_max_pos(&Y[inst].S[1], s1);
    }
}

template <class T>
__global__ void k_read_state(const InstDesc *__restrict__ D, double *__restrict__ out, int inst, int b) {
    const InstDesc &I = D[inst];
    size_t n = (size_t)I.nx * I.ny;
    const size_t plane = (size_t)I.pitch * I.ny;
    const T *Q = buf<T>(I, b);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(e % I.nx), j = (int)(e / I.nx);
        for (int k = 0; k < I.nc; ++k) out[k * n + e] = (double)Q[k * plane + (size_t)j * I.pitch + i];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class T>
void launch_band_stage(int stage, const InstDesc *D, InstDyn *Y, BandRec *R, const double *bnd, int *scratch,
                       int n_inst, int total_rec, int dir, int src, int dst, int qn, int sidx, int last,
                       cudaStream_t st) {
    int blocks = (total_rec + 127) / 128;
    switch (stage) {
        case 0: if (blocks) k_band_prep<T><<<blocks, 128, 0, st>>>(D, Y, R, n_inst, total_rec, dir, src, qn); break;
        case 1: if (blocks) k_band_sweep<T><<<blocks, 128, 0, st>>>(D, Y, R, bnd, n_inst, total_rec, dir, src); break;
        case 2: if (blocks) k_events<<<blocks, 128, 0, st>>>(D, Y, R, n_inst, total_rec); break;
        case 3: k_mix<T><<<(n_inst + 63) / 64, 64, 0, st>>>(D, Y, R, scratch, n_inst, dst, sidx); break;
        case 4: if (blocks) k_finalize<T><<<blocks, 128, 0, st>>>(D, Y, R, n_inst, total_rec, dst, last); break;
    }
}

template <class T, int DIR>
void launch_bulk_t(const InstDesc *D, InstDyn *Y, const BandRec *R, int n_inst, int total_tiles, int src, int dst,
                   int last, int grid, cudaStream_t st) {
    constexpr size_t sm = bulk_smem<T, DIR>();   // opt-in size set once by bulk_blocks_per_sm
    int g = grid < total_tiles ? grid : total_tiles;
    if (g > 0) k_bulk<T, DIR><<<g, 256, sm, st>>>(D, Y, R, n_inst, total_tiles, src, dst, last);
}

template <class T>
void launch_bulk(int dir, const InstDesc *D, InstDyn *Y, const BandRec *R, int n_inst, int total_tiles, int src,
                 int dst, int last, int grid, cudaStream_t st) {
    if (dir == 0) launch_bulk_t<T, 0>(D, Y, R, n_inst, total_tiles, src, dst, last, grid, st);
    else launch_bulk_t<T, 1>(D, Y, R, n_inst, total_tiles, src, dst, last, grid, st);
}

template <class T>
int bulk_blocks_per_sm(int dir) {
    int nb = 0;
    if (dir == 0) {
        constexpr size_t sm = bulk_smem<T, 0>();
        cudaFuncSetAttribute(k_bulk<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bulk<T, 0>, 256, sm);
    } else {
        constexpr size_t sm = bulk_smem<T, 1>();
        cudaFuncSetAttribute(k_bulk<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bulk<T, 1>, 256, sm);
    }
    return nb > 0 ? nb : 1;
}

template <class T>
void launch_write_state(const InstDesc *D, InstDyn *Y, const double *Qh, int inst, int b, cudaStream_t st) {
    k_write_state<T><<<512, 256, 0, st>>>(D, Y, Qh, inst, b);
}
template <class T>
void launch_read_state(const InstDesc *D, double *out, int inst, int b, cudaStream_t st) {
    k_read_state<T><<<512, 256, 0, st>>>(D, out, inst, b);
}

#define MB_INST(T)                                                                                                \
    template void launch_band_stage<T>(int, const InstDesc *, InstDyn *, BandRec *, const double *, int *, int, int, \
                                       int, int, int, int, int, int, cudaStream_t);                                \
    template void launch_bulk<T>(int, const InstDesc *, InstDyn *, const BandRec *, int, int, int, int, int, int,  \
                                 cudaStream_t);                                                                    \
    template int bulk_blocks_per_sm<T>(int);                                                                       \
    template void launch_write_state<T>(const InstDesc *, InstDyn *, const double *, int, int, cudaStream_t);      \
    template void launch_read_state<T>(const InstDesc *, double *, int, int, cudaStream_t);
MB_INST(float)
MB_INST(double)

}  // namespace mb
