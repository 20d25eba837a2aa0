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
            bool same = true;
            for (int q = 0; q < 4; ++q) same = same && qs[q] == qc[q];
            if (same) ps_sw = ps_step;   // first sweep of a step: one state
            else wall_state(g, qc, b.nx, b.ny, b.wx, b.wy, &rs2, &ps_sw, &u2x, &u2y);
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
// bulk sweep kernels: standard MUSCL-Hancock + HLLC update of every non-band
// cell.  Faces touching a band cell take the stabilised value its record
// holds (computed once by k_band_sweep), so every face flux is computed once.
// ---------------------------------------------------------------------------
constexpr int YSEG = 64;    // rows per thread in the y sweep

template <class T, int NC>
struct QV { T q[NC]; };

template <class T, int NC>
__device__ __forceinline__ void load_cell(const T *__restrict__ Q, size_t plane, int ci, bool flip, int in,
                                          QV<T, NC> &v) {
#pragma unroll
    for (int k = 0; k < NC; ++k) v.q[k] = __ldg(Q + k * plane + ci);
    if (NC == 4 && flip) v.q[in] = -v.q[in];
}

template <class T, int NC>
__device__ __forceinline__ void shfl_up(QV<T, NC> &o, const QV<T, NC> &v) {
#pragma unroll
    for (int k = 0; k < NC; ++k) o.q[k] = __shfl_up_sync(0xffffffffu, v.q[k], 1);
}
template <class T, int NC>
__device__ __forceinline__ void shfl_dn(QV<T, NC> &o, const QV<T, NC> &v) {
#pragma unroll
    for (int k = 0; k < NC; ++k) o.q[k] = __shfl_down_sync(0xffffffffu, v.q[k], 1);
}
template <class T, int NC>
__device__ __forceinline__ void shfl_idx(QV<T, NC> &o, const QV<T, NC> &v, int src) {
#pragma unroll
    for (int k = 0; k < NC; ++k) o.q[k] = __shfl_sync(0xffffffffu, v.q[k], src);
}

// face flux between cells (a-1, a) of a line: stabilised record value if a
// band cell is adjacent, zero next to a solid cell, HLLC otherwise
template <class T, int NC, int EQ, int DIR>
__device__ __forceinline__ void face_flux(const InstDesc &I, const BandRec *__restrict__ R, int line, int a, int n,
                                          uint8_t cl, uint8_t cr, T g, T av0, T av1, const QV<T, NC> &QRl,
                                          const QV<T, NC> &QLr, QV<T, NC> &F) {
    if ((cl | cr) & CLS_BAND) {
        bool fl;
        const int bclo = I.bc[2 * DIR], bchi = I.bc[2 * DIR + 1];
        const int pb = ghost_map(a, n, bclo, bchi, &fl), pa = ghost_map(a - 1, n, bclo, bchi, &fl);
        const int cib = DIR == 0 ? line * I.pitch + pb : pb * I.pitch + line;
        const int cia = DIR == 0 ? line * I.pitch + pa : pa * I.pitch + line;
        const bool b_real = a < n || bchi == 2;
        const bool a_real = a - 1 >= 0 || bclo == 2;
        if ((cr & CLS_BAND) && (b_real || !a_real || !(cl & CLS_BAND))) {
            const BandRec &rb = R[I.rec[cib]];
#pragma unroll
            for (int k = 0; k < NC; ++k) F.q[k] = (T)rb.Flo[k];
        } else {
            const BandRec &ra = R[I.rec[cia]];
#pragma unroll
            for (int k = 0; k < NC; ++k) F.q[k] = (T)ra.Fhi[k];
        }
        return;
    }
    if ((cl | cr) & CLS_SOLID) {
#pragma unroll
        for (int k = 0; k < NC; ++k) F.q[k] = T(0);
        return;
    }
    riemann_flux(EQ, g, DIR, av0, av1, QRl.q, QLr.q, F.q);
}

// new state of a non-band cell; wave speeds and positivity for the CFL step
template <class T, int NC, int EQ>
__device__ __forceinline__ void update_cell(T *__restrict__ Qo, size_t plane, int ci, uint8_t c0, T lam, T g, T av0,
                                            T av1, const QV<T, NC> &q, const QV<T, NC> &Flo, const QV<T, NC> &Fhi,
                                            bool last, T &s0, T &s1, int &bad) {
    if (c0 & CLS_BAND) return;
    if (c0 & CLS_SOLID) {
#pragma unroll
        for (int k = 0; k < NC; ++k) Qo[k * plane + ci] = T(NAN);
        return;
    }
    T qn[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        qn[k] = q.q[k] + lam * (Flo.q[k] - Fhi.q[k]);
        Qo[k * plane + ci] = qn[k];
    }
    if (EQ == 0) {
        T ir = fdiv(T(1), qn[0]);
        T p = (g - T(1)) * (qn[NC - 1] - T(0.5) * (qn[1 % NC] * qn[1 % NC] + qn[2 % NC] * qn[2 % NC]) * ir);
        if (!(qn[0] > T(0)) || !(p > T(0))) bad = 1;
        if (last) {
            T c = tsqrt(g * p * ir);
            s0 = fmax(s0, fabs(qn[1 % NC] * ir) + c);
            s1 = fmax(s1, fabs(qn[2 % NC] * ir) + c);
        }
    } else if (last) {
        s0 = fabs(av0);
        s1 = fabs(av1);
    }
}

template <class T>
__device__ __forceinline__ void finish_warp(InstDyn &y, bool last, T s0, T s1, int bad) {
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&y.err, ERR_UNSTABLE);
    if (last) {
        for (int o = 16; o > 0; o >>= 1) {
            s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
            s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_pos(&y.S[0], (double)s0);
            atomic_max_pos(&y.S[1], (double)s1);
        }
    }
}

__device__ __forceinline__ int find_inst_warp(const InstDesc *D, int n_inst, int gw, int dir) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (D[mid].tile_off[dir] <= gw) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// x sweep: one warp per row, lanes = 32 consecutive cells; the row is
// processed chunk by chunk, the update trailing the flux computation by one
// chunk so that the last lane finds its high face in the next chunk
template <class T, int EQ>
__global__ void __launch_bounds__(256) k_bulk_x(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                const BandRec *__restrict__ R, int n_inst, int total_warps, int src,
                                                int dst, int last) {
    constexpr int NC = EQ == 0 ? 4 : 1;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_warps) return;
    const int inst = find_inst_warp(D, n_inst, gw, 0);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    const int j = gw - I.tile_off[0];
    const int n = I.nx;
    const T lam = sizeof(T) == 4 ? (T)y.lamf : (T)y.lam;
    const T g = (T)I.gamma, av0 = (T)I.adv[0], av1 = (T)I.adv[1];
    const size_t plane = (size_t)I.pitch * I.ny;
    const T *__restrict__ Q = (const T *)I.Q[src];
    T *__restrict__ Qo = (T *)I.Q[dst];
    const int rowb = j * I.pitch;
    const int bclo = I.bc[0], bchi = I.bc[1];
    auto load = [&](int c, QV<T, NC> &v, uint8_t &cl) {
        const int a = 32 * c + lane;
        if (a < -2 || a > n + 1) {
#pragma unroll
            for (int k = 0; k < NC; ++k) v.q[k] = T(1);
            cl = CLS_SOLID;
            return;
        }
        bool fl;
        const int p = ghost_map(a, n, bclo, bchi, &fl);
        cl = I.cls[rowb + p];
        load_cell<T, NC>(Q, plane, rowb + p, fl, 1, v);
    };
    const int c_last = (n + 1) >> 5;
    QV<T, NC> Qm, Q0, Qp, QL, QR, F, Fprev, nb, nb2;
    uint8_t cm, c0, cp;
    load(-1, Qm, cm);
    load(0, Q0, c0);
    load(1, Qp, cp);
    // evolved right state of cell -1 (lane 31 of chunk -1)
    {
        shfl_up(nb, Qm);
        shfl_dn(nb2, Qm);
        QV<T, NC> t;
        shfl_idx(t, Q0, 0);
        if (lane == 31) nb2 = t;
        const int cmu = __shfl_up_sync(0xffffffffu, (int)cm, 1);
        int cmd = __shfl_down_sync(0xffffffffu, (int)cm, 1);
        const int c00 = __shfl_sync(0xffffffffu, (int)c0, 0);
        if (lane == 31) cmd = c00;
        const bool lim = !(cmu & CLS_SOLID) && !(cmd & CLS_SOLID);
        evolve(EQ, g, 0, lam, av0, av1, nb.q, Qm.q, nb2.q, lim, QL.q, QR.q);
    }
    QV<T, NC> QRc;
    shfl_idx(QRc, QR, 31);
    int cRc = __shfl_sync(0xffffffffu, (int)cm, 31);
    T s0 = T(0), s1 = T(0);
    int bad = 0;
    for (int c = 0; c <= c_last; ++c) {
        // neighbours of chunk c
        QV<T, NC> left, right, t;
        shfl_up(left, Q0);
        shfl_idx(t, Qm, 31);
        if (lane == 0) left = t;
        shfl_dn(right, Q0);
        shfl_idx(t, Qp, 0);
        if (lane == 31) right = t;
        int cl_ = __shfl_up_sync(0xffffffffu, (int)c0, 1);
        int cm31 = __shfl_sync(0xffffffffu, (int)cm, 31);
        if (lane == 0) cl_ = cm31;
        int cr_ = __shfl_down_sync(0xffffffffu, (int)c0, 1);
        int cp0 = __shfl_sync(0xffffffffu, (int)cp, 0);
        if (lane == 31) cr_ = cp0;
        const bool lim = !(cl_ & CLS_SOLID) && !(cr_ & CLS_SOLID);
        evolve(EQ, g, 0, lam, av0, av1, left.q, Q0.q, right.q, lim, QL.q, QR.q);
        // face between cells a-1 and a
        QV<T, NC> QRl;
        shfl_up(QRl, QR);
        if (lane == 0) QRl = QRc;
        const int a = 32 * c + lane;
        if (a >= 0 && a <= n) face_flux<T, NC, EQ, 0>(I, R, j, a, n, (uint8_t)cl_, c0, g, av0, av1, QRl, QL, F);
        // update chunk c-1
        if (c >= 1) {
            QV<T, NC> Fhi;
            shfl_dn(Fhi, Fprev);
            shfl_idx(t, F, 0);
            if (lane == 31) Fhi = t;
            const int ap = a - 32;
            if (ap >= 0 && ap < n)
                update_cell<T, NC, EQ>(Qo, plane, rowb + ap, cm, lam, g, av0, av1, Qm, Fprev, Fhi, last, s0, s1, bad);
        }
        shfl_idx(QRc, QR, 31);
        Fprev = F;
        Qm = Q0; cm = c0;
        Q0 = Qp; c0 = cp;
        load(c + 2, Qp, cp);
    }
    // the last chunk (its high faces were computed in the final iteration)
    {
        QV<T, NC> Fhi;
        shfl_dn(Fhi, Fprev);
        const int ap = 32 * c_last + lane;
        if (ap >= 0 && ap < n && lane < 31)
            update_cell<T, NC, EQ>(Qo, plane, rowb + ap, cm, lam, g, av0, av1, Qm, Fprev, Fhi, last, s0, s1, bad);
    }
    (void)cRc;
    finish_warp<T>(y, last != 0, s0, s1, bad);
}

// y sweep: one thread per column and segment of YSEG rows, marching upward
// with a register window; 32 consecutive columns per warp keep every load
// and store coalesced
template <class T, int EQ>
__global__ void __launch_bounds__(256, 3) k_bulk_y(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                const BandRec *__restrict__ R, int n_inst, int total_warps, int src,
                                                int dst, int last) {
    constexpr int NC = EQ == 0 ? 4 : 1;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_warps) return;
    const int inst = find_inst_warp(D, n_inst, gw, 1);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    const int local = gw - I.tile_off[1];
    const int ncg = I.tiles_x[1];
    const int cg = local % ncg, sg = local / ncg;
    const int i_raw = cg * 32 + lane;
    const bool active = i_raw < I.nx;
    const int i = active ? i_raw : I.nx - 1;
    const int n = I.ny;
    const int j0 = sg * YSEG, j1 = min(n, j0 + YSEG);
    const T lam = sizeof(T) == 4 ? (T)y.lamf : (T)y.lam;
    const T g = (T)I.gamma, av0 = (T)I.adv[0], av1 = (T)I.adv[1];
    const size_t plane = (size_t)I.pitch * I.ny;
    const T *__restrict__ Q = (const T *)I.Q[src];
    T *__restrict__ Qo = (T *)I.Q[dst];
    const int bclo = I.bc[2], bchi = I.bc[3];
    auto load = [&](int r, QV<T, NC> &v, uint8_t &cl) {
        bool fl;
        const int p = ghost_map(r, n, bclo, bchi, &fl);
        const int ci = p * I.pitch + i;
        cl = I.cls[ci];
        load_cell<T, NC>(Q, plane, ci, fl, 2, v);
    };
    QV<T, NC> qa, qm, qc, qp, qq, QL, QR, QRc, F, Fprev;
    uint8_t ca, cm, cc, cp, cq;
    load(j0 - 2, qa, ca);
    load(j0 - 1, qm, cm);
    load(j0, qc, cc);
    load(j0 + 1, qp, cp);
    load(j0 + 2, qq, cq);
    // evolved top state of row j0-1
    evolve(EQ, g, 1, lam, av0, av1, qa.q, qm.q, qc.q, !(ca & CLS_SOLID) && !(cc & CLS_SOLID), QL.q, QRc.q);
    T s0 = T(0), s1 = T(0);
    int bad = 0;
    for (int f = j0; f <= j1; ++f) {
        // window: qm = row f-1, qc = row f, qp = row f+1, qq = row f+2
        evolve(EQ, g, 1, lam, av0, av1, qm.q, qc.q, qp.q, !(cm & CLS_SOLID) && !(cp & CLS_SOLID), QL.q, QR.q);
        face_flux<T, NC, EQ, 1>(I, R, i, f, n, cm, cc, g, av0, av1, QRc, QL, F);
        if (f > j0 && active)
            update_cell<T, NC, EQ>(Qo, plane, (f - 1) * I.pitch + i, cm, lam, g, av0, av1, qm, Fprev, F, last, s0,
                                   s1, bad);
        QRc = QR;
        Fprev = F;
        qm = qc; cm = cc;
        qc = qp; cc = cp;
        qp = qq; cp = cq;
        if (f + 3 <= j1 + 1) load(f + 3, qq, cq);
    }
    finish_warp<T>(y, last != 0, s0, s1, bad);
}

template <class T, int EQ>
void bulk_attr_t(int dir) {
    if (dir == 0) cudaFuncSetAttribute(k_bulk_x<T, EQ>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    else cudaFuncSetAttribute(k_bulk_y<T, EQ>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
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

template <class T>
void launch_bulk(int dir, int eq, const InstDesc *D, InstDyn *Y, const BandRec *R, int n_inst, int total_warps,
                 int src, int dst, int last, cudaStream_t st) {
    int blocks = (total_warps + 7) / 8;
    if (blocks <= 0) return;
    if (dir == 0) {
        if (eq == 0) k_bulk_x<T, 0><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
        else k_bulk_x<T, 1><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
    } else {
        if (eq == 0) k_bulk_y<T, 0><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
        else k_bulk_y<T, 1><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
    }
}

template <class T>
int bulk_blocks_per_sm(int dir) {
    bulk_attr_t<T, 0>(dir);
    bulk_attr_t<T, 1>(dir);
    return 1;
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
    template void launch_bulk<T>(int, int, const InstDesc *, InstDyn *, const BandRec *, int, int, int, int, int,  \
                                 cudaStream_t);                                                                    \
    template int bulk_blocks_per_sm<T>(int);                                                                       \
    template void launch_write_state<T>(const InstDesc *, InstDyn *, const double *, int, int, cudaStream_t);      \
    template void launch_read_state<T>(const InstDesc *, double *, int, int, cudaStream_t);
MB_INST(float)
MB_INST(double)

}  // namespace mb
