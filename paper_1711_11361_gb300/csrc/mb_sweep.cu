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

// The band kernels run over the used band records only: boff[k] counts the
// used records of instances 0..k-1 (boff[n_inst]: all of them), and thread t
// of a launch takes the t-th, instance by instance.  -1 past the last.
__device__ __forceinline__ int band_rec_of(const InstDesc *D, const int *__restrict__ boff, int n_inst, int t) {
    if (t >= boff[n_inst]) return -1;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boff[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return D[lo].rec_base + (t - boff[lo]);
}

// one CTA of 256 threads after the geometry: boff from each instance's
// record count (capped at its capacity; an overflow is flagged elsewhere)
__global__ void __launch_bounds__(256) k_band_offsets(const InstDesc *__restrict__ D, const InstDyn *__restrict__ Y,
                                                      int n_inst, int *__restrict__ boff) {
    __shared__ int wsum[8];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n_inst; k0 += 256) {
        const int k = k0 + threadIdx.x;
        const int c = k < n_inst ? min(Y[k].band_count, D[k].rec_cap) : 0;
        int v = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = lane < 8 ? wsum[lane] : 0;
            for (int o = 1; o < 8; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < 8) wsum[lane] = w;
        }
        __syncthreads();
        if (k < n_inst) boff[k] = carry + (warp ? wsum[warp - 1] : 0) + v - c;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[7];
        __syncthreads();
    }
    if (threadIdx.x == 0) boff[n_inst] = carry;
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

// Per-instance accumulations of the band kernels (wall terms, wave speeds):
// the records a warp holds usually belong to one instance (records are
// grouped by instance), so the warp combines its threads' values and issues
// one atomic; otherwise every thread issues its own.  All 32 lanes call.
__device__ __forceinline__ bool warp_one_inst(bool act, int inst, int &i0) {
    const unsigned m = __ballot_sync(0xffffffffu, act);
    i0 = m ? __shfl_sync(0xffffffffu, inst, __ffs(m) - 1) : -1;
    return __all_sync(0xffffffffu, !act || inst == i0);
}

__device__ __forceinline__ void warp_add_to(InstDyn *Y, bool act, int inst, const double *v) {
    int i0;
    if (warp_one_inst(act, inst, i0)) {
        if (i0 < 0) return;
        for (int q = 0; q < MAXC; ++q) {
            double s = act ? v[q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&Y[i0].wall_sum[q], s);
        }
    } else if (act) {
        for (int q = 0; q < MAXC; ++q)
            if (v[q] != 0.0) atomicAdd(&Y[inst].wall_sum[q], v[q]);
    }
}

__device__ __forceinline__ void warp_max_to(InstDyn *Y, bool act, int inst, double s0, double s1) {
    int i0;
    if (warp_one_inst(act, inst, i0)) {
        if (i0 < 0) return;
        if (!act) s0 = s1 = 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
            s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomic_max_pos(&Y[i0].S[0], s0);
            atomic_max_pos(&Y[i0].S[1], s1);
        }
    } else if (act) {
        atomic_max_pos(&Y[inst].S[0], s0);
        atomic_max_pos(&Y[inst].S[1], s1);
    }
}

// ---------------------------------------------------------------------------
// k_band_prep
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void band_prep_rec(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                              BandRec *__restrict__ R, int n_inst, int r, int dir, int src, int qn) {
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
                    
#pragma unroll
                    for (int q = 0; q < MAXC; ++q)
                        if (q < I.nc) acc[q] += a * (double)QA[q * plane + c];
                }
        }
        if (ws == 0.0) {
            atomicOr(&y.err, ERR_NONBR);
            for (int q = 0; q < MAXC; ++q) b.Qp[q] = 0.0;
            b.flags &= ~RF_FLUID_A;
        } else {
            for (int q = 0; q < MAXC; ++q)
                if (q < I.nc) b.Qp[q] = acc[q] / ws;
        }
    }
    // moving-wall boundary state: advective part from the step-start state,
    // pressure from the sweep-start state
    if (b.flags & RF_FLUID_A) {
        // the cell's states in the path's type (the FP32 path stays in FP32:
        // on GB300 every FP64 conversion takes the narrow FP64 pipe)
        T qcT[MAXC], qsT[MAXC];
        const bool unc = (b.flags & RF_UNCOV) != 0;
#pragma unroll
        for (int q = 0; q < MAXC; ++q) qcT[q] = q >= I.nc ? T(0) : unc ? (T)b.Qp[q] : QA[q * plane + b.cell];
        const T n0 = QN[b.cell];
        const bool fresh = n0 != n0;
#pragma unroll
        for (int q = 0; q < MAXC; ++q) qsT[q] = q >= I.nc ? T(0) : fresh ? qcT[q] : QN[q * plane + b.cell];
        if (I.eq == 0) {
            // wall problem in the path's arithmetic type (FP64 path: double)
            const T g = (T)I.gamma;
            const T nx = (T)b.nx, ny = (T)b.ny, wx = (T)b.wx, wy = (T)b.wy;
            T rs, ps_step, usx, usy, rs2, ps_sw, u2x, u2y;
            wall_state<T>(g, qsT, nx, ny, wx, wy, &rs, &ps_step, &usx, &usy);
            bool same = true;
            for (int q = 0; q < 4; ++q) same = same && qsT[q] == qcT[q];
            if (same) ps_sw = ps_step;   // first sweep of a step: one state
            else wall_state<T>(g, qcT, nx, ny, wx, wy, &rs2, &ps_sw, &u2x, &u2y);
            T Eadv = ps_step / (g - T(1)) + T(0.5) * rs * (usx * usx + usy * usy);
            T ud = dir == 0 ? usx : usy;
            b.QB[0] = rs; b.QB[1] = rs * usx; b.QB[2] = rs * usy; b.QB[3] = Eadv;
            b.FB[0] = rs * ud;
            b.FB[1] = rs * ud * usx + (dir == 0 ? ps_sw : T(0));
            b.FB[2] = rs * ud * usy + (dir == 1 ? ps_sw : T(0));
            b.FB[3] = ud * (Eadv + ps_step);
        } else {
            b.QB[0] = (double)qsT[0];
            b.FB[0] = I.adv[dir] * (double)qsT[0];
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
            // a covered cell on a transmissive side with no fluid neighbour
            // (a body leaving the domain) passes its residual out of the
            // domain: no recipient gathers it; any other such event fails
            const bool open = (i == 0 && I.bc[0] == 0) || (i == I.nx - 1 && I.bc[1] == 0) ||
                              (j == 0 && I.bc[2] == 0) || (j == I.ny - 1 && I.bc[3] == 0);
            b.flags |= RF_NONBR;
            if (!((b.flags & RF_COVER) && open)) atomicOr(&y.err, ERR_NONBR);
            b.den = 0.0;
        } else {
            if (use8) b.flags |= RF_USE8;
            b.den = (b.flags & RF_COVER) ? den : b.aB + den;
        }
        // mark the band neighbours this event exchanges content with (all
        // eight), so that k_events gathers only where an event is near
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                int c;
                if ((di || dj) && nbr_cell(di, dj, &c) && (I.cls[c] & CLS_BAND)) atomicOr(&R[I.rec[c]].aux, 1);
            }
    }
}

template <class T>
__global__ void k_band_prep(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                            const int *__restrict__ boff, int n_inst, int dir, int src, int qn) {
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x;; t += stride) {
        const int r = band_rec_of(D, boff, n_inst, t);
        if (r < 0) break;
        band_prep_rec<T>(D, Y, R, n_inst, r, dir, src, qn);
    }
}

// the band offsets of k_band_offsets, computed by every CTA into shared
// memory (n_inst + 1 ints; the same integer sums), CTA 0 also writing them
// to boff for the later band kernels; then k_band_prep's loop over them.
// One launch fewer per sweep than k_band_offsets + k_band_prep.
template <class T>
__global__ void k_band_prep_o(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                              int *__restrict__ boff, int n_inst, int dir, int src, int qn) {
    extern __shared__ int s_boff[];
    __shared__ int wsum[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool w0 = blockIdx.x == 0;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n_inst; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const int c = k < n_inst ? min(Y[k].band_count, D[k].rec_cap) : 0;
        int v = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            if (lane < nw) wsum[lane] = w;
        }
        __syncthreads();
        if (k < n_inst) {
            const int ex = carry + (warp ? wsum[warp - 1] : 0) + v - c;
            s_boff[k] = ex;
            if (w0) boff[k] = ex;
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s_boff[n_inst] = carry;
        if (w0) boff[n_inst] = carry;
    }
    __syncthreads();
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x;; t += stride) {
        const int r = band_rec_of(D, s_boff, n_inst, t);
        if (r < 0) break;
        band_prep_rec<T>(D, Y, R, n_inst, r, dir, src, qn);
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
__device__ __forceinline__ bool band_sweep_rec(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                               BandRec *__restrict__ R, const double *__restrict__ bnd, int n_inst,
                                               int r, int dir, int src, double *wsum, int &inst_out) {
    int inst = find_inst_rec(D, n_inst, r);
    inst_out = inst;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return false;
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
    for (int q = 0; q < MAXC; ++q) {
        b.Flo[q] = Flo[q];
        b.Fhi[q] = Fhi[q];
        b.Flof[q] = (float)Flo[q];
        b.Fhif[q] = (float)Fhi[q];
    }
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
                wsum[q] += wt;
            }
            C[q] = v;
        }
    }
    for (int q = 0; q < MAXC; ++q) b.C[q] = C[q];
    return true;
}

template <class T>
__global__ void k_band_sweep(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                             const double *__restrict__ bnd, const int *__restrict__ boff, int n_inst, int dir,
                             int src) {
    const int total = boff[n_inst], stride = gridDim.x * blockDim.x;
    // whole warps iterate together (the wall-flux sum is warp-wide)
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < total; base += stride) {
        const int r = band_rec_of(D, boff, n_inst, base + (threadIdx.x & 31));
        double ws[MAXC] = {0.0, 0.0, 0.0, 0.0};
        int inst = -1;
        const bool act = r >= 0 && band_sweep_rec<T>(D, Y, R, bnd, n_inst, r, dir, src, ws, inst);
        warp_add_to(Y, act, inst, ws);
    }
}

// ---------------------------------------------------------------------------
// bulk sweep kernels: standard MUSCL-Hancock + HLLC update of every non-band
// cell.  Faces touching a band cell take the stabilised value its record
// holds (computed once by k_band_sweep), so every face flux is computed once.
// ---------------------------------------------------------------------------

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

// a non-band cell whose updated state is not physical: listed for the
// positivity safeguard (k_mix)
__device__ __forceinline__ void list_bulk_bad(InstDyn &y, int cell) {
    const int k = atomicAdd(&y.nbulk, 1);
    if (k < NBULK) y.bulkbad[k] = cell;
}

// new state of a non-band cell; wave speeds and positivity for the CFL step
template <class T, int NC, int EQ>
__device__ __forceinline__ void update_cell(T *__restrict__ Qo, size_t plane, int ci, uint8_t c0, T lam, T g, T av0,
                                            T av1, const QV<T, NC> &q, const QV<T, NC> &Flo, const QV<T, NC> &Fhi,
                                            bool last, T &s0, T &s1, InstDyn &y) {
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
        if (!(qn[0] > T(0)) || !(p > T(0))) list_bulk_bad(y, ci);
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
__device__ __forceinline__ void finish_warp(InstDyn &y, bool last, T s0, T s1) {
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
                update_cell<T, NC, EQ>(Qo, plane, rowb + ap, cm, lam, g, av0, av1, Qm, Fprev, Fhi, last, s0, s1, y);
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
            update_cell<T, NC, EQ>(Qo, plane, rowb + ap, cm, lam, g, av0, av1, Qm, Fprev, Fhi, last, s0, s1, y);
    }
    (void)cRc;
    finish_warp<T>(y, last != 0, s0, s1);
}

// y sweep: one thread per column and segment of I.yseg rows, marching upward
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
    const int j0 = sg * I.yseg, j1 = min(n, j0 + I.yseg);
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
    for (int f = j0; f <= j1; ++f) {
        // window: qm = row f-1, qc = row f, qp = row f+1, qq = row f+2
        evolve(EQ, g, 1, lam, av0, av1, qm.q, qc.q, qp.q, !(cm & CLS_SOLID) && !(cp & CLS_SOLID), QL.q, QR.q);
        face_flux<T, NC, EQ, 1>(I, R, i, f, n, cm, cc, g, av0, av1, QRc, QL, F);
        if (f > j0 && active)
            update_cell<T, NC, EQ>(Qo, plane, (f - 1) * I.pitch + i, cm, lam, g, av0, av1, qm, Fprev, F, last, s0,
                                   s1, y);
        QRc = QR;
        Fprev = F;
        qm = qc; cm = cc;
        qc = qp; cc = cp;
        qp = qq; cp = cq;
        if (f + 3 <= j1 + 1) load(f + 3, qq, cq);
    }
    finish_warp<T>(y, last != 0, s0, s1);
}

// ---------------------------------------------------------------------------
// packed FP32 Euler bulk kernels.  Every thread carries two cells (x sweep:
// two neighbours along the row; y sweep: two neighbouring columns) and runs
// the MUSCL-Hancock + HLLC arithmetic of both on FP32x2 instructions, the .x
// half for the first cell and the .y half for the second.  Same scheme and
// face ownership as the scalar kernels above; HLLC is written without
// branches (one physical flux is evaluated, then the case is selected).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 P2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}

// a pair of conserved states with 1/rho and p of each
struct S2 {
    float2 q[4];
};
struct E2 {
    float2 q[4];
    float2 ir, p;
};

__device__ __forceinline__ void prim2(float g1, const float2 *q, float2 &ir, float2 &p) {
    ir = rcp2(q[0]);
    const float2 ke = fma2(q[1], q[1], mul2(q[2], q[2]));
    p = mul2(P2(g1), fma2(mul2(P2(-0.5f), ke), ir, q[3]));
}

// prim2 of two states a, b of the same cells from one reciprocal,
// 1 / (rho_a rho_b) (the MUFU pipe is the kernels' second stall)
__device__ __forceinline__ void prim2x2(float g1, const float2 *a, const float2 *b, float2 &ira, float2 &pa,
                                        float2 &irb, float2 &pb) {
    const float2 r = rcp2(mul2(a[0], b[0]));
    ira = mul2(b[0], r);
    irb = mul2(a[0], r);
    pa = mul2(P2(g1), fma2(mul2(P2(-0.5f), fma2(a[1], a[1], mul2(a[2], a[2]))), ira, a[3]));
    pb = mul2(P2(g1), fma2(mul2(P2(-0.5f), fma2(b[1], b[1], mul2(b[2], b[2]))), irb, b[3]));
}

// physical flux along D of states q with normal velocity un and pressure p
template <int D>
__device__ __forceinline__ void flux2(const float2 *q, float2 un, float2 p, float2 *f) {
    f[0] = mul2(q[0], un);
    f[1] = D == 0 ? fma2(q[1], un, p) : mul2(q[1], un);
    f[2] = D == 1 ? fma2(q[2], un, p) : mul2(q[2], un);
    f[3] = mul2(un, add2(q[3], p));
}

__device__ __forceinline__ float2 vanleer2(float2 dm, float2 dp) {
    const float2 pr = mul2(dm, dp);
    const float2 r = mul2(add2(pr, pr), rcp2(add2(dm, dp)));
    return sel2(pr.x > 0.0f, pr.y > 0.0f, r, P2(0.0f));
}

// MUSCL-Hancock boundary states of the two cells (as evolve(): van Leer
// slopes, zero slope when lim is false, first order if an evolved state is
// not physical); also returns 1/rho and p of the evolved states
template <int D>
__device__ __forceinline__ void evolve2(float g1, float lam, const float2 *qm, const float2 *q0, const float2 *qp,
                                        bool limx, bool limy, E2 &QL, E2 &QR) {
    constexpr int in = D == 0 ? 1 : 2;
    float2 qL[4], qR[4], fL[4], fR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 sl = vanleer2(sub2(q0[k], qm[k]), sub2(qp[k], q0[k]));
        sl = sel2(limx, limy, sl, P2(0.0f));
        qL[k] = fma2(P2(-0.5f), sl, q0[k]);
        qR[k] = fma2(P2(0.5f), sl, q0[k]);
    }
    {
        float2 irL, pL, irR, pR;
        prim2x2(g1, qL, qR, irL, pL, irR, pR);
        flux2<D>(qL, mul2(qL[in], irL), pL, fL);
        flux2<D>(qR, mul2(qR[in], irR), pR, fR);
    }
    const float2 hl = P2(0.5f * lam);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 dfl = mul2(hl, sub2(fL[k], fR[k]));
        QL.q[k] = add2(qL[k], dfl);
        QR.q[k] = add2(qR[k], dfl);
    }
    prim2x2(g1, QL.q, QR.q, QL.ir, QL.p, QR.ir, QR.p);
    const bool okx = QL.q[0].x > 0.0f && QR.q[0].x > 0.0f && QL.p.x > 0.0f && QR.p.x > 0.0f;
    const bool oky = QL.q[0].y > 0.0f && QR.q[0].y > 0.0f && QL.p.y > 0.0f && QR.p.y > 0.0f;
    if (!(okx && oky)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            QL.q[k] = sel2(okx, oky, QL.q[k], q0[k]);
            QR.q[k] = sel2(okx, oky, QR.q[k], q0[k]);
        }
        prim2(g1, QL.q, QL.ir, QL.p);
        prim2(g1, QR.q, QR.ir, QR.p);
    }
}

// HLLC (Davis wave speeds) for two faces: left states L, right states R
template <int D>
__device__ __forceinline__ void hllc2(float g, const E2 &L, const E2 &R, float2 *F) {
    constexpr int in = D == 0 ? 1 : 2, it = 3 - in;
    const float2 uL = mul2(L.q[in], L.ir), uR = mul2(R.q[in], R.ir);
    const float2 cL = sqrt2(mul2(mul2(P2(g), L.p), L.ir)), cR = sqrt2(mul2(mul2(P2(g), R.p), R.ir));
    const float2 SL = min2(sub2(uL, cL), sub2(uR, cR)), SR = max2(add2(uL, cL), add2(uR, cR));
    const float2 aL = mul2(L.q[0], sub2(SL, uL)), aR = mul2(R.q[0], sub2(SR, uR));
    const float2 num = add2(sub2(R.p, L.p), sub2(mul2(aL, uL), mul2(aR, uR)));
    const float2 Ss = mul2(num, rcp2(sub2(aL, aR)));
    // side whose flux is used: L when supersonic to the right or Ss >= 0
    const bool kx = SL.x >= 0.0f || (SR.x > 0.0f && Ss.x >= 0.0f);
    const bool ky = SL.y >= 0.0f || (SR.y > 0.0f && Ss.y >= 0.0f);
    float2 q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = sel2(kx, ky, L.q[k], R.q[k]);
    const float2 iv = sel2(kx, ky, L.ir, R.ir), u = sel2(kx, ky, uL, uR), p = sel2(kx, ky, L.p, R.p);
    const float2 S = sel2(kx, ky, SL, SR), a = sel2(kx, ky, aL, aR);
    float2 f[4];
    flux2<D>(q, u, p, f);
    // a / (S - S*) and p / a from one reciprocal, 1 / (a (S - S*)) (both
    // factors are non-zero where the star state is used)
    const float2 dS = sub2(S, Ss);
    const float2 rr = rcp2(mul2(a, dS));
    const float2 fac = mul2(mul2(a, a), rr);
    const float2 pa = mul2(mul2(p, dS), rr);
    float2 qs[4];
    qs[0] = fac;
    qs[in] = mul2(fac, Ss);
    qs[it] = mul2(fac, mul2(q[it], iv));
    qs[3] = mul2(fac, fma2(sub2(Ss, u), add2(pa, Ss), mul2(q[3], iv)));
    const bool sx = SL.x >= 0.0f || SR.x <= 0.0f, sy = SL.y >= 0.0f || SR.y <= 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = sel2(sx, sy, f[k], fma2(S, sub2(qs[k], q[k]), f[k]));
}

// flux of one face (half h of F) replaced by the band record value or zero
template <int DIR>
__device__ __forceinline__ void face_override(const InstDesc &I, const BandRec *__restrict__ R, int line, int a,
                                              int n, uint8_t cl, uint8_t cr, float2 *F, int h) {
    if (!((cl | cr) & (CLS_BAND | CLS_SOLID))) return;
    float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
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
            for (int k = 0; k < 4; ++k) v[k] = rb.Flof[k];
        } else {
            const BandRec &ra = R[I.rec[cia]];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = ra.Fhif[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (h == 0) F[k].x = v[k];
        else F[k].y = v[k];
    }
}

// positivity list and CFL wave speeds of a pair of new states (cells ci and
// ci + 1; st: bit 0 first stored, bit 1 second stored).  Outside the last
// sweep only the signs are needed: rho > 0 and p > 0, i.e. 2 rho E > |m|^2,
// with no division
__device__ __forceinline__ void pair_checks(const float2 *qn, int st, int ci, bool last, float g1, float g, float &s0,
                                            float &s1, InstDyn &y) {
    if (!last) {
        const float2 m2 = fma2(qn[1], qn[1], mul2(qn[2], qn[2]));
        const float2 e2 = mul2(add2(qn[0], qn[0]), qn[3]);
        if ((st & 1) && !(qn[0].x > 0.0f && e2.x > m2.x)) list_bulk_bad(y, ci);
        if ((st & 2) && !(qn[0].y > 0.0f && e2.y > m2.y)) list_bulk_bad(y, ci + 1);
        return;
    }
    float2 ir, p;
    prim2(g1, qn, ir, p);
    if ((st & 1) && !(qn[0].x > 0.0f && p.x > 0.0f)) list_bulk_bad(y, ci);
    if ((st & 2) && !(qn[0].y > 0.0f && p.y > 0.0f)) list_bulk_bad(y, ci + 1);
    const float2 cs = sqrt2(mul2(mul2(P2(g), p), ir));
    const float2 w0 = add2(make_float2(fabsf(qn[1].x * ir.x), fabsf(qn[1].y * ir.y)), cs);
    const float2 w1 = add2(make_float2(fabsf(qn[2].x * ir.x), fabsf(qn[2].y * ir.y)), cs);
    if (st & 1) { s0 = fmaxf(s0, w0.x); s1 = fmaxf(s1, w1.x); }
    if (st & 2) { s0 = fmaxf(s0, w0.y); s1 = fmaxf(s1, w1.y); }
}

// new states of the two cells (q, fluxes Flo / Fhi through their low / high
// faces); stores the cells flagged in st (bit 0: first, bit 1: second);
// wave speeds and positivity for the CFL step
__device__ __forceinline__ void update2(float *__restrict__ Qo, size_t plane, int ci, int st, bool vec, float g1,
                                        float g, float lam, const float2 *q, const float2 *Flo, const float2 *Fhi,
                                        bool last, float &s0, float &s1, InstDyn &y) {
    float2 qn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) qn[k] = fma2(P2(lam), sub2(Flo[k], Fhi[k]), q[k]);
    if (vec) {
#pragma unroll
        for (int k = 0; k < 4; ++k) *(float2 *)(Qo + k * plane + ci) = qn[k];
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (st & 1) Qo[k * plane + ci] = qn[k].x;
            if (st & 2) Qo[k * plane + ci + 1] = qn[k].y;
        }
    }
    pair_checks(qn, st, ci, last, g1, g, s0, s1, y);
}

// asynchronous global -> shared copies of 4 or 8 bytes (completion through
// cp.async.wait_group, issued and waited for by the same thread)
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// per-warp ring of the x sweep: cell b of the row (the ghost cells -2, -1,
// n, n+1 of the boundary conditions included) sits at position b mod 64 XC;
// chunks of 64 cells arrive by cp.async XC - 2 chunks ahead of their use
template <int XC>
struct XRing {
    float q[4][64 * XC];
    unsigned char cls[64 * XC];
};

// class bits that take a cell off the plain path (solid, or a band cell whose
// faces carry stabilised fluxes)
constexpr unsigned CLS_OFF = CLS_SOLID | CLS_BAND;

// Deferred cells of a sweep (FP32 Euler).  A cell is deferred when a cell
// within three positions of it along the sweep was touched by the body
// boundary at the start pose.  The body moves by less than a cell per sweep
// and only along the sweep (k_pose sets defer_all otherwise, and for a
// rotating body), so every band cell of the sweep lies within one position
// of a touched cell, and so does every fluid cell next to a solid cell.  A
// cell that is not deferred therefore has a five-cell stencil of plain
// fluid cells (its update is the plain MUSCL-Hancock + HLLC update), or is
// solid at both poses (its state is NaN).  Neither needs the sweep's
// geometry, so the pass that stores them (mode 0) runs concurrently with the
// geometry and band-flux kernels.  The deferred cells are appended, as cell
// pairs, to a list that k_bulk_def_* work through after the band fluxes, on
// the general path; an instance with defer_all is updated by a second
// streaming pass (mode 1) instead.  The arithmetic of every cell is that of
// a single general pass.

// append this lane's pair (cell index ci of its first cell) when bits != 0;
// one atomic per warp
__device__ __forceinline__ void defer_push(const DeferList &L, InstDyn &y, int inst, int ci, int bits) {
    const unsigned m = __ballot_sync(0xffffffffu, bits != 0);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(L.count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (bits) {
        const int k = base + __popc(m & ((1u << lane) - 1u));
        if (k < L.cap) L.item[k] = make_int2(inst, ci | (bits << 28));
        else atomicOr(&y.err, ERR_DEFER_CAP);
    }
}

// deferred bits of a lane's two cells in the chunk before the current one,
// from the lane masks (bit l: lane l's pair, t0 its first cell, t1 its
// second) of touched cells in the chunks before it (p2), itself (p1) and
// after it (c)
__device__ __forceinline__ int deferred_pair(int lane, unsigned p2_0, unsigned p2_1, unsigned p1_0, unsigned p1_1,
                                             unsigned c_0, unsigned c_1) {
    // window over lanes -2 .. 33 of the chunk: bit l + 2 holds lane l
    const unsigned long long P = (unsigned long long)((p2_0 | p2_1) >> 30) |
                                 ((unsigned long long)(p1_0 | p1_1) << 2) |
                                 ((unsigned long long)(c_0 | c_1) << 34);
    const unsigned long long W1 = (unsigned long long)(p2_1 >> 30) | ((unsigned long long)p1_1 << 2) |
                                  ((unsigned long long)c_1 << 34);
    const unsigned long long W0 = (unsigned long long)(p2_0 >> 30) | ((unsigned long long)p1_0 << 2) |
                                  ((unsigned long long)c_0 << 34);
    const bool mid = ((P >> (lane + 1)) & 7ull) != 0;        // lanes l-1, l, l+1
    const bool d0 = mid || ((W1 >> lane) & 1ull);            // cell 2l-3 (lane l-2, second)
    const bool d1 = mid || ((W0 >> (lane + 4)) & 1ull);      // cell 2l+4 (lane l+2, first)
    return (d0 ? 1 : 0) | (d1 ? 2 : 0);
}

// Lines and tiles the body cannot reach (mode 0).  The body's extent over
// the sweep's poses (k_pose: every polygon, fixed or moving, at poses A, mid
// and B, widened by a cell) bounds every touched and every solid cell of the
// sweep.  A row of the x sweep outside it, or a y-sweep tile whose columns
// miss it or whose rows lie more than three rows away from it, holds only
// fluid cells with plain five-cell stencils: no class byte is needed, no
// cell is deferred and every real cell is stored.  These paths skip the
// class bytes, touch masks and deferral bookkeeping of the general loops
// below; each cell's arithmetic is the same function sequence on the same
// inputs (evolve2 with slopes on, hllc2, the update, the positivity and
// wave-speed checks), so the bits are the same.


// x sweep of row j (Q, Qo: the row's first cell) outside the body's extent,
// in the layout of k_bulk_x_p: lane l holds cells 64c + 2l, 64c + 2l + 1 of
// chunk c, the ring is filled by cp.async XC - 2 chunks ahead, the update
// trails the fluxes by one chunk
template <int XC>
__device__ __forceinline__ void bulk_x_far(const InstDesc &I, InstDyn &y, XRing<XC> &rg,
                                           const float *__restrict__ Q, float *__restrict__ Qo, int rowb, size_t plane,
                                           float lam, float g, float g1, bool last, float &s0, float &s1) {
    constexpr int XRN = 64 * XC;
    const int lane = threadIdx.x & 31;
    const int n = I.nx;
    const int c_last = (n + 1) >> 6;   // chunk holding face n
    // ghost cells of the boundary conditions: lane 0: -2, 1: -1, 2: n, 3: n+1
    float gq[4] = {1.0f, 1.0f, 1.0f, 1.0f};
    int gb = -1000000;
    if (lane < 4) {
        gb = lane < 2 ? lane - 2 : n + lane - 2;
        bool fl;
        const int p = ghost_map(gb, n, I.bc[0], I.bc[1], &fl);
#pragma unroll
        for (int k = 0; k < 4; ++k) gq[k] = __ldg(Q + k * plane + p);
        if (fl) gq[1] = -gq[1];
    }
    // ghosts of chunk c or c+1 into the ring, once those chunks' copies are
    // complete (a copy cannot overwrite them then)
    const int c_hi_ghost = (n >> 6) - 1;
    auto put_ghost = [&](int c) {
        const int gk = gb >> 6;
        if (lane < 4 && (gk == c || gk == c + 1)) {
            const int pos = gb & (XRN - 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) rg.q[k][pos] = gq[k];
        }
    };
    auto prefetch = [&](int c) {
        const int a0 = 64 * c;
        if (c >= 0 && a0 < n) {
            const int sl = a0 & (XRN - 1);
            const int a = a0 + 2 * lane;
            if (a + 1 < n) {
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async8(&rg.q[k][sl + 2 * lane], Q + k * plane + a);
            } else if (a < n) {
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async4(&rg.q[k][sl + 2 * lane], Q + k * plane + a);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int c = 0; c < XC - 2; ++c) prefetch(c);
    cp_async_wait<XC - 4>();   // chunks 0 and 1 complete
    __syncwarp();
    put_ghost(-1);
    __syncwarp();
    // evolved right state of cell -1 (all lanes alike)
    E2 QRc;
    {
        float2 qm[4], q0[4], qp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = P2(rg.q[k][XRN - 2]);
            q0[k] = P2(rg.q[k][XRN - 1]);
            qp[k] = P2(rg.q[k][0]);
        }
        E2 QL;
        evolve2<0>(g1, lam, qm, q0, qp, true, true, QL, QRc);
    }
    float2 Fprev[4];
    float2 qprev[4];   // states of the previous chunk's two cells (as loaded there)
    // new states of chunk c - 1 (F: this chunk's fluxes, whose lane 0 holds
    // the high face of the previous chunk's lane 31; tail: none)
    auto update = [&](int c, const float2 *F, bool tail) {
        const int ap = 64 * (c - 1) + 2 * lane;
        float2 qn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dn = __shfl_down_sync(0xffffffffu, Fprev[k].x, 1);
            const float nx0 = tail ? 0.0f : __shfl_sync(0xffffffffu, F[k].x, 0);
            const float2 Fhi = make_float2(Fprev[k].y, lane == 31 ? nx0 : dn);
            qn[k] = fma2(P2(lam), sub2(Fprev[k], Fhi), qprev[k]);
        }
        const int st = (ap < n ? 1 : 0) | (ap + 1 < n ? 2 : 0);
        if (st == 3) {
#pragma unroll
            for (int k = 0; k < 4; ++k) *(float2 *)(Qo + k * plane + ap) = qn[k];
        } else if (st) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qo[k * plane + ap] = qn[k].x;
        }
        pair_checks(qn, st, rowb + ap, last, g1, g, s0, s1, y);
    };
    for (int c = 0; c <= c_last; ++c) {
        __syncwarp();
        prefetch(c + XC - 2);
        cp_async_wait<XC - 3>();   // chunks up to c + 1 complete
        __syncwarp();
        if (c >= c_hi_ghost) {
            put_ghost(c);
            __syncwarp();
        }
        const int a = 64 * c + 2 * lane;
        const int pa = a & (XRN - 1), pl = (a - 1) & (XRN - 1), pr = (a + 2) & (XRN - 1);
        float2 q0[4], qm[4], qp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q0[k] = *(const float2 *)&rg.q[k][pa];
            qm[k] = make_float2(rg.q[k][pl], q0[k].x);
            qp[k] = make_float2(q0[k].y, rg.q[k][pr]);
        }
        E2 QL, QR;
        evolve2<0>(g1, lam, qm, q0, qp, true, true, QL, QR);
        // faces a (cells a-1 | a) and a+1 (cells a | a+1)
        E2 Lf;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float up = __shfl_up_sync(0xffffffffu, QR.q[k].y, 1);
            Lf.q[k] = make_float2(lane == 0 ? QRc.q[k].x : up, QR.q[k].x);
        }
        {
            const float ui = __shfl_up_sync(0xffffffffu, QR.ir.y, 1), up = __shfl_up_sync(0xffffffffu, QR.p.y, 1);
            Lf.ir = make_float2(lane == 0 ? QRc.ir.x : ui, QR.ir.x);
            Lf.p = make_float2(lane == 0 ? QRc.p.x : up, QR.p.x);
        }
        float2 F[4];
        hllc2<0>(g, Lf, QL, F);
        if (c >= 1) update(c, F, false);
#pragma unroll
        for (int k = 0; k < 4; ++k) QRc.q[k].x = __shfl_sync(0xffffffffu, QR.q[k].y, 31);
        QRc.ir.x = __shfl_sync(0xffffffffu, QR.ir.y, 31);
        QRc.p.x = __shfl_sync(0xffffffffu, QR.p.y, 31);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Fprev[k] = F[k];
            qprev[k] = q0[k];
        }
    }
    // the row's last chunk (the face past its lane 31 lies beyond face n)
    update(c_last + 1, Fprev, true);
}

// x sweep, packed: one warp per row, lane l holds cells 64c + 2l and
// 64c + 2l + 1 of chunk c; the update trails the fluxes by one chunk.
// MODE 0: the cells that are not deferred (plain arithmetic throughout);
// MODE 1: every cell of the instances with defer_all, on the general path
// (a chunk whose cells and stencil halo are all plain fluid cells still takes
// the plain arithmetic, decided by a warp-uniform ballot over the class
// bytes).  MINB: resident CTAs per SM the registers are budgeted for; XC:
// ring chunks.
template <int MINB, int XC, int MODE>
__global__ void __launch_bounds__(128, MINB) k_bulk_x_p(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                     const BandRec *__restrict__ R, int n_inst, int total_warps,
                                                     int src, int dst, int last, DeferList dl) {
    extern __shared__ __align__(16) unsigned char xsm[];
    constexpr int XRN = 64 * XC;
    constexpr bool gen = MODE != 0;
    const int lane = threadIdx.x & 31;
    XRing<XC> &rg = ((XRing<XC> *)xsm)[threadIdx.x >> 5];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_warps) return;
    const int inst = find_inst_warp(D, n_inst, gw, 0);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if ((MODE == 0) == (y.defer_all != 0)) return;
    const int j = gw - I.tile_off[0];
    const int n = I.nx;
    const int c_last = (n + 1) >> 6;   // chunk holding face n
    const float lam = y.lamf;
    const float g = (float)I.gamma, g1 = g - 1.0f;
    const size_t plane = (size_t)I.pitch * I.ny;
    const int rowb = j * I.pitch;
    const float *__restrict__ Q = (const float *)I.Q[src] + rowb;
    float *__restrict__ Qb = (float *)I.Q[dst];
    float *__restrict__ Qo = Qb + rowb;
    if (MODE == 0 && I.bc[0] != 2 && (j < y.row0 || j > y.row1)) {
        // a row outside the body's extent: plain throughout
        float s0 = 0.0f, s1 = 0.0f;
        bulk_x_far<XC>(I, y, rg, Q, Qo, rowb, plane, lam, g, g1, last != 0, s0, s1);
        finish_warp<float>(y, last != 0, s0, s1);
        return;
    }
    const unsigned char *__restrict__ cl = I.cls + rowb;
    // ghost cells of the boundary conditions: lane 0: -2, 1: -1, 2: n, 3: n+1
    float gq[4] = {1.0f, 1.0f, 1.0f, 1.0f};
    int gc = CLS_SOLID, gb = -1000000;
    if (lane < 4) {
        gb = lane < 2 ? lane - 2 : n + lane - 2;
        bool fl;
        const int p = ghost_map(gb, n, I.bc[0], I.bc[1], &fl);
#pragma unroll
        for (int k = 0; k < 4; ++k) gq[k] = __ldg(Q + k * plane + p);
        if (fl) gq[1] = -gq[1];
        gc = cl[p];
    }
    // ghosts that belong to chunk c or c+1 into the ring (after those chunks'
    // copies have completed, so that a copied class word cannot overwrite them)
    const int c_hi_ghost = (n >> 6) - 1;   // first chunk c whose chunks c, c+1 may hold ghost n or n+1
    auto put_ghost = [&](int c) {
        const int gk = gb >> 6;
        if (lane < 4 && (gk == c || gk == c + 1)) {
            const int pos = gb & (XRN - 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) rg.q[k][pos] = gq[k];
            rg.cls[pos] = (unsigned char)gc;
        }
    };
    // copies of chunk c's real cells into the ring (one commit group per call)
    auto prefetch = [&](int c) {
        const int a0 = 64 * c;
        if (c >= 0 && a0 < n) {
            const int s = a0 & (XRN - 1);
            const int a = a0 + 2 * lane;
            if (a + 1 < n) {
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async8(&rg.q[k][s + 2 * lane], Q + k * plane + a);
            } else if (a < n) {
#pragma unroll
                for (int k = 0; k < 4; ++k) cp_async4(&rg.q[k][s + 2 * lane], Q + k * plane + a);
            }
            if (lane < 16 && a0 + 4 * lane < n) cp_async4(&rg.cls[s + 4 * lane], cl + a0 + 4 * lane);
        }
        cp_async_commit();
    };
    // lane masks of chunk c's cells touched at the start pose (positions
    // outside -2 .. n + 1 hold stale ring contents and count as clear)
    auto touch_masks = [&](int c, unsigned &m0, unsigned &m1) {
        const int a = 64 * c + 2 * lane;
        const int cc = *(const unsigned short *)&rg.cls[a & (XRN - 1)];
        m0 = __ballot_sync(0xffffffffu, a >= -2 && a <= n + 1 && (cc & CLS_TOUCH));
        m1 = __ballot_sync(0xffffffffu, a + 1 >= -2 && a + 1 <= n + 1 && ((cc >> 8) & CLS_TOUCH));
    };
#pragma unroll
    for (int c = 0; c < XC - 2; ++c) prefetch(c);
    cp_async_wait<XC - 4>();   // chunks 0 and 1 complete
    __syncwarp();
    put_ghost(-1);
    __syncwarp();
    // evolved right state of cell -1 (all lanes alike)
    E2 QRc;
    {
        float2 qm[4], q0[4], qp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = P2(rg.q[k][XRN - 2]);
            q0[k] = P2(rg.q[k][XRN - 1]);
            qp[k] = P2(rg.q[k][0]);
        }
        const bool lim = !gen || (!(rg.cls[XRN - 2] & CLS_SOLID) && !(rg.cls[0] & CLS_SOLID));
        E2 QL;
        evolve2<0>(g1, lam, qm, q0, qp, lim, lim, QL, QRc);
    }
    // plain-path state of the general path: cells 64c-2, 64c-1 plain, and
    // the previous chunk entirely plain
    bool prev_hi = !((rg.cls[XRN - 2] | rg.cls[XRN - 1]) & CLS_OFF);
    bool prev_all = false;
    // touch masks of the two chunks before the current one.  Touched cells
    // lie inside the body's extent over the sweep's poses (k_pose), so rows
    // and chunks outside it skip the masks (not across a periodic side,
    // whose ghost cells mirror the far end of the row)
    unsigned tp2_0 = 0u, tp2_1 = 0u, tp1_0 = 0u, tp1_1 = 0u;
    const int ext_c0 = y.col0, ext_c1 = y.col1;
    const bool row_near = I.bc[0] == 2 || (j >= y.row0 && j <= y.row1);
    auto chunk_near = [&](int c) {
        return row_near && (I.bc[0] == 2 || (64 * c - 2 <= ext_c1 && 64 * c + 65 >= ext_c0));
    };
    if (!gen && chunk_near(-1)) touch_masks(-1, tp1_0, tp1_1);
    const int rem = n + 1 - 2 * lane;
    float s0 = 0.0f, s1 = 0.0f;
    float2 Fprev[4];
    // cells of the chunk before c that this pass stores and that are solid
    // at the start pose; mode 0 lists the deferred pairs
    auto store_bits = [&](int c, unsigned tc_0, unsigned tc_1, int cm, int &sol) {
        const int ap = 64 * (c - 1) + 2 * lane;
        const int real = (ap < n ? 1 : 0) | (ap + 1 < n ? 2 : 0);
        sol = ((cm & CLS_SOLID) ? 1 : 0) | (((cm >> 8) & CLS_SOLID) ? 2 : 0);
        if (gen) return real;
        // no touched cell within reach of chunk c-1 (the usual case): nothing deferred
        if (!(((tp2_0 | tp2_1) >> 30) | tp1_0 | tp1_1 | tc_0 | tc_1)) return real;
        const int dp = deferred_pair(lane, tp2_0, tp2_1, tp1_0, tp1_1, tc_0, tc_1) & real;
        defer_push(dl, y, inst, rowb + ap, dp);
        return real & ~dp;
    };
    // update of the chunk before c (faces Fprev, high face of lane 31 from
    // this chunk's lane 0; tail: the row's last chunk) on the general path
    auto update_general = [&](int c, const float2 *F, bool tail, int sm, int cm) {
        float2 Fhi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dn = __shfl_down_sync(0xffffffffu, Fprev[k].x, 1);
            const float nx0 = tail ? 0.0f : __shfl_sync(0xffffffffu, F[k].x, 0);
            Fhi[k] = make_float2(Fprev[k].y, lane == 31 ? nx0 : dn);
        }
        const int ap = 64 * (c - 1) + 2 * lane;
        const int pp = ap & (XRN - 1);
        S2 Qm;
#pragma unroll
        for (int k = 0; k < 4; ++k) Qm.q[k] = *(const float2 *)&rg.q[k][pp];
        const bool w0 = (sm & 1) != 0, w1 = (sm & 2) && (tail ? lane < 31 : true);
        int st = 0;
        if (w0 && !((cm & 0xff) & CLS_OFF)) st |= 1;
        if (w1 && !(((cm >> 8) & 0xff) & CLS_OFF)) st |= 2;
        if (st) update2(Qb, plane, rowb + ap, st, st == 3, g1, g, lam, Qm.q, Fprev, Fhi, last, s0, s1, y);
        if ((cm & CLS_SOLID) && w0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qo[k * plane + ap] = NAN;
        }
        if (((cm >> 8) & CLS_SOLID) && w1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qo[k * plane + ap + 1] = NAN;
        }
    };
    for (int c = 0; c <= c_last; ++c) {
        __syncwarp();
        prefetch(c + XC - 2);
        cp_async_wait<XC - 3>();   // chunks up to c + 1 complete
        __syncwarp();
        if (c >= c_hi_ghost) {
            put_ghost(c);
            __syncwarp();
        }
        const int a = 64 * c + 2 * lane;
        const int pa = a & (XRN - 1), pl = (a - 1) & (XRN - 1), pr = (a + 2) & (XRN - 1);
        const int c0 = *(const unsigned short *)&rg.cls[pa];
        bool plain = true;
        unsigned bal = 0xffffffffu;
        if (gen) {
            // plain-path test over cells 64c-2 .. 64c+64 (those up to n+1)
            const int lim = rem - 64 * c;
            const int vm = lim >= 1 ? 0x0505 : (lim == 0 ? 0x0005 : 0);
            bal = __ballot_sync(0xffffffffu, !(c0 & vm));
            const int ah = 64 * c + 64;
            const bool hclean = ah > n + 1 || !(rg.cls[ah & (XRN - 1)] & CLS_OFF);
            plain = bal == 0xffffffffu && prev_hi && hclean;
        }
        unsigned tc_0 = 0u, tc_1 = 0u;
        if (!gen && chunk_near(c)) touch_masks(c, tc_0, tc_1);
        S2 Q0;
        float2 qm[4], qp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Q0.q[k] = *(const float2 *)&rg.q[k][pa];
            qm[k] = make_float2(rg.q[k][pl], Q0.q[k].x);
            qp[k] = make_float2(Q0.q[k].y, rg.q[k][pr]);
        }
        E2 QL, QR;
        if (plain) {
            evolve2<0>(g1, lam, qm, Q0.q, qp, true, true, QL, QR);
        } else {
            const int clA = rg.cls[pl], crB = rg.cls[pr];
            const int cA = c0 & 0xff, cB = (c0 >> 8) & 0xff;
            const bool lx = !(clA & CLS_SOLID) && !(cB & CLS_SOLID);
            const bool ly = !(cA & CLS_SOLID) && !(crB & CLS_SOLID);
            evolve2<0>(g1, lam, qm, Q0.q, qp, lx, ly, QL, QR);
        }
        // faces a (cells a-1 | a) and a+1 (cells a | a+1)
        E2 Lf;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float up = __shfl_up_sync(0xffffffffu, QR.q[k].y, 1);
            Lf.q[k] = make_float2(lane == 0 ? QRc.q[k].x : up, QR.q[k].x);
        }
        {
            const float ui = __shfl_up_sync(0xffffffffu, QR.ir.y, 1), up = __shfl_up_sync(0xffffffffu, QR.p.y, 1);
            Lf.ir = make_float2(lane == 0 ? QRc.ir.x : ui, QR.ir.x);
            Lf.p = make_float2(lane == 0 ? QRc.p.x : up, QR.p.x);
        }
        float2 F[4];
        hllc2<0>(g, Lf, QL, F);
        if (!plain) {
            const int clA = rg.cls[pl];
            const int cA = c0 & 0xff, cB = (c0 >> 8) & 0xff;
            if (a <= n) face_override<0>(I, R, j, a, n, (uint8_t)clA, (uint8_t)cA, F, 0);
            if (a + 1 <= n) face_override<0>(I, R, j, a + 1, n, (uint8_t)cA, (uint8_t)cB, F, 1);
        }
        if (c >= 1) {
            const int ap = a - 64;
            const int pp = ap & (XRN - 1);
            const int cm = *(const unsigned short *)&rg.cls[pp];
            int sol;
            const int sm = store_bits(c, tc_0, tc_1, cm, sol);
            if (!gen || (prev_all && 64 * c <= n)) {
                // chunk c-1 on the plain path: the stored cells are plain, or
                // (mode 0) solid at both poses
                float2 Fhi[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float dn = __shfl_down_sync(0xffffffffu, Fprev[k].x, 1);
                    const float nx0 = __shfl_sync(0xffffffffu, F[k].x, 0);
                    Fhi[k] = make_float2(Fprev[k].y, lane == 31 ? nx0 : dn);
                }
                float2 qn[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 qo = *(const float2 *)&rg.q[k][pp];
                    qn[k] = fma2(P2(lam), sub2(Fprev[k], Fhi[k]), qo);
                }
                const int sq = sm & sol;   // solid at both poses: NaN
                if (sq) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) qn[k] = make_float2((sq & 1) ? NAN : qn[k].x, (sq & 2) ? NAN : qn[k].y);
                }
                if (sm == 3) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) *(float2 *)(Qo + k * plane + ap) = qn[k];
                } else if (sm) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (sm & 1) Qo[k * plane + ap] = qn[k].x;
                        if (sm & 2) Qo[k * plane + ap + 1] = qn[k].y;
                    }
                }
                const int st = sm & ~sol;
                pair_checks(qn, st, rowb + ap, last != 0, g1, g, s0, s1, y);
            } else {
                update_general(c, F, false, sm, cm);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) QRc.q[k].x = __shfl_sync(0xffffffffu, QR.q[k].y, 31);
        QRc.ir.x = __shfl_sync(0xffffffffu, QR.ir.y, 31);
        QRc.p.x = __shfl_sync(0xffffffffu, QR.p.y, 31);
#pragma unroll
        for (int k = 0; k < 4; ++k) Fprev[k] = F[k];
        prev_hi = (bal >> 31) != 0;
        prev_all = bal == 0xffffffffu;
        tp2_0 = tp1_0; tp2_1 = tp1_1;
        tp1_0 = tc_0; tp1_1 = tc_1;
    }
    // the row's last chunk (its high faces were computed in the final
    // iteration, except the one past lane 31 which lies beyond face n)
    {
        const int ap = 64 * c_last + 2 * lane;
        const int cm = *(const unsigned short *)&rg.cls[ap & (XRN - 1)];
        int sol;
        const int sm = store_bits(c_last + 1, 0u, 0u, cm, sol);
        update_general(c_last + 1, Fprev, true, sm, cm);
    }
    finish_warp<float>(y, last != 0, s0, s1);
}

// per-warp ring of rows for the y sweep: row r of the warp's 64 columns sits
// in slot (r - j0 + 2) % YR, prefetched YR - 2 rows ahead
constexpr int YR = 8;
struct YRing {
    float q[YR][4][64];
    unsigned char cls[YR][64];
};

// y sweep of a tile the body cannot reach (see bulk_x_far), in the layout
// of k_bulk_y_p: columns i, i+1 of this thread (st0: which exist), rows
// j0 .. j1-1 streamed through the warp's ring six rows ahead
__device__ __forceinline__ void bulk_y_far(const InstDesc &I, InstDyn &y, YRing &rg, const float *__restrict__ Q,
                                           float *__restrict__ Qo, int i, int st0, int j0, int j1, size_t plane,
                                           float lam, float g, float g1, bool last, float &s0, float &s1) {
    const int lane = threadIdx.x & 31;
    const int n = I.ny, pitch = I.pitch;
    const int bclo = I.bc[2], bchi = I.bc[3];
    // copies of row r (a ghost row of the boundary condition outside [0, n))
    // into its slot; rows past j1 + 2 are not needed (one commit group per call)
    auto prefetch = [&](int r) {
        if (r <= j1 + 2) {
            const int sl = (r - j0 + 2) & (YR - 1);
            int p = r;
            if (r < 0 || r >= n) {
                bool fl;
                p = ghost_map(r, n, bclo, bchi, &fl);
            }
            const float *src_q = Q + (size_t)p * pitch + i;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (st0 == 3) cp_async8(&rg.q[sl][k][2 * lane], src_q + k * plane);
                else if (st0 == 1) cp_async4(&rg.q[sl][k][2 * lane], src_q + k * plane);
            }
        }
        cp_async_commit();
    };
    // the pair of row r from the ring; columns past the grid read as 1,
    // ghost rows of a reflective side flip the normal momentum
    auto row = [&](int r, float2 *v) {
        const int sl = (r - j0 + 2) & (YR - 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = *(const float2 *)&rg.q[sl][k][2 * lane];
        if (st0 != 3) {
            if (!(st0 & 1)) {
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k].x = 1.0f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k].y = 1.0f;
        }
        if ((r < 0 && bclo == 1) || (r >= n && bchi == 1)) {
            v[2].x = -v[2].x;
            v[2].y = -v[2].y;
        }
    };
    for (int r = j0 - 2; r < j0 - 2 + YR; ++r) prefetch(r);
    cp_async_wait<YR - 4>();   // rows j0-2 .. j0+1 complete
    __syncwarp();
    // rows f and f+1 carry over to the next row step (as its rows f-1 and f)
    float2 qm[4], qc[4], qp[4];
    E2 QRc;
    {
        float2 qa[4];
        row(j0 - 2, qa);
        row(j0 - 1, qc);
        row(j0, qp);
        E2 QL;
        evolve2<1>(g1, lam, qa, qc, qp, true, true, QL, QRc);
    }
    float2 Fprev[4];
    float *__restrict__ wp = Qo + (size_t)(j0 - 1) * pitch + i;   // row f-1 of this thread's columns
    for (int f = j0; f <= j1; ++f, wp += pitch) {
        __syncwarp();
        prefetch(f + YR - 2);
        cp_async_wait<YR - 4>();   // rows up to f + 2 complete
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = qc[k];
            qc[k] = qp[k];
        }
        if (f + 1 < n) {
            // row f+1 (lanes past the grid compute on values that are never
            // stored)
            const int sp = (f - j0 + 3) & (YR - 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) qp[k] = *(const float2 *)&rg.q[sp][k][2 * lane];
        } else {
            row(f + 1, qp);
        }
        E2 QL, QR;
        evolve2<1>(g1, lam, qm, qc, qp, true, true, QL, QR);
        float2 F[4];
        hllc2<1>(g, QRc, QL, F);
        if (f > j0) {
            float2 qn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) qn[k] = fma2(P2(lam), sub2(Fprev[k], F[k]), qm[k]);
            if (st0 == 3) {
#pragma unroll
                for (int k = 0; k < 4; ++k) *(float2 *)(wp + k * plane) = qn[k];
            } else if (st0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) wp[k * plane] = qn[k].x;
            }
            pair_checks(qn, st0, (f - 1) * pitch + i, last, g1, g, s0, s1, y);
        }
        QRc = QR;
#pragma unroll
        for (int k = 0; k < 4; ++k) Fprev[k] = F[k];
    }
}

// y sweep, packed: one thread per pair of neighbouring columns and segment of
// I.yseg rows, marching upward; a warp covers 64 consecutive columns and
// streams its rows through a shared-memory ring filled by cp.async.  Passes
// as for the x sweep: MODE 0 stores the cells that are not deferred (no cell
// within three rows touched at the start pose) and lists the deferred pairs;
// MODE 1 updates every cell of the instances with defer_all on the general
// path, where a row step whose three rows lie inside the grid and hold only
// plain fluid cells (warp-uniform ballot) still takes the plain arithmetic.
constexpr int YCOLS_P = 64;
template <int MINB, int MODE>
__global__ void __launch_bounds__(128, MINB) k_bulk_y_p(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                     const BandRec *__restrict__ R, int n_inst, int total_warps,
                                                     int src, int dst, int last, DeferList dl) {
    extern __shared__ __align__(16) unsigned char ysm[];
    constexpr bool gen = MODE != 0;
    const int lane = threadIdx.x & 31;
    YRing &rg = ((YRing *)ysm)[threadIdx.x >> 5];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_warps) return;
    const int inst = find_inst_warp(D, n_inst, gw, 1);
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if ((MODE == 0) == (y.defer_all != 0)) return;
    const int local = gw - I.tile_off[1];
    const int ncg = I.tiles_x[1];
    const int cg = local % ncg, sg = local / ncg;
    const int col0 = cg * YCOLS_P;
    const int i = col0 + 2 * lane;     // columns i, i+1 of this thread
    const int nx = I.nx, pitch = I.pitch;
    const int st0 = (i < nx ? 1 : 0) | (i + 1 < nx ? 2 : 0);
    const int n = I.ny;
    const int j0 = sg * I.yseg, j1 = min(n, j0 + I.yseg);
    const float lam = y.lamf;
    const float g = (float)I.gamma, g1 = g - 1.0f;
    const size_t plane = (size_t)pitch * n;
    const float *__restrict__ Q = (const float *)I.Q[src];
    float *__restrict__ Qo = (float *)I.Q[dst];
    const int bclo = I.bc[2], bchi = I.bc[3];
    if (MODE == 0 && bclo != 2 && !(col0 <= y.col1 && col0 + YCOLS_P - 1 >= y.col0 && j1 + 3 >= y.row0 &&
                                    j0 - 3 <= y.row1)) {
        // a tile the body cannot reach: plain throughout
        float s0 = 0.0f, s1 = 0.0f;
        bulk_y_far(I, y, rg, Q, Qo, i, st0, j0, j1, plane, lam, g, g1, last != 0, s0, s1);
        finish_warp<float>(y, last != 0, s0, s1);
        return;
    }
    const unsigned char *__restrict__ cl = I.cls;
    const bool cls_lane = lane < 16 && col0 + 4 * lane < pitch;
    // validity mask of this lane's class pair for the plain-path test
    const int vm = st0 == 3 ? 0x0505 : (st0 == 1 ? 0x0005 : 0);
    // copies of row r (a ghost row of the boundary condition outside [0, n))
    // into its slot; rows past j1 + 2 are not needed (one commit group per call)
    auto prefetch = [&](int r) {
        if (r <= j1 + 2) {
            const int s = (r - j0 + 2) & (YR - 1);
            int p = r;
            if (r < 0 || r >= n) {
                bool fl;
                p = ghost_map(r, n, bclo, bchi, &fl);
            }
            const float *src_q = Q + (size_t)p * pitch + i;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (st0 == 3) cp_async8(&rg.q[s][k][2 * lane], src_q + k * plane);
                else if (st0 == 1) cp_async4(&rg.q[s][k][2 * lane], src_q + k * plane);
            }
            if (cls_lane) cp_async4(&rg.cls[s][4 * lane], cl + (size_t)p * pitch + col0 + 4 * lane);
        }
        cp_async_commit();
    };
    // the pair of row r from the ring; columns past the grid read as solid,
    // ghost rows of a reflective side flip the normal momentum
    auto row = [&](int r, S2 &v, int &cls) {
        const int s = (r - j0 + 2) & (YR - 1);
#pragma unroll
        for (int k = 0; k < 4; ++k) v.q[k] = *(const float2 *)&rg.q[s][k][2 * lane];
        cls = *(const unsigned short *)&rg.cls[s][2 * lane];
        if (st0 != 3) {
            if (!(st0 & 1)) {
                cls = (cls & 0xff00) | CLS_SOLID;
#pragma unroll
                for (int k = 0; k < 4; ++k) v.q[k].x = 1.0f;
            }
            cls = (cls & 0xff) | (CLS_SOLID << 8);
#pragma unroll
            for (int k = 0; k < 4; ++k) v.q[k].y = 1.0f;
        }
        if ((r < 0 && bclo == 1) || (r >= n && bchi == 1)) {
            v.q[2].x = -v.q[2].x;
            v.q[2].y = -v.q[2].y;
        }
    };
    // touched bits (start pose) of row r's two cells, from the ring; rows
    // outside -2 .. n + 1 count as clear
    auto touch_bits = [&](int r) {
        if (r < -2 || r > n + 1) return 0;
        const int c = *(const unsigned short *)&rg.cls[(r - j0 + 2) & (YR - 1)][2 * lane];
        return ((st0 & 1) && (c & CLS_TOUCH) ? 1 : 0) | ((st0 & 2) && ((c >> 8) & CLS_TOUCH) ? 2 : 0);
    };
    for (int r = j0 - 2; r < j0 - 2 + YR; ++r) prefetch(r);
    cp_async_wait<YR - 4>();   // rows j0-2 .. j0+1 complete
    __syncwarp();
    // history of touched bits per column (bit 0: the newest row); row j0-3
    // comes straight from global memory
    unsigned h0 = 0u, h1 = 0u;
    // touched cells lie inside the body's extent over the sweep's poses
    // (k_pose): a tile whose columns miss it, or whose rows are more than
    // three rows away, holds no deferred cell (not across a periodic side)
    const bool tile_near = !gen && (bclo == 2 || (col0 <= y.col1 && col0 + YCOLS_P - 1 >= y.col0 &&
                                                 j1 + 3 >= y.row0 && j0 - 3 <= y.row1));
    if (tile_near) {
        const int r = j0 - 3;
        if (r >= -2) {
            bool fl;
            const int p = (r < 0 || r >= n) ? ghost_map(r, n, bclo, bchi, &fl) : r;
            const unsigned char *cp = cl + (size_t)p * pitch + i;
            h0 = (st0 & 1) && (cp[0] & CLS_TOUCH) ? 1u : 0u;
            h1 = (st0 & 2) && (cp[1] & CLS_TOUCH) ? 1u : 0u;
        }
        for (int q = j0 - 2; q <= j0 + 1; ++q) {
            const int b = touch_bits(q);
            h0 = (h0 << 1) | (b & 1);
            h1 = (h1 << 1) | (b >> 1);
        }
    }
    E2 QRc;
    {
        S2 qa, qm, qc;
        int ca, cm, cc;
        row(j0 - 2, qa, ca);
        row(j0 - 1, qm, cm);
        row(j0, qc, cc);
        const bool lx = !gen || (!(ca & CLS_SOLID) && !(cc & CLS_SOLID));
        const bool ly = !gen || (!((ca >> 8) & CLS_SOLID) && !((cc >> 8) & CLS_SOLID));
        E2 QL;
        evolve2<1>(g1, lam, qa.q, qm.q, qc.q, lx, ly, QL, QRc);
    }
    float s0 = 0.0f, s1 = 0.0f;
    float2 Fprev[4];
    float *__restrict__ wp = Qo + (size_t)(j0 - 1) * pitch + i;   // row f-1 of this lane's columns
    for (int f = j0; f <= j1; ++f, wp += pitch) {
        __syncwarp();
        prefetch(f + YR - 2);
        cp_async_wait<YR - 4>();   // rows up to f + 2 complete
        __syncwarp();
        const int sm_ = (f - j0 + 1) & (YR - 1), sc = (f - j0 + 2) & (YR - 1), sp = (f - j0 + 3) & (YR - 1);
        const int cm = *(const unsigned short *)&rg.cls[sm_][2 * lane];
        // cells of row f-1 this pass stores; mode 0 lists the deferred pairs
        // (touched cells in rows f-4 .. f+2) and keeps the others
        int sm = st0;
        if (tile_near) {
            const int b = touch_bits(f + 2);
            h0 = (h0 << 1) | (b & 1);
            h1 = (h1 << 1) | (b >> 1);
            if (f > j0) {
                const int dp = (((h0 & 0x7Fu) ? 1 : 0) | ((h1 & 0x7Fu) ? 2 : 0)) & st0;
                defer_push(dl, y, inst, (f - 1) * pitch + i, dp);
                sm = st0 & ~dp;
            }
        }
        const int sol = ((cm & CLS_SOLID) ? 1 : 0) | (((cm >> 8) & CLS_SOLID) ? 2 : 0);
        const bool inside = f >= 1 && f + 1 < n;
        bool plain = true;
        if (gen) {
            const int cc = *(const unsigned short *)&rg.cls[sc][2 * lane];
            const int cp = *(const unsigned short *)&rg.cls[sp][2 * lane];
            plain = __all_sync(0xffffffffu, !((cm | cc | cp) & vm)) && inside;
        }
        float2 F[4];
        E2 QR;
        if (plain) {
            // rows f-1, f, f+1 (lanes past the grid compute on values that
            // are never stored)
            float2 qm[4], qc[4], qp[4];
            if (inside) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qm[k] = *(const float2 *)&rg.q[sm_][k][2 * lane];
                    qc[k] = *(const float2 *)&rg.q[sc][k][2 * lane];
                    qp[k] = *(const float2 *)&rg.q[sp][k][2 * lane];
                }
            } else {
                S2 vm_, vc, vp;
                int c_;
                row(f - 1, vm_, c_);
                row(f, vc, c_);
                row(f + 1, vp, c_);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qm[k] = vm_.q[k];
                    qc[k] = vc.q[k];
                    qp[k] = vp.q[k];
                }
            }
            E2 QL;
            evolve2<1>(g1, lam, qm, qc, qp, true, true, QL, QR);
            hllc2<1>(g, QRc, QL, F);
            if (f > j0 && __any_sync(0xffffffffu, sm != 0)) {
                float2 qn[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) qn[k] = fma2(P2(lam), sub2(Fprev[k], F[k]), qm[k]);
                const int sq = sm & sol;   // (mode 0) solid at both poses: NaN
                if (sq) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) qn[k] = make_float2((sq & 1) ? NAN : qn[k].x, (sq & 2) ? NAN : qn[k].y);
                }
                if (sm == 3) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) *(float2 *)(wp + k * plane) = qn[k];
                } else if (sm) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (sm & 1) wp[k * plane] = qn[k].x;
                        if (sm & 2) wp[k * plane + 1] = qn[k].y;
                    }
                }
                const int st = sm & ~sol;
                pair_checks(qn, st, (f - 1) * pitch + i, last != 0, g1, g, s0, s1, y);
            }
        } else {
            // rows f-1, f, f+1
            S2 qm, qc, qp;
            int cm2, cc2, cp2;
            row(f - 1, qm, cm2);
            row(f, qc, cc2);
            row(f + 1, qp, cp2);
            E2 QL;
            evolve2<1>(g1, lam, qm.q, qc.q, qp.q, !(cm2 & CLS_SOLID) && !(cp2 & CLS_SOLID),
                       !((cm2 >> 8) & CLS_SOLID) && !((cp2 >> 8) & CLS_SOLID), QL, QR);
            hllc2<1>(g, QRc, QL, F);
            if (st0 & 1) face_override<1>(I, R, i, f, n, (uint8_t)(cm2 & 0xff), (uint8_t)(cc2 & 0xff), F, 0);
            if (st0 & 2) face_override<1>(I, R, i + 1, f, n, (uint8_t)(cm2 >> 8), (uint8_t)(cc2 >> 8), F, 1);
            if (f > j0) {
                int st = 0;
                if ((sm & 1) && !((cm2 & 0xff) & CLS_OFF)) st |= 1;
                if ((sm & 2) && !(((cm2 >> 8) & 0xff) & CLS_OFF)) st |= 2;
                const int ci = (f - 1) * pitch + i;
                if (st) update2(Qo, plane, ci, st, st == 3, g1, g, lam, qm.q, Fprev, F, last, s0, s1, y);
                if ((sm & 1) && (cm2 & CLS_SOLID)) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) Qo[k * plane + ci] = NAN;
                }
                if ((sm & 2) && ((cm2 >> 8) & CLS_SOLID)) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) Qo[k * plane + ci + 1] = NAN;
                }
            }
        }
        QRc = QR;
#pragma unroll
        for (int k = 0; k < 4; ++k) Fprev[k] = F[k];
    }
    finish_warp<float>(y, last != 0, s0, s1);
}

// ---------------------------------------------------------------------------
// Geometric source of the axisymmetric Euler equations after a y sweep (a
// reading; Sec. III.E models its open-ended tube in axisymmetric form): with
// x axial and y the radius from the axis y = y0 = 0, every fluid cell gets
// Q -= dt (v / r) [rho, rho u, rho v, E + p], r at the cell centre.  One warp
// per grid row; instances of the batch without the flag return at once.  In
// FP64 every operation is rounded on its own (no contraction), in the order
// of the plain definition.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_axisym_source(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                       int n_inst, int total_warps, int buf) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_warps) return;
    const int inst = find_inst_warp(D, n_inst, gw, 0);
    const InstDesc &I = D[inst];
    if (!I.axisym || I.eq != 0) return;
    InstDyn &y = Y[inst];
    const int j = gw - I.tile_off[0];
    const size_t plane = (size_t)I.pitch * I.ny;
    T *__restrict__ Q = (T *)I.Q[buf] + (size_t)j * I.pitch;
    const double r = __dmul_rn(__dadd_rn((double)j, 0.5), I.dy);
    const double dt = y.dt;
    bool bad = false;
    for (int i = lane; i < I.nx; i += 32) {
        const T q0 = Q[i], q1 = Q[plane + i], q2 = Q[2 * plane + i], q3 = Q[3 * plane + i];
        if (!(q0 == q0)) continue;   // solid
        T n0, n1, n2, n3, pn;
        if (sizeof(T) == 8) {
            const double g1 = __dsub_rn(I.gamma, 1.0);
            const double p = __dmul_rn(g1, __dsub_rn(q3, __ddiv_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(q1, q1),
                                                                                           __dmul_rn(q2, q2))), q0)));
            const double f = __ddiv_rn(__dmul_rn(dt, __ddiv_rn(q2, q0)), r);
            n0 = (T)__dsub_rn(q0, __dmul_rn(f, q0));
            n1 = (T)__dsub_rn(q1, __dmul_rn(f, q1));
            n2 = (T)__dsub_rn(q2, __dmul_rn(f, q2));
            n3 = (T)__dsub_rn(q3, __dmul_rn(f, __dadd_rn(q3, p)));
            pn = (T)__dmul_rn(g1, __dsub_rn(n3, __ddiv_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(n1, n1),
                                                                                  __dmul_rn(n2, n2))), n0)));
        } else {
            const float g1 = (float)I.gamma - 1.0f;
            const float p = g1 * (q3 - 0.5f * (q1 * q1 + q2 * q2) / q0);
            const float f = (float)dt * (q2 / q0) / (float)r;
            n0 = q0 - f * q0;
            n1 = q1 - f * q1;
            n2 = q2 - f * q2;
            n3 = q3 - f * (q3 + p);
            pn = g1 * (n3 - 0.5f * (n1 * n1 + n2 * n2) / n0);
        }
        Q[i] = n0;
        Q[plane + i] = n1;
        Q[2 * plane + i] = n2;
        Q[3 * plane + i] = n3;
        if (!(n0 > (T)0) || !(pn > (T)0)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&y.err, ERR_UNSTABLE);
}

template <class T>
void launch_axisym_source(const InstDesc *D, InstDyn *Y, int n_inst, int total_rows, int buf, cudaStream_t st) {
    if (total_rows > 0) k_axisym_source<T><<<(total_rows + 7) / 8, 256, 0, st>>>(D, Y, n_inst, total_rows, buf);
}

// ---------------------------------------------------------------------------
// FP64 rate probe (measurement support for the FP64 path's roofline): every
// thread runs eight independent chains of FP64 fused multiply-adds, enough
// warps resident to keep the FP64 pipe of every SM busy
// ---------------------------------------------------------------------------
constexpr int FP64_PROBE_CHAINS = 8;
__global__ void __launch_bounds__(256) k_fp64_probe(double *out, int iters, double a, double b) {
    double x[FP64_PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < FP64_PROBE_CHAINS; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < FP64_PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
    }
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < FP64_PROBE_CHAINS; ++k) r += x[k];
    if (r == 12345.678) out[blockIdx.x] = r;   // keeps the chains alive; never true for these inputs
}

// FP64 fused multiply-adds per second of k_fp64_probe on the current
// device (best of three timed launches after one warm-up), or < 0 on error
double fp64_probe_rate(cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(double) * blocks, st) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    k_fp64_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-6);
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        k_fp64_probe<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-6);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = (double)blocks * threads * FP64_PROBE_CHAINS * iters / (ms * 1e-3);
        if (rate > best) best = rate;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.0;
    return best;
}

// ---------------------------------------------------------------------------
// deferred bulk cells (FP32 Euler, after the band fluxes): one thread per
// listed cell pair, the general path of the streaming kernels for its two
// cells (same functions on the same inputs, so the same bits): MUSCL-Hancock
// states of the cells around the pair, their HLLC fluxes, stabilised fluxes of
// faces touching a band cell, the update of the listed cells
// ---------------------------------------------------------------------------

// state and class of cell b of a line through the ring-free path: real and
// ghost cells (-2 .. n+1) from global memory, filler beyond
__device__ __forceinline__ void def_cell(const float *__restrict__ Q, const unsigned char *__restrict__ cl,
                                         size_t plane, int n, int stride, int comp_flip, int bclo, int bchi, int b,
                                         float *w, int &cb) {
    if (b >= -2 && b <= n + 1) {
        bool fl;
        const int p = ghost_map(b, n, bclo, bchi, &fl);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = __ldg(Q + k * plane + (size_t)p * stride);
        if (fl) w[comp_flip] = -w[comp_flip];
        cb = cl[(size_t)p * stride];
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = 1.0f;
        cb = CLS_SOLID;
    }
}

// wave speeds of a thread into its instance: one atomic per warp when the
// warp's threads share the instance
__device__ __forceinline__ void def_wave_speeds(InstDyn *__restrict__ Y, int inst, bool act, float s0, float s1) {
    const unsigned am = __activemask();
    const int i0 = __shfl_sync(am, inst, __ffs(am) - 1);
    if (__all_sync(am, inst == i0)) {
        for (int o = 16; o > 0; o >>= 1) {
            s0 = fmaxf(s0, __shfl_xor_sync(am, s0, o));
            s1 = fmaxf(s1, __shfl_xor_sync(am, s1, o));
        }
        if ((threadIdx.x & 31) == __ffs(am) - 1) {
            atomic_max_pos(&Y[i0].S[0], (double)s0);
            atomic_max_pos(&Y[i0].S[1], (double)s1);
        }
    } else if (act) {
        atomic_max_pos(&Y[inst].S[0], (double)s0);
        atomic_max_pos(&Y[inst].S[1], (double)s1);
    }
}

__global__ void __launch_bounds__(128, 5) k_bulk_def_x(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                    const BandRec *__restrict__ R, int src, int dst, int last,
                                                    DeferList dl) {
    const int cnt = min(*dl.count, dl.cap);
    const int stride = gridDim.x * blockDim.x;
    // whole warps iterate together (the wave-speed reduction is warp-wide)
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < cnt; base += stride) {
        const int t = base + (threadIdx.x & 31);
        const bool act = t < cnt;
        const int2 it = act ? dl.item[t] : dl.item[base];
        const int inst = it.x, ci = it.y & 0x0fffffff, bits = act ? (it.y >> 28) & 3 : 0;
        const InstDesc &I = D[inst];
        InstDyn &y = Y[inst];
        const int n = I.nx, j = ci / I.pitch, a = ci - j * I.pitch;
        const float lam = y.lamf;
        const float g = (float)I.gamma, g1 = g - 1.0f;
        const size_t plane = (size_t)I.pitch * I.ny;
        const int rowb = j * I.pitch;
        const float *Q = (const float *)I.Q[src] + rowb;
        float *Qb = (float *)I.Q[dst];
        const unsigned char *cl = I.cls + rowb;
        // cells a-2 .. a+3 (pairs of real cells as 8-byte loads)
        float w[6][4];
        int c[6];
        if (a >= 2 && a + 3 < n) {
#pragma unroll
            for (int m = 0; m < 6; m += 2) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 v = __ldg((const float2 *)(Q + k * plane + a - 2 + m));
                    w[m][k] = v.x;
                    w[m + 1][k] = v.y;
                }
                const unsigned short cc = __ldg((const unsigned short *)(cl + a - 2 + m));
                c[m] = cc & 0xff;
                c[m + 1] = cc >> 8;
            }
        } else {
#pragma unroll
            for (int m = 0; m < 6; ++m) def_cell(Q, cl, plane, n, 1, 1, I.bc[0], I.bc[1], a - 2 + m, w[m], c[m]);
        }
        // MUSCL-Hancock states of cells (a-1, a) and (a+1, a+2)
        float2 qm[4], q0[4], qp[4];
        E2 QLA, QRA, QLB, QRB;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = make_float2(w[0][k], w[1][k]);
            q0[k] = make_float2(w[1][k], w[2][k]);
            qp[k] = make_float2(w[2][k], w[3][k]);
        }
        evolve2<0>(g1, lam, qm, q0, qp, !(c[0] & CLS_SOLID) && !(c[2] & CLS_SOLID),
                   !(c[1] & CLS_SOLID) && !(c[3] & CLS_SOLID), QLA, QRA);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = make_float2(w[2][k], w[3][k]);
            q0[k] = make_float2(w[3][k], w[4][k]);
            qp[k] = make_float2(w[4][k], w[5][k]);
        }
        evolve2<0>(g1, lam, qm, q0, qp, !(c[2] & CLS_SOLID) && !(c[4] & CLS_SOLID),
                   !(c[3] & CLS_SOLID) && !(c[5] & CLS_SOLID), QLB, QRB);
        // faces a (cells a-1 | a), a+1 (a | a+1), a+2 (a+1 | a+2)
        E2 Rf, L2, R2;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Rf.q[k] = make_float2(QLA.q[k].y, QLB.q[k].x);
            L2.q[k] = P2(QRB.q[k].x);
            R2.q[k] = P2(QLB.q[k].y);
        }
        Rf.ir = make_float2(QLA.ir.y, QLB.ir.x);
        Rf.p = make_float2(QLA.p.y, QLB.p.x);
        L2.ir = P2(QRB.ir.x);
        L2.p = P2(QRB.p.x);
        R2.ir = P2(QLB.ir.y);
        R2.p = P2(QLB.p.y);
        float2 F[4], F2[4];
        hllc2<0>(g, QRA, Rf, F);
        hllc2<0>(g, L2, R2, F2);
        if (a <= n) face_override<0>(I, R, j, a, n, (uint8_t)c[1], (uint8_t)c[2], F, 0);
        if (a + 1 <= n) face_override<0>(I, R, j, a + 1, n, (uint8_t)c[2], (uint8_t)c[3], F, 1);
        if (a + 2 <= n) face_override<0>(I, R, j, a + 2, n, (uint8_t)c[3], (uint8_t)c[4], F2, 0);
        float2 Fhi[4], qc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Fhi[k] = make_float2(F[k].y, F2[k].x);
            qc[k] = make_float2(w[2][k], w[3][k]);
        }
        int st = 0;
        if ((bits & 1) && !(c[2] & CLS_OFF)) st |= 1;
        if ((bits & 2) && !(c[3] & CLS_OFF)) st |= 2;
        float s0 = 0.0f, s1 = 0.0f;
        if (st) update2(Qb, plane, rowb + a, st, st == 3, g1, g, lam, qc, F, Fhi, last, s0, s1, y);
        if ((bits & 1) && (c[2] & CLS_SOLID)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qb[k * plane + rowb + a] = NAN;
        }
        if ((bits & 2) && (c[3] & CLS_SOLID)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qb[k * plane + rowb + a + 1] = NAN;
        }
        if (last) def_wave_speeds(Y, inst, st != 0, s0, s1);
    }
}

__global__ void __launch_bounds__(128, 5) k_bulk_def_y(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                                    const BandRec *__restrict__ R, int src, int dst, int last,
                                                    DeferList dl) {
    const int cnt = min(*dl.count, dl.cap);
    const int stride = gridDim.x * blockDim.x;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < cnt; base += stride) {
        const int t = base + (threadIdx.x & 31);
        const bool act = t < cnt;
        const int2 it = act ? dl.item[t] : dl.item[base];
        const int inst = it.x, ci = it.y & 0x0fffffff, bits = act ? (it.y >> 28) & 3 : 0;
        const InstDesc &I = D[inst];
        InstDyn &y = Y[inst];
        const int n = I.ny, nx = I.nx, r = ci / I.pitch, i = ci - r * I.pitch;
        const int st0 = (i < nx ? 1 : 0) | (i + 1 < nx ? 2 : 0);
        const float lam = y.lamf;
        const float g = (float)I.gamma, g1 = g - 1.0f;
        const size_t plane = (size_t)I.pitch * n;
        const float *Q = (const float *)I.Q[src];
        float *Qo = (float *)I.Q[dst];
        // rows r-2 .. r+2 of columns i, i+1 (columns past the grid: filler)
        float2 w[5][4];
        int c[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const int rr = r - 2 + m;
            if (st0 == 3 && rr >= 0 && rr < n) {   // both columns real, a real row: 8-byte loads
                const size_t o = (size_t)rr * I.pitch + i;
#pragma unroll
                for (int k = 0; k < 4; ++k) w[m][k] = __ldg((const float2 *)(Q + k * plane + o));
                c[m] = __ldg((const unsigned short *)(I.cls + o));
                continue;
            }
            float a0[4], a1[4];
            int c0, c1;
            if (st0 & 1) def_cell(Q + i, I.cls + i, plane, n, I.pitch, 2, I.bc[2], I.bc[3], r - 2 + m, a0, c0);
            else { a0[0] = a0[1] = a0[2] = a0[3] = 1.0f; c0 = CLS_SOLID; }
            if (st0 & 2) def_cell(Q + i + 1, I.cls + i + 1, plane, n, I.pitch, 2, I.bc[2], I.bc[3], r - 2 + m, a1, c1);
            else { a1[0] = a1[1] = a1[2] = a1[3] = 1.0f; c1 = CLS_SOLID; }
#pragma unroll
            for (int k = 0; k < 4; ++k) w[m][k] = make_float2(a0[k], a1[k]);
            c[m] = c0 | (c1 << 8);
        }
        auto lims = [&](int m, bool &lx, bool &ly) {
            lx = !(c[m - 1] & CLS_SOLID) && !(c[m + 1] & CLS_SOLID);
            ly = !((c[m - 1] >> 8) & CLS_SOLID) && !((c[m + 1] >> 8) & CLS_SOLID);
        };
        E2 QL1, QR1, QL2, QR2, QL3, QR3;
        bool lx, ly;
        lims(1, lx, ly);
        evolve2<1>(g1, lam, w[0], w[1], w[2], lx, ly, QL1, QR1);
        lims(2, lx, ly);
        evolve2<1>(g1, lam, w[1], w[2], w[3], lx, ly, QL2, QR2);
        lims(3, lx, ly);
        evolve2<1>(g1, lam, w[2], w[3], w[4], lx, ly, QL3, QR3);
        float2 Flo[4], Fhi[4];
        hllc2<1>(g, QR1, QL2, Flo);
        hllc2<1>(g, QR2, QL3, Fhi);
        if (st0 & 1) {
            face_override<1>(I, R, i, r, n, (uint8_t)(c[1] & 0xff), (uint8_t)(c[2] & 0xff), Flo, 0);
            face_override<1>(I, R, i, r + 1, n, (uint8_t)(c[2] & 0xff), (uint8_t)(c[3] & 0xff), Fhi, 0);
        }
        if (st0 & 2) {
            face_override<1>(I, R, i + 1, r, n, (uint8_t)(c[1] >> 8), (uint8_t)(c[2] >> 8), Flo, 1);
            face_override<1>(I, R, i + 1, r + 1, n, (uint8_t)(c[2] >> 8), (uint8_t)(c[3] >> 8), Fhi, 1);
        }
        const int sm = bits & st0;
        int st = 0;
        if ((sm & 1) && !((c[2] & 0xff) & CLS_OFF)) st |= 1;
        if ((sm & 2) && !(((c[2] >> 8) & 0xff) & CLS_OFF)) st |= 2;
        float s0 = 0.0f, s1 = 0.0f;
        if (st) update2(Qo, plane, ci, st, st == 3, g1, g, lam, w[2], Flo, Fhi, last, s0, s1, y);
        if ((sm & 1) && (c[2] & CLS_SOLID)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qo[k * plane + ci] = NAN;
        }
        if ((sm & 2) && ((c[2] >> 8) & CLS_SOLID)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Qo[k * plane + ci + 1] = NAN;
        }
        if (last) def_wave_speeds(Y, inst, st != 0, s0, s1);
    }
}

template <class T, int EQ>
void bulk_attr_t(int dir) {
    if (dir == 0) cudaFuncSetAttribute(k_bulk_x<T, EQ>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    else cudaFuncSetAttribute(k_bulk_y<T, EQ>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}

// ---------------------------------------------------------------------------
// k_events: covering / uncovering, gathered by each band cell
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void events_rec(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                           BandRec *__restrict__ R, int n_inst, int r) {
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
    // only a covered or donor-uncovered cell and the neighbours k_band_prep
    // marked next to one exchange content
    const bool near_event = (x.flags & RF_COVER) || x_donor_unc || x.aux;
    for (int dj = near_event ? -1 : 2; dj <= 1; ++dj)
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
    // positivity check of the new state (in the path's type; the FP64 path
    // in FP64); a cell that kept less than MIX_COLLAPSE of its volume over
    // the sweep seeds the first merge as well (its state, content / alpha_B,
    // carries residuals of the order of its mid-pose volume)
    if (I.eq == 0 && x.aB > 0.0) {
        const T q0 = (T)(C[0] / x.aB), q1 = (T)(C[1] / x.aB), q2 = (T)(C[2] / x.aB), q3 = (T)(C[3] / x.aB);
        const T p = ((T)I.gamma - T(1)) * (q3 - T(0.5) * (q1 * q1 + q2 * q2) / q0);
        bool ok = q0 > T(0) && p > T(0) && isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(q3);
        if (x.aB < MIX_COLLAPSE * x.aA) ok = false;
        if (!ok) {
            x.flags |= RF_BAD;
            int k = atomicAdd(&y.nbad, 1);
            if (k < 16) y.badlist[k] = r;
        }
    }
}

template <class T>
__global__ void k_events(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                         const int *__restrict__ boff, int n_inst) {
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x;; t += stride) {
        const int r = band_rec_of(D, boff, n_inst, t);
        if (r < 0) break;
        events_rec<T>(D, Y, R, n_inst, r);
    }
}

// ---------------------------------------------------------------------------
// k_mix: positivity safeguard (a reading; the paper gives none): every cluster
// of non-physical cells and their fluid face neighbours shares its total
// content in proportion to volume.  One warp per instance; runs only when the
// instance flagged a bad cell.  Also advances the instance's clock.
//
// The cluster bookkeeping (union-find over the cells involved) lives in
// shared memory.  Every lane follows the same control flow on the same data;
// lane 0 writes the shared arrays, and the searches, the scans of the band
// records and the loads of the cluster members are spread over the lanes.
// Sums over a cluster run in cell order on every lane alike, so the result
// does not depend on the lanes.
// ---------------------------------------------------------------------------
constexpr int MIXCAP = 1024;
constexpr int MIX_SMEM = 2 * (1 + MAXC) * MIXCAP * (int)sizeof(double);   // k_mix's node cache and sums
constexpr int MIX_LAYERS = 8;   // merges per sweep (cells still non-physical seed the next)

template <class T>
__global__ void __launch_bounds__(32) k_mix(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                            BandRec *__restrict__ R, int n_inst, int dst, int sidx) {
    __shared__ int node[MIXCAP];   // cell of each node
    __shared__ int par[MIXCAP];    // union-find parent (node index), later the root's cell
    __shared__ int nxt[MIXCAP];    // seeds of the merge; scratch of the root pass
    __shared__ unsigned char nbm[MIXCAP];   // each seed's fluid face neighbours (bit m: neighbour m)
    // each node's volume fraction and content, read once per merge and
    // replaced by the merged content as it is written (dynamic, MIX_SMEM bytes)
    extern __shared__ double mixc[];
    double *vol_s = mixc, *cont_s = mixc + MIXCAP;   // cont_s[q * MIXCAP + node]
    double *acc_s = mixc + (1 + MAXC) * MIXCAP;      // cluster sums by slot: volume, then the components
    const int inst = blockIdx.x, lane = threadIdx.x;
    if (inst >= n_inst) return;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    const int nbad = y.nbad, nbulk = y.nbulk;
    __syncwarp();
    if (lane == 0) {
        // advance pose and clock
        y.X = y.XB;
        y.Y = y.YB;
        y.th = y.thB;
        if (sidx == 1) {
            y.t += y.dt;
            y.step += 1;
        }
    }
    if (nbad == 0 && nbulk == 0) return;
    if (nbulk > NBULK) {
        if (lane == 0) y.err |= ERR_UNSTABLE | ERR_MIX_CAP;
        return;
    }
    int nn = 0;   // nodes (the same on every lane)
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Qo = bufw<T>(I, dst);
    auto find_node = [&](int cell) -> int {
        for (int k0 = 0; k0 < nn; k0 += 32) {
            const int k = k0 + lane;
            const unsigned m = __ballot_sync(0xffffffffu, k < nn && node[k] == cell);
            if (m) return k0 + __ffs(m) - 1;
        }
        if (nn >= MIXCAP) return -1;
        if (lane == 0) {
            node[nn] = cell;
            par[nn] = nn;
        }
        __syncwarp();
        return nn++;
    };
    auto root = [&](int k) { while (par[k] != k) k = par[k]; return k; };
    auto alpha_B = [&](int c) -> double {
        const uint8_t cl = I.cls[c];
        return (cl & CLS_BAND) ? R[I.rec[c]].aB : ((cl & CLS_SOLID) ? 0.0 : 1.0);
    };
    const int dd[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    auto nbr = [&](int i, int j, int m, int &c) -> bool {
        int ii = i + dd[m][0], jj = j + dd[m][1];
        if (I.bc[0] == 2) { ii %= I.nx; if (ii < 0) ii += I.nx; }
        if (I.bc[2] == 2) { jj %= I.ny; if (jj < 0) jj += I.ny; }
        if (ii < 0 || ii >= I.nx || jj < 0 || jj >= I.ny) return false;
        c = jj * I.pitch + ii;
        return true;
    };
    // a non-physical cell joins the clusters of its fluid face neighbours
    // (msk: which of them are fluid, found beforehand)
    auto seed = [&](int cell, unsigned msk) -> bool {
        const int kb = find_node(cell);
        if (kb < 0) return false;
        const int i = cell % I.pitch, j = cell / I.pitch;
        for (int m = 0; m < 4; ++m) {
            int c;
            if (!((msk >> m) & 1u) || !nbr(i, j, m, c)) continue;
            const int kn = find_node(c);
            if (kn < 0) return false;
            const int ra = root(kb), rb = root(kn);
            if (ra != rb) {
                if (lane == 0) {
                    if (ra < rb) par[rb] = ra; else par[ra] = rb;
                }
                __syncwarp();
            }
        }
        return true;
    };
    // the ns seeds in nxt, in order; their neighbours' volume fractions are
    // looked up by all lanes at once (classes and records do not change here)
    auto seed_all = [&](int ns) -> bool {
        for (int q = lane; q < ns; q += 32) {
            const int c = nxt[q], i = c % I.pitch, j = c / I.pitch;
            unsigned msk = 0u;
            for (int m = 0; m < 4; ++m) {
                int cn;
                if (nbr(i, j, m, cn) && alpha_B(cn) > 0.0) msk |= 1u << m;
            }
            nbm[q] = (unsigned char)msk;
        }
        __syncwarp();
        for (int q = 0; q < ns; ++q)
            if (!seed(nxt[q], nbm[q])) return false;
        return true;
    };
    auto sort_int = [](int *v, int m) {
        for (int x = 1; x < m; ++x) {
            const int t = v[x];
            int z = x;
            while (z > 0 && v[z - 1] > t) { v[z] = v[z - 1]; --z; }
            v[z] = t;
        }
    };
    // physical state of node k's content after a merge (the cached values
    // are those written: a band cell's content, a bulk cell's state in the
    // path's type)
    auto physical = [&](int k) -> bool {
        double q[MAXC];
        if (I.cls[node[k]] & CLS_BAND) {
            const double aB = vol_s[k];
            if (!(aB > 0.0)) return true;
            for (int m = 0; m < I.nc; ++m) q[m] = cont_s[m * MIXCAP + k] / aB;
        } else {
            for (int m = 0; m < I.nc; ++m) q[m] = cont_s[m * MIXCAP + k];
        }
        const double pm = (I.gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
        return q[0] > 0.0 && pm > 0.0 && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
    };
    int nnext = 0;
    bool overflow = false;
    for (int layer = 0; layer < MIX_LAYERS; ++layer) {
        nn = 0;
        int ns = nnext;   // later merges: the cells still non-physical, in cell order
        if (layer == 0) {
            // flagged band records by cell, then listed bulk cells
            int seeds[16 + NBULK];
            int nl = 0;
            ns = 0;
            if (nbad <= 16) {
                for (int q = 0; q < nbad; ++q) seeds[nl++] = R[y.badlist[q]].cell;
                sort_int(seeds, nl);
                if (lane == 0)
                    for (int q = 0; q < nl; ++q) nxt[q] = seeds[q];
                ns = nl;
            } else {
                // every flagged record, in record order
                const int nrec = min(y.band_count, I.rec_cap);
                for (int q0 = 0; q0 < nrec; q0 += 32) {
                    const int q = q0 + lane;
                    const bool bad = q < nrec && (R[I.rec_base + q].flags & RF_BAD);
                    const unsigned m = __ballot_sync(0xffffffffu, bad);
                    const int at = ns + __popc(m & ((1u << lane) - 1u));
                    if (bad && at < MIXCAP) nxt[at] = R[I.rec_base + q].cell;
                    ns += __popc(m);
                }
            }
            nl = 0;
            for (int q = 0; q < nbulk; ++q) seeds[nl++] = y.bulkbad[q];
            sort_int(seeds, nl);
            if (lane == 0)
                for (int q = 0; q < nl && ns + q < MIXCAP; ++q) nxt[ns + q] = seeds[q];
            ns += nl;
            __syncwarp();
        }
        // more seeds than nodes fit: the merge would overflow
        overflow = ns > MIXCAP || !seed_all(ns);
        if (overflow) {
            if (lane == 0) y.err |= ERR_UNSTABLE | ERR_MIX_CAP;
            return;
        }
        __syncwarp();
        // nodes in cell order with the cell of their cluster root, so that the
        // cluster sums run in a fixed order
        for (int k = lane; k < nn; k += 32) nxt[k] = node[root(k)];
        __syncwarp();
        for (int k = lane; k < nn; k += 32) par[k] = nxt[k];
        __syncwarp();
        if (lane == 0) {
            for (int x = 1; x < nn; ++x) {
                const int c = node[x], r = par[x];
                int z = x;
                while (z > 0 && node[z - 1] > c) { node[z] = node[z - 1]; par[z] = par[z - 1]; --z; }
                node[z] = c;
                par[z] = r;
            }
        }
        __syncwarp();
        // every node's volume fraction and content, one read each
        for (int m = lane; m < nn; m += 32) {
            const int c = node[m];
            double vv = 1.0, cv[MAXC] = {0, 0, 0, 0};
            if (I.cls[c] & CLS_BAND) {
                const BandRec &bb = R[I.rec[c]];
                vv = bb.aB;
                for (int q = 0; q < I.nc; ++q) cv[q] = bb.C2[q];
            } else {
                for (int q = 0; q < I.nc; ++q) cv[q] = (double)Qo[q * plane + c];
            }
            vol_s[m] = vv;
            for (int q = 0; q < MAXC; ++q) cont_s[q * MIXCAP + m] = cv[q];
        }
        __syncwarp();
        // each node's cluster slot: the position of its root cell among the
        // nodes (sorted by cell); the slots' sums start at zero
        for (int m = lane; m < nn; m += 32) {
            const int rc = par[m];
            int lo = 0, hi = nn - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (node[mid] < rc) lo = mid + 1; else hi = mid;
            }
            nxt[m] = lo;
            for (int q = 0; q <= MAXC; ++q) acc_s[q * MIXCAP + m] = 0.0;
        }
        __syncwarp();
        // the cluster sums: every cluster's members added in cell order
        if (lane == 0) {
            for (int m = 0; m < nn; ++m) {
                const int r = nxt[m];
                acc_s[r] += vol_s[m];
                for (int q = 0; q < MAXC; ++q) acc_s[(q + 1) * MIXCAP + r] += cont_s[q * MIXCAP + m];
            }
        }
        __syncwarp();
        // each member's share, in proportion to its volume
        for (int m = lane; m < nn; m += 32) {
            const int r = nxt[m], c = node[m];
            const double vol = acc_s[r];
            if (I.cls[c] & CLS_BAND) {
                BandRec &bb = R[I.rec[c]];
                for (int q = 0; q < I.nc; ++q) {
                    const double v = bb.aB * (acc_s[(q + 1) * MIXCAP + r] / vol);
                    bb.C2[q] = v;
                    cont_s[q * MIXCAP + m] = v;
                }
            } else {
                for (int q = 0; q < I.nc; ++q) {
                    const T v = (T)(acc_s[(q + 1) * MIXCAP + r] / vol);
                    Qo[q * plane + c] = v;
                    cont_s[q * MIXCAP + m] = (double)v;
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            y.mixed += nn;
            y.mixed_total += nn;
        }
        // cells still non-physical, in cell order
        nnext = 0;
        for (int k0 = 0; k0 < nn; k0 += 32) {
            const int k = k0 + lane;
            const bool bad = k < nn && !physical(k);
            const unsigned m = __ballot_sync(0xffffffffu, bad);
            if (bad) nxt[nnext + __popc(m & ((1u << lane) - 1u))] = node[k];
            nnext += __popc(m);
        }
        __syncwarp();
        if (nnext == 0) return;
    }
    // still non-physical after the last merge
    if (lane == 0) y.err |= ERR_UNSTABLE | ERR_MIX_BULK;
}

// ---------------------------------------------------------------------------
// k_finalize: new state of band cells, class bytes of the end pose
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ bool finalize_rec(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y,
                                             BandRec *__restrict__ R, int n_inst, int r, int dst, int last,
                                             double &s0, double &s1, int &inst_out) {
    int inst = find_inst_rec(D, n_inst, r);
    inst_out = inst;
    const InstDesc &I = D[inst];
    InstDyn &y = Y[inst];
    if (r - I.rec_base >= y.band_count) return false;
    BandRec &b = R[r];
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Qo = bufw<T>(I, dst);
    if (b.aB > 0.0) {
        // the state divides the content by the volume fraction in FP64; the
        // positivity check and the wave speeds run in the path's type (on
        // GB300 every FP64 instruction takes the narrow FP64 pipe)
        T q[MAXC];
        for (int k = 0; k < I.nc; ++k) {
            q[k] = (T)(b.C2[k] / b.aB);
            Qo[k * plane + b.cell] = q[k];
        }
        if (I.eq == 0) {
            const T g = (T)I.gamma;
            T p = (g - T(1)) * (q[3] - T(0.5) * (q[1] * q[1] + q[2] * q[2]) / q[0]);
            bool ok = q[0] > T(0) && p > T(0) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
            if (!ok) atomicOr(&y.err, ERR_UNSTABLE | ERR_MIX_BAND);
            if (last) {
                T c = tsqrt(g * p / q[0]);
                s0 = (double)(fabs(q[1] / q[0]) + c);
                s1 = (double)(fabs(q[2] / q[0]) + c);
                // non-finite or negative speeds force the smallest step
                if (!(s0 >= 0.0)) s0 = 1e300;
                if (!(s1 >= 0.0)) s1 = 1e300;
            }
        } else if (last) {
            s0 = fabs(I.adv[0]);
            s1 = fabs(I.adv[1]);
        }
    } else {
        for (int k = 0; k < I.nc; ++k) Qo[k * plane + b.cell] = T(NAN);
    }
    const bool tB = (b.flags & RF_TOUCH_B) != 0;
    I.cls[b.cell] = (uint8_t)((b.aB == 0.0 ? CLS_SOLID : 0) | (tB && b.aB > 0.0 ? CLS_CUT : 0) | (tB ? CLS_TOUCH : 0) |
                              ((b.flags & RF_MOV_B) ? CLS_MOVT : 0));
    I.alpha[b.cell] = b.aB;
    I.rec[b.cell] = -1;
    return true;
}

template <class T>
__global__ void k_finalize(const InstDesc *__restrict__ D, InstDyn *__restrict__ Y, BandRec *__restrict__ R,
                           const int *__restrict__ boff, int n_inst, int dst, int last) {
    const int total = boff[n_inst], stride = gridDim.x * blockDim.x;
    // whole warps iterate together (the wave-speed reduction is warp-wide)
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < total; base += stride) {
        const int r = band_rec_of(D, boff, n_inst, base + (threadIdx.x & 31));
        double s0 = 0.0, s1 = 0.0;
        int inst = -1;
        const bool act = r >= 0 && finalize_rec<T>(D, Y, R, n_inst, r, dst, last, s0, s1, inst);
        if (last) warp_max_to(Y, act, inst, s0, s1);
    }
}

// ---------------------------------------------------------------------------
// state initialisation and the CFL wave speeds of a state; state read-back.
// One CTA per STATE_ROWS rows of one instance (instance inst0 + blockIdx.y),
// threads along the row; the FP64 host layout lives in a device staging
// buffer (one per instance, or one per batch with a pointer per instance).
// ---------------------------------------------------------------------------
constexpr int STATE_ROWS = 8;
constexpr int STATE_THREADS = 128;

// Sources: srcs[blockIdx.y] (srcs != nullptr; a null entry skips that
// instance) or src1.  The first step's wave speeds are the FP64 maxima over
// the stored (T-rounded) states.  With T = float each cell's speeds are
// first formed in FP32; a cell goes through the FP64 formula only if one of
// its FP32 speeds comes within 1e-4 of the largest the thread has seen, or
// if its pressure is small against its energy (p <= E/20, where the FP32
// error could exceed 1e-5), and its state differs from the last state the
// thread took through the FP64 formula.  Elsewhere the FP32 speeds are
// within 1e-5 of the FP64 ones, so no skipped cell can hold the maximum,
// and the result is that of the FP64 formula over every cell.  H: the
// element type of the host layout (FP64 or FP32 states).
template <class T, class H>
__global__ void __launch_bounds__(STATE_THREADS) k_write_state(const InstDesc *__restrict__ D,
                                                               InstDyn *__restrict__ Y,
                                                               const H *const *__restrict__ srcs,
                                                               const H *__restrict__ src1, int inst0, int b) {
    const int inst = inst0 + blockIdx.y;
    const H *__restrict__ Qh = srcs ? srcs[blockIdx.y] : src1;
    if (!Qh) return;
    const InstDesc &I = D[inst];
    const int j0 = blockIdx.x * STATE_ROWS;
    if (j0 >= I.ny) return;
    const size_t n = (size_t)I.nx * I.ny;
    const size_t plane = (size_t)I.pitch * I.ny;
    T *Q = bufw<T>(I, b);
    const float gf = (float)I.gamma;
    float m0 = -1.0f, m1 = -1.0f;   // FP32 maxima of the trusted cells (T = float)
    unsigned lq[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};   // last state taken in FP64
    double s0 = 0.0, s1 = 0.0;
    bool fluid = false;
    const int j1 = min(j0 + STATE_ROWS, I.ny);
    for (int j = j0; j < j1; ++j) {
        for (int i = threadIdx.x; i < I.nx; i += STATE_THREADS) {
            const int c = j * I.pitch + i;
            const size_t e = (size_t)j * I.nx + i;
            const bool solid = I.cls[c] & CLS_SOLID;
            T q[MAXC] = {T(0), T(0), T(0), T(0)};
            for (int k = 0; k < I.nc; ++k) {
                q[k] = (T)Qh[k * n + e];
                Q[k * plane + c] = solid ? T(NAN) : q[k];
            }
            if (solid) continue;
            fluid = true;
            if (I.eq == 0) {
                bool exact = true;
                if (sizeof(T) == 4) {
                    const float r = (float)q[0], u = (float)q[1], v = (float)q[2], E = (float)q[3];
                    const unsigned b[4] = {__float_as_uint(r), __float_as_uint(u), __float_as_uint(v),
                                           __float_as_uint(E)};
                    const bool same = b[0] == lq[0] && b[1] == lq[1] && b[2] == lq[2] && b[3] == lq[3];
                    const float pf = (gf - 1.0f) * (E - 0.5f * (u * u + v * v) / r);
                    const bool trusted = r > 0.0f && pf > 0.05f * E && isfinite(pf) && isfinite(u) && isfinite(v);
                    if (trusted) {
                        const float cf = sqrtf(gf * pf / r);
                        const float f0 = fabsf(u / r) + cf, f1 = fabsf(v / r) + cf;
                        exact = f0 >= m0 * (1.0f - 1e-4f) || f1 >= m1 * (1.0f - 1e-4f);
                        m0 = fmaxf(m0, f0);
                        m1 = fmaxf(m1, f1);
                    }
                    exact = exact && !same;
                    if (exact)
                        for (int k = 0; k < 4; ++k) lq[k] = b[k];
                }
                if (exact) {
                    const double d0 = (double)q[0], d1 = (double)q[1], d2 = (double)q[2], d3 = (double)q[3];
                    const double p = (I.gamma - 1.0) * (d3 - 0.5 * (d1 * d1 + d2 * d2) / d0);
                    const double c2 = sqrt(I.gamma * p / d0);
                    s0 = fmax(s0, fabs(d1 / d0) + c2);
                    s1 = fmax(s1, fabs(d2 / d0) + c2);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 = fmax(s0, __shfl_xor_sync(0xffffffffu, s0, o));
        s1 = fmax(s1, __shfl_xor_sync(0xffffffffu, s1, o));
    }
    fluid = __any_sync(0xffffffffu, fluid);
    if ((threadIdx.x & 31) == 0 && fluid) {
        // advection: the constant speeds
        atomic_max_pos(&Y[inst].S[0], I.eq == 0 ? s0 : fabs(I.adv[0]));
        atomic_max_pos(&Y[inst].S[1], I.eq == 0 ? s1 : fabs(I.adv[1]));
    }
}

// Destinations: dsts[blockIdx.y] (null entry: skip) or dst1; nc planes of
// nx*ny values of type H (FP64 or FP32), solid cells NaN.
template <class T, class H>
__global__ void __launch_bounds__(STATE_THREADS) k_read_state(const InstDesc *__restrict__ D,
                                                              H *const *__restrict__ dsts,
                                                              H *__restrict__ dst1, int inst0, int b) {
    const int inst = inst0 + blockIdx.y;
    H *__restrict__ out = dsts ? dsts[blockIdx.y] : dst1;
    if (!out) return;
    const InstDesc &I = D[inst];
    const int j0 = blockIdx.x * STATE_ROWS;
    if (j0 >= I.ny) return;
    const size_t n = (size_t)I.nx * I.ny;
    const size_t plane = (size_t)I.pitch * I.ny;
    const T *Q = buf<T>(I, b);
    const int j1 = min(j0 + STATE_ROWS, I.ny);
    for (int j = j0; j < j1; ++j)
        for (int i = threadIdx.x; i < I.nx; i += STATE_THREADS)
            for (int k = 0; k < I.nc; ++k)
                out[k * n + (size_t)j * I.nx + i] = (H)Q[k * plane + (size_t)j * I.pitch + i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// stage 0 first counts the sweep's used band records (boff, n_inst + 1
// ints); the record kernels then run grid-stride over those only
template <class T>
void launch_band_stage(int stage, const InstDesc *D, InstDyn *Y, BandRec *R, const double *bnd, int *boff, int n_inst,
                       int total_rec, int dir, int src, int dst, int qn, int sidx, int last, cudaStream_t st) {
    constexpr int BAND_BLOCKS = 1216;   // 8 CTAs of 128 threads per SM
    const int blocks = std::min((total_rec + 127) / 128, BAND_BLOCKS);
    switch (stage) {
        case 0:
            if (!blocks) break;
            if ((size_t)(n_inst + 1) * sizeof(int) <= 32768) {
                k_band_prep_o<T><<<blocks, 128, (n_inst + 1) * sizeof(int), st>>>(D, Y, R, boff, n_inst, dir, src, qn);
            } else {
                k_band_offsets<<<1, 256, 0, st>>>(D, Y, n_inst, boff);
                k_band_prep<T><<<blocks, 128, 0, st>>>(D, Y, R, boff, n_inst, dir, src, qn);
            }
            break;
        case 1: if (blocks) k_band_sweep<T><<<blocks, 128, 0, st>>>(D, Y, R, bnd, boff, n_inst, dir, src); break;
        case 2: if (blocks) k_events<T><<<blocks, 128, 0, st>>>(D, Y, R, boff, n_inst); break;
        case 3: k_mix<T><<<n_inst, 32, MIX_SMEM, st>>>(D, Y, R, n_inst, dst, sidx); break;
        case 4: if (blocks) k_finalize<T><<<blocks, 128, 0, st>>>(D, Y, R, boff, n_inst, dst, last); break;
    }
}

// bulk passes of one sweep.  FP32 Euler (the FP32x2 kernels): mode 0 is the
// pass over the cells that need no band data (it lists the deferred cell
// pairs in dl), mode 1 the deferred pairs and, when any instance may have
// defer_all (any_defer_all), the streaming pass over those instances.  Other
// kernels: one pass, launched for mode 0 only.
template <class T>
void launch_bulk(int dir, int eq, const InstDesc *D, InstDyn *Y, const BandRec *R, int n_inst, int total_warps,
                 int src, int dst, int last, int shape, int mode, DeferList dl, int any_defer_all, cudaStream_t st) {
    const int cta = shape & 1023;
    const int wpc = cta / 32;   // warps per CTA of the FP32x2 kernels
    int blocks = (total_warps + 7) / 8;
    if (blocks <= 0) return;
    const bool packed = sizeof(T) == 4 && eq == 0;   // FP32 Euler: the FP32x2 kernels
    if (!packed && mode != 0) return;
    const int pg = (total_warps + wpc - 1) / wpc;
    const bool m4 = (shape & SHAPE_MINB4) != 0, r8 = (shape & SHAPE_RING8) != 0;
    constexpr int DEF_BLOCKS = 760;   // 5 resident CTAs of 128 threads per SM, grid-stride over the list
    if (dir == 0) {
        if (packed) {
            const size_t sm = wpc * (r8 ? sizeof(XRing<8>) : sizeof(XRing<4>));
            if (mode == 1) {
                k_bulk_def_x<<<DEF_BLOCKS, 128, 0, st>>>(D, Y, R, src, dst, last, dl);
                if (any_defer_all)
                    k_bulk_x_p<4, 4, 1><<<pg, cta, wpc * sizeof(XRing<4>), st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            } else if (m4 && r8) k_bulk_x_p<4, 8, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            else if (m4) k_bulk_x_p<4, 4, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            else if (r8) k_bulk_x_p<5, 8, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            else k_bulk_x_p<5, 4, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
        } else if (eq == 0) k_bulk_x<T, 0><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
        else k_bulk_x<T, 1><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
    } else {
        if (packed) {
            const size_t sm = wpc * sizeof(YRing);
            if (mode == 1) {
                k_bulk_def_y<<<DEF_BLOCKS, 128, 0, st>>>(D, Y, R, src, dst, last, dl);
                if (any_defer_all)
                    k_bulk_y_p<4, 1><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            } else if (m4) k_bulk_y_p<4, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
            else k_bulk_y_p<5, 0><<<pg, cta, sm, st>>>(D, Y, R, n_inst, total_warps, src, dst, last, dl);
        } else if (eq == 0) k_bulk_y<T, 0><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
        else k_bulk_y<T, 1><<<blocks, 256, 0, st>>>(D, Y, R, n_inst, total_warps, src, dst, last);
    }
}

template <class T>
int bulk_blocks_per_sm(int dir) {
    cudaFuncSetAttribute(k_mix<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MIX_SMEM);
    bulk_attr_t<T, 0>(dir);
    bulk_attr_t<T, 1>(dir);
    if (sizeof(T) == 4) {   // the FP32x2 kernels' shared-memory rings (4 warps per CTA at most)
        if (dir == 0) {
            const int s4 = (int)(4 * sizeof(XRing<4>)), s8 = (int)(4 * sizeof(XRing<8>));
            cudaFuncSetAttribute(k_bulk_x_p<5, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4);
            cudaFuncSetAttribute(k_bulk_x_p<4, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4);
            cudaFuncSetAttribute(k_bulk_x_p<5, 8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8);
            cudaFuncSetAttribute(k_bulk_x_p<4, 8, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8);
            cudaFuncSetAttribute(k_bulk_x_p<4, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4);
        } else {
            const int sy = (int)(4 * sizeof(YRing));
            cudaFuncSetAttribute(k_bulk_y_p<5, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
            cudaFuncSetAttribute(k_bulk_y_p<4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
            cudaFuncSetAttribute(k_bulk_y_p<4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sy);
        }
    }
    return 1;
}

// instances inst0 .. inst0+ninst-1 (max_ny: their largest ny); per-instance
// pointers in the device array ptrs, or one pointer p1 (ninst == 1)
template <class T, class H>
void launch_write_state(const InstDesc *D, InstDyn *Y, const H *const *ptrs, const H *p1, int inst0, int ninst,
                        int max_ny, int b, cudaStream_t st) {
    const dim3 grid((max_ny + STATE_ROWS - 1) / STATE_ROWS, ninst);
    if (ninst > 0 && max_ny > 0) k_write_state<T, H><<<grid, STATE_THREADS, 0, st>>>(D, Y, ptrs, p1, inst0, b);
}
template <class T, class H>
void launch_read_state(const InstDesc *D, H *const *ptrs, H *p1, int inst0, int ninst, int max_ny, int b,
                       cudaStream_t st) {
    const dim3 grid((max_ny + STATE_ROWS - 1) / STATE_ROWS, ninst);
    if (ninst > 0 && max_ny > 0) k_read_state<T, H><<<grid, STATE_THREADS, 0, st>>>(D, ptrs, p1, inst0, b);
}

#define MB_INST(T)                                                                                                \
    template void launch_band_stage<T>(int, const InstDesc *, InstDyn *, BandRec *, const double *, int *,          \
                                       int, int, int, int, int, int, int, int, cudaStream_t);                     \
    template void launch_bulk<T>(int, int, const InstDesc *, InstDyn *, const BandRec *, int, int, int, int, int,  \
                                 int, int, DeferList, int, cudaStream_t);                                               \
    template int bulk_blocks_per_sm<T>(int);                                                                       \
    template void launch_axisym_source<T>(const InstDesc *, InstDyn *, int, int, int, cudaStream_t);               \
    template void launch_write_state<T, double>(const InstDesc *, InstDyn *, const double *const *, const double *, \
                                                int, int, int, int, cudaStream_t);                                 \
    template void launch_write_state<T, float>(const InstDesc *, InstDyn *, const float *const *, const float *,    \
                                               int, int, int, int, cudaStream_t);                                  \
    template void launch_read_state<T, double>(const InstDesc *, double *const *, double *, int, int, int, int,    \
                                               cudaStream_t);                                                      \
    template void launch_read_state<T, float>(const InstDesc *, float *const *, float *, int, int, int, int,       \
                                              cudaStream_t);
MB_INST(float)
MB_INST(double)

}  // namespace mb
