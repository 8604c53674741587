// kernels_struct.cu -- the persistent engine on the slack-structured form of
// the explicit inverse (engine LP_ENGINE_STRUCTURED).
//
// Let R be the constraint rows whose slack is nonbasic and k = |R|.  With the
// basis columns ordered as structurals then slacks, B = [[A_RJ, 0], [A_SJ, I]]
// and B^-1 = [[A_RJ^-1, 0], [-A_SJ A_RJ^-1, I]]: every column of B^-1 that
// belongs to a row with a basic slack s is the unit vector e_pos(s), and
// y = c_B^T B^-1 is zero on those rows (c_s = 0).  Step 8's update keeps this
// exactly: for such a column rho_s = 0, so B^-1[i][s] - alpha_i * 0 is
// unchanged, and when the slack of row e enters, its column becomes
// B^-1[i][e] - alpha_i * (rho_e / alpha_r) = alpha_i - alpha_i * 1 = 0 off row r
// and y_e + d_q * 1 = y_e - y_e = 0.  The method of Section 2.1 therefore only
// ever changes k columns of B^-1 and k entries of y, and
//   PRICE   d_j = c_j - sum_{i in R} y_i A_ij                       (k n FMAs)
//   FTRAN   alpha_i = sum_{i' in R} B^-1[i][i'] a_q[i'] + a_q[s_i]   (k m FMAs)
//           where s_i is the row of the slack basic at position i, if any
//   UPDATE  B^-1[i][R] -= alpha_i rho_R / alpha_r                    (k m FMAs)
// compute the same quantities as the dense (m + n) m work per pivot, up to the
// order in which the nonzero terms of each sum are added.
//
// Layout: constraint rows live in "slots" (a permutation kept in slot_row /
// row_slot); the rows of R occupy slots [0, k).  A_p holds A with its rows in
// slot order (column-major like A_cm), bp holds the B^-1 columns of the live
// slots (row-major, column t = slot t), yp holds y in slot order.  A pivot
// changes R by at most one row in and one row out:
//   the leaving variable is the slack of row `join`: its row moves to slot k
//     (swapped with the row there) and k grows; its new B^-1 column is
//     e_r - (alpha - e_r) / alpha_r, i.e. the update formula applied to the
//     old unit column e_r with rho = 1;
//   the entering variable is the slack of row `ent`: its column becomes e_r
//     and is dropped; the last live slot moves into its place and k shrinks.
// A_p rows, the slot maps, yp and rho move with the slots; the slot maps are
// double-buffered (read the current copy, write the next) so that no CTA reads
// a map entry another CTA is changing.
//
// The kernel is k_iterate's phase structure (grid barriers between (1) the
// pivot's vectors and bookkeeping, (2) PRICE + CHUZC, (3) UPDATE + FTRAN +
// ratios, (4) CHUZR) over the live slots only.  Reinversion stays the dense
// structure-aware rebuild; k_struct_layout / k_struct_gather_* then gather the
// live columns of the rebuilt B^-1 into bp.
#include "lpgb_internal.cuh"
#include "iter_common.cuh"
#include "../../include/lpgb.h"

#include <cfloat>

namespace lpgb {

namespace {

// The slot moves of one pivot (every CTA computes the same values).
struct SlotMoves {
    int join, ent;   // rows entering / leaving R (-1: none)
    int k0, k1, kn;  // live slots before, after the join, after the drop
    int tl;          // old slot of `join`
    int u;           // row displaced from slot k0 by the join
    int te;          // slot of `ent`, which receives row w
    int w;           // row moved into slot te
    int J;           // new slot of the joining row's column (-1: none)
    int src_te;      // old slot whose column moves to te (-1: none or the join)
};

__device__ SlotMoves slot_moves(const DevState& s, int leave, int q, int k, int par) {
    const Params& P = s.p;
    const int32_t* sr = s.slot_row + (size_t)par * P.m;
    const int32_t* rs = s.row_slot + (size_t)par * P.m;
    SlotMoves v;
    v.join = leave >= P.n ? leave - P.n : -1;
    v.ent = q >= P.n ? q - P.n : -1;
    v.k0 = k;
    v.tl = v.join >= 0 ? __ldcg(rs + v.join) : -1;
    v.u = v.join >= 0 ? __ldcg(sr + k) : -1;
    v.k1 = k + (v.join >= 0 ? 1 : 0);
    v.te = v.ent >= 0 ? __ldcg(rs + v.ent) : -1;
    v.w = v.ent >= 0 ? (v.join >= 0 ? v.join : __ldcg(sr + k - 1)) : -1;
    v.kn = v.k1 - (v.ent >= 0 ? 1 : 0);
    v.J = v.join >= 0 ? (v.ent >= 0 ? v.te : v.k0) : -1;
    v.src_te = (v.ent >= 0 && v.join < 0) ? v.k0 - 1 : -1;
    return v;
}

// new slot_row entry of slot t / new row_slot entry of row x
__device__ __forceinline__ int moved_slot_row(const SlotMoves& v, int t, int old) {
    if (v.ent >= 0 && t == v.te) return v.w;
    if (v.ent >= 0 && t == v.k1 - 1) return v.ent;
    if (v.join >= 0 && t == v.k0) return v.join;
    if (v.join >= 0 && t == v.tl) return v.u;
    return old;
}
__device__ __forceinline__ int moved_row_slot(const SlotMoves& v, int x, int old) {
    if (v.ent >= 0 && x == v.ent) return v.k1 - 1;
    if (v.ent >= 0 && x == v.w) return v.te;
    if (v.join >= 0 && x == v.join) return v.J;
    if (v.join >= 0 && x == v.u) return v.tl;
    return old;
}

// Source of slot t's rho and y after the moves: an old slot, or -2 for the
// joining row (rho = 1, y = 0: its old column is e_r and its y is zero).
__device__ __forceinline__ int vec_src(const SlotMoves& v, int t) {
    if (t == v.J) return -2;
    if (t == v.te && v.src_te >= 0) return v.src_te;
    return t;
}

// Step 8 on the block's rows of the live B^-1 columns (new slot order), fused
// with the FTRAN of the next entering column and the Step 6 ratios.  A CTA
// always owns the same rows, so its own rows are read through L1; A_p, whose
// rows move during the launch, is read through L2.  aq: the
// entering structural column of A_p (nullptr for a slack, whose unit vector
// sits at live slot aq_unit).  rh: rho / alpha_r in new slot order, zero past
// kn.  Returns, in lane 0 of each warp, the smallest ratio of its rows.
__device__ double update_block_s(const DevState& s, const SlotMoves& v, int r, bool do_upd, bool do_ftran,
                                 const double* acur, double* anxt, const double* aq, int aq_unit, const double* rh) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kn = v.kn;
    const int kh = (kn + 1) >> 1;  // double2 units covering the live slots
    const double2* aq2 = reinterpret_cast<const double2*>(aq);
    const double2* rh2 = reinterpret_cast<const double2*>(rh);
    double tmin = DBL_MAX;
    const int G = gridDim.x;
    const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
    for (int l = warp; l < owned; l += nw) {
        const int i = blockIdx.x + G * l;
        double* rowd = s.bp + (size_t)i * P.ld;
        double2* row = reinterpret_cast<double2*>(rowd);
        // the unit term of FTRAN: the row of the slack basic at position i
        const int us = (do_ftran && aq) ? __ldcg(s.uslot + i) : -1;
        const double aus = us >= 0 ? __ldcg(aq + us) : 0.0;
        double a0 = 0.0, a1 = 0.0;
        if (do_upd && i == r) {
            // row r becomes rho / alpha_r (every slot, the moved ones included)
            for (int k = lane; k < kh; k += 32) {
                const double2 nv = rh2[k];
                __stcs(row + k, nv);
                if (do_ftran) {
                    const int t0 = 2 * k, t1 = t0 + 1;
                    const double2 w = aq ? __ldcg(aq2 + k) : make_double2(t0 == aq_unit ? 1.0 : 0.0, t1 == aq_unit ? 1.0 : 0.0);
                    a0 = fma(nv.x, w.x, a0);
                    if (t1 < kn) a1 = fma(nv.y, w.y, a1);
                }
            }
        } else {
            const double na = do_upd ? -__ldcg(acur + i) : 0.0;
            const bool st = na != 0.0;
            // old value of the column that moves into slot te (read before any store)
            const double bte = (do_upd && v.src_te >= 0) ? __ldcg(rowd + v.src_te) : 0.0;
            for (int k0 = lane; k0 < kh; k0 += 32 * kS) {
                double2 o[kS];
#pragma unroll
                for (int t = 0; t < kS; ++t)
                    if (k0 + 32 * t < kh) o[t] = __ldcs(row + k0 + 32 * t);
#pragma unroll
                for (int t = 0; t < kS; ++t) {
                    const int k = k0 + 32 * t;
                    if (k >= kh) break;
                    const int t0 = 2 * k, t1 = t0 + 1;
                    double2 nv = o[t];
                    if (do_upd) {
                        const double2 p = rh2[k];
                        const double b0 = t0 == v.J ? 0.0 : (t0 == v.te && v.src_te >= 0 ? bte : o[t].x);
                        const double b1 = t1 == v.J ? 0.0 : (t1 == v.te && v.src_te >= 0 ? bte : o[t].y);
                        nv.x = fma(na, p.x, b0);
                        nv.y = fma(na, p.y, b1);
                        if (st) __stcs(row + k, nv);
                    }
                    if (do_ftran) {
                        const double2 w = aq ? __ldcg(aq2 + k) : make_double2(t0 == aq_unit ? 1.0 : 0.0, t1 == aq_unit ? 1.0 : 0.0);
                        a0 = fma(nv.x, w.x, a0);
                        if (t1 < kn) a1 = fma(nv.y, w.y, a1);
                    }
                }
            }
            if (do_upd && !st && lane == 0) {
                // alpha_i = 0: only the moved columns change
                if (v.J >= 0) rowd[v.J] = 0.0;
                if (v.src_te >= 0) rowd[v.te] = bte;
            }
        }
        if (do_ftran) {
            const double al = warp_sum(a0 + a1) + aus;
            if (lane == 0) {
                anxt[i] = al;
                double th = DBL_MAX;
                if (al > P.tol_piv) th = __ldcg(s.bbar + i) / al;
                s.theta[i] = th;
                s.row_var[i] = __ldcg(s.basis + i);
                tmin = fmin(tmin, th);
            }
        }
    }
    return tmin;
}

__global__ void __launch_bounds__(kUpdateThreads, 1) k_iterate_s(DevState s, int iters) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    extern __shared__ double sh[];  // y and rho / alpha_r in slot order (ld doubles each)
    __shared__ IterState S;
    __shared__ volatile int fail;
    __shared__ double gmin_sh;
    __shared__ int nflag;
    __shared__ int flg[kMaxFlagged];
    __shared__ double tb_sh;
    __shared__ RowPart rec_sh;
    __shared__ SlotMoves mv;  // this step's slot moves (thread 0 writes them in phase 1)
    unsigned epoch = 0;
    const bool lead = blockIdx.x == 0;
    const int G = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = G * blockDim.x;
    if (threadIdx.x == 0) {
        fail = 0;
        S.status = C->status; S.it = C->it; S.q = C->q; S.r = C->r; S.tcount = C->tcount;
        S.abuf = C->abuf; S.pending = C->pending; S.flags = C->flags; S.degen_run = C->degen_run;
        S.bland = C->bland; S.dq = C->dq; S.theta = C->theta; S.alpha_r = C->alpha_r;
        S.leave = (S.r >= 0 && S.r < P.m) ? s.basis[S.r] : -1;
        S.nsb = C->nsb; S.n_degenerate = C->n_degenerate; S.n_tabu = C->n_tabu; S.n_bland = C->n_bland;
        S.n_asp = C->n_asp; S.n_price = C->n_price; S.n_update = C->n_update;
        S.z = C->z; S.bytes_price = C->bytes_price; S.bytes_update = C->bytes_update;
        S.k = C->k_live; S.par = C->map_par;
    }
    if (!grid_barrier(s.gbar, epoch, &fail)) {
        if (lead && threadIdx.x == 0) C->err = kErrTimeout;
        return;
    }
    double* ysh = sh;
    double* rh = sh + P.ld;
    for (int step = 0; step < iters; ++step) {
        // ---- (1) the pivot chosen by the last ratio test: slot moves, rho, y, bbar, bookkeeping
        const bool piv = S.status == kRunning && S.r >= 0 && S.r < P.m && S.q >= 0;
        {
            const int r = S.r;
            const double* acur = s.alpha + (size_t)S.abuf * P.ld;
            const double ar = S.alpha_r, th = S.theta, dq = S.dq;
            const int par = S.par;
            if (threadIdx.x == 0) {
                if (piv) {
                    mv = slot_moves(s, S.leave, S.q, S.k, par);
                } else {
                    mv.join = mv.ent = -1;
                    mv.k0 = mv.k1 = mv.kn = S.k;
                    mv.tl = mv.u = mv.te = mv.w = mv.J = mv.src_te = -1;
                }
            }
            __syncthreads();  // the moves are visible and every thread has read the state
            if (piv) {
            if (threadIdx.x == 0) {
                if (lead) {
                    // the positions whose basic slack changed slot
                    s.uslot[r] = mv.ent >= 0 ? mv.k1 - 1 : -1;
                    if (mv.join >= 0 && mv.tl != mv.k0) s.uslot[__ldcg(s.pos + P.n + mv.u)] = mv.tl;
                }
                pivot_bookkeeping(s, S, lead);
                S.k = mv.kn;
                S.par = par ^ 1;
            }
            const int32_t* sr0 = s.slot_row + (size_t)par * P.m;
            const int32_t* rs0 = s.row_slot + (size_t)par * P.m;
            int32_t* sr1 = s.slot_row + (size_t)(par ^ 1) * P.m;
            int32_t* rs1 = s.row_slot + (size_t)(par ^ 1) * P.m;
            const double* brow = s.bp + (size_t)r * P.ld;
            for (int x = tid; x < P.m; x += stride) {
                // next slot maps; bbar (by basis position)
                const int a = __ldcg(sr0 + x), b = __ldcg(rs0 + x);
                const double bb = __ldcg(s.bbar + x), ak = __ldcg(acur + x);
                sr1[x] = moved_slot_row(mv, x, a);
                rs1[x] = moved_row_slot(mv, x, b);
                s.bbar[x] = (x == r) ? th : __dsub_rn(bb, __dmul_rn(ak, th));
            }
            for (int t = tid; t < mv.kn; t += stride) {
                // rho / alpha_r and y in the new slot order
                const int src = vec_src(mv, t);
                const double rv = src >= 0 ? __ldcg(brow + src) : 1.0;
                const double yv = src >= 0 ? __ldcg(s.yp + src) : 0.0;
                const double rn = rv / ar;
                s.rho[t] = rn;
                s.yp[t] = __dadd_rn(yv, __dmul_rn(dq, rn));
            }
            if (mv.join >= 0 || mv.ent >= 0) {
                // A_p rows follow their slots (at most three slots change)
                int dst[3], src[3], nm = 0;
                if (mv.ent >= 0 && mv.join >= 0) {
                    dst[0] = mv.te; src[0] = mv.tl;
                    dst[1] = mv.k0; src[1] = mv.te;
                    nm = 2;
                    if (mv.tl != mv.k0) { dst[2] = mv.tl; src[2] = mv.k0; nm = 3; }
                } else if (mv.ent >= 0) {
                    if (mv.te != mv.k0 - 1) { dst[0] = mv.te; src[0] = mv.k0 - 1; dst[1] = mv.k0 - 1; src[1] = mv.te; nm = 2; }
                } else if (mv.tl != mv.k0) {
                    dst[0] = mv.k0; src[0] = mv.tl; dst[1] = mv.tl; src[1] = mv.k0; nm = 2;
                }
                for (int j = tid; j < P.n && nm > 0; j += stride) {
                    double* col = s.A_p + (size_t)j * P.ld;
                    double val[3];
                    for (int e = 0; e < nm; ++e) val[e] = __ldcg(col + src[e]);
                    for (int e = 0; e < nm; ++e) col[dst[e]] = val[e];
                }
            }
            if (!grid_barrier(s.gbar, epoch, &fail)) break;
            if (S.status == kReinvert) break;
            }
        }
        const int kn = S.k;
        const int kk = min(P.ld, (kn + 63) & ~63);  // live slots rounded up to a double2 sweep
        // ---- (2) PRICE + CHUZC over the live slots
        if (S.status == kRunning) {
            const bool stage_rh = S.pending != 0;
            for (int t = threadIdx.x; t < kk; t += blockDim.x) {
                ysh[t] = t < kn ? __ldcg(s.yp + t) : 0.0;
                if (stage_rh) rh[t] = t < kn ? __ldcg(s.rho + t) : 0.0;
            }
            __syncthreads();
            const int32_t* sr = s.slot_row + (size_t)S.par * P.m;
            const Cand bc = price_block<true>(s, S.it, ysh, s.A_p, kk >> 1, sr, kn);
            if (threadIdx.x == 0) s.price_part[blockIdx.x] = to_price_cand(bc);
            if (!grid_barrier(s.gbar, epoch, &fail)) break;
            const Cand g = reduce_price_parts(s.price_part, G);
            if (threadIdx.x == 0) {
                const Chuzc d = chuzc_decide(g, S.bland != 0, P.tol_d);
                if (d.optimal) {
                    S.status = kOptimal;
                    S.q = -1;
                } else {
                    S.q = d.q;
                    S.dq = d.dq;
                    S.flags |= d.flags;
                }
                if (lead) {
                    S.bytes_price += 8.0 * kn * (double)(P.n - S.nsb);
                    S.n_price++;
                    S.n_asp += d.asp;
                }
            }
            __syncthreads();
        } else if (S.pending != 0) {
            for (int t = threadIdx.x; t < kk; t += blockDim.x) rh[t] = t < kn ? __ldcg(s.rho + t) : 0.0;
            __syncthreads();
        }
        // ---- (3) UPDATE of the pending pivot + FTRAN of the new column + ratios
        const bool do_upd = S.pending != 0 && S.r >= 0 && S.r < P.m;
        const bool do_ftran = S.status == kRunning && S.q >= 0 && S.q < P.n + P.m;
        if (!do_upd && !do_ftran) break;
        const double* aq = (do_ftran && S.q < P.n) ? s.A_p + (size_t)S.q * P.ld : nullptr;
        const int aq_unit = (do_ftran && S.q >= P.n) ? __ldcg(s.row_slot + (size_t)S.par * P.m + (S.q - P.n)) : -1;
        const double* acur = s.alpha + (size_t)S.abuf * P.ld;
        double* anxt = s.alpha + (size_t)(S.abuf ^ 1) * P.ld;
        const double tb = block_min(update_block_s(s, mv, S.r, do_upd, do_ftran, acur, anxt, aq, aq_unit, rh));
        if (threadIdx.x == 0) {
            tb_sh = tb;
            if (lead) {
                S.bytes_update += (do_upd ? 16.0 : (do_ftran ? 8.0 : 0.0)) * P.m * (double)kn;
                S.n_update++;
            }
        }
        __syncthreads();
        if (do_ftran) {
            const double tbl = tb_sh;
            const double thr_b = tbl + P.tol_tie * fmax(1.0, fabs(tbl));
            const bool blandb = S.bland != 0;
            RowCand lb = {0.0, 0, -1, 0.0};
            int lc = 0;
            if (tbl != DBL_MAX) {
                const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
                for (int l = threadIdx.x; l < owned; l += blockDim.x) {
                    const int i = blockIdx.x + G * l;
                    const double al = anxt[i], th = s.theta[i];  // written by this CTA
                    if (al > P.tol_piv && th <= thr_b) {
                        lc++;
                        RowCand c = {al, s.row_var[i], i, th};
                        if (row_beats(c, lb, blandb)) lb = c;
                    }
                }
            }
            lb = block_row_best(lb, lc, blandb);
            if (threadIdx.x == 0) {
                RowPart rp;
                rp.tmin = tbl; rp.a = lb.a; rp.th = lb.th; rp.var = lb.var; rp.row = lb.row; rp.cnt = lc; rp.pad_ = 0;
                s.row_part[blockIdx.x] = rp;
            }
        }
        if (!do_ftran) {
            if (threadIdx.x == 0) S.pending = 0;
            break;
        }
        if (!grid_barrier(s.gbar, epoch, &fail)) break;
        // ---- (4) CHUZR: minimum ratio, tie set, leaving row (every CTA)
        RowPart rec;
        rec.tmin = DBL_MAX;
        if ((int)threadIdx.x < G) {
            const RowPart* rp = s.row_part + threadIdx.x;
            rec.tmin = __ldcg(&rp->tmin); rec.a = __ldcg(&rp->a); rec.th = __ldcg(&rp->th);
            rec.var = __ldcg(&rp->var); rec.row = __ldcg(&rp->row); rec.cnt = __ldcg(&rp->cnt);
        }
        const double mine = rec.tmin;
        double tg = block_min(mine);
        if (threadIdx.x == 0) {
            gmin_sh = tg;
            nflag = 0;
        }
        __syncthreads();
        const double gmin = gmin_sh;
        if (gmin == DBL_MAX) {
            if (threadIdx.x == 0) {
                S.status = kUnbounded;
                S.pending = 0;
            }
            break;
        }
        const double thr = gmin + P.tol_tie * fmax(1.0, fabs(gmin));
        if ((int)threadIdx.x < G && mine <= thr) {
            const int k = atomicAdd(&nflag, 1);
            if (k < kMaxFlagged) flg[k] = threadIdx.x;
            rec_sh = rec;
        }
        __syncthreads();
        const bool bland = S.bland != 0;
        RowCand best = {0.0, 0, -1, 0.0};
        int cnt = 0;
        if (nflag == 1) {
            if (threadIdx.x == 0) {
                best.a = rec_sh.a; best.var = rec_sh.var; best.row = rec_sh.row; best.th = rec_sh.th;
                cnt = rec_sh.cnt;
            }
        } else if (nflag <= kMaxFlagged) {
            const int per = (P.m + G - 1) / G;
            for (int e = threadIdx.x; e < nflag * per; e += blockDim.x) {
                const int b = flg[e / per], l = e % per;
                const int i = b + G * l;
                if (i >= P.m) continue;
                const double al = __ldcg(anxt + i), th = __ldcg(s.theta + i);
                if (al > P.tol_piv && th <= thr) {
                    cnt++;
                    RowCand c = {al, __ldcg(s.row_var + i), i, th};
                    if (row_beats(c, best, bland)) best = c;
                }
            }
        } else {
            for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
                const double al = __ldcg(anxt + i), th = __ldcg(s.theta + i);
                if (al > P.tol_piv && th <= thr) {
                    cnt++;
                    RowCand c = {al, __ldcg(s.row_var + i), i, th};
                    if (row_beats(c, best, bland)) best = c;
                }
            }
        }
        const RowCand b = nflag == 1 ? best : block_row_best(best, cnt, bland);
        if (threadIdx.x == 0) {
            S.pending = 0;
            if (b.row < 0) {
                S.status = kUnbounded;
                if (lead) C->err = kErrBadIndex;
            } else {
                S.r = b.row;
                S.leave = b.var;
                S.theta = b.th;
                S.alpha_r = b.a;
                S.tcount = cnt;
                if (cnt > 1) S.flags |= kTfTieSet;
                S.abuf ^= 1;
            }
        }
        __syncthreads();
        if (S.status != kRunning) break;
    }
    if (lead && threadIdx.x == 0) {
        iterate_flush(s, S);
        if (fail) C->err = kErrTimeout;
    }
}

// ---- entering the structured form from the dense state ------------------------------
// One block: the live rows R (nonbasic slack), a check that the current slot
// map holds exactly R in slots [0, k) (rebuilt, R then the other rows in
// increasing order, when it does not or when force is set), the basic-slack
// slot of every basis position, and a fresh start at PRICE.
__global__ void __launch_bounds__(1024) k_struct_layout(DevState s, int force, int32_t* relayout) {
    const Params& P = s.p;
    Ctrl* C = s.ctrl;
    const int par = C->map_par;
    int32_t* sr = s.slot_row + (size_t)par * P.m;
    int32_t* rs = s.row_slot + (size_t)par * P.m;
    __shared__ int wc[32];
    __shared__ int tot_sh, bad_sh;
    // k = |R|, and the live rows the current map holds in its first k slots
    int live = 0;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) live += s.pos[P.n + i] < 0;
    for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = live;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wc[w];
        tot_sh = t;
        bad_sh = force;
    }
    __syncthreads();
    const int k = tot_sh;
    for (int t = threadIdx.x; t < k; t += blockDim.x)
        if (s.pos[P.n + sr[t]] >= 0) bad_sh = 1;
    __syncthreads();
    const bool rebuild = bad_sh != 0;
    if (rebuild) {
        // stable partition of the rows: R first, then the rows with a basic slack
        int base_live = 0, base_dead = k;
        for (int c0 = 0; c0 < P.m; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            const int isl = i < P.m && s.pos[P.n + i] < 0;
            const unsigned bal = __ballot_sync(0xffffffffu, isl);
            const unsigned balv = __ballot_sync(0xffffffffu, i < P.m);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(bal) | (__popc(balv) << 16);
            __syncthreads();
            int bl = 0, bd = 0, cl = 0, cd = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const int nl = wc[w] & 0xffff, nv = wc[w] >> 16;
                if (w < (int)(threadIdx.x >> 5)) { bl += nl; bd += nv - nl; }
                cl += nl; cd += nv - nl;
            }
            const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
            if (i < P.m) {
                const int sl = isl ? base_live + bl + __popc(bal & below)
                                   : base_dead + bd + __popc(~bal & balv & below);
                sr[sl] = i;
                rs[i] = sl;
            }
            base_live += cl;
            base_dead += cd;
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P.m; p += blockDim.x) {
        const int v = s.basis[p];
        s.uslot[p] = v >= P.n ? rs[v - P.n] : -1;
    }
    if (threadIdx.x == 0) {
        *relayout = rebuild ? 1 : 0;
        C->k_live = k;
        C->q = -1;
        C->r = -1;
        C->pending = 0;
    }
}

// A_p = A_cm with its rows in slot order (only after a rebuilt map)
__global__ void k_struct_gather_A(DevState s, const int32_t* relayout) {
    if (*relayout == 0) return;
    const Params& P = s.p;
    const int32_t* sr = s.slot_row + (size_t)s.ctrl->map_par * P.m;
    const size_t total = (size_t)P.n * P.ld;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t j = e / P.ld;
        const int t = (int)(e % P.ld);
        s.A_p[e] = t < P.m ? s.A_cm[j * P.ld + sr[t]] : 0.0;
    }
}

// the live columns of the dense B^-1 and the live entries of y
__global__ void k_struct_gather_B(DevState s) {
    const Params& P = s.p;
    const int k = s.ctrl->k_live;
    const int32_t* sr = s.slot_row + (size_t)s.ctrl->map_par * P.m;
    const size_t total = (size_t)P.m * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / k;
        const int t = (int)(e % k);
        s.bp[i * P.ld + t] = s.binv[i * P.ld + sr[t]];
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.ld; t += gridDim.x * blockDim.x)
        s.yp[t] = t < k ? s.y[sr[t]] : 0.0;
}

// dense y (and its FP32 copy) from the slot-order y, for the solution and every
// dense consumer
__global__ void k_struct_scatter_y(DevState s) {
    const Params& P = s.p;
    const int k = s.ctrl->k_live;
    const int32_t* rs = s.row_slot + (size_t)s.ctrl->map_par * P.m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.ld; i += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (i < P.m) {
            const int t = rs[i];
            if (t < k) v = s.yp[t];
        }
        s.y[i] = v;
        s.y32[i] = (float)v;
    }
}

// identity slot maps (both copies)
__global__ void k_struct_init_maps(DevState s) {
    const Params& P = s.p;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * P.m; e += gridDim.x * blockDim.x) {
        s.slot_row[e] = e % P.m;
        s.row_slot[e] = e % P.m;
    }
}

}  // namespace

size_t iterate_s_smem_bytes(int ld) { return 2 * (size_t)ld * sizeof(double); }

int occupancy_iterate_s(int ld) {
    cudaFuncSetAttribute(k_iterate_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)iterate_s_smem_bytes(ld));
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_s, kUpdateThreads, iterate_s_smem_bytes(ld));
    return nb;
}

cudaError_t launch_iterate_s(const DevState& s, int blocks, int iters, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s.gbar, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kUpdateThreads);
    cfg.dynamicSmemBytes = iterate_s_smem_bytes(s.p.ld);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_iterate_s, s, iters);
}

void launch_struct_enter(const DevState& s, int force, int32_t* relayout, cudaStream_t st) {
    k_struct_layout<<<1, 1024, 0, st>>>(s, force, relayout);
    k_struct_gather_A<<<1024, 256, 0, st>>>(s, relayout);
    k_struct_gather_B<<<1024, 256, 0, st>>>(s);
}

void launch_struct_scatter_y(const DevState& s, cudaStream_t st) {
    k_struct_scatter_y<<<64, 256, 0, st>>>(s);
}

void launch_struct_init_maps(const DevState& s, cudaStream_t st) {
    k_struct_init_maps<<<64, 256, 0, st>>>(s);
}

}  // namespace lpgb
