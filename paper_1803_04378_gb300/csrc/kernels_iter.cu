// kernels_iter.cu -- one simplex iteration as three kernels, all decisions on
// the device so that many iterations can run from one captured CUDA graph.
//
//   k_pivot   Step 7/8 bookkeeping of the pending pivot (q, r): the new row r
//             rho = B^-1[r,:] / alpha_r, the row-0 update y += d_q * rho, the
//             bbar update, basis exchange, tabu rule (Sections 2.2/3.4),
//             Bland safety net, trace, iteration counter, reinversion trigger.
//   k_price   Step 3 PRICE d_j = c_j - y^T a_j over nonbasic structural j
//             (d = -y_i for slacks) fused with Step 4 CHUZC: per-block
//             candidates, final choice by the last block to finish.
//   k_update  Step 8 B^-1 update  B^-1[i,:] -= alpha_i * rho (row r := rho),
//             fused with the next Step 5 FTRAN alpha' = B^-1 a_q' while each
//             row is in registers, the Step 6 ratios theta_i = bbar_i/alpha'_i
//             and, in the last block, the ratio-test tie set and the leaving
//             row.
//
// Section 3.1 avoids an `if i == r` branch inside a 2-D thread block; here a
// whole warp owns one row, so the row-r case is a warp-uniform branch and costs
// nothing.
#include "lpgb_internal.cuh"
#include "iter_common.cuh"
#include "../../include/lpgb.h"

#include <cfloat>

namespace lpgb {

namespace {


// ---- initial slack basis (Step 1 with B = I) -------------------------------------
__global__ void k_init_slack(DevState s) {
    const Params& P = s.p;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t total = (size_t)P.m * P.ld;
    for (size_t e = tid; e < total; e += stride) {
        const size_t i = e / P.ld, k = e % P.ld;
        s.binv[e] = (i == k) ? 1.0 : 0.0;
    }
    for (size_t i = tid; i < (size_t)P.ld; i += stride) {
        s.y[i] = 0.0;
        s.y32[i] = 0.f;
        s.rho[i] = 0.0;
        s.alpha[i] = 0.0;
        s.alpha[P.ld + i] = 0.0;
    }
    for (size_t i = tid; i < (size_t)P.m; i += stride) {
        s.bbar[i] = s.b[i];
        s.basis[i] = P.n + (int)i;
    }
    for (size_t j = tid; j < (size_t)(P.n + P.m); j += stride) {
        s.pos[j] = j < (size_t)P.n ? -1 : (int)(j - P.n);
        s.tabu_until[j] = 0;
    }
    if (tid == 0) {
        Ctrl c = {};
        c.map_par = s.ctrl->map_par;  // the slot map copy that matches A_p survives a reset
        c.status = P.max_iters > 0 ? kRunning : kIterLimit;
        c.q = -1;
        c.r = -1;
        *s.ctrl = c;
    }
}

// ---- k_pivot -----------------------------------------------------------------------
__global__ void __launch_bounds__(kPivotThreads) k_pivot(DevState s) {
    pdl_enter();
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    if (C->status != kRunning || C->r < 0 || C->r >= P.m || C->q < 0) return;
    const int r = C->r;
    const double* acur = s.alpha + (size_t)C->abuf * P.ld;
    const double ar = acur[r];
    const double th = C->theta;  // bbar_r / alpha_r, computed by the ratio test
    const double dq = C->dq;
    const double* brow = s.prow ? s.prow : s.binv + (size_t)r * P.ld;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    // new row r of the tableau and the row-0 (dual) update
    for (int k = tid; k < P.ld; k += stride) {
        const double rn = brow[k] / ar;
        s.rho[k] = rn;
        const double yn = __dadd_rn(s.y[k], __dmul_rn(dq, rn));
        s.y[k] = yn;
        s.y32[k] = (float)yn;
    }
    for (int i = tid; i < P.m; i += stride) {
        if (i == r) s.bbar[i] = th;
        else s.bbar[i] = __dsub_rn(s.bbar[i], __dmul_rn(acur[i], th));
    }
    if (!is_last_block(&C->ticket_pivot) || threadIdx.x != 0) return;
    __threadfence();
    // scalar bookkeeping, one thread
    C->ticket_pivot = 0;
    const int it = C->it;
    const int q = C->q;
    const int leave = s.basis[r];
    int flags = C->flags;
    const bool degenerate = th <= P.tol_tie;
    if (degenerate) { flags |= kTfDegenerate; C->n_degenerate++; }
    if (P.tabu_tenure > 0 && (C->tcount > 1 || degenerate)) {
        s.tabu_until[leave] = it + 1 + P.tabu_tenure;
        flags |= kTfTabuPush;
        C->n_tabu++;
    }
    if (it < P.trace_cap) {
        s.trace.q[it] = q;
        s.trace.r[it] = r;
        s.trace.theta[it] = th;
        s.trace.dq[it] = dq;
        s.trace.flags[it] = flags;
    }
    C->z = __dadd_rn(C->z, __dmul_rn(dq, th));
    s.pos[leave] = -1;
    s.basis[r] = q;
    s.pos[q] = r;
    C->nsb += (q < P.n ? 1 : 0) - (leave < P.n ? 1 : 0);
    const int it1 = it + 1;
    C->it = it1;
    C->degen_run = degenerate ? C->degen_run + 1 : 0;
    if (C->bland && !degenerate) C->bland = 0;
    if (!C->bland && P.bland_after > 0 && C->degen_run >= P.bland_after) {
        C->bland = 1;
        C->n_bland++;
    }
    C->flags = 0;
    C->pending = 1;  // at a reinversion too: the next k_update applies it (B^-1 stays that of the basis)
    if (P.reinvert_every > 0 && it1 % P.reinvert_every == 0) C->status = kReinvert;
    else if (it1 >= P.max_iters) C->status = kIterLimit;
    __threadfence();
}

// ---- k_price: PRICE + CHUZC -----------------------------------------------------
__global__ void __launch_bounds__(kPriceThreads, 1) k_price(DevState s) {
    pdl_enter();
    Ctrl* C = s.ctrl;
    if (C->status != kRunning) return;
    const Params& P = s.p;
    // price_mode 1: this full FP64 pass only runs when the BF16 screen found no
    // improving candidate, or under the Bland safety net
    if (P.price_mode == 1 && !C->need_full && !C->bland) return;
    extern __shared__ double ysh[];
    for (int k = threadIdx.x; k < P.ld; k += blockDim.x) ysh[k] = s.y[k];
    __syncthreads();
    const Cand bc = (P.price_mode == 2 ? price_block_csc(s, C->it, ysh, no_patch()) : price_block(s, C->it, ysh, s.A_cm, P.ld >> 1, nullptr, P.m, no_patch()));
    if (threadIdx.x == 0) s.price_part[blockIdx.x] = to_price_cand(bc);
    if (!is_last_block(&C->ticket_price)) return;
    // last block: reduce all partials and decide
    const Cand g = reduce_price_parts(s.price_part, gridDim.x);
    if (threadIdx.x == 0) {
        C->ticket_price = 0;
        C->bytes_price += (P.price_mode == 2 ? 12.0 * P.nnz / P.n : 8.0 * P.m) * (double)(P.n - C->nsb);
        C->n_price++;
        if (P.price_mode == 1) {
            C->need_full = 0;
            C->n_full++;
        }
        const Chuzc d = chuzc_decide(g, C->bland != 0, P.tol_d);
        if (d.optimal) {
            C->status = kOptimal;
            C->q = -1;
        } else {
            C->q = d.q;
            C->dq = d.dq;
            C->flags |= d.flags;
            C->n_asp += d.asp;
        }
        __threadfence();
    }
}

// ---- UPDATE of one block's rows (k_update and k_iterate) ----------------------------
// Step 8 on the block's rows of B^-1 (row r := rho) fused with the FTRAN of
// the next entering column (aq) and the Step 6 ratios.  Returns, in lane 0 of
// each warp, the smallest ratio of its rows.  snapshot: also record the basic
// variable of each row for a ratio test that runs while the basis changes.
// aq_unit >= 0: the entering column is the slack unit vector e_{aq_unit}
// (generated, aq unused).

__device__ double update_block(const DevState& s, int r, bool do_upd, bool do_ftran, const double* acur,
                               double* anxt, const double* aq, const double* rh, bool snapshot, int aq_unit = -1) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = P.ld >> 1;
    const double2* aq2 = reinterpret_cast<const double2*>(aq);
    const double2* rh2 = reinterpret_cast<const double2*>(rh);
    auto aqv = [&](int k) -> double2 {
        if (aq_unit < 0) return aq2[k];
        return make_double2(2 * k == aq_unit ? 1.0 : 0.0, 2 * k + 1 == aq_unit ? 1.0 : 0.0);
    };
    double tmin = DBL_MAX;
    // Rows are dealt to blocks round-robin (block b owns i = b, b+G, ...) so
    // every SM gets the same share, and to the block's warps one row at a
    // time, which spreads them evenly over the SM's four schedulers.  Each
    // warp keeps kS 512-byte reads of its row in flight.
    const int G = gridDim.x;
    const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
    for (int l = warp; l < owned; l += nw) {
        const int i = blockIdx.x + G * l;
        double2* row = reinterpret_cast<double2*>(s.binv + (size_t)i * P.ld);
        double a0 = 0.0, a1 = 0.0;
        if (do_upd && i == r) {
            // the pivot row becomes rho (no read of the old row)
            for (int k = lane; k < half; k += 32) {
                const double2 v = rh2[k];
                __stcs(row + k, v);
                if (do_ftran) {
                    const double2 w = aqv(k);
                    a0 = fma(v.x, w.x, a0); a1 = fma(v.y, w.y, a1);
                }
            }
        } else {
            const double na = do_upd ? -__ldcg(acur + i) : 0.0;
            const bool st = na != 0.0;
            if (st || do_ftran) {
                for (int k0 = lane; k0 < half; k0 += 32 * kS) {
                    double2 v[kS];
#pragma unroll
                    for (int t = 0; t < kS; ++t)
                        if (k0 + 32 * t < half) v[t] = __ldcs(row + k0 + 32 * t);
#pragma unroll
                    for (int t = 0; t < kS; ++t) {
                        const int k = k0 + 32 * t;
                        if (k >= half) break;
                        if (st) {
                            const double2 p = rh2[k];
                            v[t].x = fma(na, p.x, v[t].x); v[t].y = fma(na, p.y, v[t].y);
                            __stcs(row + k, v[t]);
                        }
                        if (do_ftran) {
                            const double2 w = aqv(k);
                            a0 = fma(v[t].x, w.x, a0); a1 = fma(v[t].y, w.y, a1);
                        }
                    }
                }
            }
        }
        if (do_ftran) {
            const double al = warp_sum(a0 + a1);
            if (lane == 0) {
                anxt[i] = al;
                double th = DBL_MAX;
                if (al > P.tol_piv) th = __ldcg(s.bbar + i) / al;
                s.theta[i] = th;
                if (snapshot) s.row_var[i] = __ldcg(s.basis + i);
                tmin = fmin(tmin, th);
            }
        }
    }
    return tmin;
}

// block minimum (result in thread 0)
// Lexicographic comparison of rows i and r of B^-1, each divided by its alpha
// (alpha' of the current FTRAN), by one warp: -1 if row i comes first, +1 if
// row r does, 0 if every column is equal within tau relative (the result in
// every lane).  64 columns per round trip; a column where both entries are
// zero is passed on integer tests, the others are compared as x_i a_r vs
// x_r a_i (both alphas are positive), so no division runs on the FP64 pipe.
__device__ int lex_cmp_warp(const DevState& s, const double* anxt, int i, int r, double tau) {
    const int lane = threadIdx.x & 31;
    const double ai = __ldcg(anxt + i), ar = __ldcg(anxt + r);
    const double2* bi = reinterpret_cast<const double2*>(s.binv + (size_t)i * s.p.ld);
    const double2* br = reinterpret_cast<const double2*>(s.binv + (size_t)r * s.p.ld);
    const double aa = ai * ar;
    for (int c0 = 0; c0 < s.p.m; c0 += 64) {
        const double2 xi = __ldcg(bi + (c0 >> 1) + lane), xr = __ldcg(br + (c0 >> 1) + lane);
        int code = 0;  // 1 + element index of the first difference; sign in bit 2
#pragma unroll
        for (int e = 1; e >= 0; --e) {
            const double x = e ? xi.y : xi.x, y = e ? xr.y : xr.x;
            const bool zz = ((__double_as_longlong(x) | __double_as_longlong(y)) << 1) == 0;
            if (!zz) {
                const double u = x * ar, v = y * ai;
                if (fabs(u - v) > tau * fmax(aa, fmax(fabs(u), fabs(v)))) code = (e + 1) | (u < v ? 4 : 0);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, code != 0);
        if (bal) {
            const int src = __ffs(bal) - 1;
            const int cd = __shfl_sync(0xffffffffu, code, src);
            return (cd & 4) ? -1 : 1;
        }
    }
    return 0;
}

// ---- k_update: B^-1 update + FTRAN + ratio test -------------------------------------
__global__ void __launch_bounds__(kUpdateThreads, 1) k_update(DevState s) {
    pdl_enter();
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    const int status = C->status;
    const int q = C->q;
    const int r = C->r;
    const int ab = C->abuf;
    const bool do_upd = C->pending != 0 && r >= 0 && r < P.m;
    const bool do_ftran = status == kRunning && q >= 0 && q < P.n + P.m;
    if (!do_upd && !do_ftran) return;
    extern __shared__ double sh[];
    double* aq = sh;            // column q' of [A | I]
    double* rh = sh + P.ld;     // new row r (rho)
    if (do_ftran) {
        if (q < P.n) {
            const double* col = s.A_cm + (size_t)q * P.ld;
            for (int k = threadIdx.x; k < P.ld; k += blockDim.x) aq[k] = col[k];
        } else {
            for (int k = threadIdx.x; k < P.ld; k += blockDim.x) aq[k] = (k == q - P.n) ? 1.0 : 0.0;
        }
    }
    if (do_upd)
        for (int k = threadIdx.x; k < P.ld; k += blockDim.x) rh[k] = s.rho[k];
    __syncthreads();
    const double* acur = s.alpha + (size_t)ab * P.ld;
    double* anxt = s.alpha + (size_t)(ab ^ 1) * P.ld;
    const double tmin = block_min(update_block(s, r, do_upd, do_ftran, acur, anxt, aq, rh, false));
    if (!do_ftran) {
        // only the pending update was applied; the last block clears the flag
        if (!is_last_block(&C->ticket_update)) return;
        if (threadIdx.x == 0) {
            C->ticket_update = 0;
            C->pending = 0;
            C->bytes_update += 16.0 * P.m * (double)P.m;
            C->n_update++;
            __threadfence();
        }
        return;
    }
    if (threadIdx.x == 0) s.upd_part[blockIdx.x] = tmin;
    if (!is_last_block(&C->ticket_update)) return;
    // last block: global minimum, tie set and leaving row
    __shared__ double s_tmin;
    double t = DBL_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fmin(t, __ldcg(s.upd_part + b));
    t = block_min(t);
    if (threadIdx.x == 0) s_tmin = t;
    __syncthreads();
    const double gmin = s_tmin;
    if (threadIdx.x == 0) {
        C->bytes_update += (do_upd ? 16.0 : 8.0) * P.m * (double)P.m;
        C->n_update++;
    }
    if (gmin == DBL_MAX) {
        if (threadIdx.x == 0) {
            C->ticket_update = 0;
            C->pending = 0;
            C->status = kUnbounded;
            __threadfence();
        }
        return;
    }
    const double thr = gmin + P.tol_tie * fmax(1.0, fabs(gmin));
    const bool bland = C->bland != 0;
    RowCand best = {0.0, 0, -1, 0.0};
    int cnt = 0;
    // all loads of a chunk are issued before any is tested: one L2 round trip per chunk
    constexpr int kU = 8;
    for (int base = 0; base < P.m; base += kU * (int)blockDim.x) {
        double al[kU], th[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = base + u * blockDim.x + threadIdx.x;
            al[u] = i < P.m ? __ldcg(anxt + i) : 0.0;
            th[u] = i < P.m ? __ldcg(s.theta + i) : DBL_MAX;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = base + u * blockDim.x + threadIdx.x;
            if (i < P.m && al[u] > P.tol_piv && th[u] <= thr) {
                cnt++;
                RowCand c = {al[u], s.basis[i], i, th[u]};
                if (row_beats(c, best, bland)) best = c;
            }
        }
    }
    RowCand b = block_row_best(best, cnt, bland);
    if (P.lex) {
        // Lexicographic rule: the tie set's row of B^-1 / alpha_i that is
        // lexicographically smallest leaves; a pairwise tournament over the
        // tied rows (listed in lex_rows), exact ties to the smaller basic index.
        __shared__ int lex_n;
        if (threadIdx.x == 0) lex_n = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
            const double al = __ldcg(anxt + i), th = __ldcg(s.theta + i);
            if (al > P.tol_piv && th <= thr) s.lex_rows[atomicAdd(&lex_n, 1)] = i;
        }
        __syncthreads();
        const int nt = lex_n;
        if (nt > 1) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            for (int w = 1; w < nt; w *= 2) {
                for (int e = warp * 2 * w; e + w < nt; e += nw * 2 * w) {
                    const int i = __ldcg(s.lex_rows + e), r2 = __ldcg(s.lex_rows + e + w);
                    const int cmp = lex_cmp_warp(s, anxt, i, r2, P.tol_tie);
                    if (lane == 0 && (cmp > 0 || (cmp == 0 && s.basis[r2] < s.basis[i]))) s.lex_rows[e] = r2;
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const int rr = __ldcg(s.lex_rows);
                b.row = rr;
                b.a = __ldcg(anxt + rr);
                b.th = __ldcg(s.theta + rr);
                b.var = s.basis[rr];
            }
        }
    }
    if (threadIdx.x == 0) {
        C->ticket_update = 0;
        C->pending = 0;
        if (b.row < 0) {  // cannot happen for finite data; stop rather than pivot on garbage
            C->status = kUnbounded;
            C->err = kErrBadIndex;
            __threadfence();
            return;
        }
        C->r = b.row;
        C->theta = b.th;
        C->alpha_r = b.a;
        C->tcount = cnt;
        if (cnt > 1) C->flags |= kTfTieSet;
        C->abuf = ab ^ 1;
        __threadfence();
    }
}

// ---- k_iterate: many pivots in one cooperative launch (price_mode 0 and 2) -----------
//
// The three kernels above, as phases of one persistent kernel with one CTA per
// SM: (1) apply the chosen pivot (rho, y, bbar slices; the bookkeeping), (2)
// PRICE, (3) CHUZC + UPDATE/FTRAN/ratios, then the ratio test, each phase
// behind a grid barrier.  Decisions that a last block took alone (CHUZC, the
// leaving row, the bookkeeping scalars) are computed by every CTA from the
// same partials in global memory, so all CTAs follow the same path and no
// single block is left working while the others idle; block 0 alone writes
// the shared state and the control block.  Data another CTA wrote in this
// launch is read through L2 (__ldcg).  The ratio test reads the basic
// variable of each row from the snapshot taken by the FTRAN (row_var), since
// block 0 may already be exchanging the basis.

// kCsc: PRICE over the sparse copy of A (price_mode 2), a separate instantiation so
// that the dense PRICE keeps its registers.
template <bool kCsc>
__global__ void __launch_bounds__(kUpdateThreads, 1) k_iterate(DevState s, int iters) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    extern __shared__ double sh[];  // y and rho (ld doubles each)
    __shared__ IterState S;
    __shared__ volatile int fail;
    __shared__ double gmin_sh;
    __shared__ int nflag;
    __shared__ int flg[kMaxFlagged];
    __shared__ double tb_sh;
    __shared__ RowPart rec_sh;
    unsigned epoch = 0;
    const bool lead = blockIdx.x == 0;
    const int G = gridDim.x;
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
    // every CTA has its copy of the control block before block 0 changes it
    if (!grid_barrier(s.gbar, epoch, &fail)) {
        if (lead && threadIdx.x == 0) C->err = kErrTimeout;
        return;
    }
    for (int step = 0; step < iters; ++step) {
        // ---- (1) the pivot chosen by the last ratio test: rho, y, bbar, bookkeeping
        bool rh_staged = false;
        if (S.status == kRunning && S.r >= 0 && S.r < P.m && S.q >= 0) {
            const int r = S.r;
            const double* acur = s.alpha + (size_t)S.abuf * P.ld;
            const double ar = S.alpha_r, th = S.theta, dq = S.dq;
            __syncthreads();  // every thread has read the state before thread 0 advances it
            // the bookkeeping's dependent loads overlap the slices below
            if (threadIdx.x == 0) pivot_bookkeeping(s, S, lead);
            const double* brow = s.binv + (size_t)r * P.ld;
            const int tid = blockIdx.x * blockDim.x + threadIdx.x;
            const int stride = G * blockDim.x;
            for (int k = tid; k < P.ld; k += stride) {
                // all four loads first: one round trip (m <= ld)
                const double bk = __ldcg(brow + k), yk = __ldcg(s.y + k);
                const double bb = k < P.m ? __ldcg(s.bbar + k) : 0.0, ak = k < P.m ? __ldcg(acur + k) : 0.0;
                const double rn = bk / ar;
                s.rho[k] = rn;
                const double yn = __dadd_rn(yk, __dmul_rn(dq, rn));
                s.y[k] = yn;
                s.y32[k] = (float)yn;
                if (k < P.m) s.bbar[k] = (k == r) ? th : __dsub_rn(bb, __dmul_rn(ak, th));
            }
            if (!grid_barrier(s.gbar, epoch, &fail)) break;
        }
        double* rh = sh + P.ld;  // rho for UPDATE, staged with y
        // ---- (2) PRICE + CHUZC
        if (S.status == kRunning) {
            const bool stage_rh = S.pending != 0;
            for (int k = threadIdx.x; k < P.ld; k += blockDim.x) {
                sh[k] = __ldcg(s.y + k);
                if (stage_rh) rh[k] = __ldcg(s.rho + k);
            }
            rh_staged = stage_rh;
            __syncthreads();
            const Cand bc = kCsc ? price_block_csc(s, S.it, sh, no_patch()) : price_block(s, S.it, sh, s.A_cm, P.ld >> 1, nullptr, P.m, no_patch());
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
                    S.bytes_price += (P.price_mode == 2 ? 12.0 * P.nnz / P.n : 8.0 * P.m) * (double)(P.n - S.nsb);
                    S.n_price++;
                    S.n_asp += d.asp;
                }
            }
            __syncthreads();
        }
        // ---- (3) UPDATE of the pending pivot + FTRAN of the new column + ratios
        const bool do_upd = S.pending != 0 && S.r >= 0 && S.r < P.m;
        const bool do_ftran = S.status == kRunning && S.q >= 0 && S.q < P.n + P.m;
        if (!do_upd && !do_ftran) break;
        // a structural entering column is read by every warp straight from A
        // (it stays in L1); a slack column e_i is generated
        const double* aq = (do_ftran && S.q < P.n) ? s.A_cm + (size_t)S.q * P.ld : nullptr;
        const int aq_unit = (do_ftran && S.q >= P.n) ? S.q - P.n : -1;
        if (do_upd && !rh_staged)
            for (int k = threadIdx.x; k < P.ld; k += blockDim.x) rh[k] = __ldcg(s.rho + k);
        __syncthreads();
        const double* acur = s.alpha + (size_t)S.abuf * P.ld;
        double* anxt = s.alpha + (size_t)(S.abuf ^ 1) * P.ld;
        const double tb = block_min(update_block(s, S.r, do_upd, do_ftran, acur, anxt, aq, rh, true, aq_unit));
        if (threadIdx.x == 0) {
            tb_sh = tb;
            if (lead) {
                S.bytes_update += (do_upd ? 16.0 : (do_ftran ? 8.0 : 0.0)) * P.m * (double)P.m;
                S.n_update++;
            }
        }
        __syncthreads();
        if (do_ftran) {
            // this CTA's best row and tie count under its own smallest ratio's
            // threshold; when one CTA holds the global minimum this is the answer
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
            // the pending update of the last pivot was applied (optimal, iteration limit or reinversion)
            if (threadIdx.x == 0) S.pending = 0;
            break;
        }
        if (!grid_barrier(s.gbar, epoch, &fail)) break;
        // ---- (4) CHUZR: minimum ratio, tie set, leaving row (every CTA)
        // one record per CTA (G <= blockDim): smallest ratio, best row, tie count
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
        // CTAs whose smallest ratio lies within the tie tolerance hold the tie set
        if ((int)threadIdx.x < G && mine <= thr) {
            const int k = atomicAdd(&nflag, 1);
            if (k < kMaxFlagged) flg[k] = threadIdx.x;
            rec_sh = rec;  // read only when this CTA is the only one (nflag == 1)
        }
        __syncthreads();
        const bool bland = S.bland != 0;
        RowCand best = {0.0, 0, -1, 0.0};
        int cnt = 0;
        if (nflag == 1) {
            // one CTA holds the minimum, so its threshold is the global one and
            // its record is the tie set's best row and size
            if (threadIdx.x == 0) {
                best.a = rec_sh.a; best.var = rec_sh.var; best.row = rec_sh.row; best.th = rec_sh.th;
                cnt = rec_sh.cnt;
            }
        } else if (nflag <= kMaxFlagged) {
            const int per = (P.m + G - 1) / G;  // rows of the fullest CTA
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
            if (b.row < 0) {  // cannot happen for finite data; stop rather than pivot on garbage
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

// Self-test of the bounded wait: the barrier expects one CTA more than the
// grid has, so no CTA is ever released; every CTA must give up after the spin
// limit and report kErrTimeout instead of waiting forever.
__global__ void k_barrier_selftest(uint32_t* bar, int32_t* err) {
    __shared__ volatile int fail;
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    unsigned epoch = 0;
    if (!grid_barrier(bar, epoch, &fail, gridDim.x + 1u) && threadIdx.x == 0) atomicExch(err, kErrTimeout);
}

}  // namespace

size_t price_smem_bytes(int ld) { return (size_t)ld * sizeof(double); }
size_t update_smem_bytes(int ld) { return 2 * (size_t)ld * sizeof(double); }

void configure_iter_kernels(int ld) {
    cudaFuncSetAttribute(k_price, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)price_smem_bytes(ld));
    cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem_bytes(ld));
}

void launch_init_slack(const DevState& s, cudaStream_t st) {
    k_init_slack<<<1024, 256, 0, st>>>(s);
}

void launch_pivot(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl) {
    launch_k(k_pivot, dim3(g.pivot_blocks), dim3(kPivotThreads), 0, st, pdl, s);
}

void launch_price_lp(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl);

void launch_price(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl) {
    if (s.p.price_mode == 1) {
        launch_price_lp(s, g, st, pdl);
        pdl = g.pdl != 0;  // k_price directly follows k_price_lp
    }
    launch_k(k_price, dim3(g.price_blocks), dim3(kPriceThreads), price_smem_bytes(s.p.ld), st, pdl, s);
}

void launch_update(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl) {
    launch_k(k_update, dim3(g.update_blocks), dim3(kUpdateThreads), update_smem_bytes(s.p.ld), st, pdl, s);
}

int occupancy_price(int ld) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_price, kPriceThreads, price_smem_bytes(ld));
    return nb;
}

size_t iterate_smem_bytes(int ld) { return 2 * (size_t)ld * sizeof(double); }

int occupancy_iterate(int ld) {
    cudaFuncSetAttribute(k_iterate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)iterate_smem_bytes(ld));
    cudaFuncSetAttribute(k_iterate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)iterate_smem_bytes(ld));
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate<false>, kUpdateThreads, iterate_smem_bytes(ld));
    return nb;
}

cudaError_t launch_iterate(const DevState& s, int blocks, int iters, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s.gbar, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kUpdateThreads);
    cfg.dynamicSmemBytes = iterate_smem_bytes(s.p.ld);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return s.p.price_mode == 2 ? cudaLaunchKernelEx(&cfg, k_iterate<true>, s, iters)
                               : cudaLaunchKernelEx(&cfg, k_iterate<false>, s, iters);
}

int barrier_selftest(int blocks, cudaStream_t st) {
    uint32_t* bar = nullptr;
    int32_t* err = nullptr;
    if (cudaMallocAsync(&bar, 2 * sizeof(uint32_t), st) != cudaSuccess) return LP_ERR_CUDA;
    if (cudaMallocAsync(&err, sizeof(int32_t), st) != cudaSuccess) {
        cudaFreeAsync(bar, st);
        return LP_ERR_CUDA;
    }
    cudaMemsetAsync(bar, 0, 2 * sizeof(uint32_t), st);
    cudaMemsetAsync(err, 0, sizeof(int32_t), st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_barrier_selftest, bar, err);
    int32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(bar, st);
    cudaFreeAsync(err, st);
    cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LP_ERR_CUDA;
    return h == kErrTimeout ? LP_ERR_TIMEOUT : LP_OK;
}

int occupancy_update(int ld) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update, kUpdateThreads, update_smem_bytes(ld));
    return nb;
}

}  // namespace lpgb
