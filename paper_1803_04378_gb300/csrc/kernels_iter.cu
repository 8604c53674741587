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

#include <cfloat>

namespace lpgb {

namespace {

constexpr int kPriceThreads = 512;
constexpr int kUpdateThreads = 512;
constexpr int kPivotThreads = 64;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- CHUZC candidate ---------------------------------------------------------
struct Cand {
    double d_all; int j_all;
    double d_nt;  int j_nt;
    double d_min; int j_min;
    double d_pr;  int j_pr; int k_pr;
};

__device__ __forceinline__ void cand_init(Cand& c) {
    c.d_all = -DBL_MAX; c.j_all = -1;
    c.d_nt = -DBL_MAX; c.j_nt = -1;
    c.d_min = 0.0; c.j_min = -1;
    c.d_pr = 0.0; c.j_pr = -1; c.k_pr = kNoRank;
}

// a beats b: larger d, exact ties to the smaller index.
__device__ __forceinline__ bool beats(double da, int ja, double db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

__device__ __forceinline__ void cand_offer(Cand& c, double d, int j, bool nontabu, double tol_d, int rank) {
    if (beats(d, j, c.d_all, c.j_all)) { c.d_all = d; c.j_all = j; }
    if (nontabu && beats(d, j, c.d_nt, c.j_nt)) { c.d_nt = d; c.j_nt = j; }
    if (d > tol_d && (c.j_min < 0 || j < c.j_min)) { c.d_min = d; c.j_min = j; }
    // guided rule: Dantzig restricted to the listed (priority) columns
    if (nontabu && d > tol_d && rank != kNoRank && beats(d, j, c.d_pr, c.j_pr)) { c.d_pr = d; c.j_pr = j; c.k_pr = rank; }
}

__device__ __forceinline__ void cand_merge(Cand& c, const Cand& o) {
    if (beats(o.d_all, o.j_all, c.d_all, c.j_all)) { c.d_all = o.d_all; c.j_all = o.j_all; }
    if (beats(o.d_nt, o.j_nt, c.d_nt, c.j_nt)) { c.d_nt = o.d_nt; c.j_nt = o.j_nt; }
    if (o.j_min >= 0 && (c.j_min < 0 || o.j_min < c.j_min)) { c.d_min = o.d_min; c.j_min = o.j_min; }
    if (beats(o.d_pr, o.j_pr, c.d_pr, c.j_pr)) { c.d_pr = o.d_pr; c.j_pr = o.j_pr; c.k_pr = o.k_pr; }
}

__device__ __forceinline__ Cand cand_shfl(const Cand& c, int off) {
    Cand o;
    o.d_all = __shfl_xor_sync(0xffffffffu, c.d_all, off);
    o.j_all = __shfl_xor_sync(0xffffffffu, c.j_all, off);
    o.d_nt = __shfl_xor_sync(0xffffffffu, c.d_nt, off);
    o.j_nt = __shfl_xor_sync(0xffffffffu, c.j_nt, off);
    o.d_min = __shfl_xor_sync(0xffffffffu, c.d_min, off);
    o.j_min = __shfl_xor_sync(0xffffffffu, c.j_min, off);
    o.d_pr = __shfl_xor_sync(0xffffffffu, c.d_pr, off);
    o.j_pr = __shfl_xor_sync(0xffffffffu, c.j_pr, off);
    o.k_pr = __shfl_xor_sync(0xffffffffu, c.k_pr, off);
    return o;
}

// Block-wide reduction; the result is valid in thread 0.
__device__ Cand cand_block_reduce(Cand c) {
    __shared__ Cand sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cand_merge(c, cand_shfl(c, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = c;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        if (lane < nw) c = sh[lane]; else cand_init(c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cand_merge(c, cand_shfl(c, o));
    }
    return c;
}

// Leaving-row candidate of the ratio test: largest alpha, exact ties to the
// smallest basic variable index (Bland mode: smallest basic variable index).
struct RowCand { double a; int var; int row; };

__device__ __forceinline__ bool row_beats(const RowCand& x, const RowCand& y, bool bland) {
    if (x.row < 0) return false;
    if (y.row < 0) return true;
    if (bland) return x.var < y.var;
    return x.a > y.a || (x.a == y.a && x.var < y.var);
}

__device__ __forceinline__ bool is_last_block(int32_t* ticket) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int t = atomicAdd(ticket, 1);
        last = (t == (int)gridDim.x - 1);
    }
    __syncthreads();
    return last != 0;
}

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
        c.status = P.max_iters > 0 ? kRunning : kIterLimit;
        c.q = -1;
        c.r = -1;
        *s.ctrl = c;
    }
}

// ---- k_pivot -----------------------------------------------------------------------
__global__ void __launch_bounds__(kPivotThreads) k_pivot(DevState s) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    if (C->status != kRunning || C->r < 0 || C->r >= P.m || C->q < 0) return;
    const int r = C->r;
    const double* acur = s.alpha + (size_t)C->abuf * P.ld;
    const double ar = acur[r];
    const double th = C->theta;  // bbar_r / alpha_r, computed by the ratio test
    const double dq = C->dq;
    const double* brow = s.binv + (size_t)r * P.ld;
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
    if (P.reinvert_every > 0 && it1 % P.reinvert_every == 0) {
        C->status = kReinvert;
        C->pending = 0;
    } else {
        C->pending = 1;
        if (it1 >= P.max_iters) C->status = kIterLimit;
    }
    __threadfence();
}

// ---- k_price: PRICE + CHUZC -----------------------------------------------------
__global__ void __launch_bounds__(kPriceThreads, 2) k_price(DevState s) {
    Ctrl* C = s.ctrl;
    if (C->status != kRunning) return;
    const Params& P = s.p;
    // price_mode 1: this full FP64 pass only runs when the BF16 screen found no
    // improving candidate, or under the Bland safety net
    if (P.price_mode == 1 && !C->need_full && !C->bland) return;
    extern __shared__ double ysh[];
    for (int k = threadIdx.x; k < P.ld; k += blockDim.x) ysh[k] = s.y[k];
    __syncthreads();
    const int it = C->it;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = P.ld >> 1;
    const double2* y2 = reinterpret_cast<const double2*>(ysh);
    Cand cand;
    cand_init(cand);
    // Columns are dealt to blocks round-robin (block b owns j = b, b+G, b+2G,
    // ...) so every SM gets the same share; each warp takes two owned columns
    // at a time, so one shared-memory load of y feeds four FMAs.
    const int G = gridDim.x;
    const int owned = (P.n - (int)blockIdx.x + G - 1) / G;
    for (int l = 2 * warp; l < owned; l += 2 * nw) {
        const int jA = blockIdx.x + G * l;
        const int jB = (l + 1 < owned) ? jA + G : -1;
        const bool nbA = s.pos[jA] < 0;
        const bool nbB = jB >= 0 && s.pos[jB] < 0;
        if (nbA && nbB) {
            const double2* ca = reinterpret_cast<const double2*>(s.A_cm + (size_t)jA * P.ld);
            const double2* cb = reinterpret_cast<const double2*>(s.A_cm + (size_t)jB * P.ld);
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
            int k = lane;
#pragma unroll 2
            for (; k + 32 < half; k += 64) {
                const double2 u0 = __ldcs(ca + k), u1 = __ldcs(ca + k + 32);
                const double2 v0 = __ldcs(cb + k), v1 = __ldcs(cb + k + 32);
                const double2 y0 = y2[k], y1 = y2[k + 32];
                a0 = fma(u0.x, y0.x, a0); a1 = fma(u0.y, y0.y, a1);
                a2 = fma(u1.x, y1.x, a2); a3 = fma(u1.y, y1.y, a3);
                b0 = fma(v0.x, y0.x, b0); b1 = fma(v0.y, y0.y, b1);
                b2 = fma(v1.x, y1.x, b2); b3 = fma(v1.y, y1.y, b3);
            }
            for (; k < half; k += 32) {
                const double2 u0 = __ldcs(ca + k), v0 = __ldcs(cb + k), y0 = y2[k];
                a0 = fma(u0.x, y0.x, a0); a1 = fma(u0.y, y0.y, a1);
                b0 = fma(v0.x, y0.x, b0); b1 = fma(v0.y, y0.y, b1);
            }
            const double da = s.c[jA] - warp_sum((a0 + a1) + (a2 + a3));
            const double db = s.c[jB] - warp_sum((b0 + b1) + (b2 + b3));
            cand_offer(cand, da, jA, s.tabu_until[jA] <= it, P.tol_d, s.rank[jA]);
            cand_offer(cand, db, jB, s.tabu_until[jB] <= it, P.tol_d, s.rank[jB]);
        } else if (nbA || nbB) {
            const int j = nbA ? jA : jB;
            const double2* col = reinterpret_cast<const double2*>(s.A_cm + (size_t)j * P.ld);
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int k = lane;
#pragma unroll 4
            for (; k + 32 < half; k += 64) {
                const double2 u = __ldcs(col + k), v = __ldcs(col + k + 32);
                const double2 yu = y2[k], yv = y2[k + 32];
                a0 = fma(u.x, yu.x, a0); a1 = fma(u.y, yu.y, a1);
                a2 = fma(v.x, yv.x, a2); a3 = fma(v.y, yv.y, a3);
            }
            for (; k < half; k += 32) {
                const double2 u = __ldcs(col + k), yu = y2[k];
                a0 = fma(u.x, yu.x, a0); a1 = fma(u.y, yu.y, a1);
            }
            const double d = s.c[j] - warp_sum((a0 + a1) + (a2 + a3));
            cand_offer(cand, d, j, s.tabu_until[j] <= it, P.tol_d, s.rank[j]);
        }
    }
    // slack columns: d_{n+i} = -y_i
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.m; i += gridDim.x * blockDim.x) {
        const int j = P.n + i;
        if (s.pos[j] >= 0) continue;
        cand_offer(cand, -ysh[i], j, s.tabu_until[j] <= it, P.tol_d, s.rank[j]);
    }
    Cand bc = cand_block_reduce(cand);
    if (threadIdx.x == 0) {
        PriceCand pc;
        pc.d_all = bc.d_all; pc.j_all = bc.j_all;
        pc.d_nt = bc.d_nt; pc.j_nt = bc.j_nt;
        pc.d_min = bc.d_min; pc.j_min = bc.j_min;
        pc.d_pr = bc.d_pr; pc.j_pr = bc.j_pr; pc.k_pr = bc.k_pr;
        pc.pad_ = 0;
        s.price_part[blockIdx.x] = pc;
    }
    if (!is_last_block(&C->ticket_price)) return;
    // last block: reduce all partials and decide
    Cand g;
    cand_init(g);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const PriceCand* pp = s.price_part + b;
        Cand o;
        o.d_all = __ldcg(&pp->d_all); o.j_all = __ldcg(&pp->j_all);
        o.d_nt = __ldcg(&pp->d_nt); o.j_nt = __ldcg(&pp->j_nt);
        o.d_min = __ldcg(&pp->d_min); o.j_min = __ldcg(&pp->j_min);
        o.d_pr = __ldcg(&pp->d_pr); o.j_pr = __ldcg(&pp->j_pr); o.k_pr = __ldcg(&pp->k_pr);
        cand_merge(g, o);
    }
    g = cand_block_reduce(g);
    if (threadIdx.x == 0) {
        C->ticket_price = 0;
        C->bytes_price += 8.0 * P.m * (double)(P.n - C->nsb);
        C->n_price++;
        if (P.price_mode == 1) {
            C->need_full = 0;
            C->n_full++;
        }
        if (g.j_all < 0 || !(g.d_all > P.tol_d)) {
            C->status = kOptimal;
            C->q = -1;
        } else {
            int q;
            double dq;
            if (C->bland) {
                q = g.j_min; dq = g.d_min;
                C->flags |= kTfBland;
            } else if (g.j_pr >= 0) {
                // guided entering rule: Dantzig's choice among the listed columns
                q = g.j_pr; dq = g.d_pr;
                C->flags |= kTfGuided;
            } else if (g.j_nt >= 0 && g.d_nt > P.tol_d) {
                q = g.j_nt; dq = g.d_nt;
            } else {
                q = g.j_all; dq = g.d_all;
                C->flags |= kTfAspiration;
                C->n_asp++;
            }
            C->q = q;
            C->dq = dq;
        }
        __threadfence();
    }
}

// ---- k_update: B^-1 update + FTRAN + ratio test -------------------------------------
__global__ void __launch_bounds__(kUpdateThreads) k_update(DevState s) {
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
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = P.ld >> 1;
    const double2* aq2 = reinterpret_cast<const double2*>(aq);
    const double2* rh2 = reinterpret_cast<const double2*>(rh);
    double tmin = DBL_MAX;
    // Rows are dealt to blocks round-robin (block b owns i = b, b+G, ...) so
    // every SM gets the same share; each warp takes two owned rows at a time.
    const int G = gridDim.x;
    const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
    for (int l = 2 * warp; l < owned; l += 2 * nw) {
        const int i0 = blockIdx.x + G * l;
        const int i1 = (l + 1 < owned) ? i0 + G : -1;
        double al0 = 0.0, al1 = 0.0;
        const bool pair = i1 >= 0 && !(do_upd && (i0 == r || i1 == r));
        if (pair) {
            double2* r0 = reinterpret_cast<double2*>(s.binv + (size_t)i0 * P.ld);
            double2* r1 = reinterpret_cast<double2*>(s.binv + (size_t)i1 * P.ld);
            double a0 = 0.0, a1 = 0.0, c0 = 0.0, c1 = 0.0;
            if (do_upd) {
                const double na0 = -acur[i0], na1 = -acur[i1];
                const bool st0 = na0 != 0.0, st1 = na1 != 0.0;
                if (do_ftran) {
#pragma unroll 2
                    for (int k = lane; k < half; k += 32) {
                        double2 v = __ldcs(r0 + k), u = __ldcs(r1 + k);
                        const double2 p = rh2[k], w = aq2[k];
                        v.x = fma(na0, p.x, v.x); v.y = fma(na0, p.y, v.y);
                        u.x = fma(na1, p.x, u.x); u.y = fma(na1, p.y, u.y);
                        if (st0) __stcs(r0 + k, v);
                        if (st1) __stcs(r1 + k, u);
                        a0 = fma(v.x, w.x, a0); a1 = fma(v.y, w.y, a1);
                        c0 = fma(u.x, w.x, c0); c1 = fma(u.y, w.y, c1);
                    }
                } else {
#pragma unroll 2
                    for (int k = lane; k < half; k += 32) {
                        double2 v = __ldcs(r0 + k), u = __ldcs(r1 + k);
                        const double2 p = rh2[k];
                        v.x = fma(na0, p.x, v.x); v.y = fma(na0, p.y, v.y);
                        u.x = fma(na1, p.x, u.x); u.y = fma(na1, p.y, u.y);
                        if (st0) __stcs(r0 + k, v);
                        if (st1) __stcs(r1 + k, u);
                    }
                }
            } else {
#pragma unroll 4
                for (int k = lane; k < half; k += 32) {
                    const double2 v = __ldcs(r0 + k), u = __ldcs(r1 + k), w = aq2[k];
                    a0 = fma(v.x, w.x, a0); a1 = fma(v.y, w.y, a1);
                    c0 = fma(u.x, w.x, c0); c1 = fma(u.y, w.y, c1);
                }
            }
            if (do_ftran) {
                al0 = warp_sum(a0 + a1);
                al1 = warp_sum(c0 + c1);
            }
        } else {
            // single rows: the pivot row, or the odd row left over
            for (int h = 0; h < 2; ++h) {
                const int i = h == 0 ? i0 : i1;
                if (i < 0) continue;
                double2* row = reinterpret_cast<double2*>(s.binv + (size_t)i * P.ld);
                double a0 = 0.0, a1 = 0.0;
                if (do_upd && i == r) {
                    for (int k = lane; k < half; k += 32) {
                        const double2 v = rh2[k];
                        __stcs(row + k, v);
                        const double2 w = aq2[k];
                        a0 = fma(v.x, w.x, a0); a1 = fma(v.y, w.y, a1);
                    }
                } else {
                    const double na = do_upd ? -acur[i] : 0.0;
                    const bool st = na != 0.0;
                    for (int k = lane; k < half; k += 32) {
                        double2 v = __ldcs(row + k);
                        if (st) {
                            const double2 p = rh2[k];
                            v.x = fma(na, p.x, v.x); v.y = fma(na, p.y, v.y);
                            __stcs(row + k, v);
                        }
                        const double2 w = aq2[k];
                        a0 = fma(v.x, w.x, a0); a1 = fma(v.y, w.y, a1);
                    }
                }
                const double al = warp_sum(a0 + a1);
                if (h == 0) al0 = al; else al1 = al;
            }
        }
        if (do_ftran && lane == 0) {
            for (int h = 0; h < 2; ++h) {
                const int i = h == 0 ? i0 : i1;
                if (i < 0) continue;
                const double al = h == 0 ? al0 : al1;
                anxt[i] = al;
                double th = DBL_MAX;
                if (al > P.tol_piv) th = s.bbar[i] / al;
                s.theta[i] = th;
                tmin = fmin(tmin, th);
            }
        }
    }
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
    // block minimum of theta
    __shared__ double shm[32];
    for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    if (lane == 0) shm[threadIdx.x >> 5] = tmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = DBL_MAX;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmin(t, shm[w]);
        s.upd_part[blockIdx.x] = t;
    }
    if (!is_last_block(&C->ticket_update)) return;
    // last block: global minimum, tie set and leaving row
    __shared__ double s_tmin;
    double t = DBL_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fmin(t, __ldcg(s.upd_part + b));
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    __syncthreads();
    if (lane == 0) shm[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = DBL_MAX;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u = fmin(u, shm[w]);
        s_tmin = u;
    }
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
    RowCand best = {0.0, 0, -1};
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
                RowCand c = {al[u], s.basis[i], i};
                if (row_beats(c, best, bland)) best = c;
            }
        }
    }
    // block reduce (best, cnt)
    for (int o = 16; o > 0; o >>= 1) {
        RowCand oc;
        oc.a = __shfl_xor_sync(0xffffffffu, best.a, o);
        oc.var = __shfl_xor_sync(0xffffffffu, best.var, o);
        oc.row = __shfl_xor_sync(0xffffffffu, best.row, o);
        if (row_beats(oc, best, bland)) best = oc;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    __shared__ RowCand shr[32];
    __shared__ int shc[32];
    if (lane == 0) { shr[threadIdx.x >> 5] = best; shc[threadIdx.x >> 5] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        RowCand b = shr[0];
        int total = shc[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            if (row_beats(shr[w], b, bland)) b = shr[w];
            total += shc[w];
        }
        C->ticket_update = 0;
        C->pending = 0;
        if (b.row < 0) {  // cannot happen for finite data; stop rather than pivot on garbage
            C->status = kUnbounded;
            C->err = kErrBadIndex;
            __threadfence();
            return;
        }
        C->r = b.row;
        C->theta = __ldcg(s.theta + b.row);
        C->alpha_r = b.a;
        C->tcount = total;
        if (total > 1) C->flags |= kTfTieSet;
        C->abuf = ab ^ 1;
        __threadfence();
    }
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

void launch_pivot(const DevState& s, const Geometry& g, cudaStream_t st) {
    k_pivot<<<g.pivot_blocks, kPivotThreads, 0, st>>>(s);
}

void launch_price_lp(const DevState& s, const Geometry& g, cudaStream_t st);

void launch_price(const DevState& s, const Geometry& g, cudaStream_t st) {
    if (s.p.price_mode == 1) launch_price_lp(s, g, st);
    k_price<<<g.price_blocks, kPriceThreads, price_smem_bytes(s.p.ld), st>>>(s);
}

void launch_update(const DevState& s, const Geometry& g, cudaStream_t st) {
    k_update<<<g.update_blocks, kUpdateThreads, update_smem_bytes(s.p.ld), st>>>(s);
}

int occupancy_price(int ld) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_price, kPriceThreads, price_smem_bytes(ld));
    return nb;
}

int occupancy_update(int ld) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_update, kUpdateThreads, update_smem_bytes(ld));
    return nb;
}

}  // namespace lpgb
