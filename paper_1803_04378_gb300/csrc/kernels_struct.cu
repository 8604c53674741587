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

constexpr int kMaxOwnedRows = 256;  // rows of B^-1 per CTA (ratio-test records kept in shared memory)

// Step 8 on the block's rows of the live B^-1 columns (new slot order), fused
// with the FTRAN of the next entering column and the Step 6 ratios.  A CTA
// always owns the same rows (i = b, b + G, ...), so it reads its own rows
// through L1.  aqs: the entering structural column of A_p staged in shared
// memory (all m slots: the live ones for the dot product, the others for the
// unit columns of the basic slacks), or nullptr for a slack, whose unit vector
// sits at live slot aq_unit.  rh: rho / alpha_r in new slot order, zero past
// kn.  Row l of the CTA leaves alpha', bbar_i and its basic variable in
// ral/rb/rvar[l] (alpha' and the variable also in global memory for the ratio
// test of other CTAs); the ratios themselves are formed in row_record.
// Warp sum of a + b over the 32 lanes (every lane gets it) in 64-bit fixed
// point.  The values are aligned to the warp's largest binary exponent E
// (one redux): a value is t 2^(E - 1079) with |t| < 2^57, rounded to nearest;
// the t are added exactly by integer shuffles, and the sum is rounded to
// binary64 once (ll_scaled).  Relative to 2^(E - 1022), which bounds every
// |value|, the error is below 2^-51 plus the final rounding -- no more than
// the FP64 butterfly's -- and the sum does not depend on the lane order.  It
// spends no FP64 instruction (each holds the FP64 pipe for ~64 cycles on this
// chip, and the butterfly needs six per row).  Subnormal, infinite and NaN
// inputs take the FP64 butterfly.
__device__ __forceinline__ double warp_sum2_fixed(double a, double b) {
    const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
    const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
    const bool odd = (ea == 0 && (ua << 1) != 0) || (eb == 0 && (ub << 1) != 0) || ea == 0x7ff || eb == 0x7ff;
    const unsigned emax = __reduce_max_sync(0xffffffffu, (unsigned)max(ea, eb));
    if (__any_sync(0xffffffffu, odd) || emax == 0) return warp_sum(a + b);
    auto fix = [emax](unsigned long long u, int e) -> long long {
        if (e == 0) return 0;  // +-0
        const long long mant = (long long)((u & 0xFFFFFFFFFFFFFull) | (1ull << 52));
        const int sh = e - (int)emax + 4;  // at most 4
        long long t = 0;
        if (sh >= 0) t = mant << sh;
        else if (sh > -60) t = (mant + (1ll << (-sh - 1))) >> (-sh);
        return (u >> 63) ? -t : t;
    };
    long long t = fix(ua, ea) + fix(ub, eb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t == 0 ? 0.0 : ll_scaled(t, (int)emax - 1079);
}

// upd: which rows take the pending rank-1 update here -- kUpdAll, kUpdRowR
// (only row r: the others were updated by the update warps while the rest of
// the CTA priced), kUpdButR (every row but r, no FTRAN: the update warps), or
// kUpdNone.  Warps w0 .. w0 + nwarps - 1 share the CTA's rows.
enum { kUpdNone = 0, kUpdAll = 1, kUpdRowR = 2, kUpdButR = 3 };

__device__ void update_block_s(const DevState& s, const SlotMoves& v, int r, int q_new, int upd, bool do_ftran,
                               const double* acur, double* anxt, const double* aqs, int aq_unit, const double* rh,
                               double* ral, double* rb, int* rvar, int w0, int nwarps) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31;
    const int warp = (int)(threadIdx.x >> 5) - w0, nw = nwarps;
    const int kn = v.kn;
    const int kh = (kn + 1) >> 1;  // double2 units covering the live slots
    const double2* aq2 = reinterpret_cast<const double2*>(aqs);
    const double2* rh2 = reinterpret_cast<const double2*>(rh);
    const int G = gridDim.x;
    const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
    for (int l = warp; l < owned; l += nw) {
        const int i = blockIdx.x + G * l;
        const bool do_upd = upd == kUpdAll || (upd == kUpdRowR && i == r) || (upd == kUpdButR && i != r);
        if (!do_upd && !do_ftran) continue;
        double* rowd = s.bp + (size_t)i * P.ld;
        double2* row = reinterpret_cast<double2*>(rowd);
        // per-row scalars, all issued before the row streams in
        const int us = (do_ftran && aqs) ? __ldcg(s.uslot + i) : -1;
        const double na = (do_upd && i != r) ? -__ldcg(acur + i) : 0.0;
        const double bte = (do_upd && i != r && v.src_te >= 0) ? __ldcg(rowd + v.src_te) : 0.0;
        const double bb = do_ftran ? __ldcg(s.bbar + i) : 0.0;
        const int var = do_ftran ? (i == r && upd != kUpdNone ? q_new : __ldcg(s.basis + i)) : 0;
        double a0 = 0.0, a1 = 0.0;
        if (do_upd && i == r) {
            // row r becomes rho / alpha_r (every slot, the moved ones included)
            for (int k = lane; k < kh; k += 32) {
                const double2 nv = rh2[k];
                __stcs(row + k, nv);
                if (do_ftran) {
                    const int t0 = 2 * k, t1 = t0 + 1;
                    const double2 w = aqs ? aq2[k] : make_double2(t0 == aq_unit ? 1.0 : 0.0, t1 == aq_unit ? 1.0 : 0.0);
                    a0 = fma(nv.x, w.x, a0);
                    if (t1 < kn) a1 = fma(nv.y, w.y, a1);
                }
            }
        } else {
            const bool st = na != 0.0;
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
                        if (st) {
                            if (do_ftran) __stcs(row + k, nv);
                            else __stcg(row + k, nv);  // read again by the next FTRAN
                        }
                    }
                    if (do_ftran) {
                        const double2 w = aqs ? aq2[k] : make_double2(t0 == aq_unit ? 1.0 : 0.0, t1 == aq_unit ? 1.0 : 0.0);
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
            const double al = warp_sum2_fixed(a0, a1);
            if (lane == 0) {
                const double alf = al + (us >= 0 ? aqs[us] : 0.0);
                anxt[i] = alf;
                s.row_var[i] = var;
                ral[l] = alf;
                rb[l] = bb;
                rvar[l] = var;
            }
        }
    }
}

// The CTA's ratio-test record from its rows' (alpha', bbar, variable): its
// smallest ratio, and its best row and tie count under that ratio's tie
// threshold (one warp, one lane per row).  On this chip every FP64
// instruction holds a scheduler's FP64 pipe for 64 cycles whatever the number
// of active lanes, so the ratios of 32 rows are formed by one warp-wide
// division; the minimum, the tie band and the largest pivot are taken on
// integer keys, across the warp by redux (a dependent shuffle costs more).
__device__ void row_record(const Params& P, int owned, bool bland, const double* ral, const double* rb,
                           const int* rvar, RowRec* out) {
    const int lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const long long kpiv = dkey(P.tol_piv), kbig = dkey(DBL_MAX);
    // pass 1: ratios and their minimum
    long long kmin_l = kbig;
    double th0 = DBL_MAX;  // the first 32 rows' ratios, kept for pass 2
    for (int l0 = 0; l0 < owned; l0 += 32) {
        const int l = l0 + lane;
        const double al = l < owned ? ral[l] : 0.0;
        const bool ok = l < owned && dkey(al) > kpiv;
        const double th = ok ? rb[l] / al : DBL_MAX;
        if (l0 == 0) th0 = th;
        kmin_l = min(kmin_l, dkey(th));
    }
    const long long kmin = warp_min_key(kmin_l);
    const double tmin = kdouble(kmin);
    const double thr = kmin == kbig ? DBL_MAX : tmin + P.tol_tie * fmax(1.0, fabs(tmin));
    const long long kthr = dkey(thr);
    // pass 2: the tie band, its size and best row (largest pivot, then smallest
    // basic index; Bland: smallest basic index), lane by lane
    long long ka = LLONG_MIN;
    int bvar = INT_MAX, bl = -1, cnt = 0;
    double bth = 0.0;
    if (kmin != kbig) {
        for (int l0 = 0; l0 < owned; l0 += 32) {
            const int l = l0 + lane;
            const double al = l < owned ? ral[l] : 0.0;
            const long long kal = dkey(al);
            const bool ok = l < owned && kal > kpiv;
            const double th = l0 == 0 ? th0 : (ok ? rb[l] / al : DBL_MAX);
            if (ok && dkey(th) <= kthr) {
                cnt++;
                const int v = rvar[l];
                const bool better = bl < 0 || (bland ? v < bvar : (kal > ka || (kal == ka && v < bvar)));
                if (better) { ka = kal; bvar = v; bl = l; bth = th; }
            }
        }
    }
    const int tot = __reduce_add_sync(0xffffffffu, cnt);
    long long kbest;
    const int win = bland ? warp_argmin_index(bvar, bl >= 0)
                          : warp_argmax_key(ka, bvar, bl >= 0, kbest);
    if (win < 0 ? lane == 0 : lane == win) {
        RowRec rp;
        rp.tmin = kmin; rp.thr = kthr;
        rp.a = win >= 0 ? kdouble(ka) : 0.0;
        rp.th = win >= 0 ? bth : 0.0;
        rp.var = win >= 0 ? bvar : 0; rp.row = win >= 0 ? (int)blockIdx.x + G * bl : -1;
        rp.cnt = tot; rp.pad_ = 0;
        *out = rp;
    }
}

// ---- lexicographic leaving rule on the slack-structured inverse ---------------------
// Row i of B^-1 at constraint k is bp[i][slot(k)] when row k is live (slot <
// kn), else the unit column of row k's basic slack: 1 where that slack is the
// basic variable of position i, 0 elsewhere.  Rows i and r, each divided by its
// alpha, are compared in constraint order by one warp, kLexPer x 32 constraints
// per round trip (all loads of a round issued before any test), as x_i a_r
// against x_r a_i (both alphas are positive): -1 if row i comes first, +1 if
// row r does, 0 if every entry agrees within tau relative (the result in every
// lane).
constexpr int kLexPer = 8;

__device__ int lex_cmp_s(const DevState& s, const double* anxt, const int32_t* rs, int kn, int i, int r,
                         double tau) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31;
    const double ai = __ldcg(anxt + i), ar = __ldcg(anxt + r);
    const int vi = __ldcg(s.row_var + i), vr = __ldcg(s.row_var + r);
    const double* bi = s.bp + (size_t)i * P.ld;
    const double* br = s.bp + (size_t)r * P.ld;
    const double aa = ai * ar;
    for (int k0 = 0; k0 < P.m; k0 += 32 * kLexPer) {
        int slot[kLexPer];
#pragma unroll
        for (int u = 0; u < kLexPer; ++u) {
            const int k = k0 + 32 * u + lane;
            slot[u] = k < P.m ? __ldcg(rs + k) : -1;
        }
        double x[kLexPer], y[kLexPer];
#pragma unroll
        for (int u = 0; u < kLexPer; ++u) {
            const int k = k0 + 32 * u + lane;
            if (slot[u] >= 0 && slot[u] < kn) {
                x[u] = __ldcg(bi + slot[u]);
                y[u] = __ldcg(br + slot[u]);
            } else {
                x[u] = vi == P.n + k ? 1.0 : 0.0;
                y[u] = vr == P.n + k ? 1.0 : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < kLexPer; ++u) {
            int code = 0;  // 1 for a difference, sign in bit 2
            if (slot[u] >= 0 && ((__double_as_longlong(x[u]) | __double_as_longlong(y[u])) << 1) != 0) {
                const double a = x[u] * ar, b = y[u] * ai;
                if (fabs(a - b) > tau * fmax(aa, fmax(fabs(a), fabs(b)))) code = 1 | (a < b ? 4 : 0);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, code != 0);
            if (bal) {
                const int cd = __shfl_sync(0xffffffffu, code, __ffs(bal) - 1);
                return (cd & 4) ? -1 : 1;
            }
        }
    }
    return 0;
}

// row c leaves before row b: lexicographically smaller, exact ties to the smaller basic index
__device__ __forceinline__ bool lex_before_s(const DevState& s, const double* anxt, const int32_t* rs, int kn,
                                             int c, int b, double tau) {
    const int cmp = lex_cmp_s(s, anxt, rs, kn, c, b, tau);
    return cmp < 0 || (cmp == 0 && __ldcg(s.row_var + c) < __ldcg(s.row_var + b));
}

// The tie set's lexicographically smallest row (every thread of the CTA; the
// result in every thread).  The tie set is that of the ratio test: alpha_i >
// tol_piv and bbar_i <= thr alpha_i.  Warp w scans its contiguous range of
// rows in order, keeping the row that leaves first; the warps' rows then meet
// in a binary tree in warp order.  The comparisons follow the same fixed
// schedule in every CTA, so every CTA picks the same row.
__device__ int lex_pick_s(const DevState& s, const double* anxt, const int32_t* rs, int kn, double thr) {
    const Params& P = s.p;
    __shared__ int wbest[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per = (P.m + nw - 1) / nw;
    const int r0 = warp * per, r1 = min(P.m, r0 + per);
    int best = -1;
    for (int base = r0; base < r1; base += 32) {
        const int i = base + lane;
        bool tied = false;
        if (i < r1) {
            const double al = __ldcg(anxt + i), bb = __ldcg(s.bbar + i);
            tied = al > P.tol_piv && bb <= thr * al;
        }
        unsigned bal = __ballot_sync(0xffffffffu, tied);
        while (bal) {
            const int c = base + __ffs(bal) - 1;
            bal &= bal - 1;
            if (best < 0 || lex_before_s(s, anxt, rs, kn, c, best, P.tol_tie)) best = c;
        }
    }
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    for (int h = 1; h < nw; h *= 2) {
        // round h: warp w (a multiple of 2h) meets warp w + h
        if (warp % (2 * h) == 0 && warp + h < nw) {
            const int a = wbest[warp], c = wbest[warp + h];
            int win = a;
            if (c >= 0 && (a < 0 || lex_before_s(s, anxt, rs, kn, c, a, P.tol_tie))) win = c;
            __syncwarp();
            if (lane == 0) wbest[warp] = win;
        }
        __syncthreads();
    }
    return wbest[0];
}

__device__ __forceinline__ PriceRec to_price_rec(const Cand& c) {
    PriceRec r;
    r.d_all = c.d_all; r.d_nt = c.d_nt;  // keys
    r.j_all = c.j_all; r.j_nt = c.j_nt; r.j_min = c.j_min; r.j_pr = c.j_pr;
    r.d_min = c.d_min; r.d_pr = c.d_pr;
    r.k_pr = c.k_pr; r.pad_[0] = r.pad_[1] = r.pad_[2] = 0;
    return r;
}

// CHUZC over the per-CTA partials (result in thread 0): the warps that hold
// them take one record per lane (four 16-byte loads), reduce it across the
// warp by redux, and warp 0 reduces the warps' results the same way.
// cand_warp_reduce restricted to the categories a step can use: the smallest
// improving index only under the Bland safety net, the priority candidate only
// while a priority list is set (otherwise no candidate carries one).  The
// categories left out keep their initial values, which are also what a full
// reduction would give for them.
__device__ Cand cand_warp_reduce_sel(const Cand& c, bool need_min, bool need_pr) {
    Cand g;
    cand_init(g);
    long long kb;
    int w = warp_argmax_key(c.d_all, c.j_all, c.j_all >= 0, kb);
    if (w >= 0) { g.d_all = kb; g.j_all = __shfl_sync(0xffffffffu, c.j_all, w); }
    w = warp_argmax_key(c.d_nt, c.j_nt, c.j_nt >= 0, kb);
    if (w >= 0) { g.d_nt = kb; g.j_nt = __shfl_sync(0xffffffffu, c.j_nt, w); }
    if (need_min) {
        w = warp_argmin_index(c.j_min, c.j_min >= 0);
        if (w >= 0) { g.j_min = __shfl_sync(0xffffffffu, c.j_min, w); g.d_min = __shfl_sync(0xffffffffu, c.d_min, w); }
    }
    if (need_pr) {
        w = warp_argmax_key(c.d_pr, c.j_pr, c.j_pr >= 0, kb);
        if (w >= 0) {
            g.d_pr = kb;
            g.j_pr = __shfl_sync(0xffffffffu, c.j_pr, w);
            g.k_pr = __shfl_sync(0xffffffffu, c.k_pr, w);
        }
    }
    return g;
}

__device__ Cand reduce_price_parts_s(const PriceRec* part, int nparts, bool need_min, bool need_pr) {
    __shared__ Cand wsh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwu = (nparts + 31) >> 5;  // warps holding partials
    Cand g;
    cand_init(g);
    if (warp < nwu) {
        for (int b = threadIdx.x; b < nparts; b += nwu * 32) {
            const longlong2* p2 = reinterpret_cast<const longlong2*>(part + b);
            const int4* p4 = reinterpret_cast<const int4*>(part + b);
            const longlong2 w0 = __ldcg(p2);
            const int4 w1 = __ldcg(p4 + 1);
            const longlong2 w2 = __ldcg(p2 + 2);
            const int4 w3 = __ldcg(p4 + 3);
            Cand o;
            o.d_all = w0.x; o.d_nt = w0.y;
            o.j_all = w1.x; o.j_nt = w1.y; o.j_min = w1.z; o.j_pr = w1.w;
            o.d_min = w2.x; o.d_pr = w2.y;
            o.k_pr = w3.x;
            cand_merge(g, o);
        }
        g = cand_warp_reduce_sel(g, need_min, need_pr);
        if (lane == 0) wsh[warp] = g;
    }
    __syncthreads();
    if (warp == 0) {
        if (lane < nwu) g = wsh[lane];
        else cand_init(g);
        g = cand_warp_reduce_sel(g, need_min, need_pr);
    }
    return g;
}

__device__ PricePatch pivot_patch(const SlotMoves& v, int q, int leave, bool push, int tabu_until) {
    PricePatch p = no_patch();
    p.basic_j = q;
    p.free_j = leave;
    if (push) { p.tabu_j = leave; p.tabu_until = tabu_until; }
    // the slot -> row entries that differ from the current map, in the
    // precedence order of moved_slot_row
    if (v.ent >= 0) {
        p.sp_slot[p.nsp] = v.te; p.sp_row[p.nsp] = v.w; ++p.nsp;
        p.sp_slot[p.nsp] = v.k1 - 1; p.sp_row[p.nsp] = v.ent; ++p.nsp;
    }
    if (v.join >= 0) {
        p.sp_slot[p.nsp] = v.k0; p.sp_row[p.nsp] = v.join; ++p.nsp;
        p.sp_slot[p.nsp] = v.tl; p.sp_row[p.nsp] = v.u; ++p.nsp;
    }
    return p;
}

// One step = apply the pivot chosen by the last ratio test and price (A),
// grid barrier, CHUZC + UPDATE/FTRAN + the CTA's ratio-test record (B), grid
// barrier, CHUZR (C).  Step (A) needs no barrier of its own: every CTA
// computes y and rho / alpha_r in the new slot order for itself from the
// pivot row of B^-1 (final since the last barrier), moves the A_p rows of the
// columns it prices and updates bbar on the rows it owns; the pivot's
// changes to pos, tabu_until and the slot map reach PRICE as a patch while
// the lead CTA writes them to memory (visible to all after the next barrier).
// The y of the next step is written by the lead CTA to the other half of a
// double buffer.
// ---- exact PRICE through an FP32 screen ---------------------------------------------
// FP32 runs at about 58x the FP64 rate on this chip.  Every listed column j is
// first priced in FP32 -- s~_j = sum_t y32_t a32_tj with y32, a32 the FP32
// roundings -- together with S~_j = sum_t |y32_t| |a32_tj|.  With u = 2^-24,
// k summed rows and |y|, |a| within [2^-100, 2^40] or zero, the FP32 result
// satisfies |s~_j - y^T a_j| <= gamma_{d+2} / ((1 - u)^2 (1 - gamma_d)) S~_j,
// where gamma_n = n u / (1 - n u) and d = T + 5 bounds the roundings any term
// goes through: the T fused multiply-adds of its lane's chain (T = 4 per 128
// rows) and the five butterfly levels; the +2 are the roundings of y and a to
// FP32, and the denominator turns the computed S~_j into an upper bound of
// sum |y_t a_tj| (Higham, Accuracy and Stability of Numerical Algorithms,
// ch. 3, for sums along any tree).  (d + 3) u 1.01 S~_j covers it for
// d u < 1e-3 and (k + 8) 2^-100 covers underflow.  The interval
// [c_j - s~_j - E_j, c_j - s~_j + E_j] is formed in FP32 with directed
// rounding from c_j rounded down and up (kept per column), so it contains d_j
// and costs no FP64 instruction.
// A column can be the block's exact argmax of a category (all nonbasic,
// non-tabu, non-tabu prioritised) only if its interval reaches the largest
// lower end of the category; exactly those columns are re-priced in FP64 with
// the arithmetic of the full PRICE (same segments, lanes and pairing order), so
// the block's candidates -- and the pivots -- are bit-identical to it.  The
// smallest-index rule of the safety net needs every improving column, so
// under it the full FP64 PRICE runs.
constexpr int kScreenMaxList = kPriceThreads;

// order-preserving integer image of a float (no NaN; -0 and +0 share one key)
__device__ __forceinline__ int fkey(float x) {
    int b = __float_as_int(x);
    if ((b & 0x7fffffff) == 0) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffff);
}

// kNC columns at once: s[c] = sum y a_c and a[c] = sum |y| |a_c| over the n4
// float4 groups, lane-strided, then across the warp by butterflies (every lane
// gets the sums): per lane a chain of 4 fused multiply-adds per float4 in
// increasing k, then five butterfly levels, as the screen's error bound counts.
template <int kNC>
__device__ __forceinline__ void dotn_f32(const float4* const (&col)[kNC], const float4* y4, int n4, int lane,
                                         float (&sv)[kNC], float (&av)[kNC]) {
#pragma unroll
    for (int c = 0; c < kNC; ++c) sv[c] = av[c] = 0.f;
#pragma unroll 2
    for (int k = lane; k < n4; k += 32) {
        const float4 y = y4[k];
        float4 u[kNC];
#pragma unroll
        for (int c = 0; c < kNC; ++c) u[c] = __ldcg(col[c] + k);
#pragma unroll
        for (int c = 0; c < kNC; ++c) {
            sv[c] = fmaf(u[c].x, y.x, sv[c]); sv[c] = fmaf(u[c].y, y.y, sv[c]);
            sv[c] = fmaf(u[c].z, y.z, sv[c]); sv[c] = fmaf(u[c].w, y.w, sv[c]);
            av[c] = fmaf(fabsf(u[c].x), fabsf(y.x), av[c]); av[c] = fmaf(fabsf(u[c].y), fabsf(y.y), av[c]);
            av[c] = fmaf(fabsf(u[c].z), fabsf(y.z), av[c]); av[c] = fmaf(fabsf(u[c].w), fabsf(y.w), av[c]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < kNC; ++c) {
            sv[c] += __shfl_xor_sync(0xffffffffu, sv[c], o);
            av[c] += __shfl_xor_sync(0xffffffffu, av[c], o);
        }
    }
}

// k_iterate_s prices with warps 0 .. kPriceWarpsS-1 while the others apply the
// pending rank-1 update to the CTA's rows; the pricing warps synchronise on
// named barrier 1 (kPT threads), never on the block barrier.
constexpr int kPriceWarpsS = 20;
constexpr int kScreenCols = 2;  // columns one warp screens at a time
constexpr int kPriceGroupS = 32 * kPriceWarpsS;

template <int kPT>
__device__ __forceinline__ void group_sync() {
    if (kPT == kUpdateThreads) __syncthreads();
    else asm volatile("bar.sync 1, %0;\n" ::"n"(kPT) : "memory");
}

// The block's list of nonbasic owned columns kept from the last step (jl, jc,
// jt, jr, count): the pivot made column basic_j basic and free_j nonbasic (each
// only if it is a structural this block owns), and free_j carries its patched
// tabu expiry; no other listed entry changes.  Entry order is immaterial to the
// screened PRICE (every candidate comparison breaks ties by column index).
template <int kPT>
__device__ int list_patch(const DevState& s, const PricePatch& pp, int* jl, double* jc, int* jt, int* jr,
                          int* cnt_sh) {
    __shared__ int rm_sh;
    const int G = gridDim.x;
    const int bj = pp.basic_j, fj = pp.free_j;
    const bool rm = bj >= 0 && bj < s.p.n && bj % G == (int)blockIdx.x;
    const bool add = fj >= 0 && fj < s.p.n && fj % G == (int)blockIdx.x;
    const int cnt = *cnt_sh;
    // the joining column's cost, tabu expiry and priority, loaded before the search
    double fc = 0.0;
    int ft = 0, fr = kNoRank;
    if (threadIdx.x == 0 && add) {
        fc = s.c[fj];
        ft = patched_tabu(s, pp, fj);
        fr = s.rank[fj];
    }
    if (threadIdx.x == 0) rm_sh = -1;
    group_sync<kPT>();
    if (rm)
        for (int e = threadIdx.x; e < cnt; e += kPT)
            if (jl[e] == bj) rm_sh = e;
    group_sync<kPT>();
    if (threadIdx.x == 0) {
        int c = cnt;
        const int e = rm_sh;
        if (e >= 0) {
            --c;
            jl[e] = jl[c]; jc[e] = jc[c]; jt[e] = jt[c]; jr[e] = jr[c];
        }
        if (add) {
            jl[c] = fj; jc[c] = fc; jt[c] = ft; jr[c] = fr;
            ++c;
        }
        *cnt_sh = c;
    }
    group_sync<kPT>();
    return *cnt_sh;
}

// Lists, in order, the nonbasic columns among the block's owned columns
// lb .. lb+kPT-1 (block b owns j = b, b+G, ...), with their cost, tabu
// expiry and priority, all loaded in the same round trip, by the kPT pricing
// threads.  Returns the count.
template <int kPT>
__device__ int list_nonbasic_g(const DevState& s, const PricePatch& pp, int lb, int owned, int* jl, double* jc,
                               int* jt, int* jr, int* wcnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    const int l = lb + (int)threadIdx.x;
    const int jj = (int)blockIdx.x + G * l;
    bool nb = false;
    double cj = 0.0;
    int tj = 0, rj = kNoRank;
    if (l < owned) {
        const int pj = __ldcg(s.pos + jj);
        cj = s.c[jj];
        tj = patched_tabu(s, pp, jj);
        rj = s.rank[jj];
        nb = jj == pp.basic_j ? false : (jj == pp.free_j ? true : pj < 0);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, nb);
    if (lane == 0) wcnt[warp] = __popc(bal);
    group_sync<kPT>();
    int before = 0, cnt = 0;
    for (int w = 0; w < kPT / 32; ++w) {
        const int cw = wcnt[w];
        if (w < warp) before += cw;
        cnt += cw;
    }
    if (nb) {
        const int e = before + __popc(bal & ((1u << lane) - 1u));
        jl[e] = jj;
        jc[e] = cj;
        jt[e] = tj;
        jr[e] = rj;
    }
    group_sync<kPT>();
    return cnt;
}

// cand_block_reduce over the kPT pricing threads (the result in thread 0);
// the screened PRICE never runs under the Bland safety net
template <int kPT>
__device__ Cand cand_group_reduce(Cand c, bool need_pr) {
    __shared__ Cand csh[32];
    c = cand_warp_reduce_sel(c, false, need_pr);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    group_sync<kPT>();
    if (lane == 0) csh[wid] = c;
    group_sync<kPT>();
    if (wid == 0) {
        if (lane < kPT / 32) c = csh[lane];
        else cand_init(c);
        c = cand_warp_reduce_sel(c, false, need_pr);
    }
    return c;
}

// list_ok (shared, in the calling kernel): the list of the last step is
// current up to this step's pivot (set here after a one-chunk list; the caller
// clears it when a step prices by the full FP64 path or a launch begins).
template <int kPT>
__device__ Cand price_block_screened(const DevState& s, int it, const double* ysh, const float* ysh32, int kk,
                                     const int32_t* slack_rows, int nslack, const PricePatch& pp, int* list_ok) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPT >> 5;
    const int G = gridDim.x;
    const int half = P.ld >> 1;
    const long long ktol = dkey(P.tol_d);
    __shared__ int jl[kScreenMaxList];
    __shared__ double jc[kScreenMaxList];
    __shared__ int jt[kScreenMaxList], jr[kScreenMaxList];
    __shared__ int wcnt[kPriceThreads / 32];
    __shared__ int klo[kScreenMaxList], khi[kScreenMaxList];
    __shared__ int bandsh[3][32];
    __shared__ int rl[kScreenMaxList];
    __shared__ int nrl;
    __shared__ double part[2][kPriceThreads / 64];
    __shared__ int list_cnt;  // entries of the kept list
    Cand cand;
    cand_init(cand);
    // slack candidates: exact (d = -y), offered directly, loads issued first
    int sj = -1;
    const int si = blockIdx.x + G * threadIdx.x;
    if (si < nslack) {
        int row = -1;
        for (int e = 0; e < pp.nsp && row < 0; ++e)
            if (pp.sp_slot[e] == si) row = pp.sp_row[e];
        if (row < 0) row = __ldcg(slack_rows + si);
        sj = P.n + row;
    }
    // its tabu expiry and priority, loaded now and used twice below
    const int sj_tabu = sj >= 0 ? patched_tabu(s, pp, sj) : 0;
    const int sj_rank = sj >= 0 ? s.rank[sj] : kNoRank;
    const int n4 = kk >> 2;
    const int depth = 4 * ((n4 + 31) >> 5) + 5;  // fused multiply-adds per lane + butterfly levels
    const float umul = __fmul_ru((float)(depth + 3), 6.0200691e-8f);  // (d + 3) u 1.01, rounded up
    const float uabs = __fmul_ru((float)(kk + 8), 7.8886091e-31f);     // (k + 8) 2^-100: underflow
    const int owned = (P.n - (int)blockIdx.x + G - 1) / G;
    const bool keep = owned <= kPT;  // one chunk: the list is kept from step to step
    const float4* y4 = reinterpret_cast<const float4*>(ysh32);
    for (int lb = 0; lb < owned; lb += kPT) {
        const int cnt = (keep && *list_ok) ? list_patch<kPT>(s, pp, jl, jc, jt, jr, &list_cnt)
                                           : list_nonbasic_g<kPT>(s, pp, lb, owned, jl, jc, jt, jr, wcnt);
        if (keep && threadIdx.x == 0) list_cnt = cnt;
        // (1) FP32 screen, kScreenCols listed columns per warp (the last
        // group repeats its final column; the repeat writes the same keys)
        for (int e0 = kScreenCols * warp; e0 < cnt; e0 += kScreenCols * nw) {
            const float4* cp[kScreenCols];
            float cl[kScreenCols], ch[kScreenCols];
#pragma unroll
            for (int c = 0; c < kScreenCols; ++c) {
                const int j = jl[min(e0 + c, cnt - 1)];
                cp[c] = reinterpret_cast<const float4*>(s.A_p32 + (size_t)j * P.ld);
                cl[c] = ch[c] = 0.f;
                if (lane == 0) { cl[c] = __ldg(s.c32lo + j); ch[c] = __ldg(s.c32hi + j); }
            }
            float sv[kScreenCols], av[kScreenCols];
            dotn_f32<kScreenCols>(cp, y4, n4, lane, sv, av);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < kScreenCols; ++c) {
                    const int e = min(e0 + c, cnt - 1);
                    const float E = __fmaf_ru(umul, av[c], uabs);
                    klo[e] = fkey(__fsub_rd(cl[c], __fadd_ru(sv[c], E)));
                    khi[e] = fkey(__fadd_ru(__fsub_ru(ch[c], sv[c]), E));
                }
            }
        }
        group_sync<kPT>();
        // (2) the largest lower end of each category (slacks exact)
        int b0 = INT_MIN, b1 = INT_MIN, b2 = INT_MIN;
        for (int e = threadIdx.x; e < cnt; e += kPT) {
            const int lo = klo[e];
            const bool nt = jt[e] <= it;
            b0 = max(b0, lo);
            if (nt) b1 = max(b1, lo);
            if (nt && jr[e] != kNoRank) b2 = max(b2, lo);
        }
        if (lb == 0 && sj >= 0) {
            const int kd = fkey(__double2float_rd(-ysh[si]));  // exact value, its lower FP32 bound
            const bool nt = sj_tabu <= it;
            b0 = max(b0, kd);
            if (nt) b1 = max(b1, kd);
            if (nt && sj_rank != kNoRank) b2 = max(b2, kd);
        }
        // across the warp, then across the 32 warps, by redux
        b0 = __reduce_max_sync(0xffffffffu, b0);
        b1 = __reduce_max_sync(0xffffffffu, b1);
        b2 = __reduce_max_sync(0xffffffffu, b2);
        if (lane == 0) { bandsh[0][warp] = b0; bandsh[1][warp] = b1; bandsh[2][warp] = b2; }
        if (threadIdx.x == 0) nrl = 0;
        group_sync<kPT>();
        const int L0 = __reduce_max_sync(0xffffffffu, lane < nw ? bandsh[0][lane] : INT_MIN);
        const int L1 = __reduce_max_sync(0xffffffffu, lane < nw ? bandsh[1][lane] : INT_MIN);
        const int L2 = __reduce_max_sync(0xffffffffu, lane < nw ? bandsh[2][lane] : INT_MIN);
        // (3) the columns whose interval reaches a category's lower end
        for (int e = threadIdx.x; e < cnt; e += kPT) {
            const int hi = khi[e];
            const bool nt = jt[e] <= it;
            if (hi >= L0 || (nt && hi >= L1) || (nt && jr[e] != kNoRank && hi >= L2)) rl[atomicAdd(&nrl, 1)] = e;
        }
        group_sync<kPT>();
        // (4) exact FP64 re-price, two warps (the two row segments) per column
        const int nr = nrl;
        const int nch = (kk >> 1) >> 5;
        const int seg = warp & 1;
        const int k0 = 32 * (seg * nch / 2), k1 = 32 * ((seg + 1) * nch / 2);
        const double2* A2 = reinterpret_cast<const double2*>(s.A_p);
        const double2* y2 = reinterpret_cast<const double2*>(ysh);
        for (int r0 = 0; r0 < nr; r0 += nw / 2) {
            const int slot = warp >> 1;
            const int ri = r0 + slot;
            if (ri < nr) {
                const int col = jl[rl[ri]];
                double acc[1];
                dot_cols<1, true>(A2, &col, half, y2, k0, k1, lane, acc);
                const double t = pair_sum(acc[0]);
                if (lane == 0) part[seg][slot] = t;
            }
            group_sync<kPT>();
            if ((int)threadIdx.x < nw / 2 && r0 + (int)threadIdx.x < nr) {
                const int e = rl[r0 + threadIdx.x];
                const double sum = part[0][threadIdx.x] + part[1][threadIdx.x];
                cand_offer(cand, jc[e] - sum, jl[e], jt[e] <= it, ktol, jr[e]);
            }
            group_sync<kPT>();
        }
    }
    if (threadIdx.x == 0) *list_ok = keep ? 1 : 0;  // every thread read it before the loop's barriers
    if (sj >= 0) cand_offer(cand, -ysh[si], sj, sj_tabu <= it, ktol, sj_rank);
    for (int i = si + G * kPT; i < nslack; i += G * kPT) {
        int row = -1;
        for (int e = 0; e < pp.nsp && row < 0; ++e)
            if (pp.sp_slot[e] == i) row = pp.sp_row[e];
        if (row < 0) row = __ldcg(slack_rows + i);
        const int j = P.n + row;
        cand_offer(cand, -ysh[i], j, patched_tabu(s, pp, j) <= it, ktol, s.rank[j]);
    }
    return cand_group_reduce<kPT>(cand, P.prio != 0);
}

__global__ void __launch_bounds__(kUpdateThreads, 1) k_iterate_s(DevState s, int iters) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    extern __shared__ double sh[];  // y, rho / alpha_r, entering column (ld doubles each)
    __shared__ IterState S;
    __shared__ volatile int fail;
    __shared__ SlotMoves mv;
    __shared__ PricePatch ppat;
    __shared__ int nflag, flagged;
    __shared__ long long wmin_sh[32], wthr_sh[32];
    __shared__ double rinv_sh;
    __shared__ int screen_sh;
    __shared__ int list_ok;  // the screened PRICE's list of nonbasic columns is current
    __shared__ int wcnt_sh[32];
    __shared__ double ral[kMaxOwnedRows], rb[kMaxOwnedRows];
    __shared__ int rvar[kMaxOwnedRows];
    unsigned epoch = 0;
    const bool lead = blockIdx.x == 0;
    const int G = gridDim.x;
    const int owned = (P.m - (int)blockIdx.x + G - 1) / G;
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
        screen_sh = P.screen && C->screen_off == 0;
        list_ok = 0;
    }
    if (!grid_barrier(s.gbar, epoch, &fail)) {
        if (lead && threadIdx.x == 0) C->err = kErrTimeout;
        return;
    }
    const bool screen_ok = screen_sh != 0;
    double* ysh = sh;
    double* rh = sh + P.ld;
    double* aqs = sh + 2 * (size_t)P.ld;
    float* ysh32 = reinterpret_cast<float*>(sh + 3 * (size_t)P.ld);  // y in FP32 for the screen
    for (int step = 0; step < iters; ++step) {
        // ---- (A) apply the pivot chosen by the last ratio test, then PRICE
        const bool piv = S.status == kRunning && S.r >= 0 && S.r < P.m && S.q >= 0;
        const int r = S.r, q = S.q, par = S.par;
        const double* acur = s.alpha + (size_t)S.abuf * P.ld;
        const double ar = S.alpha_r, th = S.theta, dq = S.dq;
        // this thread's first pair of the pivot row of B^-1 and of the old y,
        // loaded before the slot moves are known (k grows by one at most)
        const int kpre = min(P.ld, (S.k + 1 + 63) & ~63);
        double2 pre_rb = make_double2(0.0, 0.0), pre_yb = make_double2(0.0, 0.0);
        if (2 * (int)threadIdx.x < kpre) {
            if (piv) pre_rb = __ldcg(reinterpret_cast<const double2*>(s.bp + (size_t)r * P.ld) + threadIdx.x);
            pre_yb = __ldcg(reinterpret_cast<const double2*>(s.yp + (size_t)par * P.ld) + threadIdx.x);
        }
        if (threadIdx.x == 0) {
            if (piv) {
                mv = slot_moves(s, S.leave, S.q, S.k, par);
                const bool degenerate = th <= P.tol_tie;
                const bool push = P.tabu_tenure > 0 && (S.tcount > 1 || degenerate);
                ppat = pivot_patch(mv, S.q, S.leave, push, S.it + 1 + P.tabu_tenure);
                rinv_sh = 1.0 / ar;
            } else {
                mv.join = mv.ent = -1;
                mv.k0 = mv.k1 = mv.kn = S.k;
                mv.tl = mv.u = mv.te = mv.w = mv.J = mv.src_te = -1;
                ppat = no_patch();
            }
        }
        __syncthreads();  // the moves are visible and every thread has read the state
        const int kn = mv.kn;
        const int kk = min(P.ld, (kn + 63) & ~63);  // live slots rounded up to a double2 sweep
        const double rinv = rinv_sh;
        if (threadIdx.x == 0) {
            if (piv) {
                if (lead) {
                    // the positions whose basic slack changed slot
                    s.uslot[r] = mv.ent >= 0 ? mv.k1 - 1 : -1;
                    if (mv.join >= 0 && mv.tl != mv.k0) s.uslot[__ldcg(s.pos + P.n + mv.u)] = mv.tl;
                }
                pivot_bookkeeping(s, S, lead);
                S.k = kn;
                S.par = par ^ 1;
            }
        }
        int ybig = 0;
        {
            // y and rho / alpha_r in the new slot order (every CTA, into shared memory)
            const double* yold = s.yp + (size_t)par * P.ld;
            double* ynew = s.yp + (size_t)(par ^ 1) * P.ld;
            const double* brow = s.bp + (size_t)(piv ? r : 0) * P.ld;
            // slot pairs in 16-byte loads; a moved slot reads its source itself
            for (int p = threadIdx.x; 2 * p < kk; p += blockDim.x) {
                const bool first = p == (int)threadIdx.x;  // kk <= kpre: prefetched above
                const double2 rb = first ? pre_rb
                                         : (piv ? __ldcg(reinterpret_cast<const double2*>(brow) + p) : make_double2(0.0, 0.0));
                const double2 yb = first ? pre_yb : __ldcg(reinterpret_cast<const double2*>(yold) + p);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int t = 2 * p + e;
                    double rn = 0.0, yv = 0.0;
                    if (t < kn) {
                        const int src = piv ? vec_src(mv, t) : t;
                        double rv = e ? rb.y : rb.x, yo = e ? yb.y : yb.x;
                        if (src == -2) { rv = 1.0; yo = 0.0; }
                        else if (src != t) { rv = __ldcg(brow + src); yo = __ldcg(yold + src); }
                        if (piv) {
                            rn = rv * rinv;  // one reciprocal per pivot: a division per slot in every CTA would load the FP64 pipe
                            yv = __dadd_rn(yo, __dmul_rn(dq, rn));
                        } else {
                            yv = yo;
                        }
                        if (lead && piv) ynew[t] = yv;
                    }
                    rh[t] = rn;
                    ysh[t] = yv;
                    ysh32[t] = (float)yv;
                    // screen range: |y| <= 2^40 (exponent field test, no FP64 instruction)
                    ybig |= ((__double_as_longlong(yv) >> 52) & 0x7ff) > 1023 + 40;
                }
            }
        }
        if (piv) {
            if (lead) {
                // the next copy of the slot maps
                const int32_t* sr0 = s.slot_row + (size_t)par * P.m;
                const int32_t* rs0 = s.row_slot + (size_t)par * P.m;
                int32_t* sr1 = s.slot_row + (size_t)(par ^ 1) * P.m;
                int32_t* rs1 = s.row_slot + (size_t)(par ^ 1) * P.m;
                for (int x = threadIdx.x; x < P.m; x += blockDim.x) {
                    const int a = __ldcg(sr0 + x), b = __ldcg(rs0 + x);
                    sr1[x] = moved_slot_row(mv, x, a);
                    rs1[x] = moved_row_slot(mv, x, b);
                }
            }
            if (mv.join >= 0 || mv.ent >= 0) {
                // A_p rows of the columns this CTA prices follow their slots
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
                for (int j = blockIdx.x + G * threadIdx.x; j < P.n && nm > 0; j += G * blockDim.x) {
                    double* col = s.A_p + (size_t)j * P.ld;
                    float* col32 = s.A_p32 + (size_t)j * P.ld;
                    double val[3];
                    float v32[3];
                    for (int e = 0; e < nm; ++e) { val[e] = __ldcg(col + src[e]); v32[e] = __ldcg(col32 + src[e]); }
                    for (int e = 0; e < nm; ++e) { col[dst[e]] = val[e]; col32[dst[e]] = v32[e]; }
                }
            }
            // bbar on the rows this CTA owns (their ratios are computed here too)
            for (int l = threadIdx.x; l < owned; l += blockDim.x) {
                const int i = blockIdx.x + G * l;
                const double bb = __ldcg(s.bbar + i), ak = __ldcg(acur + i);
                s.bbar[i] = (i == r) ? th : __dsub_rn(bb, __dmul_rn(ak, th));
            }
        }
        const bool yrange = __syncthreads_or(ybig) == 0;  // y, rho, the A_p moves and thread 0's bookkeeping are done
        bool upd_early = false;  // the rows but r took the pivot's update while the others priced
        if (S.status == kRunning) {
            const int32_t* sr = s.slot_row + (size_t)par * P.m;  // + the patch: the map after the moves
            // the FP32 screen unless the safety net needs every improving column
            // or y leaves the screen's range (then the full FP64 PRICE)
            const bool scr = screen_ok && yrange && !S.bland;
            if (scr) {
                // warps 0 .. kPriceWarpsS-1 price; the others apply the pivot's
                // rank-1 update to the CTA's rows but r (row r is read by every
                // CTA for its rho in this step, so it changes after the barrier)
                if ((int)(threadIdx.x >> 5) < kPriceWarpsS) {
                    const Cand bc =
                        price_block_screened<kPriceGroupS>(s, S.it, ysh, ysh32, kk, sr, kn, ppat, &list_ok);
                    if (threadIdx.x == 0) s.price_rec[blockIdx.x] = to_price_rec(bc);
                } else if (piv) {
                    update_block_s(s, mv, r, q, kUpdButR, false, acur, nullptr, nullptr, -1, rh, nullptr, nullptr,
                                   nullptr, kPriceWarpsS, kUpdateThreads / 32 - kPriceWarpsS);
                }
                upd_early = piv;
            } else {
                const Cand bc = price_block<true>(s, S.it, ysh, s.A_p, kk >> 1, sr, kn, ppat);
                if (threadIdx.x == 0) {
                    list_ok = 0;  // this step's pivot is not in the kept list
                    s.price_rec[blockIdx.x] = to_price_rec(bc);
                }
            }
            if (!grid_barrier(s.gbar, epoch, &fail)) break;
            // ---- (B) CHUZC (every CTA), then UPDATE + FTRAN + ratios
            const Cand g = reduce_price_parts_s(s.price_rec, G, S.bland != 0, P.prio != 0);
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
        }
        const bool do_upd = piv;
        const bool do_ftran = S.status == kRunning && S.q >= 0 && S.q < P.n + P.m;
        if (!do_upd && !do_ftran) break;
        if (do_upd && S.status != kRunning) {
            // no PRICE barrier in this step (the pivot's bookkeeping stopped the
            // run: a reinversion is due or the iteration limit is reached), yet
            // the owner of row r overwrites it below: every CTA must have read
            // it for its rho first (the status is the same in every CTA)
            if (!grid_barrier(s.gbar, epoch, &fail)) break;
        }
        const double* aqp = nullptr;
        int aq_unit = -1;
        if (do_ftran) {
            if (S.q < P.n) {
                // the entering column of A_p (every slot), staged in shared memory
                const double2* col = reinterpret_cast<const double2*>(s.A_p + (size_t)S.q * P.ld);
                double2* a2 = reinterpret_cast<double2*>(aqs);
                for (int t = threadIdx.x; t < (P.ld >> 1); t += blockDim.x) a2[t] = __ldcg(col + t);
                aqp = aqs;
            } else {
                const int row = S.q - P.n;
                aq_unit = moved_row_slot(mv, row, __ldcg(s.row_slot + (size_t)par * P.m + row));
            }
        }
        __syncthreads();
        const double* acur2 = s.alpha + (size_t)S.abuf * P.ld;
        double* anxt = s.alpha + (size_t)(S.abuf ^ 1) * P.ld;
        update_block_s(s, mv, r, q, do_upd ? (upd_early ? kUpdRowR : kUpdAll) : kUpdNone, do_ftran, acur2, anxt, aqp,
                       aq_unit, rh, ral, rb, rvar, 0, kUpdateThreads / 32);
        if (lead && threadIdx.x == 0) {
            S.bytes_update += (do_upd ? 16.0 : (do_ftran ? 8.0 : 0.0)) * P.m * (double)kn;
            S.n_update++;
        }
        if (!do_ftran) {
            if (threadIdx.x == 0) S.pending = 0;
            break;
        }
        __syncthreads();
        if (threadIdx.x < 32) row_record(P, owned, S.bland != 0, ral, rb, rvar, s.row_rec + blockIdx.x);
        if (!grid_barrier(s.gbar, epoch, &fail)) break;
        // ---- (C) CHUZR: minimum ratio, tie set, leaving row (every CTA), on
        // integer keys; the tie threshold comes with the record that holds
        // the minimum
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        RowRec rec;
        rec.tmin = dkey(DBL_MAX);
        rec.thr = rec.tmin;
        if ((int)threadIdx.x < G) {
            const longlong2* p2 = reinterpret_cast<const longlong2*>(s.row_rec + threadIdx.x);
            const longlong2 w0 = __ldcg(p2);
            const double2 w1 = __ldcg(reinterpret_cast<const double2*>(p2 + 1));
            const int4 w2 = __ldcg(reinterpret_cast<const int4*>(p2 + 2));
            rec.tmin = w0.x; rec.thr = w0.y; rec.a = w1.x; rec.th = w1.y;
            rec.var = w2.x; rec.row = w2.y; rec.cnt = w2.z;
        }
        const int nwu = (G + 31) >> 5;
        if (warp < nwu) {
            // (the threshold is a function of the minimum: any lane holding it has it)
            const long long wm = warp_min_key(rec.tmin);
            const unsigned hold = __ballot_sync(0xffffffffu, rec.tmin == wm);
            if (lane == __ffs(hold) - 1) { wmin_sh[warp] = wm; wthr_sh[warp] = rec.thr; }
        }
        __syncthreads();
        long long gmin = wmin_sh[0], gthr = wthr_sh[0];
        for (int w = 1; w < nwu; ++w)
            if (wmin_sh[w] < gmin) { gmin = wmin_sh[w]; gthr = wthr_sh[w]; }
        if (gmin == dkey(DBL_MAX)) {
            if (threadIdx.x == 0) {
                S.status = kUnbounded;
                S.pending = 0;
            }
            break;
        }
        const double thr = kdouble(gthr);
        // CTAs whose smallest ratio lies within the tie tolerance hold the tie set
        const bool fl = (int)threadIdx.x < G && rec.tmin <= gthr;
        const unsigned bal = __ballot_sync(0xffffffffu, fl);
        if (lane == 0 && warp < nwu) wcnt_sh[warp] = __popc(bal);
        if (fl) flagged = threadIdx.x;  // read only when this CTA is the only one
        __syncthreads();
        int nf = 0;
        for (int w = 0; w < nwu; ++w) nf += wcnt_sh[w];
        const bool bland = S.bland != 0;
        RowCand b = {0.0, 0, -1, 0.0};
        int cnt = 0;
        if (nf == 1) {
            // one CTA holds the minimum, so its threshold is the global one and
            // its record is the tie set's best row and size
            if ((int)threadIdx.x == flagged) {
                nflag = rec.row < 0 ? -1 : 1;
                if (rec.row >= 0) {
                    S.r = rec.row; S.leave = rec.var; S.theta = rec.th; S.alpha_r = rec.a; S.tcount = rec.cnt;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                S.pending = 0;
                if (nflag < 0) {
                    S.status = kUnbounded;
                    if (lead) C->err = kErrBadIndex;
                } else {
                    if (S.tcount > 1) S.flags |= kTfTieSet;
                    S.abuf ^= 1;
                }
            }
        } else {
            // the tie set spans several CTAs: scan the rows of all CTAs
            for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
                const double al = __ldcg(anxt + i), bb = __ldcg(s.bbar + i);
                if (al > P.tol_piv && bb <= thr * al) {
                    cnt++;
                    RowCand c = {al, __ldcg(s.row_var + i), i, 0.0};
                    if (row_beats(c, b, bland)) b = c;
                }
            }
            b = block_row_best(b, cnt, bland);
            if (threadIdx.x == 0) {
                S.pending = 0;
                if (b.row < 0) {
                    S.status = kUnbounded;
                    if (lead) C->err = kErrBadIndex;
                } else {
                    S.r = b.row;
                    S.leave = b.var;
                    S.theta = __ldcg(s.bbar + b.row) / b.a;
                    S.alpha_r = b.a;
                    S.tcount = cnt;
                    if (cnt > 1) S.flags |= kTfTieSet;
                    S.abuf ^= 1;
                }
            }
        }
        __syncthreads();
        if (S.status != kRunning) break;
        if (P.lex && S.tcount > 1) {
            // lexicographic rule: the tie set's row of B^-1 / alpha_i that is
            // lexicographically smallest leaves instead
            const int rr = lex_pick_s(s, anxt, s.row_slot + (size_t)S.par * P.m, kn, thr);
            if (threadIdx.x == 0 && rr >= 0) {
                const double al = __ldcg(anxt + rr);
                S.r = rr;
                S.leave = __ldcg(s.row_var + rr);
                S.theta = __ldcg(s.bbar + rr) / al;
                S.alpha_r = al;
            }
            __syncthreads();
        }
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

// A_p = A_cm with its rows in slot order and its FP32 copy (only after a
// rebuilt map); the screen is switched off when a nonzero of A lies outside
// [2^-100, 2^40] in magnitude.
__global__ void k_struct_gather_A(DevState s, const int32_t* relayout) {
    if (*relayout == 0) return;
    const Params& P = s.p;
    const int32_t* sr = s.slot_row + (size_t)s.ctrl->map_par * P.m;
    const size_t total = (size_t)P.n * P.ld;
    int off = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t j = e / P.ld;
        const int t = (int)(e % P.ld);
        const double a = t < P.m ? s.A_cm[j * P.ld + sr[t]] : 0.0;
        s.A_p[e] = a;
        s.A_p32[e] = (float)a;
        const int ex = (int)((__double_as_longlong(a) >> 52) & 0x7ff);
        off |= a != 0.0 && (ex > 1023 + 40 || ex < 1023 - 100);
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
        s.c32lo[j] = __double2float_rd(s.c[j]);
        s.c32hi[j] = __double2float_ru(s.c[j]);
        const int ex = (int)((__double_as_longlong(s.c[j]) >> 52) & 0x7ff);
        off |= ex > 1023 + 100;  // c within FP32 range
    }
    if (__syncthreads_or(off) && threadIdx.x == 0) atomicOr(&s.ctrl->screen_off, 1);
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
    double* yp = s.yp + (size_t)s.ctrl->map_par * P.ld;  // the current half of the double buffer
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.ld; t += gridDim.x * blockDim.x)
        yp[t] = t < k ? s.y[sr[t]] : 0.0;
}

// The live columns straight from a reinversion's compact result, without the
// dense B^-1: column t is row R_a = slot_row[t] of B^-1, which is W[b][a] on
// the structural position of index b and C[g][a] on the position of the slack
// of the g-th row with a basic slack (the same values k_assemble_rows writes).
__global__ void k_struct_gather_B_compact(DevState s) {
    const Params& P = s.p;
    const int k = s.ctrl->k_live;
    const int32_t* sr = s.slot_row + (size_t)s.ctrl->map_par * P.m;
    const double* W = s.rv_W;
    const double* Cs = s.rv_W + (size_t)k * k;
    const size_t total = (size_t)P.m * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), t = (int)(e % k);
        const int a = s.rv_row_index[sr[t]];
        const int v = s.basis[i];
        s.bp[(size_t)i * P.ld + t] = v < P.n ? W[(size_t)s.rv_b_of_pos[i] * k + a]
                                             : Cs[(size_t)s.rv_g_of_row[v - P.n] * k + a];
    }
    double* yp = s.yp + (size_t)s.ctrl->map_par * P.ld;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < P.ld; t += gridDim.x * blockDim.x)
        yp[t] = t < k ? s.y[sr[t]] : 0.0;
}

// dense y (and its FP32 copy) from the slot-order y, for the solution and every
// dense consumer
__global__ void k_struct_scatter_y(DevState s) {
    const Params& P = s.p;
    const int k = s.ctrl->k_live;
    const int32_t* rs = s.row_slot + (size_t)s.ctrl->map_par * P.m;
    const double* yp = s.yp + (size_t)s.ctrl->map_par * P.ld;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.ld; i += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (i < P.m) {
            const int t = rs[i];
            if (t < k) v = yp[t];
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

size_t iterate_s_smem_bytes(int ld) { return 3 * (size_t)ld * sizeof(double) + (size_t)ld * sizeof(float); }

bool struct_engine_fits(int m, int ld, int ctas) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_iterate_s) != cudaSuccess) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return fa.sharedSizeBytes + iterate_s_smem_bytes(ld) <= (size_t)optin && (m + ctas - 1) / ctas <= kMaxOwnedRows;
}

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

void launch_struct_enter(const DevState& s, int force, int32_t* relayout, cudaStream_t st, bool compact) {
    k_struct_layout<<<1, 1024, 0, st>>>(s, force, relayout);
    k_struct_gather_A<<<1024, 256, 0, st>>>(s, relayout);
    if (compact)
        k_struct_gather_B_compact<<<1024, 256, 0, st>>>(s);
    else
        k_struct_gather_B<<<1024, 256, 0, st>>>(s);
}

void launch_struct_scatter_y(const DevState& s, cudaStream_t st) {
    k_struct_scatter_y<<<64, 256, 0, st>>>(s);
}

void launch_struct_init_maps(const DevState& s, cudaStream_t st) {
    k_struct_init_maps<<<64, 256, 0, st>>>(s);
}

}  // namespace lpgb
