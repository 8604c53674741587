// iter_common.cuh -- device building blocks shared by the persistent engines
// (k_iterate on the dense explicit inverse, k_iterate_s on its slack-structured
// form) and the per-phase kernels: warp/block reductions, the CHUZC candidate
// of Step 4 with the tabu mask (Sections 2.2 and 3.4), the blocked PRICE of
// Step 3, the ratio-test candidate of Step 6, the bounded grid barrier and the
// Step 7/8 bookkeeping of a pivot.  Included by one translation unit per
// engine; everything lives in an anonymous namespace.
#pragma once
#include "lpgb_internal.cuh"

#include <cfloat>
#include <climits>

namespace lpgb {
namespace {

constexpr int kPriceThreads = 1024;
constexpr int kOct = 4;   // columns per warp in k_price
constexpr int kSeg = 2;   // row segments per column in k_price
constexpr int kPriceCols = kPriceThreads / 32 / kSeg * kOct;  // columns per block per round
constexpr int kUpdateThreads = 1024;
constexpr int kPivotThreads = 64;
constexpr int kMaxFlagged = 64;  // k_iterate: CTAs scanned for the ratio-test tie set
constexpr int kS = 4;  // 512-byte reads in flight per warp (UPDATE)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum in the pairing order of k_price's transposed reduction (lanes
// 16 apart, then 8, 1, 2, 4), so that a column's d_j does not depend on the
// width of the group it was priced in.
__device__ __forceinline__ double pair_sum(double t) {
    t += __shfl_xor_sync(0xffffffffu, t, 16);
    t += __shfl_xor_sync(0xffffffffu, t, 8);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    return t;
}

// acc[c] = sum over this lane's elements k0+lane, k0+lane+32, ... < k1 of
// column cols[c] (double2 units) times y.  Register double buffering: the W
// loads of the next step are issued before the FMAs of the current one, so a
// warp always has a step's worth of reads in flight while it computes.
// kL2: the columns change during the launch (another SM may hold a stale L1
// line), so they are read through L2.
template <int W, bool kL2 = false>
__device__ __forceinline__ double2 ld_col(const double2* p) {
    return kL2 ? __ldcg(p) : __ldcs(p);
}

template <int W, bool kL2 = false>
__device__ __forceinline__ void dot_cols(const double2* __restrict__ A2, const int* cols, int half,
                                         const double2* y2, int k0, int k1, int lane, double (&acc)[W]) {
    const double2* p[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
        p[c] = A2 + (size_t)cols[c] * half;
        acc[c] = 0.0;
    }
    int k = k0 + lane;
    if (k >= k1) return;
    double2 nx[W];
#pragma unroll
    for (int c = 0; c < W; ++c) nx[c] = ld_col<W, kL2>(p[c] + k);
#pragma unroll 1
    for (; k < k1; k += 32) {
        double2 cur[W];
#pragma unroll
        for (int c = 0; c < W; ++c) cur[c] = nx[c];
        if (k + 32 < k1) {
#pragma unroll
            for (int c = 0; c < W; ++c) nx[c] = ld_col<W, kL2>(p[c] + k + 32);
        }
        const double2 yv = y2[k];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(cur[c].y, yv.y, fma(cur[c].x, yv.x, acc[c]));
    }
}

// ---- warp reductions on 64-bit keys by 32-bit redux ------------------------------
// On this chip a dependent warp shuffle costs about 110 cycles and a redux
// about 90: a five-level butterfly of a 64-bit key takes ten shuffles in
// sequence, these take two or three reduxes (the high half, then the low
// half among the lanes that hold the extreme high half).  Keys are the
// order-preserving integer images of doubles (dkey); every lane gets the result.
__device__ __forceinline__ long long key_join(int hi, unsigned lo) {
    return (long long)(((unsigned long long)(unsigned)hi << 32) | lo);
}
__device__ __forceinline__ long long warp_min_key(long long k) {
    const int hi = (int)(k >> 32);
    const int h = __reduce_min_sync(0xffffffffu, hi);
    const unsigned lo = __reduce_min_sync(0xffffffffu, hi == h ? (unsigned)k : 0xffffffffu);
    return key_join(h, lo);
}
// maximum over the lanes with `valid` (LLONG_MIN when there is none)
__device__ __forceinline__ long long warp_max_key(long long k, bool valid) {
    const int hi = valid ? (int)(k >> 32) : INT_MIN;
    const int h = __reduce_max_sync(0xffffffffu, hi);
    const unsigned lo = __reduce_max_sync(0xffffffffu, (valid && hi == h) ? (unsigned)k : 0u);
    return key_join(h, lo);
}
// The lane holding the largest key, exact ties to the smallest index, among
// the lanes with `valid` (-1 when there is none); kbest gets the key.
__device__ __forceinline__ int warp_argmax_key(long long k, int idx, bool valid, long long& kbest) {
    kbest = warp_max_key(k, valid);
    const bool top = valid && k == kbest;
    const int imin = __reduce_min_sync(0xffffffffu, top ? idx : INT_MAX);
    const unsigned b = __ballot_sync(0xffffffffu, top && idx == imin);
    return b ? __ffs(b) - 1 : -1;
}
// The lane holding the smallest index among the lanes with `valid` (-1: none).
__device__ __forceinline__ int warp_argmin_index(int idx, bool valid) {
    const int imin = __reduce_min_sync(0xffffffffu, valid ? idx : INT_MAX);
    const unsigned b = __ballot_sync(0xffffffffu, valid && idx == imin);
    return b ? __ffs(b) - 1 : -1;
}

// ---- CHUZC candidate ---------------------------------------------------------
// Reduced costs are compared through their order-preserving integer images
// (dkey, kdouble in lpgb_internal.cuh).

// d_* fields hold dkey images of reduced costs.
struct Cand {
    long long d_all; int j_all;
    long long d_nt;  int j_nt;
    long long d_min; int j_min;
    long long d_pr;  int j_pr; int k_pr;
};

__device__ __forceinline__ void cand_init(Cand& c) {
    c.d_all = LLONG_MIN; c.j_all = -1;
    c.d_nt = LLONG_MIN; c.j_nt = -1;
    c.d_min = 0; c.j_min = -1;
    c.d_pr = 0; c.j_pr = -1; c.k_pr = kNoRank;
}

// a beats b: larger d, exact ties to the smaller index.
__device__ __forceinline__ bool beats(long long da, int ja, long long db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

// ktol = dkey(tol_d)
__device__ __forceinline__ void cand_offer(Cand& c, double dval, int j, bool nontabu, long long ktol, int rank) {
    const long long d = dkey(dval);
    if (beats(d, j, c.d_all, c.j_all)) { c.d_all = d; c.j_all = j; }
    if (nontabu && beats(d, j, c.d_nt, c.j_nt)) { c.d_nt = d; c.j_nt = j; }
    if (d > ktol && (c.j_min < 0 || j < c.j_min)) { c.d_min = d; c.j_min = j; }
    // guided rule: Dantzig restricted to the listed (priority) columns
    if (nontabu && d > ktol && rank != kNoRank && beats(d, j, c.d_pr, c.j_pr)) { c.d_pr = d; c.j_pr = j; c.k_pr = rank; }
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

// Warp-wide cand_merge of every lane's candidate, by redux (see the warp
// reductions above): the four categories reduce independently, each to its
// largest key with exact ties to the smallest index (j_min: the smallest
// index); the payloads come from the winning lanes.  Every lane gets the result.
__device__ Cand cand_warp_reduce(const Cand& c) {
    Cand g;
    cand_init(g);
    long long kb;
    int w = warp_argmax_key(c.d_all, c.j_all, c.j_all >= 0, kb);
    if (w >= 0) { g.d_all = kb; g.j_all = __shfl_sync(0xffffffffu, c.j_all, w); }
    w = warp_argmax_key(c.d_nt, c.j_nt, c.j_nt >= 0, kb);
    if (w >= 0) { g.d_nt = kb; g.j_nt = __shfl_sync(0xffffffffu, c.j_nt, w); }
    w = warp_argmin_index(c.j_min, c.j_min >= 0);
    if (w >= 0) { g.j_min = __shfl_sync(0xffffffffu, c.j_min, w); g.d_min = __shfl_sync(0xffffffffu, c.d_min, w); }
    w = warp_argmax_key(c.d_pr, c.j_pr, c.j_pr >= 0, kb);
    if (w >= 0) {
        g.d_pr = kb;
        g.j_pr = __shfl_sync(0xffffffffu, c.j_pr, w);
        g.k_pr = __shfl_sync(0xffffffffu, c.k_pr, w);
    }
    return g;
}

// Block-wide reduction; the result is valid in thread 0.
__device__ Cand cand_block_reduce(Cand c) {
    __shared__ Cand sh[32];
    c = cand_warp_reduce(c);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = c;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        if (lane < nw) c = sh[lane]; else cand_init(c);
        c = cand_warp_reduce(c);
    }
    return c;
}

// Leaving-row candidate of the ratio test: largest alpha, exact ties to the
// smallest basic variable index (Bland mode: smallest basic variable index).
struct RowCand { double a; int var; int row; double th; };  // th: the row's ratio

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
// ---- PRICE of one block's columns (k_price, k_iterate, k_iterate_s) ------------------
// Changes of the pivot being applied that a CTA has not necessarily seen in
// memory yet (k_iterate_s applies a pivot without a grid barrier before
// PRICE): column basic_j entered the basis, column free_j left it and is tabu
// until tabu_until when tabu_j == free_j, and the slot -> row entries listed
// in sp_* override the slot map (first match wins).
struct PricePatch {
    int basic_j, free_j, tabu_j, tabu_until;
    int nsp;
    int sp_slot[4], sp_row[4];
};

__device__ __forceinline__ PricePatch no_patch() {
    PricePatch p;
    p.basic_j = p.free_j = p.tabu_j = -1;
    p.tabu_until = 0;
    p.nsp = 0;
    return p;
}

__device__ __forceinline__ int patched_tabu(const DevState& s, const PricePatch& pp, int j) {
    return j == pp.tabu_j ? pp.tabu_until : __ldcg(s.tabu_until + j);
}

// Lists, in order, the nonbasic columns among the block's owned columns
// lb .. lb+kPriceThreads-1 (block b owns j = b, b+G, ...), with their cost,
// tabu expiry and priority, all loaded in the same round trip.  Returns the
// count; ends with a block barrier.
__device__ int list_nonbasic(const DevState& s, const PricePatch& pp, int lb, int owned, int* jl, double* jc,
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
    __syncthreads();
    int before = 0, cnt = 0;
    for (int w = 0; w < kPriceThreads / 32; ++w) {
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
    __syncthreads();
    return cnt;
}

// ysh holds y; each column j contributes its first 2*len_half rows of Acol
// (column stride ld; kL2: read through L2).  pos and tabu_until, which the
// bookkeeping of a persistent launch writes from another block, are read
// through L2.  slack_rows: the rows of the nonbasic slacks, entry i holding
// the row of ysh[i] (nslack of them); otherwise every row is a slack
// candidate and basic slacks are skipped.  Returns the block's candidate in
// thread 0.
template <bool kL2 = false>
__device__ Cand price_block(const DevState& s, int it, const double* ysh, const double* Acol, int len_half,
                            const int32_t* slack_rows, int nslack, const PricePatch& pp) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int half = P.ld >> 1;  // column stride in double2
    const double2* y2 = reinterpret_cast<const double2*>(ysh);
    const int G = gridDim.x;
    const long long ktol = dkey(P.tol_d);
    // Slack candidates are dealt to blocks round-robin too; their loads are
    // issued first so that they complete under the column work.
    int sj = -1;
    {
        const int i = blockIdx.x + G * threadIdx.x;
        if (i < nslack) {
            int row = i;
            if (slack_rows) {
                row = -1;
                for (int e = 0; e < pp.nsp && row < 0; ++e)
                    if (pp.sp_slot[e] == i) row = pp.sp_row[e];
                if (row < 0) row = __ldcg(slack_rows + i);
            }
            sj = P.n + row;
        }
    }
    // Columns are dealt to blocks round-robin (block b owns j = b, b+G, ...)
    // so every SM gets the same share.  The block first lists its nonbasic
    // columns (with their cost, tabu state and priority, loaded in the same
    // round trip); then each warp takes kOct listed columns over one of kSeg
    // row segments, so one shared-memory load of y feeds 2*kOct FMAs, 2*kOct
    // independent 512-byte loads are in flight per step, and the kOct partial
    // sums leave the warp through one transposed reduction (6 adds for 4
    // columns instead of 5 per column).  The segment sums of a column are
    // added in a fixed order, so d_j does not depend on where j was listed.
    // Candidates live in shared memory (one per offering thread) so that no
    // registers are held across the streaming loops.
    __shared__ Cand csh[kPriceCols];
    __shared__ int jl[kPriceThreads];
    __shared__ double jc[kPriceThreads];
    __shared__ int jt[kPriceThreads], jr[kPriceThreads];
    __shared__ double part[kSeg][kPriceCols];
    __shared__ int wcnt[kPriceThreads / 32];
    if (threadIdx.x < kPriceCols) cand_init(csh[threadIdx.x]);
    const int owned = (P.n - (int)blockIdx.x + G - 1) / G;
    const int nch = len_half >> 5;  // 32-double2 chunks priced per column
    // Warp w runs on scheduler w % 4.  When the column's chunks do not split
    // evenly the two segments differ by one chunk, so the segments alternate
    // between the warp pairs of consecutive groups: every scheduler gets the
    // same FP64 work (the partial sums are combined in the same order).
    static_assert(kSeg == 2, "segment interleave assumes two segments");
    const int seg = (warp & 1) ^ ((warp >> 2) & 1), gi = warp / kSeg;
    const int k0 = 32 * (seg * nch / kSeg), k1 = 32 * ((seg + 1) * nch / kSeg);
    const double2* A2 = reinterpret_cast<const double2*>(Acol);
    for (int lb = 0; lb < owned; lb += kPriceThreads) {
        const int cnt = list_nonbasic(s, pp, lb, owned, jl, jc, jt, jr, wcnt);
        // Groups of 4 listed columns, and of 3 where cnt is not a multiple of 4,
        // so that every warp streams 3 or 4 columns at a time (a lone column
        // would run latency-bound long after the others); only lists shorter
        // than the 3-groups they would need fall back to groups of 1 or 2.
        const int n3 = (4 - (cnt & 3)) & 3;
        const bool mixed = cnt >= 3 * n3;
        const int n4 = mixed ? (cnt - 3 * n3) / 4 : cnt / 4;
        const int ngrp = mixed ? n4 + n3 : (cnt + 3) / 4;
        for (int gb = 0; gb < ngrp; gb += kPriceThreads / 32 / kSeg) {
            const int g = gb + gi;
            int e0 = 0, width = 0;
            if (g < ngrp) {
                if (!mixed) { e0 = 4 * g; width = min(4, cnt - e0); }
                else if (g < n4) { e0 = 4 * g; width = 4; }
                else { e0 = 4 * n4 + 3 * (g - n4); width = 3; }
            }
            const int slot = gi * kOct;  // part[] slots of this warp's group
            if (width == 4) {
                double acc[4];
                dot_cols<4, kL2>(A2, jl + e0, half, y2, k0, k1, lane, acc);
                // transposed reduction: lane L ends with column ((L>>4)&1)*2 + ((L>>3)&1)
                const bool h16 = lane & 16, h8 = lane & 8;
                double r2[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const double send = h16 ? acc[i] : acc[2 + i];
                    const double keep = h16 ? acc[2 + i] : acc[i];
                    r2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
                const double send = h8 ? r2[0] : r2[1];
                double r1 = (h8 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, send, 8);
                r1 += __shfl_xor_sync(0xffffffffu, r1, 1);
                r1 += __shfl_xor_sync(0xffffffffu, r1, 2);
                r1 += __shfl_xor_sync(0xffffffffu, r1, 4);
                const int c = (h16 ? 2 : 0) + (h8 ? 1 : 0);
                if ((lane & 7) == 0) part[seg][slot + c] = r1;
            } else if (width == 3) {
                double acc[3];
                dot_cols<3, kL2>(A2, jl + e0, half, y2, k0, k1, lane, acc);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double t = pair_sum(acc[c]);
                    if (lane == 0) part[seg][slot + c] = t;
                }
            } else if (width == 2) {
                double acc[2];
                dot_cols<2, kL2>(A2, jl + e0, half, y2, k0, k1, lane, acc);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double t = pair_sum(acc[c]);
                    if (lane == 0) part[seg][slot + c] = t;
                }
            } else if (width == 1) {
                double acc[1];
                dot_cols<1, kL2>(A2, jl + e0, half, y2, k0, k1, lane, acc);
                const double t = pair_sum(acc[0]);
                if (lane == 0) part[seg][slot] = t;
            }
            __syncthreads();
            // thread t < kPriceCols: column t of this round = group t/4, member t%4
            if (threadIdx.x < kPriceCols) {
                const int gg = gb + (int)threadIdx.x / kOct, c = (int)threadIdx.x % kOct;
                int ee = -1;
                if (gg < ngrp) {
                    if (!mixed) ee = (4 * gg + c < cnt) ? 4 * gg + c : -1;
                    else if (gg < n4) ee = 4 * gg + c;
                    else ee = c < 3 ? 4 * n4 + 3 * (gg - n4) + c : -1;
                }
                if (ee >= 0) {
                    double sum = part[0][threadIdx.x];
#pragma unroll
                    for (int t = 1; t < kSeg; ++t) sum += part[t][threadIdx.x];
                    Cand cc = csh[threadIdx.x];
                    cand_offer(cc, jc[ee] - sum, jl[ee], jt[ee] <= it, ktol, jr[ee]);
                    csh[threadIdx.x] = cc;
                }
            }
            __syncthreads();
        }
    }
    Cand cand;
    cand_init(cand);
    if (threadIdx.x < kPriceCols) cand = csh[threadIdx.x];
    // slack columns: d_{n+i} = -y_i
    for (int i = blockIdx.x + G * threadIdx.x; i < nslack; i += G * blockDim.x) {
        int j = sj;
        if (i != (int)(blockIdx.x + G * threadIdx.x)) {
            int row = i;
            if (slack_rows) {
                row = -1;
                for (int e = 0; e < pp.nsp && row < 0; ++e)
                    if (pp.sp_slot[e] == i) row = pp.sp_row[e];
                if (row < 0) row = __ldcg(slack_rows + i);
            }
            j = P.n + row;
        }
        if (!slack_rows && (j == pp.basic_j ? true : (j == pp.free_j ? false : __ldcg(s.pos + j) >= 0))) continue;
        cand_offer(cand, -ysh[i], j, patched_tabu(s, pp, j) <= it, ktol, s.rank[j]);
    }
    return cand_block_reduce(cand);
}

// PRICE of the block's columns from the compressed sparse column copy of A
// (price_mode 2): each warp takes one listed column at a time and its lanes
// stride over the column's nonzeros (four independent loads in flight per
// lane), gathering y by row index from shared memory; the lane sums are added
// in a fixed order.  Slack candidates as in price_block.
__device__ Cand price_block_csc(const DevState& s, int it, const double* ysh, const PricePatch& pp) {
    const Params& P = s.p;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int G = gridDim.x;
    const long long ktol = dkey(P.tol_d);
    __shared__ int jl[kPriceThreads];
    __shared__ double jc[kPriceThreads];
    __shared__ int jt[kPriceThreads], jr[kPriceThreads];
    __shared__ int wcnt[kPriceThreads / 32];
    Cand cand;
    cand_init(cand);
    const int owned = (P.n - (int)blockIdx.x + G - 1) / G;
    for (int lb = 0; lb < owned; lb += kPriceThreads) {
        const int cnt = list_nonbasic(s, pp, lb, owned, jl, jc, jt, jr, wcnt);
        for (int e = warp; e < cnt; e += nw) {
            const int j = jl[e];
            const long long p0 = __ldg(s.csc_ptr + j), p1 = __ldg(s.csc_ptr + j + 1);
            // four independent nonzeros per lane per step (eight loads in flight;
            // deeper unrolling spills in the persistent kernel)
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            long long p = p0 + lane;
            for (; p + 96 < p1; p += 128) {
                const int r0 = __ldg(s.csc_row + p), r1 = __ldg(s.csc_row + p + 32);
                const int r2 = __ldg(s.csc_row + p + 64), r3 = __ldg(s.csc_row + p + 96);
                const double v0 = __ldg(s.csc_val + p), v1 = __ldg(s.csc_val + p + 32);
                const double v2 = __ldg(s.csc_val + p + 64), v3 = __ldg(s.csc_val + p + 96);
                a0 = fma(v0, ysh[r0], a0);
                a1 = fma(v1, ysh[r1], a1);
                a2 = fma(v2, ysh[r2], a2);
                a3 = fma(v3, ysh[r3], a3);
            }
            for (; p < p1; p += 32) a0 = fma(__ldg(s.csc_val + p), ysh[__ldg(s.csc_row + p)], a0);
            const double t = pair_sum((a0 + a1) + (a2 + a3));
            if (lane == 0) cand_offer(cand, jc[e] - t, j, jt[e] <= it, ktol, jr[e]);
        }
        __syncthreads();  // the list is rebuilt for the next round
    }
    for (int i = blockIdx.x + G * threadIdx.x; i < P.m; i += G * blockDim.x) {
        const int j = P.n + i;
        if (j == pp.basic_j ? true : (j == pp.free_j ? false : __ldcg(s.pos + j) >= 0)) continue;
        cand_offer(cand, -ysh[i], j, patched_tabu(s, pp, j) <= it, ktol, s.rank[j]);
    }
    return cand_block_reduce(cand);
}

__device__ __forceinline__ PriceCand to_price_cand(const Cand& bc) {
    PriceCand pc;
    pc.d_all = kdouble(bc.d_all); pc.j_all = bc.j_all;
    pc.d_nt = kdouble(bc.d_nt); pc.j_nt = bc.j_nt;
    pc.d_min = kdouble(bc.d_min); pc.j_min = bc.j_min;
    pc.d_pr = kdouble(bc.d_pr); pc.j_pr = bc.j_pr; pc.k_pr = bc.k_pr;
    pc.pad_ = 0;
    return pc;
}

// the global candidate from the per-block partials (all threads; result in thread 0)
__device__ Cand reduce_price_parts(const PriceCand* part, int nparts) {
    Cand g;
    cand_init(g);
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const PriceCand* pp = part + b;
        Cand o;
        o.d_all = dkey(__ldcg(&pp->d_all)); o.j_all = __ldcg(&pp->j_all);
        o.d_nt = dkey(__ldcg(&pp->d_nt)); o.j_nt = __ldcg(&pp->j_nt);
        o.d_min = dkey(__ldcg(&pp->d_min)); o.j_min = __ldcg(&pp->j_min);
        o.d_pr = dkey(__ldcg(&pp->d_pr)); o.j_pr = __ldcg(&pp->j_pr); o.k_pr = __ldcg(&pp->k_pr);
        cand_merge(g, o);
    }
    return cand_block_reduce(g);
}

// Step 4 CHUZC on the global candidate: optimality over all nonbasic columns,
// then Bland (safety net), the guided rule, Dantzig among non-tabu columns,
// or aspiration (every improving column tabu).
struct Chuzc {
    int optimal, q, flags, asp;
    double dq;
};

__device__ Chuzc chuzc_decide(const Cand& g, bool bland, double tol_d) {
    Chuzc o = {0, -1, 0, 0, 0.0};
    const long long ktol = dkey(tol_d);
    if (g.j_all < 0 || !(g.d_all > ktol)) {
        o.optimal = 1;
    } else if (bland) {
        o.q = g.j_min; o.dq = kdouble(g.d_min); o.flags = kTfBland;
    } else if (g.j_pr >= 0) {
        o.q = g.j_pr; o.dq = kdouble(g.d_pr); o.flags = kTfGuided;
    } else if (g.j_nt >= 0 && g.d_nt > ktol) {
        o.q = g.j_nt; o.dq = kdouble(g.d_nt);
    } else {
        o.q = g.j_all; o.dq = kdouble(g.d_all); o.flags = kTfAspiration; o.asp = 1;
    }
    return o;
}

__device__ double block_min(double v) {
    __shared__ double shm[32];
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = DBL_MAX;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmin(t, shm[w]);
    return t;
}

// block reduce of the ratio-test candidate and the tie-set count (result in thread 0)
__device__ RowCand block_row_best(RowCand best, int& cnt, bool bland) {
    __shared__ RowCand shr[32];
    __shared__ int shc[32];
    for (int o = 16; o > 0; o >>= 1) {
        RowCand oc;
        oc.a = __shfl_xor_sync(0xffffffffu, best.a, o);
        oc.var = __shfl_xor_sync(0xffffffffu, best.var, o);
        oc.row = __shfl_xor_sync(0xffffffffu, best.row, o);
        oc.th = __shfl_xor_sync(0xffffffffu, best.th, o);
        if (row_beats(oc, best, bland)) best = oc;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { shr[threadIdx.x >> 5] = best; shc[threadIdx.x >> 5] = cnt; }
    __syncthreads();
    RowCand b = shr[0];
    int total = shc[0];
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            if (row_beats(shr[w], b, bland)) b = shr[w];
            total += shc[w];
        }
    cnt = total;
    return b;
}

struct IterState {
    int status, it, q, r, leave, tcount, abuf, pending, flags, degen_run, bland;
    double dq, theta, alpha_r;
    // kept by block 0 during the launch, written back to the control block at its end
    int nsb, n_degenerate, n_tabu, n_bland, n_asp, n_price, n_update;
    int k, par;  // slack-structured engine: live slots, current slot map
    double z, bytes_price, bytes_update;
};

constexpr unsigned kBarrierSpins = 1u << 21;  // about a second of polling, then the launch gives up

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of a cooperative launch: one cumulative arrival counter.  Each
// CTA adds its arrival with a release reduction (no round trip) and polls the
// counter with acquire loads until every CTA of this barrier has arrived
// (epoch * CTAs).  Waits are bounded; a CTA that gives up reports it, and the
// launch ends with kErrTimeout.
__device__ __forceinline__ void red_release_add(uint32_t* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ bool grid_barrier(uint32_t* bar, unsigned& epoch, volatile int* fail, unsigned parties = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        ++epoch;
        const unsigned target = epoch * (parties ? parties : gridDim.x);
        red_release_add(bar, 1u);
        unsigned spins = 0;
        while (ld_acquire_u32(bar) < target) {
            if (++spins > kBarrierSpins) {
                *fail = 1;
                break;
            }
        }
    }
    __syncthreads();
    return *fail == 0;
}

// Step 7/8 bookkeeping of the pivot (q, r): identical scalar updates in every
// CTA; the lead CTA also writes the basis exchange, tabu list, trace and
// counters (the same rules as k_pivot).
__device__ void pivot_bookkeeping(const DevState& s, IterState& S, bool lead) {
    const Params& P = s.p;
    const int it = S.it, q = S.q, r = S.r, leave = S.leave;
    const double th = S.theta, dq = S.dq;
    int flags = S.flags;
    const bool degenerate = th <= P.tol_tie;
    if (degenerate) flags |= kTfDegenerate;
    const bool push = P.tabu_tenure > 0 && (S.tcount > 1 || degenerate);
    if (push) flags |= kTfTabuPush;
    if (lead) {
        // stores only: the leaving variable comes from the ratio test, the
        // counters and the objective stay in S until the launch ends
        if (degenerate) S.n_degenerate++;
        if (push) {
            s.tabu_until[leave] = it + 1 + P.tabu_tenure;
            S.n_tabu++;
        }
        if (it < P.trace_cap) {
            s.trace.q[it] = q;
            s.trace.r[it] = r;
            s.trace.theta[it] = th;
            s.trace.dq[it] = dq;
            s.trace.flags[it] = flags;
        }
        S.z = __dadd_rn(S.z, __dmul_rn(dq, th));
        s.pos[leave] = -1;
        s.basis[r] = q;
        s.pos[q] = r;
        S.nsb += (q < P.n ? 1 : 0) - (leave < P.n ? 1 : 0);
    }
    const int it1 = it + 1;
    S.it = it1;
    S.degen_run = degenerate ? S.degen_run + 1 : 0;
    if (S.bland && !degenerate) S.bland = 0;
    if (!S.bland && P.bland_after > 0 && S.degen_run >= P.bland_after) {
        S.bland = 1;
        if (lead) S.n_bland++;
    }
    S.flags = 0;
    S.pending = 1;  // at a reinversion too: the update is applied before the launch stops
    if (P.reinvert_every > 0 && it1 % P.reinvert_every == 0) {
        S.status = kReinvert;
    } else if (it1 >= P.max_iters) {
        S.status = kIterLimit;
    }
}

// The state block 0 kept during the launch, into the control block.
__device__ void iterate_flush(const DevState& s, const IterState& S) {
    Ctrl* C = s.ctrl;
    C->status = S.status; C->it = S.it; C->q = S.q; C->r = S.r; C->tcount = S.tcount; C->abuf = S.abuf;
    C->pending = S.pending; C->flags = S.flags; C->degen_run = S.degen_run; C->bland = S.bland;
    C->dq = S.dq; C->theta = S.theta; C->alpha_r = S.alpha_r;
    C->nsb = S.nsb; C->n_degenerate = S.n_degenerate; C->n_tabu = S.n_tabu; C->n_bland = S.n_bland;
    C->n_asp = S.n_asp; C->n_price = S.n_price; C->n_update = S.n_update;
    C->z = S.z; C->bytes_price = S.bytes_price; C->bytes_update = S.bytes_update;
    C->k_live = S.k; C->map_par = S.par;
}

}  // namespace
}  // namespace lpgb
