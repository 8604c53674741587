// kernels_reinv.cu -- periodic reinversion: rebuild B^-1 from the basis columns.
//
// The paper only updates B^-1 (Step 8); this design rebuilds it every
// `reinvert_every` pivots to stop rounding drift.  The basis matrix of
// max c^T x, Ax <= b has slack columns e_s for some rows: with k structural
// basic columns J (at basis positions P) and R the k rows whose slack is
// nonbasic, B is, up to permutation,
//       [ B11  0 ]        B11 = A[R, J]   (k x k)
//       [ A_SJ I ]        A_SJ = A[S, J]  (S = rows with a basic slack)
// so  B^-1 rows of structural positions = [ B11^-1 | 0 ] and rows of slack
// positions (slack of row s) = [ -A[s, J] B11^-1 | e_s ].  Only B11 is
// inverted (2k^3 flops) plus one (m-k) x k x k product, instead of 2m^3.
//
// At a periodic reinversion B11^-1 comes from one Newton-Schulz refinement
// step of the updated inverse when that is close enough (k_refine_* below);
// otherwise from in-place Gauss-Jordan elimination with partial pivoting
// (row pivots chosen among rows not yet used, no physical swaps), blocked in
// panels of columns (k_gj_panel + k_gj_trail below); per-step kernels remain
// for a device that refuses the cluster launch.  The matrix lives
// column-major.  With pivot row p_t for column t, the stored matrix M satisfies
//       B11^-1[b][p_t] = M[p_b][t].
#include "lpgb_internal.cuh"

#include <cooperative_groups.h>

#include <cfloat>

namespace lpgb {

namespace {

constexpr int kClassifyThreads = 1024;
constexpr int kStepThreads = 256;

// The three lists in increasing position order (and J, c_J with the
// structural positions), each thread taking a run of consecutive positions:
// counts, one block scan of the three counts, then the writes.
__global__ void __launch_bounds__(kClassifyThreads) k_classify(DevState s, int k_expect) {
    pdl_enter();
    __shared__ int wsum[3][32];
    const int m = s.p.m, n = s.p.n;
    const int per = (m + (int)blockDim.x - 1) / (int)blockDim.x;
    const int p0 = min(m, (int)threadIdx.x * per), p1 = min(m, p0 + per);
    int cs = 0, cl = 0;
    for (int p = p0; p < p1; ++p) {
        cs += s.basis[p] < n ? 1 : 0;
        cl += s.pos[n + p] >= 0 ? 1 : 0;
    }
    const int cr = (p1 - p0) - cl;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int is = cs, il = cl, ir = cr;  // inclusive scans within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, is, o), b = __shfl_up_sync(0xffffffffu, il, o),
                  c = __shfl_up_sync(0xffffffffu, ir, o);
        if (lane >= o) { is += a; il += b; ir += c; }
    }
    if (lane == 31) { wsum[0][w] = is; wsum[1][w] = il; wsum[2][w] = ir; }
    __syncthreads();
    if (w == 0) {
        int a = lane < nw ? wsum[0][lane] : 0, b = lane < nw ? wsum[1][lane] : 0, c = lane < nw ? wsum[2][lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ua = __shfl_up_sync(0xffffffffu, a, o), ub = __shfl_up_sync(0xffffffffu, b, o),
                      uc = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) { a += ua; b += ub; c += uc; }
        }
        if (lane < nw) { wsum[0][lane] = a; wsum[1][lane] = b; wsum[2][lane] = c; }
    }
    __syncthreads();
    // rows (index p used as a row here): slack basic -> S list, else R list
    int ks = (w ? wsum[0][w - 1] : 0) + is - cs;
    int kl = (w ? wsum[1][w - 1] : 0) + il - cl;
    int kr = (w ? wsum[2][w - 1] : 0) + ir - cr;
    for (int p = p0; p < p1; ++p) {
        const int var = s.basis[p];
        if (var < n) {
            s.rv_struct_pos[ks] = p;
            s.rv_J[ks] = var;
            s.rv_cJ[ks] = s.c[var];
            s.rv_b_of_pos[p] = ks++;
        } else {
            s.rv_b_of_pos[p] = -1;
        }
        if (s.pos[n + p] >= 0) {
            s.rv_slack_pos[kl] = p;
            s.rv_g_of_row[p] = kl++;
            s.rv_row_index[p] = -1;
        } else {
            s.rv_g_of_row[p] = -1;
            s.rv_row_index[p] = kr;
            s.rv_rows[kr++] = p;
        }
    }
    if (threadIdx.x == 0) {
        const int ts = wsum[0][nw - 1], tl = wsum[1][nw - 1], tr = wsum[2][nw - 1];
        s.ctrl->k_struct = ts;
        s.ctrl->refine_rej = 0;
        s.ctrl->refine_res = 0.0;
        if (ts != tr || ts + tl != m || (k_expect >= 0 && ts != k_expect)) s.ctrl->err = kErrBadIndex;
    }
}

// B11[a][t] = A[R[a], J[t]] stored column-major: M[t*k + a].
__global__ void k_gather(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const size_t total = (size_t)k * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(e / k), a = (int)(e % k);
        const int j = s.basis[s.rv_struct_pos[t]];
        s.rv_M[e] = s.A_cm[(size_t)j * s.p.ld + s.rv_rows[a]];
    }
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
        s.rv_rowdone[a] = 0;
        s.rv_pivrow[a] = -1;
    }
}

// Pivot search on column `t` (already up to date) for elimination step `t`;
// one block.  Publishes the column into f and the pivot row into pivrow[t].
__device__ void search_publish(DevState& s, int k, int t) {
    __shared__ double sv[32];
    __shared__ int si[32];
    const double* col = s.rv_M + (size_t)t * k;
    double best = -1.0;
    int bi = -1;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        if (s.rv_rowdone[a]) continue;
        const double v = fabs(col[a]);
        if (v > best || (v == best && a < bi)) { best = v; bi = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (ov > best || (ov == best && (bi < 0 || oi < bi)))) { best = ov; bi = oi; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sv[w] = best; si[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = -1.0;
        int p = -1;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            if (si[i] >= 0 && (sv[i] > b || (sv[i] == b && si[i] < p))) { b = sv[i]; p = si[i]; }
        if (!(b > 0.0)) {
            s.ctrl->err = kErrSingular;
            p = -1;
        } else {
            s.rv_rowdone[p] = 1;
        }
        s.rv_pivrow[t] = p;
    }
    __syncthreads();
    double* f = s.rv_f + (size_t)(t & 1) * k;
    for (int a = threadIdx.x; a < k; a += blockDim.x) f[a] = col[a];
}

__global__ void __launch_bounds__(kStepThreads) k_gj_search0(DevState s, int k) {
    search_publish(s, k, 0);
}

// Elimination step j on every column, then the owner of column j+1 publishes
// the pivot of step j+1.
__global__ void __launch_bounds__(kStepThreads) k_gj_step(DevState s, int k, int j) {
    const int p = s.rv_pivrow[j];
    if (p < 0 || p >= k || s.ctrl->err != kErrNone) return;  // singular: flagged by the search
    const double* f = s.rv_f + (size_t)(j & 1) * k;
    const double pv = f[p];
    __shared__ double g_sh;
    for (int t = blockIdx.x; t < k; t += gridDim.x) {
        double* col = s.rv_M + (size_t)t * k;
        if (t == j) {
            for (int a = threadIdx.x; a < k; a += blockDim.x)
                col[a] = (a == p) ? 1.0 / pv : -f[a] / pv;
        } else {
            if (threadIdx.x == 0) g_sh = col[p] / pv;
            __syncthreads();
            const double g = g_sh;
            for (int a = threadIdx.x; a < k; a += blockDim.x)
                col[a] = (a == p) ? g : fma(-f[a], g, col[a]);
        }
        __syncthreads();
        if (t == j + 1) search_publish(s, k, t);
        __syncthreads();
    }
}

// Blocked Gauss-Jordan elimination of B11, panels of kNB columns.
//
// One cluster of kPCS CTAs eliminates the pivots of a panel on the k x kNB
// panel alone (its rows split evenly over the CTAs, held in shared memory).
// The product T of the panel's elementary transforms differs from the
// identity only in the columns of the panel's pivot rows p_t, and column t of
// the eliminated panel is T e_{p_t}; so every other column v of the matrix
// becomes
//     T v = (v with rows p_t set to 0) + Panel * v[p_0 .. p_{w-1}],
// a GEMM of inner dimension kNB run over the whole GPU (k_gj_trail).  A
// panel column has received every earlier transform before its pivot is
// searched, so the pivots are those of the unblocked elimination.
//
// Inside a panel the steps are pipelined around one hardware cluster barrier
// per step, split into arrive and wait.  Each CTA publishes its best
// candidate for the next pivot (|value| as an ordered integer key, smaller row
// on equal keys) in its own shared memory; after the barrier every CTA reads
// all candidates and the pivot row through distributed shared memory.  Only
// the next column and the candidate row are needed before the barrier, so
// warp 0 updates those two first (lookahead), publishes and arrives; the
// other warps arrive at once and eliminate the rest of the panel while the
// barrier completes.  No row but a CTA's own candidate is ever read by another
// CTA, and the owner of the pivot row leaves it untouched during the step
// (others are reading it) and folds the scaling into its update of the next
// step.  The arithmetic of every entry is the same as in the unpipelined
// order, so the result does not depend on the schedule.
constexpr int kPCS = 16;
constexpr int kNB = 32;
constexpr int kPLD = kNB + 1;  // padded row stride of the panel in shared memory
constexpr int kPanelThreads = 256;
constexpr size_t kPanelMaxSmem = 200 * 1024;

__device__ __forceinline__ unsigned long long mag_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return u > 0x7ff0000000000000ull ? 0ull : u;  // a NaN never becomes a pivot
}

__device__ __forceinline__ bool cand_better(unsigned long long ka, int ra, unsigned long long kb, int rb) {
    return ka > kb || (ka == kb && ra < rb);
}

// Warp-wide best candidate (largest key, then smallest row) with three
// reductions: the high half of the key, the low half among the lanes that
// hold the largest high half, the row among the lanes that hold the largest
// key.  The result is in every lane.
__device__ __forceinline__ void warp_best(unsigned long long& bk, int& br) {
    const unsigned hi = (unsigned)(bk >> 32), lo = (unsigned)bk;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    br = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? br : 0x7fffffff);
    bk = ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory"); }
// warp 0 hands the next column and the candidate row to the other warps
__device__ __forceinline__ void handoff_arrive() { asm volatile("bar.arrive 1, %0;\n" ::"n"(kPanelThreads) : "memory"); }
__device__ __forceinline__ void handoff_wait() { asm volatile("bar.sync 1, %0;\n" ::"n"(kPanelThreads) : "memory"); }

size_t gj_panel_smem(int k) {
    const size_t rpc = (size_t)((k + kPCS - 1) / kPCS);
    return rpc * kPLD * sizeof(double) + rpc * sizeof(double) + rpc * sizeof(int);
}

__global__ void __launch_bounds__(kPanelThreads) k_gj_panel(DevState s, int k, int c0, int w) {
    namespace cg = cooperative_groups;
    // Read before the first cluster barrier, so all CTAs see the same value
    // (this kernel writes err only after that barrier).
    if (s.ctrl->err != kErrNone) return;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int rpc = (k + kPCS - 1) / kPCS;
    const int a0 = rank * rpc;
    const int nr = max(0, min(rpc, k - a0));
    const int lane = threadIdx.x & 31;
    const bool w0 = threadIdx.x < 32;
    extern __shared__ double psm[];
    double* pan = psm;                                          // rpc x kPLD, row-major
    double* fcol = pan + (size_t)rpc * kPLD;                    // column t of the local rows before step t
    int* done = reinterpret_cast<int*>(fcol + rpc);             // row already a pivot
    __shared__ double g[3][kNB];                                // scaled pivot row of step t in g[t % 3]
    __shared__ unsigned long long ckey[2];                      // published candidate of step t in [t & 1]
    __shared__ int crow[2];
    __shared__ int piv[kNB];
    __shared__ int cand_sh;                                     // local row of the published candidate, or -1
    __shared__ int fail_sh;
    for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
        const int r = e % nr, t = e / nr;
        pan[r * kPLD + t] = s.rv_M[(size_t)(c0 + t) * k + a0 + r];
    }
    for (int r = threadIdx.x; r < nr; r += blockDim.x) done[r] = s.rv_rowdone[a0 + r];
    if (threadIdx.x == 0) fail_sh = 0;
    __syncthreads();
    if (w0) {  // candidate of step 0: column c0 is up to date
        unsigned long long bk = 0ull;
        int br = 0x7fffffff;
        for (int r = lane; r < nr; r += 32) {
            if (done[r]) continue;
            const unsigned long long kk = mag_key(pan[r * kPLD]);
            if (cand_better(kk, a0 + r, bk, br)) { bk = kk; br = a0 + r; }
        }
        warp_best(bk, br);
        if (lane == 0) { ckey[0] = bk; crow[0] = br; }
    }
    cluster_arrive();
    int prev_local = -1;  // local row of the previous step's pivot, if owned here
    bool fail = false;
    for (int t = 0; t < w; ++t) {
        const int gb = t % 3, gp = (t + 2) % 3;  // g of this step and of the previous one
        cluster_wait();
        if (w0) {
            unsigned long long bk = 0ull;
            int br = 0x7fffffff;
            if (lane < kPCS) {
                bk = *cl.map_shared_rank(&ckey[t & 1], lane);
                br = *cl.map_shared_rank(&crow[t & 1], lane);
            }
            warp_best(bk, br);
            if (bk == 0ull || br < 0 || br >= k) {
                if (lane == 0) fail_sh = 1;
            } else {
                const int owner = br / rpc;
                const double* src = cl.map_shared_rank(pan, owner) + (size_t)(br - owner * rpc) * kPLD;
                const double pr = lane < w ? src[lane] : 0.0;
                const double pv = __shfl_sync(0xffffffffu, pr, t);
                const double ri = 1.0 / pv;
                if (lane < w) g[gb][lane] = (lane == t) ? ri : pr * ri;
                if (lane == 0) piv[t] = br;
            }
        }
        __syncthreads();  // g, piv; the other warps are done with step t-1
        if (fail_sh) {
            fail = true;
            break;
        }
        const int p = piv[t];
        const int lp = (p >= a0 && p < a0 + nr) ? p - a0 : -1;
        const bool next = t + 1 < w;
        if (w0) {
            // column t of every local row before the step, then column t+1
            // after it (not the pivot row) and the candidate for step t+1
            unsigned long long bk = 0ull;
            int br = 0x7fffffff;
            for (int r = lane; r < nr; r += 32) {
                const bool pr_row = r == prev_local;
                const double f = pr_row ? g[gp][t] : pan[r * kPLD + t];
                fcol[r] = f;
                if (next && r != lp) {
                    const double old = pr_row ? g[gp][t + 1] : pan[r * kPLD + t + 1];
                    const double v = fma(-f, g[gb][t + 1], old);
                    pan[r * kPLD + t + 1] = v;
                    if (!done[r]) {
                        const unsigned long long kk = mag_key(v);
                        if (cand_better(kk, a0 + r, bk, br)) { bk = kk; br = a0 + r; }
                    }
                }
            }
            int cand = -1;
            if (next) {
                warp_best(bk, br);
                if (bk != 0ull) cand = br - a0;
                __syncwarp();
                if (cand >= 0 && lane < w && lane != t + 1) {  // the candidate row, complete
                    const double f = fcol[cand];
                    double* e = pan + cand * kPLD + lane;
                    *e = (lane == t) ? -f * g[gb][t] : fma(-f, g[gb][lane], *e);
                }
                if (lane == 0) { ckey[(t + 1) & 1] = bk; crow[(t + 1) & 1] = br; }
            }
            if (lane == 0) {
                cand_sh = cand;
                if (lp >= 0) done[lp] = 1;
            }
            handoff_arrive();
            cluster_arrive();
        } else {
            handoff_wait();
            cluster_arrive();
            const int cand = cand_sh;
            const double ri = g[gb][t];
            for (int e = threadIdx.x - 32; e < nr * w; e += blockDim.x - 32) {
                const int r = e / w, j = e - r * w;
                if (r == lp || r == cand || j == t + 1) continue;  // pivot row: read by the other CTAs
                const double f = fcol[r];
                const double old = (r == prev_local) ? g[gp][j] : pan[r * kPLD + j];
                pan[r * kPLD + j] = (j == t) ? -f * ri : fma(-f, g[gb][j], old);
            }
        }
        prev_local = lp;
    }
    if (fail) cluster_arrive();
    cluster_wait();  // every CTA has read the last pivot row
    __syncthreads();
    if (!fail && prev_local >= 0) {
        const int lw = (w - 1) % 3;
        for (int j = threadIdx.x; j < w; j += blockDim.x) pan[prev_local * kPLD + j] = g[lw][j];
    }
    __syncthreads();
    if (fail) {
        if (rank == 0 && threadIdx.x == 0) s.ctrl->err = kErrSingular;
        return;
    }
    for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
        const int r = e % nr, t = e / nr;
        s.rv_M[(size_t)(c0 + t) * k + a0 + r] = pan[r * kPLD + t];
    }
    if (rank == 0)
        for (int t = threadIdx.x; t < w; t += blockDim.x) {
            s.rv_pivrow[c0 + t] = piv[t];
            s.rv_rowdone[piv[t]] = 1;
        }
    // rows p_t of every column outside the panel: copy to rv_W (t-major), then zero
    const int nout = k - w;
    const size_t tot = (size_t)w * nout;
    for (size_t e = (size_t)rank * blockDim.x + threadIdx.x; e < tot; e += (size_t)kPCS * blockDim.x) {
        const int t = (int)(e / nout), o = (int)(e % nout);
        const int j = o < c0 ? o : o + w;
        double* src = s.rv_M + (size_t)j * k + piv[t];
        s.rv_W[(size_t)t * k + j] = *src;
        *src = 0.0;
    }
}

// M[:, j] += Panel * R[:, j] for every column j outside the panel (R = rows
// p_t of those columns, saved by k_gj_panel); a warp's lanes are 32
// consecutive rows, each thread accumulates 4 columns over the panel.
constexpr int kTM = 32, kTN = 16, kTrailThreads = 128;
__global__ void __launch_bounds__(kTrailThreads) k_gj_trail(DevState s, int k, int c0, int w) {
    if (s.ctrl->err != kErrNone) return;
    __shared__ double As[kNB][kTM];
    __shared__ double Bs[kNB][kTN];
    const int nout = k - w;
    const int a0 = blockIdx.y * kTM, o0 = blockIdx.x * kTN;
    for (int e = threadIdx.x; e < kTM * w; e += blockDim.x) {
        const int r = e % kTM, t = e / kTM;
        const int a = a0 + r;
        As[t][r] = a < k ? s.rv_M[(size_t)(c0 + t) * k + a] : 0.0;
    }
    for (int e = threadIdx.x; e < kTN * w; e += blockDim.x) {
        const int c = e % kTN, t = e / kTN;
        const int o = o0 + c;
        Bs[t][c] = o < nout ? s.rv_W[(size_t)t * k + (o < c0 ? o : o + w)] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, c4 = (threadIdx.x >> 5) * 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t < w; ++t) {
        const double av = As[t][lane];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = fma(av, Bs[t][c4 + c], acc[c]);
    }
    const int a = a0 + lane;
    if (a >= k) return;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int o = o0 + c4 + c;
        if (o >= nout) continue;
        double* dst = s.rv_M + (size_t)(o < c0 ? o : o + w) * k + a;
        *dst += acc[c];
    }
}

// ---- Reinversion by refinement ---------------------------------------------
// A periodic reinversion starts from the updated inverse of the same basis
// (the engines apply the last pivot's update before they stop for it), which
// after at most reinvert_every rank-1 updates is close to B^-1.  One step of
// the Newton-Schulz iteration for the matrix inverse (G. Schulz, 1933),
//     Y1 = Y0 + Y0 (I - B11 Y0),   I - B11 Y1 = (I - B11 Y0)^2,
// squares the residual of B11^-1: from ||I - B11 Y0||_inf <= kRefineTol the
// new residual is below the rounding of the products, as after a fresh
// elimination, for two k x k x k FP64 products instead of k sequential pivot
// steps.  The slack rows -A[S, J] B11^-1 then follow from Y1 as after an
// elimination.  A larger residual (or a NaN) falls back to Gauss-Jordan.
//
// Scratch: B11 (column-major, as k_gather writes it), Y0 and R = I - B11 Y0
// (row-major) in rv_M, which needs 3 k^2 <= m^2; per-tile partial row sums of
// |R| after the first k^2 entries of rv_W; Y1 into rv_W, where the
// elimination leaves B11^-1.

// B11 (as k_gather) and Y0[b][a] = stored B^-1[P_b][R_a]: the dense inverse,
// or the live column of row R_a in the slack-structured state (slot map
// `par`, `k_live` live slots).
__global__ void k_refine_extract(DevState s, int k, int from_struct, int k_live, int par) {
    pdl_enter();
    if (s.ctrl->err != kErrNone) return;
    const size_t total = (size_t)k * k;
    double* Y = s.rv_M + total;
    const int32_t* rs = s.row_slot + (size_t)par * s.p.m;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        {
            // B11 (column-major, as k_gather)
            const int t = (int)(e / k), a = (int)(e % k);
            s.rv_M[e] = s.A_cm[(size_t)s.rv_J[t] * s.p.ld + s.rv_rows[a]];
        }
        const int b = (int)(e / k), a = (int)(e % k);
        const size_t prow = (size_t)s.rv_struct_pos[b] * s.p.ld;
        const int i = s.rv_rows[a];
        double v = 0.0;
        if (from_struct) {
            const int sl = rs[i];
            if (sl >= 0 && sl < k_live) v = s.bp[prow + sl];
        } else {
            v = s.binv[prow + i];
        }
        Y[e] = v;
    }
}

// kMode 0: R[i][c] = [i == c] - sum_l B11[i][l] Y0[l][c], and the sum of |R|
//          over the tile's columns (in column order) per row into the partials;
// kMode 1: Y1[i][c] = Y0[i][c] + sum_l Y0[i][l] R[l][c], into rv_W.
// Each output is one fused multiply-add chain in increasing l, so the result
// does not depend on the launch shape.  kRT x kRT tiles keep the SMs' shares
// within one small tile of each other at k of a few hundred.
constexpr int kRT = 8;
template <int kMode>
__global__ void __launch_bounds__(kRT * kRT) k_refine_gemm(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const size_t kk = (size_t)k * k;
    const double* B11 = s.rv_M;
    const double* Y0 = s.rv_M + kk;
    double* R = s.rv_M + 2 * kk;
    const int tx = threadIdx.x % kRT, ty = threadIdx.x / kRT;
    const int i = blockIdx.y * kRT + ty, c = blockIdx.x * kRT + tx;
    const bool in = i < k && c < k;
    double acc = 0.0;
    if (in) {
        if (kMode == 0) {
            const double* x = B11 + i;  // B11[i][l] at l*k + i
            const double* z = Y0 + c;   // Y0[l][c] at l*k + c
#pragma unroll 8
            for (int l = 0; l < k; ++l) acc = fma(x[(size_t)l * k], z[(size_t)l * k], acc);
        } else {
            const double* x = Y0 + (size_t)i * k;  // Y0[i][l]
            const double* z = R + c;               // R[l][c] at l*k + c
#pragma unroll 8
            for (int l = 0; l < k; ++l) acc = fma(x[l], z[(size_t)l * k], acc);
        }
    }
    if (kMode == 0) {
        __shared__ double rabs[kRT][kRT];
        double v = 0.0;
        if (in) {
            v = (i == c ? 1.0 : 0.0) - acc;
            R[(size_t)i * k + c] = v;
        }
        rabs[ty][tx] = fabs(v);
        __syncthreads();
        if (tx == 0 && i < k) {
            double t = 0.0;
#pragma unroll
            for (int u = 0; u < kRT; ++u) t += rabs[ty][u];
            s.rv_W[kk + (size_t)i * gridDim.x + blockIdx.x] = t;
        }
    } else if (in) {
        s.rv_W[(size_t)i * k + c] = Y0[(size_t)i * k + c] + acc;
    }
}

// Tensor-core form of the two products (reinvert_tc, k <= 1024): the exact
// 7-bit-sliced products of ozaki.cu give P = -(B11 Y0) into R's place and
// P = Y0 R into rv_W; these kernels finish them.
// R = I - B11 Y0 = I + P in place, and ||R||_inf into ctrl->refine_res (reset
// to 0 by the classification): each row's sum of |R| (columns in order, one
// warp per row; NaN counts as DBL_MAX) by an atomic max on the bits of the
// non-negative doubles, which order as unsigned integers.
__global__ void __launch_bounds__(256) k_refine_finish_residual(DevState s, int k) {
    pdl_enter();
    if (s.ctrl->err != kErrNone) return;
    const size_t kk = (size_t)k * k;
    double* R = s.rv_M + 2 * kk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + warp; i < k; i += gridDim.x * nw) {
        double t = 0.0;
        for (int c = lane; c < k; c += 32) {
            double v = R[(size_t)i * k + c];
            if (c == i) {
                v = 1.0 + v;
                R[(size_t)i * k + c] = v;
            }
            t += fabs(v);
        }
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(&s.ctrl->refine_res),
                      (unsigned long long)__double_as_longlong(t >= 0.0 ? t : DBL_MAX));
    }
}

// Y1 = Y0 + P, P = Y0 R in rv_W
__global__ void k_refine_add(DevState s, int k) {
    pdl_enter();
    if (s.ctrl->err != kErrNone) return;
    const size_t kk = (size_t)k * k;
    const double* Y0 = s.rv_M + kk;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk; e += (size_t)gridDim.x * blockDim.x)
        s.rv_W[e] = Y0[e] + s.rv_W[e];
}

// ||R||_inf from the partial row sums (each row summed in tile order) into
// ctrl->refine_res; a NaN row counts as infinite.
__global__ void __launch_bounds__(1024) k_refine_norm(DevState s, int k, int ntc) {
    __shared__ double wmax[32];
    const double* part = s.rv_W + (size_t)k * k;
    double mx = 0.0;
    if (s.ctrl->err == kErrNone)
        for (int a = threadIdx.x; a < k; a += blockDim.x) {
            double r = 0.0;
            for (int t = 0; t < ntc; ++t) r += part[(size_t)a * ntc + t];
            if (!(r >= 0.0)) r = DBL_MAX;  // NaN
            mx = fmax(mx, r);
        }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
        s.ctrl->refine_res = s.ctrl->err == kErrNone ? m : DBL_MAX;
    }
}

// pinv[pivrow[t]] = t (stored over rv_rowdone, no longer needed)
__global__ void k_pivinv(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        const int p = s.rv_pivrow[t];
        if (p >= 0 && p < k) s.rv_rowdone[p] = t;
    }
}

// After an elimination, the dense B11^-1 (row b, column a) = M[pinv[a]*k +
// pivrow[b]] (a refinement writes it directly)
__global__ void k_b11i(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const size_t total = (size_t)k * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / k), a = (int)(e % k);
        s.rv_W[e] = s.rv_M[(size_t)s.rv_rowdone[a] * k + s.rv_pivrow[b]];
    }
}

// C (nslack x k, after B11^-1 in rv_W) = -A[S, J] B11^-1; S rows in increasing
// order so that a tile's gathers from a column of A are close together.
// 32 x 32 tiles (2 x 2 outputs per thread): with k of a few hundred, the
// (m-k) x k output gives several tiles per SM, so the SMs' shares differ by a
// small fraction of a tile.
constexpr int kGM = 32, kGN = 32, kGK = 16;
__global__ void __launch_bounds__(256) k_slack_gemm(DevState s, int k, int nslack) {
    if (s.ctrl->err != kErrNone) return;
    __shared__ double As[kGK][kGM + 1];
    __shared__ double Bs[kGK][kGN + 1];
    const double* B11i = s.rv_W;
    double* Cs = s.rv_W + (size_t)k * k;
    const int row0 = blockIdx.y * kGM, col0 = blockIdx.x * kGN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {};
    const int ld = s.p.ld;
    for (int b0 = 0; b0 < k; b0 += kGK) {
        for (int e = threadIdx.x; e < kGM * kGK; e += blockDim.x) {
            const int rr = e % kGM, bb = e / kGM;
            const int gr = row0 + rr, gb = b0 + bb;
            As[bb][rr] = (gr < nslack && gb < k) ? s.A_cm[(size_t)s.rv_J[gb] * ld + s.rv_slack_pos[gr]] : 0.0;
        }
        for (int e = threadIdx.x; e < kGN * kGK; e += blockDim.x) {
            const int cc = e % kGN, bb = e / kGN;
            const int gc = col0 + cc, gb = b0 + bb;
            Bs[bb][cc] = (gc < k && gb < k) ? B11i[(size_t)gb * k + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < kGK; ++bb) {
            const double a0 = As[bb][ty * 2], a1 = As[bb][ty * 2 + 1];
            const double b0v = Bs[bb][tx * 2], b1v = Bs[bb][tx * 2 + 1];
            acc[0][0] = fma(a0, b0v, acc[0][0]); acc[0][1] = fma(a0, b1v, acc[0][1]);
            acc[1][0] = fma(a1, b0v, acc[1][0]); acc[1][1] = fma(a1, b1v, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int gr = row0 + ty * 2 + i;
        if (gr >= nslack) continue;
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int gc = col0 + tx * 2 + jj;
            if (gc < k) Cs[(size_t)gr * k + gc] = -acc[i][jj];
        }
    }
}

// Every row of B^-1 in one coalesced pass (warp per row): structural position
// -> row b of B11^-1 on the R columns; slack of row s -> row of C on the R
// columns and 1 in column s; zero elsewhere (padding included).
__global__ void k_assemble_rows(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int m = s.p.m, n = s.p.n, ld = s.p.ld;
    for (int p = gw; p < m; p += nw) {
        const int v = s.basis[p];
        const double* src;
        int unit = -1;
        if (v < n) {
            src = s.rv_W + (size_t)s.rv_b_of_pos[p] * k;
        } else {
            unit = v - n;
            src = s.rv_W + (size_t)k * k + (size_t)s.rv_g_of_row[unit] * k;
        }
        double* row = s.binv + (size_t)p * ld;
        for (int col = lane; col < ld; col += 32) {
            double val = 0.0;
            if (col < m) {
                const int a = s.rv_row_index[col];
                if (a >= 0) val = src[a];
                else if (col == unit) val = 1.0;
            }
            __stcs(row + col, val);
        }
    }
}

// bbar from the structure: structural position of b: sum_a B11^-1[b][a] b[R[a]];
// slack of row s: b[s] + sum_a C[g][a] b[R[a]] (warp per basis position; the
// part's blocks bid = 0 .. nb-1)
__device__ void bbar_struct_part(const DevState& s, int k, int bid, int nb) {
    const int lane = threadIdx.x & 31;
    const int gw = (bid * (int)blockDim.x + (int)threadIdx.x) >> 5;
    const int nw = (nb * (int)blockDim.x) >> 5;
    const int m = s.p.m, n = s.p.n;
    for (int p = gw; p < m; p += nw) {
        const int v = s.basis[p];
        const double* src;
        double base = 0.0;
        if (v < n) {
            src = s.rv_W + (size_t)s.rv_b_of_pos[p] * k;
        } else {
            base = s.b[v - n];
            src = s.rv_W + (size_t)k * k + (size_t)s.rv_g_of_row[v - n] * k;
        }
        double acc = 0.0;
        for (int a = lane; a < k; a += 32) acc = fma(src[a], s.b[s.rv_rows[a]], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s.bbar[p] = base + acc;
    }
}

// y[R[a]] = sum_b c_J[b] B11^-1[b][a] (one warp per a: lane-strided partial
// sums in increasing b, combined in a fixed shuffle order); y = 0 on rows with
// a basic slack
__device__ void duals_struct_part(const DevState& s, int k, int bid, int nb) {
    const int m = s.p.m;
    for (int i = bid * (int)blockDim.x + (int)threadIdx.x; i < s.p.ld; i += nb * (int)blockDim.x) {
        if (i >= m || s.rv_row_index[i] < 0) {
            s.y[i] = 0.0;
            s.y32[i] = 0.f;
        }
    }
    const int lane = threadIdx.x & 31;
    const int gw = (bid * (int)blockDim.x + (int)threadIdx.x) >> 5, nw = (nb * (int)blockDim.x) >> 5;
    for (int a = gw; a < k; a += nw) {
        double acc = 0.0;
        for (int b = lane; b < k; b += 32) acc = fma(s.rv_cJ[b], s.rv_W[(size_t)b * k + a], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int i = s.rv_rows[a];
            s.y[i] = acc;
            s.y32[i] = (float)acc;
        }
    }
}

constexpr int kFinishThreads = 256;
constexpr int kCloseLanes = 1024;  // the objective is summed as by 1024 threads (32 warp totals in order)

// bbar (blocks 0 .. nb_bbar-1) and y (the others) of the rebuilt basis; the
// last block to finish then takes the objective, the feasibility of the
// rebuilt basis, the verdict on a refinement (tol >= 0: its residual against
// tol) and the status for the next iteration.
__global__ void __launch_bounds__(kFinishThreads) k_reinv_finish(DevState s, int k, int nb_bbar, int check_feasible,
                                                                 double tol) {
    pdl_enter();
    __shared__ double sz[kCloseLanes / 32];
    __shared__ int sbad[kCloseLanes / 32];
    __shared__ int last;
    if (s.ctrl->err == kErrNone) {
        if ((int)blockIdx.x < nb_bbar) bbar_struct_part(s, k, blockIdx.x, nb_bbar);
        else duals_struct_part(s, k, blockIdx.x - nb_bbar, gridDim.x - nb_bbar);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&s.ctrl->ticket_reinv, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int m = s.p.m, n = s.p.n;
    constexpr int kVirt = kCloseLanes / kFinishThreads;  // virtual threads t + j kFinishThreads
    double z[kVirt];
    int bad[kVirt];
#pragma unroll
    for (int j = 0; j < kVirt; ++j) {
        z[j] = 0.0;
        bad[j] = 0;
        for (int p = threadIdx.x + j * kFinishThreads; p < m; p += kCloseLanes) {
            const int var = s.basis[p];
            const double v = __ldcg(s.bbar + p);
            if (var < n) z[j] = fma(s.c[var], v, z[j]);
            if (v < -1e-9 * s.p.b_scale) bad[j] = 1;
        }
        for (int o = 16; o > 0; o >>= 1) {
            z[j] += __shfl_xor_sync(0xffffffffu, z[j], o);
            bad[j] |= __shfl_xor_sync(0xffffffffu, bad[j], o);
        }
        const int vw = (threadIdx.x >> 5) + j * (kFinishThreads / 32);
        if ((threadIdx.x & 31) == 0) { sz[vw] = z[j]; sbad[vw] = bad[j]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int b = 0;
        for (int w = 0; w < kCloseLanes / 32; ++w) { t += sz[w]; b |= sbad[w]; }
        Ctrl* C = s.ctrl;
        C->ticket_reinv = 0;
        if (tol >= 0.0) C->refine_rej = (C->err == kErrNone && C->refine_res <= tol) ? 0 : 1;
        C->z = t;
        if (!C->refine_rej) C->n_reinv++;  // a rejected refinement is redone by elimination
        C->nsb = C->k_struct;
        C->pending = 0;
        C->ticket_price = C->ticket_update = C->ticket_pivot = 0;
        if (check_feasible && b && C->err == kErrNone && !C->refine_rej) C->err = kErrInfeasibleStart;
        C->status = (C->refine_rej || C->err != kErrNone) ? kRebuildStopped
                    : (C->it >= s.p.max_iters) ? kIterLimit : kRunning;
    }
}

}  // namespace

void launch_reinv_classify(const DevState& s, int k_expect, cudaStream_t st) {
    launch_k(k_classify, dim3(1), dim3(kClassifyThreads), 0, st, true, s, k_expect);
}

int reinv_gj_launches(int k) {
    if (k <= 0) return 0;
    if (gj_panel_smem(k) > kPanelMaxSmem) return k + 3;
    const int panels = (k + kNB - 1) / kNB;
    return 2 + panels + (k > kNB ? panels : 0);
}

void launch_reinv_gj(const DevState& s, int k, const Geometry& g, cudaStream_t st) {
    if (k <= 0) return;
    {
        const size_t total = (size_t)k * k;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_gather<<<blocks, 256, 0, st>>>(s, k);
    }
    const size_t smem = gj_panel_smem(k);
    if (smem <= kPanelMaxSmem) {
        cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelMaxSmem);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kPCS, 1, 1);
        cfg.blockDim = dim3(kPanelThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kPCS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        bool ok = true;
        for (int c0 = 0; c0 < k && ok; c0 += kNB) {
            const int w = k - c0 < kNB ? k - c0 : kNB;
            if (cudaLaunchKernelEx(&cfg, k_gj_panel, s, k, c0, w) != cudaSuccess) {
                ok = false;
                break;
            }
            if (w < k) {
                const dim3 grid((k - w + kTN - 1) / kTN, (k + kTM - 1) / kTM);
                k_gj_trail<<<grid, kTrailThreads, 0, st>>>(s, k, c0, w);
            }
        }
        if (ok) {
            k_pivinv<<<(k + 255) / 256, 256, 0, st>>>(s, k);
            return;
        }
        // A refused cluster launch: redo the elimination from a fresh B11
        // with the per-step kernels.
        (void)cudaGetLastError();
        {
            const size_t total = (size_t)k * k;
            int blocks = (int)((total + 255) / 256);
            if (blocks > 4096) blocks = 4096;
            k_gather<<<blocks, 256, 0, st>>>(s, k);
        }
    }
    k_gj_search0<<<1, kStepThreads, 0, st>>>(s, k);
    int blocks = k < 2 * g.sms ? k : 2 * g.sms;
    for (int j = 0; j < k; ++j) k_gj_step<<<blocks, kStepThreads, 0, st>>>(s, k, j);
    k_pivinv<<<(k + 255) / 256, 256, 0, st>>>(s, k);
}

bool refine_fits(int k, int m) { return k > 0 && 3 * (size_t)k * k <= (size_t)m * m; }

static bool refine_on_tc(const DevState& s, int k) { return s.p.reinvert_tc && s.oz_xs && oz_fits(k); }

// Returns the number of kernels launched.
int launch_refine_residual(const DevState& s, int k, int from_struct, int k_live, int par, cudaStream_t st) {
    const size_t kk = (size_t)k * k;
    int blocks = (int)((kk + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    launch_k(k_refine_extract, dim3(blocks), dim3(256), 0, st, true, s, k, from_struct, k_live, par);
    if (refine_on_tc(s, k) &&
        oz_refine_residual_product(s.rv_M, s.rv_M + kk, k, s.rv_M + 2 * kk, s.oz_xs, s.oz_ys, s.oz_ex, s.oz_ey,
                                   &s.ctrl->err, st) == cudaSuccess) {
        launch_k(k_refine_finish_residual, dim3((k + 7) / 8), dim3(256), 0, st, true, s, k);
        return 5;
    }
    (void)cudaGetLastError();
    const int nt = (k + kRT - 1) / kRT;
    k_refine_gemm<0><<<dim3(nt, nt), kRT * kRT, 0, st>>>(s, k);
    k_refine_norm<<<1, 1024, 0, st>>>(s, k, nt);
    return 3;
}

int launch_refine_apply(const DevState& s, int k, cudaStream_t st) {
    const size_t kk = (size_t)k * k;
    if (refine_on_tc(s, k) &&
        oz_refine_update_product(s.rv_M + kk, s.rv_M + 2 * kk, k, s.rv_W, s.oz_xs, s.oz_ys, s.oz_ex, s.oz_ey,
                                 &s.ctrl->err, st) == cudaSuccess) {
        int blocks = (int)((kk + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        launch_k(k_refine_add, dim3(blocks), dim3(256), 0, st, true, s, k);
        return 4;
    }
    (void)cudaGetLastError();
    const int nt = (k + kRT - 1) / kRT;
    k_refine_gemm<1><<<dim3(nt, nt), kRT * kRT, 0, st>>>(s, k);
    return 1;
}

// Returns 1 when the slack-row product ran on the tensor cores.  dense_rows:
// write the dense B^-1 (the slack-structured engine gathers its live columns
// from W and C instead).
int launch_reinv_assemble(const DevState& s, int k, const Geometry& g, cudaStream_t st, int from_gj,
                          bool dense_rows) {
    const int nslack = s.p.m - k;
    int tc = 0;
    if (k > 0) {
        const size_t kk = (size_t)k * k;
        int blocks = (int)((kk + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        if (from_gj) k_b11i<<<blocks, 256, 0, st>>>(s, k);
        if (nslack > 0) {
            if (s.p.reinvert_tc && s.oz_xs && oz_fits(k) &&
                oz_slack_product(s.A_cm, s.p.ld, s.rv_J, s.rv_slack_pos, s.rv_W, k, nslack, s.rv_W + kk, s.oz_xs,
                                 s.oz_ys, s.oz_ex, s.oz_ey, &s.ctrl->err, st) == cudaSuccess) {
                tc = 1;
            } else {
                (void)cudaGetLastError();
                dim3 grid((k + kGN - 1) / kGN, (nslack + kGM - 1) / kGM);
                k_slack_gemm<<<grid, 256, 0, st>>>(s, k, nslack);
            }
        }
    }
    if (dense_rows) k_assemble_rows<<<g.sms * 4, 256, 0, st>>>(s, k);
    return tc;
}

void launch_reinv_finish(const DevState& s, int k, const Geometry& g, cudaStream_t st, int check_feasible,
                         double refine_tol) {
    launch_k(k_reinv_finish, dim3(g.sms * 4), dim3(kFinishThreads), 0, st, true, s, k, g.sms * 2, check_feasible,
             refine_tol);
}

}  // namespace lpgb
