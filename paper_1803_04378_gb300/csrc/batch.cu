// batch.cu -- many small LPs in persistent launches (lp_batch_* in include/lpgb.h).
//
// Each CTA solves whole LPs, one at a time, taking the next one from an atomic
// work queue: the full revised simplex of Section 2.1 (Steps 3-8, Figure 1
// tableau with the explicit B^-1), the tabu rule of Sections 2.2/3.4 with the
// same aspiration and Bland safety net as the single-LP solver, and
// structure-aware reinversion every `reinvert_every` pivots.  LPs are grouped
// into size buckets (m <= 64, 128, 192, 256); every bucket has its own
// persistent kernel whose thread count and B^-1 residency (shared memory or
// an L2-resident global slot per CTA) come from the autotuner.  The bucket
// kernels run side by side on forked streams, captured together as one CUDA
// graph, so the tail of one bucket overlaps the others.  Inside a bucket the
// largest LPs go first so the tail is made of small ones.
//
// PRICE (price_mode 1, the default for batches): a BF16 copy of A screens the
// columns with FP32 FMAs, the top k are re-priced in FP64, and the full FP64
// PRICE runs whenever no candidate improves or Bland's rule is on.  FTRAN, the
// ratio test, the B^-1 update and reinversion are FP64.
//
// B^-1 is stored column-major (element (i, k) at Binv[k*m + i]) so that a
// thread per row reads consecutive addresses in FTRAN.
#include "lpgb_internal.cuh"
#include "../../include/lpgb.h"

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace lpgb {

struct BatchLP {
    int32_t m, n;
    int64_t a_off;   // into A (row-major m x n) and A_lp
    int32_t r_off;   // into b / y (m values)
    int32_t c_off;   // into c / x (n values)
};

struct BatchParams {
    int32_t reinvert_every, tabu_tenure, max_iters, bland_after, price_mode, topk, trace_cap;
    double tol_d, tol_piv, tol_tie;
};

struct BatchState {
    BatchParams p;
    const BatchLP* lps;
    const int32_t* order;       // LP indices, bucket by bucket, largest first
    const double* A;
    const uint16_t* A_lp;       // BF16 copy (price_mode 1)
    const double* b;
    const double* c;
    int32_t* status;
    int32_t* iters;
    double* obj;
    double* x;
    double* y;
    int32_t* queue;             // one counter per bucket
    double* scratch[4];         // per bucket, per-CTA slots: [B^-1 if global] [reinversion block]
    int64_t slot_doubles[4];    // 2 * (bucket's largest m)^2
    int32_t* trace_q;
    int32_t* trace_r;
};

constexpr int kBuckets = 4;
static_assert(sizeof(BatchState::scratch) / sizeof(double*) == kBuckets, "one scratch area per bucket");
constexpr int kBucketM[kBuckets] = {64, 128, 192, 256};
constexpr int kBatchMaxM = 256;
constexpr int kBatchMaxN = 512;
constexpr int kBatchTopk = 8;
constexpr int kSlotsPerSm = 8;  // scratch slots per SM and bucket (CTAs per SM at most)

namespace {

// ---------------------------------------------------------------- reductions
// Values are ordered through their integer images (dkey): every FP64 compare
// or min would hold the FP64 pipe as long as an FMA on this chip.
struct BCand { long long d; int j; };  // d: dkey image

__device__ __forceinline__ bool bc_beats(long long da, int ja, long long db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

// Block argmax of (d, j) with exact ties to the smallest j; result broadcast.
template <int T>
__device__ BCand block_best(BCand c, BCand* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        BCand x;
        x.d = __shfl_xor_sync(0xffffffffu, c.d, o);
        x.j = __shfl_xor_sync(0xffffffffu, c.j, o);
        if (bc_beats(x.d, x.j, c.d, c.j)) c = x;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = c;
    __syncthreads();
    BCand r = sh[0];
    for (int i = 1; i < T / 32; ++i)
        if (bc_beats(sh[i].d, sh[i].j, r.d, r.j)) r = sh[i];
    __syncthreads();
    return r;
}

template <int T>
__device__ int block_sum_int(int v, int* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int r = 0;
    for (int i = 0; i < T / 32; ++i) r += sh[i];
    __syncthreads();
    return r;
}

// Block minimum of dkey images; thread 0 also forms the ratio test's tie
// threshold of the minimum (one FP64 evaluation per block), broadcast in *thr.
template <int T>
__device__ long long block_min_key(long long v, long long* sh, double tol_tie, long long* thr) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    long long r = sh[0];
    for (int i = 1; i < T / 32; ++i) r = min(r, sh[i]);
    if (threadIdx.x == 0) {
        const double t = kdouble(r);
        *thr = t == DBL_MAX ? r : dkey(t + tol_tie * fmax(1.0, fabs(t)));
    }
    __syncthreads();
    return r;
}

template <int T>
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < T / 32; ++i) r += sh[i];
    __syncthreads();
    return r;
}

// Leaving-row candidate: largest alpha, ties to the smallest basic variable
// (Bland: smallest basic variable).
struct RCand { long long a; int var; int row; };  // a: dkey image of alpha

__device__ __forceinline__ bool rc_beats(const RCand& x, const RCand& y, bool bland) {
    if (x.row < 0) return false;
    if (y.row < 0) return true;
    if (bland) return x.var < y.var;
    return x.a > y.a || (x.a == y.a && x.var < y.var);
}

template <int T>
__device__ RCand block_row(RCand c, bool bland, RCand* sh, int& cnt, int* shc) {
    for (int o = 16; o > 0; o >>= 1) {
        RCand x;
        x.a = __shfl_xor_sync(0xffffffffu, c.a, o);
        x.var = __shfl_xor_sync(0xffffffffu, c.var, o);
        x.row = __shfl_xor_sync(0xffffffffu, c.row, o);
        if (rc_beats(x, c, bland)) c = x;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[w] = c; shc[w] = cnt; }
    __syncthreads();
    RCand r = sh[0];
    int total = shc[0];
    for (int i = 1; i < T / 32; ++i) {
        if (rc_beats(sh[i], r, bland)) r = sh[i];
        total += shc[i];
    }
    __syncthreads();
    cnt = total;
    return r;
}

__device__ __forceinline__ float bf16f(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }

// Scalars of the LP being solved (shared memory).
struct LPScal {
    int status, it, q, r, tcount, degen_run, bland, flags, k, err;
    double dq, theta, z;
};

struct Red {
    BCand bc[32];
    RCand rc[32];
    double dv[32];
    long long kv[33];  // keys; kv[32]: the tie threshold
    int iv[32];
    int kj[16 * kBatchTopk];   // top-K selection: each warp's kept columns
    float kd[16 * kBatchTopk];
};

// ---------------------------------------------------------------- one LP
// Top K (K <= kBatchTopk) screened columns, best first, in the order
// (larger d, then smaller j); entries of -FLT_MAX are not candidates.  Each
// warp ranks its columns among themselves by counting the columns that beat
// them (no barrier), keeps ranks below K, and warp 0 ranks the kept columns of
// all warps the same way: cand[t] is the t-th best (-1 when fewer exist).
template <int T>
__device__ void batch_topk(const float* dts, int n, int K, int* cand, int* kj, float* kd) {
    constexpr int W = T / 32;
    constexpr int V = (kBatchMaxN + T - 1) / T;  // columns per lane
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto beats = [](float da, int ja, float db, int jb) { return da > db || (da == db && ja < jb); };
    float d[V];
    int j[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        j[v] = (int)threadIdx.x + T * v;
        d[v] = j[v] < n ? dts[j[v]] : -FLT_MAX;
        if (d[v] == -FLT_MAX) j[v] = -1;
    }
    if (lane < K) kj[w * K + lane] = -1;
    __syncwarp();
    int rank[V];
#pragma unroll
    for (int v = 0; v < V; ++v) rank[v] = 0;
    for (int src = 0; src < 32; ++src) {
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const float od = __shfl_sync(0xffffffffu, d[u], src);
            const int oj = __shfl_sync(0xffffffffu, j[u], src);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (oj >= 0 && j[v] >= 0 && beats(od, oj, d[v], j[v])) rank[v]++;
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
        if (j[v] >= 0 && rank[v] < K) {
            kj[w * K + rank[v]] = j[v];
            kd[w * K + rank[v]] = d[v];
        }
    __syncthreads();
    if (w == 0) {
        constexpr int C = (W * kBatchTopk + 31) / 32;  // kept columns per lane
        float cd[C];
        int cj[C], cr[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int e = lane + 32 * c;
            cj[c] = e < W * K ? kj[e] : -1;
            cd[c] = cj[c] >= 0 ? kd[e] : -FLT_MAX;
            cr[c] = 0;
        }
        for (int src = 0; src < 32; ++src) {
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const float od = __shfl_sync(0xffffffffu, cd[u], src);
                const int oj = __shfl_sync(0xffffffffu, cj[u], src);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    if (oj >= 0 && cj[c] >= 0 && beats(od, oj, cd[c], cj[c])) cr[c]++;
            }
        }
        if (lane < K) cand[lane] = -1;
        __syncwarp();
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (cj[c] >= 0 && cr[c] < K) cand[cr[c]] = cj[c];
    }
    __syncthreads();
}

template <int T, bool SMEM>
__device__ void solve_one(const BatchState& s, int lp, unsigned char* smem, double* slot, int mmax, int nmax) {
    const BatchParams& P = s.p;
    const BatchLP L = s.lps[lp];
    const int m = L.m, n = L.n, N = n + m;
    const double* A = s.A + L.a_off;
    const uint16_t* Alp = s.A_lp ? s.A_lp + L.a_off : nullptr;
    const double* b = s.b + L.r_off;
    const double* c = s.c + L.c_off;
    const int tid = threadIdx.x;

    // shared-memory carve-up (sizes by the bucket maximum)
    double* dp = reinterpret_cast<double*>(smem);
    double* Binv;
    if (SMEM) { Binv = dp; dp += (size_t)mmax * mmax; }
    else { Binv = slot; slot += (size_t)mmax * mmax; }
    double* W = slot;  // reinversion block, k x k column-major (global slot)
    double* y = dp; dp += mmax;
    double* bbar = dp; dp += mmax;
    double* al = dp; dp += mmax;
    double* rho = dp; dp += mmax;
    double* aq = dp; dp += mmax;
    double* th = dp; dp += mmax;
    float* y32 = reinterpret_cast<float*>(dp);
    float* dts = y32 + mmax;                       // nmax screened values
    int* ip = reinterpret_cast<int*>(dts + nmax);
    int* basis = ip; ip += mmax;
    int* pos = ip; ip += nmax + mmax;
    int* tabu = ip; ip += nmax + mmax;
    int* lstP = ip; ip += mmax;
    int* lstR = ip; ip += mmax;
    int* pivrow = ip; ip += mmax;
    int* pinv = ip; ip += mmax;
    int* cand = ip; ip += kBatchTopk + 1;
    double* cand_d = reinterpret_cast<double*>(((uintptr_t)ip + 7) & ~(uintptr_t)7);

    __shared__ LPScal S;
    __shared__ Red R;

    // Step 1: slack basis
    for (int e = tid; e < m * m; e += T) Binv[e] = (e / m == e % m) ? 1.0 : 0.0;
    for (int i = tid; i < m; i += T) {
        y[i] = 0.0;
        y32[i] = 0.f;
        bbar[i] = b[i];
        basis[i] = n + i;
    }
    for (int j = tid; j < N; j += T) {
        pos[j] = j < n ? -1 : j - n;
        tabu[j] = 0;
    }
    if (tid == 0) {
        S.status = kRunning; S.it = 0; S.q = -1; S.r = -1; S.tcount = 0;
        S.degen_run = 0; S.bland = 0; S.flags = 0; S.err = 0; S.z = 0.0; S.dq = 0.0; S.theta = 0.0;
    }
    __syncthreads();

    for (;;) {
        if (S.it >= P.max_iters) {
            if (tid == 0) S.status = kIterLimit;
            __syncthreads();
            break;
        }
        const int it = S.it;
        const bool bland = S.bland != 0;
        // ---- Step 3/4: PRICE + CHUZC
        bool have_q = false;
        if (P.price_mode == 1 && !bland && Alp != nullptr) {
            // BF16 screen over nonbasic, non-tabu structural columns
            // four lanes per column, rows dealt round-robin, two chains each
            for (int base = 0; base < n; base += T / 4) {
                const int j = base + (tid >> 2), g = tid & 3;
                const bool live = j < n && pos[j] < 0 && tabu[j] <= it;
                float a0 = 0.f, a1 = 0.f;
                if (live) {
                    int i = g;
                    for (; i + 4 < m; i += 8) {
                        a0 = fmaf(y32[i], bf16f(__ldg(Alp + (size_t)i * n + j)), a0);
                        a1 = fmaf(y32[i + 4], bf16f(__ldg(Alp + (size_t)(i + 4) * n + j)), a1);
                    }
                    for (; i < m; i += 4) a0 = fmaf(y32[i], bf16f(__ldg(Alp + (size_t)i * n + j)), a0);
                }
                float acc = a0 + a1;
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (g == 0 && j < n) dts[j] = live ? (float)c[j] - acc : -FLT_MAX;
            }
            __syncthreads();
            const int K = P.topk < kBatchTopk ? P.topk : kBatchTopk;
            batch_topk<T>(dts, n, K, cand, R.kj, R.kd);
            // exact FP64 re-price: one warp per candidate
            const int warp = tid >> 5, lane = tid & 31;
            for (int t = warp; t < K; t += T / 32) {
                const int j = cand[t];
                if (j < 0) continue;
                double acc = 0.0;
                for (int i = lane; i < m; i += 32) acc = fma(y[i], __ldg(A + (size_t)i * n + j), acc);
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) cand_d[t] = c[j] - acc;
            }
            // best exact slack (non-tabu)
            BCand bs = {LLONG_MIN, -1};
            for (int i = tid; i < m; i += T) {
                const int j = n + i;
                const long long kd = dkey(-y[i]);
                if (pos[j] < 0 && tabu[j] <= it && bc_beats(kd, j, bs.d, bs.j)) bs = {kd, j};
            }
            __syncthreads();
            bs = block_best<T>(bs, R.bc);
            if (tid == 0) {
                BCand best = bs;
                for (int t = 0; t < K; ++t)
                    if (cand[t] >= 0 && bc_beats(dkey(cand_d[t]), cand[t], best.d, best.j)) best = {dkey(cand_d[t]), cand[t]};
                if (best.j >= 0 && best.d > dkey(P.tol_d)) {
                    S.q = best.j;
                    S.dq = kdouble(best.d);
                    R.iv[0] = 1;
                } else {
                    R.iv[0] = 0;
                }
            }
            __syncthreads();
            have_q = R.iv[0] != 0;
            __syncthreads();
        }
        if (!have_q) {
            // full FP64 PRICE (the oracle's rule, tabu and aspiration included)
            BCand ball = {LLONG_MIN, -1}, bnt = {LLONG_MIN, -1};
            int jmin = -1;
            const long long ktol = dkey(P.tol_d);
            auto offer = [&](double dv, int j) {
                const long long d = dkey(dv);
                if (bc_beats(d, j, ball.d, ball.j)) ball = {d, j};
                if (tabu[j] <= it && bc_beats(d, j, bnt.d, bnt.j)) bnt = {d, j};
                if (d > ktol && (jmin < 0 || j < jmin)) jmin = j;
            };
            // structural columns: four lanes per column
            for (int base = 0; base < n; base += T / 4) {
                const int j = base + (tid >> 2), g = tid & 3;
                const bool live = j < n && pos[j] < 0;
                double a0 = 0.0, a1 = 0.0;
                if (live) {
                    int i = g;
                    for (; i + 4 < m; i += 8) {
                        a0 = fma(y[i], __ldg(A + (size_t)i * n + j), a0);
                        a1 = fma(y[i + 4], __ldg(A + (size_t)(i + 4) * n + j), a1);
                    }
                    for (; i < m; i += 4) a0 = fma(y[i], __ldg(A + (size_t)i * n + j), a0);
                }
                double acc = a0 + a1;
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (g == 0 && live) offer(c[j] - acc, j);
            }
            for (int i = tid; i < m; i += T)
                if (pos[n + i] < 0) offer(-y[i], n + i);
            ball = block_best<T>(ball, R.bc);
            bnt = block_best<T>(bnt, R.bc);
            // smallest improving index: reduce as argmax of (-j)
            BCand bm = {jmin >= 0 ? -(long long)jmin : LLONG_MIN, jmin};
            bm = block_best<T>(bm, R.bc);
            if (tid == 0) {
                if (ball.j < 0 || !(ball.d > ktol)) {
                    S.status = kOptimal;
                } else if (bland) {
                    // d of the smallest improving index: recompute exactly below
                    S.q = bm.j;
                    S.flags |= kTfBland;
                } else if (bnt.j >= 0 && bnt.d > ktol) {
                    S.q = bnt.j;
                    S.dq = kdouble(bnt.d);
                } else {
                    S.q = ball.j;
                    S.dq = kdouble(ball.d);
                    S.flags |= kTfAspiration;
                }
            }
            __syncthreads();
            if (S.status != kRunning) break;
            if (bland) {
                // exact d of the Bland choice (same arithmetic as above)
                const int j = S.q;
                if (tid == 0) {
                    if (j < n) {
                        double acc = 0.0;
                        for (int i = 0; i < m; ++i) acc = fma(y[i], __ldg(A + (size_t)i * n + j), acc);
                        S.dq = c[j] - acc;
                    } else {
                        S.dq = -y[j - n];
                    }
                }
                __syncthreads();
            }
        }
        const int q = S.q;
        // ---- Step 5: FTRAN alpha = B^-1 a_q
        for (int k = tid; k < m; k += T) aq[k] = q < n ? __ldg(A + (size_t)k * n + q) : (k == q - n ? 1.0 : 0.0);
        __syncthreads();
        if (q < n) {
            // four lanes per row, columns of B^-1 dealt round-robin
            for (int base = 0; base < m; base += T / 4) {
                const int i = base + (tid >> 2), g = tid & 3;
                double a0 = 0.0, a1 = 0.0;
                if (i < m) {
                    int k = g;
                    for (; k + 4 < m; k += 8) {
                        a0 = fma(Binv[(size_t)k * m + i], aq[k], a0);
                        a1 = fma(Binv[(size_t)(k + 4) * m + i], aq[k + 4], a1);
                    }
                    for (; k < m; k += 4) a0 = fma(Binv[(size_t)k * m + i], aq[k], a0);
                }
                double acc = a0 + a1;
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (g == 0 && i < m) al[i] = acc;
            }
        } else {
            for (int i = tid; i < m; i += T) al[i] = Binv[(size_t)(q - n) * m + i];
        }
        __syncthreads();
        // ratios one row per lane: a warp-wide division covers 32 rows
        const long long kpiv = dkey(P.tol_piv);
        long long tl = dkey(DBL_MAX);
        for (int i = tid; i < m; i += T) {
            const double a = al[i];
            const double t = dkey(a) > kpiv ? bbar[i] / a : DBL_MAX;
            th[i] = t;
            tl = min(tl, dkey(t));
        }
        // ---- Step 6: CHUZR with the tie set (on integer keys)
        const long long kmin = block_min_key<T>(tl, R.kv, P.tol_tie, &R.kv[32]);
        if (kmin == dkey(DBL_MAX)) {
            if (tid == 0) S.status = kUnbounded;
            __syncthreads();
            break;
        }
        const long long kthr = R.kv[32];
        RCand rc = {0, 0, -1};
        int cnt = 0;
        for (int i = tid; i < m; i += T) {
            const long long ka = dkey(al[i]);
            if (ka > kpiv && dkey(th[i]) <= kthr) {
                cnt++;
                RCand x = {ka, basis[i], i};
                if (rc_beats(x, rc, bland)) rc = x;
            }
        }
        rc = block_row<T>(rc, bland, R.rc, cnt, R.iv);  // best row and tie-set size together
        const int r = rc.row;
        const double ar = al[r];
        const double theta = th[r];
        const double dq = S.dq;
        // ---- Step 7/8 bookkeeping (tabu, trace, objective, basis)
        if (tid == 0) {
            int flags = S.flags;
            const int leave = basis[r];
            const bool degenerate = theta <= P.tol_tie;
            if (degenerate) flags |= kTfDegenerate;
            if (P.tabu_tenure > 0 && (cnt > 1 || degenerate)) {
                tabu[leave] = it + 1 + P.tabu_tenure;
                flags |= kTfTabuPush;
            }
            if (cnt > 1) flags |= kTfTieSet;
            if (s.trace_q && it < P.trace_cap) {
                s.trace_q[(size_t)lp * P.trace_cap + it] = q;
                s.trace_r[(size_t)lp * P.trace_cap + it] = r;
            }
            S.z = __dadd_rn(S.z, __dmul_rn(dq, theta));
            pos[leave] = -1;
            basis[r] = q;
            pos[q] = r;
            S.it = it + 1;
            S.degen_run = degenerate ? S.degen_run + 1 : 0;
            if (S.bland && !degenerate) S.bland = 0;
            if (!S.bland && P.bland_after > 0 && S.degen_run >= P.bland_after) S.bland = 1;
            S.flags = 0;
        }
        // ---- Step 8: tableau pivot (row r / alpha_r, row i - alpha_i * row r)
        for (int k = tid; k < m; k += T) rho[k] = Binv[(size_t)k * m + r] / ar;
        __syncthreads();
        for (int k = tid; k < m; k += T) {
            y[k] = __dadd_rn(y[k], __dmul_rn(dq, rho[k]));
            y32[k] = (float)y[k];
        }
        for (int i = tid; i < m; i += T)
            bbar[i] = (i == r) ? theta : __dsub_rn(bbar[i], __dmul_rn(al[i], theta));
        {
            // element e = k*m + i walks by T: advance (k, i) without dividing
            const int dk = T / m, di = T - dk * m;
            int k = tid / m, i = tid - k * m;
            for (int e = tid; e < m * m; e += T) {
                Binv[e] = (i == r) ? rho[k] : fma(-al[i], rho[k], Binv[e]);
                k += dk;
                i += di;
                if (i >= m) { i -= m; ++k; }
            }
        }
        __syncthreads();
        // ---- periodic reinversion (structure-aware, as in the single-LP solver)
        if (P.reinvert_every > 0 && S.it % P.reinvert_every == 0) {
            if (tid == 0) {
                int k = 0, kr = 0;
                for (int p = 0; p < m; ++p)
                    if (basis[p] < n) lstP[k++] = p;
                for (int i = 0; i < m; ++i)
                    if (pos[n + i] < 0) lstR[kr++] = i;
                S.k = k;
                if (k != kr) S.err = 1;
            }
            __syncthreads();
            const int k = S.k;
            if (S.err) { if (tid == 0) S.status = -1; __syncthreads(); break; }
            for (int e = tid; e < k * k; e += T) {
                const int t = e / k, a = e - t * k;
                W[e] = __ldg(A + (size_t)lstR[a] * n + basis[lstP[t]]);
            }
            for (int a = tid; a < k; a += T) { pinv[a] = 0; pivrow[a] = -1; }  // pinv doubles as "row used"
            __syncthreads();
            for (int j = 0; j < k; ++j) {
                BCand pc = {LLONG_MIN, -1};
                for (int a = tid; a < k; a += T)
                    if (!pinv[a]) {
                        const long long v = dkey(fabs(W[(size_t)j * k + a]));
                        if (bc_beats(v, a, pc.d, pc.j)) pc = {v, a};
                    }
                pc = block_best<T>(pc, R.bc);
                if (pc.j < 0 || !(pc.d > 0)) {
                    if (tid == 0) S.err = 2;
                    __syncthreads();
                    break;
                }
                const int p = pc.j;
                for (int a = tid; a < k; a += T) rho[a] = W[(size_t)j * k + a];  // pivot column f
                __syncthreads();
                const double pv = rho[p];
                for (int t = tid; t < k; t += T) aq[t] = W[(size_t)t * k + p] / pv;  // g_t (row p / pivot)
                if (tid == 0) { pivrow[j] = p; pinv[p] = 1; }
                __syncthreads();
                for (int e = tid; e < k * k; e += T) {
                    const int t = e / k, a = e - t * k;
                    if (t == j) W[e] = (a == p) ? 1.0 / pv : -rho[a] / pv;
                    else W[e] = (a == p) ? aq[t] : fma(-rho[a], aq[t], W[e]);
                }
                __syncthreads();
            }
            if (S.err) { if (tid == 0) S.status = -1; __syncthreads(); break; }
            for (int t = tid; t < k; t += T) pinv[pivrow[t]] = t;
            for (int e = tid; e < m * m; e += T) Binv[e] = 0.0;
            __syncthreads();
            // B11^-1[bb][a] = W[pinv[a]*k + pivrow[bb]]
            for (int e = tid; e < k * k; e += T) {
                const int bb = e / k, a = e - bb * k;
                Binv[(size_t)lstR[a] * m + lstP[bb]] = W[(size_t)pinv[a] * k + pivrow[bb]];
            }
            // slack positions: B^-1[p, s] = 1, B^-1[p, R[a]] = -sum_b A[s, J[b]] B11^-1[b][a]
            for (int e = tid; e < m * k; e += T) {
                const int p = e / (k > 0 ? k : 1), a = e - p * k;
                if (k == 0 || basis[p] < n) continue;
                const int sr = basis[p] - n;
                double acc = 0.0;
                for (int bb = 0; bb < k; ++bb)
                    acc = fma(__ldg(A + (size_t)sr * n + basis[lstP[bb]]), W[(size_t)pinv[a] * k + pivrow[bb]], acc);
                Binv[(size_t)lstR[a] * m + p] = -acc;
            }
            for (int p = tid; p < m; p += T)
                if (basis[p] >= n) Binv[(size_t)(basis[p] - n) * m + p] = 1.0;
            __syncthreads();
            for (int p = tid; p < m; p += T) {
                double acc = 0.0;
                for (int kk = 0; kk < m; ++kk) acc = fma(Binv[(size_t)kk * m + p], b[kk], acc);
                bbar[p] = acc;
            }
            for (int sr = tid; sr < m; sr += T) {
                double acc = 0.0;
                for (int p = 0; p < m; ++p)
                    if (basis[p] < n) acc = fma(c[basis[p]], Binv[(size_t)sr * m + p], acc);
                y[sr] = acc;
                y32[sr] = (float)acc;
            }
            __syncthreads();
            double zz = 0.0;
            for (int p = tid; p < m; p += T)
                if (basis[p] < n) zz = fma(c[basis[p]], bbar[p], zz);
            zz = block_sum<T>(zz, R.dv);
            if (tid == 0) S.z = zz;
            __syncthreads();
        }
    }
    // ---- outputs
    double* xo = s.x + L.c_off;
    double* yo = s.y + L.r_off;
    for (int j = tid; j < n; j += T) xo[j] = 0.0;
    __syncthreads();
    for (int p = tid; p < m; p += T)
        if (basis[p] < n) xo[basis[p]] = bbar[p];
    for (int i = tid; i < m; i += T) yo[i] = y[i];
    if (tid == 0) {
        s.status[lp] = S.status;
        s.iters[lp] = S.it;
        s.obj[lp] = S.z;
    }
    __syncthreads();
}

template <int T, bool SMEM>
__global__ void __launch_bounds__(T, 1024 / T) k_batch(BatchState s, int bucket, int begin, int count, int mmax, int nmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* slot = s.scratch[bucket] + (size_t)blockIdx.x * s.slot_doubles[bucket];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(s.queue + bucket, 1);
        __syncthreads();
        const int k = next;
        __syncthreads();
        if (k >= count) break;
        solve_one<T, SMEM>(s, s.order[begin + k], smem, slot, mmax, nmax);
    }
}

}  // namespace

size_t batch_smem_bytes(int mmax, int nmax, bool smem_binv) {
    size_t d = (smem_binv ? (size_t)mmax * mmax : 0) + 6 * (size_t)mmax;
    size_t f = (size_t)mmax + nmax;
    size_t i = 3 * (size_t)mmax + 2 * ((size_t)nmax + mmax) + 2 * (size_t)mmax + kBatchTopk + 1;
    return d * 8 + f * 4 + i * 4 + 8 + (kBatchTopk + 1) * 8 + 64;
}

using BatchKernel = void (*)(BatchState, int, int, int, int, int);

BatchKernel batch_kernel(int threads, bool smem_binv) {
    switch (threads) {
        case 128: return smem_binv ? k_batch<128, true> : k_batch<128, false>;
        case 256: return smem_binv ? k_batch<256, true> : k_batch<256, false>;
        default: return smem_binv ? k_batch<512, true> : k_batch<512, false>;
    }
}

}  // namespace lpgb

using namespace lpgb;

// ---------------------------------------------------------------- host side
struct lp_batch {
    int device = 0;
    int count = 0;
    lp_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    size_t smem_optin = 0;
    std::vector<void*> allocs;
    std::vector<BatchLP> lps;
    std::vector<int32_t> order;
    int bucket_begin[kBuckets + 1] = {};
    int cfg_threads[kBuckets] = {256, 256, 256, 256};
    int cfg_smem[kBuckets] = {1, 1, 0, 0};
    int64_t sum_m = 0, sum_n = 0;
    BatchState st{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the buckets run side by side on their own streams, forked from and
    // joined back into `stream`; the whole solve is one captured CUDA graph
    cudaStream_t bstream[kBuckets] = {};
    cudaEvent_t fork = nullptr, join[kBuckets] = {};
    cudaGraphExec_t graph = nullptr;
    bool solved = false;
    double fp64_flops_per_iter_avg = 0.0;
};

namespace {

int bfail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA; }

#define BCK(x)                                     \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return bfail(e_);   \
    } while (0)

template <typename T>
int balloc(lp_batch* h, T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return bfail(e);
    h->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return LP_OK;
}

void bfree(lp_batch* h) {
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->e0) cudaEventDestroy(h->e0);
    if (h->e1) cudaEventDestroy(h->e1);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->fork) cudaEventDestroy(h->fork);
    for (int bk = 0; bk < kBuckets; ++bk) {
        if (h->join[bk]) cudaEventDestroy(h->join[bk]);
        if (h->bstream[bk]) cudaStreamDestroy(h->bstream[bk]);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

bool cfg_valid(const lp_batch* h, int bucket, int threads, int smem) {
    if (threads != 128 && threads != 256 && threads != 512) return false;
    const size_t need = batch_smem_bytes(kBucketM[bucket], kBatchMaxN, smem != 0);
    return need <= h->smem_optin;
}

int grid_for(const lp_batch* h, int bucket, int* grid, size_t* smem) {
    const int T = h->cfg_threads[bucket];
    const bool sm = h->cfg_smem[bucket] != 0;
    *smem = batch_smem_bytes(kBucketM[bucket], kBatchMaxN, sm);
    BatchKernel k = batch_kernel(T, sm);
    BCK(cudaFuncSetAttribute(reinterpret_cast<const void*>(k), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
    int occ = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, T, *smem));
    *grid = h->sms * std::max(1, occ);
    return LP_OK;
}

struct BucketLaunch {
    int grid = 0;
    size_t smem = 0;
};

// Grid and shared memory of every non-empty bucket in [b0, b1).
int plan_buckets(lp_batch* h, int b0, int b1, BucketLaunch* out) {
    for (int bk = b0; bk < b1; ++bk) {
        const int cnt = h->bucket_begin[bk + 1] - h->bucket_begin[bk];
        out[bk] = BucketLaunch{};
        if (cnt == 0) continue;
        int rc = grid_for(h, bk, &out[bk].grid, &out[bk].smem);
        if (rc != LP_OK) return rc;
        out[bk].grid = std::min(std::min(out[bk].grid, h->sms * kSlotsPerSm), cnt);
    }
    return LP_OK;
}

// Launch the buckets in [b0, b1), largest first: one after another on
// `stream`, or (concurrent) each on its own stream between a fork and a join,
// so that a bucket's tail overlaps the next bucket.  Every bucket has its own
// scratch slots, so concurrent buckets never share one.
int launch_buckets(lp_batch* h, int b0, int b1, const BucketLaunch* plan, bool concurrent) {
    BCK(cudaMemsetAsync(h->st.queue, 0, sizeof(int32_t) * kBuckets, h->stream));
    if (concurrent) BCK(cudaEventRecord(h->fork, h->stream));
    for (int bk = b1 - 1; bk >= b0; --bk) {
        const int begin = h->bucket_begin[bk], cnt = h->bucket_begin[bk + 1] - begin;
        if (cnt == 0 || plan[bk].grid == 0) continue;
        cudaStream_t st = h->stream;
        if (concurrent) {
            st = h->bstream[bk];
            BCK(cudaStreamWaitEvent(st, h->fork, 0));
        }
        BatchKernel k = batch_kernel(h->cfg_threads[bk], h->cfg_smem[bk] != 0);
        k<<<plan[bk].grid, h->cfg_threads[bk], plan[bk].smem, st>>>(h->st, bk, begin, cnt, kBucketM[bk], kBatchMaxN);
        BCK(cudaGetLastError());
        if (concurrent) {
            BCK(cudaEventRecord(h->join[bk], st));
            BCK(cudaStreamWaitEvent(h->stream, h->join[bk], 0));
        }
    }
    return LP_OK;
}

// (Re)capture the whole solve as one graph after a change of the tuning.
int capture_batch_graph(lp_batch* h) {
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    BucketLaunch plan[kBuckets];
    int rc = plan_buckets(h, 0, kBuckets, plan);
    if (rc != LP_OK) return rc;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rc = launch_buckets(h, 0, kBuckets, plan, true);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != LP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BCK(e);
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    BCK(e);
    return LP_OK;
}

}  // namespace

extern "C" {

int lp_batch_create(lp_batch** out, int32_t count, const int32_t* m, const int32_t* n, const double* A,
                    const double* b, const double* c, int32_t on_device, const lp_options* opt) {
    if (!out) return LP_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !m || !n || !A || !b || !c) return LP_ERR_INVALID_ARG;
    lp_options o;
    lp_default_options(&o);
    o.price_mode = 1;
    o.topk = kBatchTopk;
    if (opt) o = *opt;
    if (o.price_mode < 0 || o.price_mode > 1 || o.topk < 1 || o.max_iters < 0 || o.reinvert_every < 0 ||
        o.tabu_tenure < 0 || o.bland_after < 0 || o.trace_cap < 0)
        return LP_ERR_INVALID_ARG;
    lp_batch* h = new (std::nothrow) lp_batch();
    if (!h) return LP_ERR_OOM;
    h->opt = o;
    h->count = count;
    int rc = LP_OK;
    auto fail = [&](int code) {
        bfree(h);
        delete h;
        return code;
    };
    h->lps.resize(count);
    int64_t aoff = 0, roff = 0, coff = 0;
    for (int k = 0; k < count; ++k) {
        if (m[k] < 1 || m[k] > kBatchMaxM || n[k] < 1 || n[k] > kBatchMaxN) return fail(LP_ERR_INVALID_ARG);
        h->lps[k] = {m[k], n[k], aoff, (int32_t)roff, (int32_t)coff};
        aoff += (int64_t)m[k] * n[k];
        roff += m[k];
        coff += n[k];
        if (roff > INT32_MAX || coff > INT32_MAX) return fail(LP_ERR_INVALID_ARG);
    }
    h->sum_m = roff;
    h->sum_n = coff;
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(LP_ERR_CUDA);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return fail(LP_ERR_CUDA);
    h->sms = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    if (o.cuda_stream) {
        h->stream = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(LP_ERR_CUDA);
        h->own_stream = true;
    }
    if (cudaEventCreate(&h->e0) != cudaSuccess || cudaEventCreate(&h->e1) != cudaSuccess) return fail(LP_ERR_CUDA);
    if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) return fail(LP_ERR_CUDA);
    for (int bk = 0; bk < kBuckets; ++bk)
        if (cudaStreamCreateWithFlags(&h->bstream[bk], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join[bk], cudaEventDisableTiming) != cudaSuccess)
            return fail(LP_ERR_CUDA);
    // host-side validation of host inputs
    if (!on_device) {
        for (int64_t e = 0; e < aoff; ++e)
            if (!std::isfinite(A[e])) return fail(LP_ERR_INVALID_ARG);
        for (int64_t e = 0; e < roff; ++e)
            if (!std::isfinite(b[e]) || b[e] < 0) return fail(LP_ERR_INVALID_ARG);
        for (int64_t e = 0; e < coff; ++e)
            if (!std::isfinite(c[e])) return fail(LP_ERR_INVALID_ARG);
    }
    // buckets by m, largest work first inside a bucket
    std::vector<int> idx(count);
    for (int k = 0; k < count; ++k) idx[k] = k;
    auto bucket_of = [&](int k) {
        for (int bk = 0; bk < kBuckets; ++bk)
            if (h->lps[k].m <= kBucketM[bk]) return bk;
        return kBuckets - 1;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int bb) {
        const int ba = bucket_of(a), bb2 = bucket_of(bb);
        if (ba != bb2) return ba < bb2;
        const int64_t wa = (int64_t)h->lps[a].m * (h->lps[a].m + h->lps[a].n);
        const int64_t wb = (int64_t)h->lps[bb].m * (h->lps[bb].m + h->lps[bb].n);
        return wa > wb;
    });
    h->order = idx;
    {
        int k = 0;
        for (int bk = 0; bk < kBuckets; ++bk) {
            h->bucket_begin[bk] = k;
            while (k < count && bucket_of(idx[k]) == bk) ++k;
        }
        h->bucket_begin[kBuckets] = count;
    }
    for (int bk = 0; bk < kBuckets; ++bk)
        if (!cfg_valid(h, bk, h->cfg_threads[bk], h->cfg_smem[bk])) h->cfg_smem[bk] = 0;
    // device buffers
    BatchState& S = h->st;
    S.p = {o.reinvert_every, o.tabu_tenure, o.max_iters, o.bland_after, o.price_mode, o.topk, o.trace_cap,
           o.tol_d, o.tol_piv, o.tol_tie};
    BatchLP* dl;
    int32_t *dord, *dst, *dit, *dq;
    double *dA, *db, *dc, *dob, *dx, *dy, *dscr;
    if ((rc = balloc(h, &dl, count)) || (rc = balloc(h, &dord, count)) || (rc = balloc(h, &dst, count)) ||
        (rc = balloc(h, &dit, count)) || (rc = balloc(h, &dq, kBuckets)) || (rc = balloc(h, &dA, aoff)) ||
        (rc = balloc(h, &db, roff)) || (rc = balloc(h, &dc, coff)) || (rc = balloc(h, &dob, count)) ||
        (rc = balloc(h, &dx, coff)) || (rc = balloc(h, &dy, roff)))
        return fail(rc);
    // per-CTA slots of each non-empty bucket: B^-1 (global residency) + reinversion block
    for (int bk = 0; bk < kBuckets; ++bk) {
        S.slot_doubles[bk] = 2 * (int64_t)kBucketM[bk] * kBucketM[bk];
        S.scratch[bk] = nullptr;
        if (h->bucket_begin[bk + 1] == h->bucket_begin[bk]) continue;
        if ((rc = balloc(h, &dscr, (size_t)S.slot_doubles[bk] * h->sms * kSlotsPerSm))) return fail(rc);
        S.scratch[bk] = dscr;
    }
    S.lps = dl; S.order = dord; S.status = dst; S.iters = dit; S.queue = dq;
    S.A = dA; S.b = db; S.c = dc; S.obj = dob; S.x = dx; S.y = dy;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(dl, h->lps.data(), sizeof(BatchLP) * count, cudaMemcpyHostToDevice, h->stream) ||
        cudaMemcpyAsync(dord, idx.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, h->stream) ||
        cudaMemcpyAsync(dA, A, sizeof(double) * aoff, kind, h->stream) ||
        cudaMemcpyAsync(db, b, sizeof(double) * roff, kind, h->stream) ||
        cudaMemcpyAsync(dc, c, sizeof(double) * coff, kind, h->stream))
        return fail(LP_ERR_CUDA);
    if (o.price_mode == 1) {
        uint16_t* lp16;
        if ((rc = balloc(h, &lp16, aoff))) return fail(rc);
        launch_to_bf16(dA, lp16, (size_t)aoff, h->stream);
        S.A_lp = lp16;
    }
    if (o.trace_cap > 0) {
        int32_t *tq, *tr;
        if ((rc = balloc(h, &tq, (size_t)count * o.trace_cap)) || (rc = balloc(h, &tr, (size_t)count * o.trace_cap)))
            return fail(rc);
        S.trace_q = tq;
        S.trace_r = tr;
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LP_ERR_CUDA);
    if (on_device) {
        // device inputs: validate with the same rules on a host copy of b (small)
        std::vector<double> hb(roff);
        if (cudaMemcpy(hb.data(), db, sizeof(double) * roff, cudaMemcpyDeviceToHost)) return fail(LP_ERR_CUDA);
        for (double v : hb)
            if (!std::isfinite(v) || v < 0) return fail(LP_ERR_INVALID_ARG);
    }
    *out = h;
    return LP_OK;
}

int lp_batch_solve(lp_batch* h, lp_batch_result* res) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->graph) {
        int rc = capture_batch_graph(h);
        if (rc != LP_OK) return rc;
    }
    BCK(cudaEventRecord(h->e0, h->stream));
    BCK(cudaGraphLaunch(h->graph, h->stream));
    BCK(cudaEventRecord(h->e1, h->stream));
    BCK(cudaEventSynchronize(h->e1));
    h->solved = true;
    if (res) {
        std::vector<int32_t> st(h->count), it(h->count);
        BCK(cudaMemcpy(st.data(), h->st.status, sizeof(int32_t) * h->count, cudaMemcpyDeviceToHost));
        BCK(cudaMemcpy(it.data(), h->st.iters, sizeof(int32_t) * h->count, cudaMemcpyDeviceToHost));
        memset(res, 0, sizeof(*res));
        double fl = 0.0;
        for (int k = 0; k < h->count; ++k) {
            if (st[k] == kOptimal) res->solved++;
            else if (st[k] == kUnbounded) res->unbounded++;
            else if (st[k] == kIterLimit) res->iter_limit++;
            else res->failed++;
            res->iterations += it[k];
            const double mm = h->lps[k].m;
            // FP64 work per pivot: FTRAN + update (2 m^2 FMA) + top-k re-price (k m FMA) or full PRICE (m n FMA)
            const double price = h->opt.price_mode == 1 ? (double)h->opt.topk * mm : mm * h->lps[k].n;
            fl += it[k] * 2.0 * (2.0 * mm * mm + price);
        }
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, h->e0, h->e1));
        res->seconds = ms * 1e-3;
        res->fp64_flops = fl;
    }
    return LP_OK;
}

int lp_batch_get(const lp_batch* h, int32_t* status, int32_t* iterations, double* objective, double* x,
                 double* y) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->solved) return LP_ERR_STATE;
    if (status) BCK(cudaMemcpy(status, h->st.status, sizeof(int32_t) * h->count, cudaMemcpyDeviceToHost));
    if (iterations) BCK(cudaMemcpy(iterations, h->st.iters, sizeof(int32_t) * h->count, cudaMemcpyDeviceToHost));
    if (objective) BCK(cudaMemcpy(objective, h->st.obj, sizeof(double) * h->count, cudaMemcpyDeviceToHost));
    if (x) BCK(cudaMemcpy(x, h->st.x, sizeof(double) * h->sum_n, cudaMemcpyDeviceToHost));
    if (y) BCK(cudaMemcpy(y, h->st.y, sizeof(double) * h->sum_m, cudaMemcpyDeviceToHost));
    return LP_OK;
}

int lp_batch_get_trace(const lp_batch* h, int32_t k, int32_t* q, int32_t* r, int32_t cap, int32_t* count) {
    if (!h || k < 0 || k >= h->count || cap < 0) return LP_ERR_INVALID_ARG;
    if (!h->solved || h->opt.trace_cap <= 0) return LP_ERR_STATE;
    int32_t it = 0;
    BCK(cudaMemcpy(&it, h->st.iters + k, sizeof(int32_t), cudaMemcpyDeviceToHost));
    const int n = std::min(std::min(it, h->opt.trace_cap), cap);
    if (count) *count = n;
    if (n > 0 && q) BCK(cudaMemcpy(q, h->st.trace_q + (size_t)k * h->opt.trace_cap, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (n > 0 && r) BCK(cudaMemcpy(r, h->st.trace_r + (size_t)k * h->opt.trace_cap, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    return LP_OK;
}

int lp_batch_set_tuning(lp_batch* h, const int32_t* table) {
    if (!h || !table) return LP_ERR_INVALID_ARG;
    for (int bk = 0; bk < kBuckets; ++bk)
        if (!cfg_valid(h, bk, table[2 * bk], table[2 * bk + 1])) return LP_ERR_INVALID_ARG;
    for (int bk = 0; bk < kBuckets; ++bk) {
        h->cfg_threads[bk] = table[2 * bk];
        h->cfg_smem[bk] = table[2 * bk + 1];
    }
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return LP_OK;
}

int lp_batch_tune(lp_batch* h, int32_t* table, int32_t trials) {
    if (!h || trials < 1) return LP_ERR_INVALID_ARG;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    const int threads[3] = {128, 256, 512};
    for (int bk = 0; bk < kBuckets; ++bk) {
        if (h->bucket_begin[bk + 1] == h->bucket_begin[bk]) continue;
        float best = 1e30f;
        int bt = h->cfg_threads[bk], bs = h->cfg_smem[bk];
        for (int sm = 1; sm >= 0; --sm) {
            for (int t : threads) {
                if (!cfg_valid(h, bk, t, sm)) continue;
                h->cfg_threads[bk] = t;
                h->cfg_smem[bk] = sm;
                float tot = 0.f;
                BucketLaunch plan[kBuckets];
                int rc = plan_buckets(h, bk, bk + 1, plan);
                if (rc != LP_OK) return rc;
                for (int r = 0; r < trials; ++r) {
                    BCK(cudaEventRecord(h->e0, h->stream));
                    rc = launch_buckets(h, bk, bk + 1, plan, false);
                    if (rc != LP_OK) return rc;
                    BCK(cudaEventRecord(h->e1, h->stream));
                    BCK(cudaEventSynchronize(h->e1));
                    float ms = 0.f;
                    BCK(cudaEventElapsedTime(&ms, h->e0, h->e1));
                    tot += ms;
                }
                if (tot < best) { best = tot; bt = t; bs = sm; }
            }
        }
        h->cfg_threads[bk] = bt;
        h->cfg_smem[bk] = bs;
    }
    if (table)
        for (int bk = 0; bk < kBuckets; ++bk) { table[2 * bk] = h->cfg_threads[bk]; table[2 * bk + 1] = h->cfg_smem[bk]; }
    return LP_OK;
}

void lp_batch_destroy(lp_batch* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    bfree(h);
    delete h;
}

}  // extern "C"
