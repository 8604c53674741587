// ooc.cu -- Case 2 of Section 3 (Figure 4): the tableau does not fit the
// device memory granted to it.
//
// The explicit inverse B^-1 (the part of the tableau Step 8 rewrites every
// pivot) then lives in pinned host memory and passes through the device in
// blocks of consecutive rows: every pivot, each block is copied in, updated
// (Step 8 of the previous pivot) fused with the FTRAN of the next entering
// column and the ratios, and copied back, one cudaMemcpyAsync per block on
// copy streams of their own while the other block buffer is computed.  The
// blocks are visited in alternating order, so the block updated last stays
// on the device and is the first of the next pivot (the paper keeps the last
// part for the next update), and row r of the updated inverse, which every
// row of the next update needs, is fetched once.  PRICE (A stays resident),
// the pivot bookkeeping and the ratio-test choice are the kernels of the
// captured-graph engine; the per-row arithmetic below is that of its UPDATE
// (kernels_iter.cu), so the pivots and values are the same bit for bit.
#include "lpgb_internal.cuh"
#include "iter_common.cuh"

#include <cfloat>

namespace lpgb {
namespace {

// Step 8 on the rows i0..i1-1 held in win (row i at win + (i - i0) ld) fused
// with the FTRAN of the next entering column and the ratios theta_i.
__global__ void __launch_bounds__(kUpdateThreads, 1) k_ooc_update(DevState s, double* win, int i0, int i1) {
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
    double* aq = sh;         // column q' of [A | I]
    double* rh = sh + P.ld;  // new row r (rho)
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = P.ld >> 1;
    const double2* aq2 = reinterpret_cast<const double2*>(aq);
    const double2* rh2 = reinterpret_cast<const double2*>(rh);
    for (int i = i0 + (int)blockIdx.x * nw + warp; i < i1; i += (int)gridDim.x * nw) {
        double2* row = reinterpret_cast<double2*>(win + (size_t)(i - i0) * P.ld);
        double a0 = 0.0, a1 = 0.0;
        if (do_upd && i == r) {
            for (int k = lane; k < half; k += 32) {
                const double2 v = rh2[k];
                __stcs(row + k, v);
                if (do_ftran) {
                    const double2 w = aq2[k];
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
                            const double2 w = aq2[k];
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
            }
        }
    }
}

// Step 6 over all rows once every block is done: the minimum ratio, the tie
// set and the leaving row (largest pivot, then smallest basic index; Bland:
// smallest basic index), as the last block of k_update decides it.
__global__ void __launch_bounds__(1024, 1) k_ooc_chuzr(DevState s) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    const int status = C->status;
    const int q = C->q;
    const int r = C->r;
    const int ab = C->abuf;
    const bool do_upd = C->pending != 0 && r >= 0 && r < P.m;
    const bool do_ftran = status == kRunning && q >= 0 && q < P.n + P.m;
    if (!do_upd && !do_ftran) return;
    if (!do_ftran) {
        if (threadIdx.x == 0) {
            C->pending = 0;
            C->bytes_update += 16.0 * P.m * (double)P.m;
            C->n_update++;
        }
        return;
    }
    const double* anxt = s.alpha + (size_t)(ab ^ 1) * P.ld;
    __shared__ double s_tmin;
    double t = DBL_MAX;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) t = fmin(t, __ldcg(s.theta + i));
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
            C->pending = 0;
            C->status = kUnbounded;
        }
        return;
    }
    const double thr = gmin + P.tol_tie * fmax(1.0, fabs(gmin));
    const bool bland = C->bland != 0;
    RowCand best = {0.0, 0, -1, 0.0};
    int cnt = 0;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) {
        const double al = __ldcg(anxt + i), th = __ldcg(s.theta + i);
        if (al > P.tol_piv && th <= thr) {
            cnt++;
            RowCand c = {al, s.basis[i], i, th};
            if (row_beats(c, best, bland)) best = c;
        }
    }
    const RowCand b = block_row_best(best, cnt, bland);
    if (threadIdx.x == 0) {
        C->pending = 0;
        if (b.row < 0) {  // cannot happen for finite data; stop rather than pivot on garbage
            C->status = kUnbounded;
            C->err = kErrBadIndex;
            return;
        }
        C->r = b.row;
        C->theta = b.th;
        C->alpha_r = b.a;
        C->tcount = cnt;
        if (cnt > 1) C->flags |= kTfTieSet;
        C->abuf = ab ^ 1;
    }
}

// Row r of the updated inverse for the next pivot's bookkeeping (k_pivot reads
// s.prow): from the block still on the device (rows w0..w1-1 in win) or from
// the host copy, which the device reads over the host link.
__global__ void k_ooc_fetch_row(DevState s, const double* host_binv, const double* win, int w0, int w1,
                                double* prow) {
    const Ctrl* C = s.ctrl;
    const Params& P = s.p;
    const int r = C->r;
    if (C->status != kRunning || r < 0 || r >= P.m) return;
    const double* src = (r >= w0 && r < w1) ? win + (size_t)(r - w0) * P.ld : host_binv + (size_t)r * P.ld;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.ld; k += gridDim.x * blockDim.x) prow[k] = src[k];
}

}  // namespace

void launch_ooc_update(const DevState& s, const Geometry& g, double* win, int i0, int i1, cudaStream_t st) {
    const int rows = i1 - i0;
    int blocks = (rows + kUpdateThreads / 32 - 1) / (kUpdateThreads / 32);
    if (blocks > g.update_blocks) blocks = g.update_blocks;
    if (blocks < 1) blocks = 1;
    k_ooc_update<<<blocks, kUpdateThreads, update_smem_bytes(s.p.ld), st>>>(s, win, i0, i1);
}

void launch_ooc_chuzr(const DevState& s, cudaStream_t st) { k_ooc_chuzr<<<1, 1024, 0, st>>>(s); }

void launch_ooc_fetch_row(const DevState& s, const double* host_binv, const double* win, int w0, int w1,
                          double* prow, cudaStream_t st) {
    k_ooc_fetch_row<<<8, 256, 0, st>>>(s, host_binv, win, w0, w1, prow);
}

int configure_ooc_kernels(int ld) {
    return cudaFuncSetAttribute(k_ooc_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)update_smem_bytes(ld)) == cudaSuccess
               ? 0
               : -1;
}

}  // namespace lpgb
