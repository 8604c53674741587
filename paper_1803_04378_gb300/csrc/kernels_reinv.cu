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
// B11^-1 comes from in-place Gauss-Jordan elimination with partial pivoting
// (row pivots chosen among rows not yet used, no physical swaps).  The matrix
// lives column-major; each CTA owns whole columns, and the CTA that owns
// column j+1 searches and publishes the pivot of step j+1 while step j is
// applied, so one launch per elimination step is the only synchronisation.
// With pivot row p_t for column t, the stored matrix M satisfies
//       B11^-1[b][p_t] = M[p_b][t].
#include "lpgb_internal.cuh"

#include <cfloat>

namespace lpgb {

namespace {

constexpr int kClassifyThreads = 1024;
constexpr int kStepThreads = 256;

// exclusive prefix sum of a 0/1 flag across a 1024-thread block
__device__ int block_excl_scan(int flag, int* total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    const int inwarp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    const int excl = (w ? wsum[w - 1] : 0) + inwarp;
    *total = wsum[nw - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kClassifyThreads) k_classify(DevState s) {
    const int m = s.p.m, n = s.p.n;
    int ks = 0, kr = 0, kl = 0;
    for (int c0 = 0; c0 < m; c0 += blockDim.x) {
        const int p = c0 + threadIdx.x;
        const int var = p < m ? s.basis[p] : 0;
        const int fs = (p < m && var < n) ? 1 : 0;
        const int fl = (p < m && var >= n) ? 1 : 0;
        int tot;
        const int e1 = block_excl_scan(fs, &tot);
        if (fs) s.rv_struct_pos[ks + e1] = p;
        ks += tot;
        const int e2 = block_excl_scan(fl, &tot);
        if (fl) s.rv_slack_pos[kl + e2] = p;
        kl += tot;
        const int fr = (p < m && s.pos[n + p] < 0) ? 1 : 0;
        const int e3 = block_excl_scan(fr, &tot);
        if (p < m) s.rv_row_index[p] = fr ? kr + e3 : -1;
        if (fr) s.rv_rows[kr + e3] = p;
        kr += tot;
    }
    if (threadIdx.x == 0) {
        s.ctrl->k_struct = ks;
        if (ks != kr || ks + kl != m) s.ctrl->err = kErrBadIndex;
    }
}

// B11[a][t] = A[R[a], J[t]] stored column-major: M[t*k + a].
__global__ void k_gather(DevState s, int k) {
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

// pinv[pivrow[t]] = t (stored over rv_rowdone, no longer needed)
__global__ void k_pivinv(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        const int p = s.rv_pivrow[t];
        if (p >= 0 && p < k) s.rv_rowdone[p] = t;
    }
}

__global__ void k_zero(double* x, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        x[e] = 0.0;
}

// B11^-1[b][a] with the pivot bookkeeping of the in-place elimination
__device__ __forceinline__ double b11inv(const DevState& s, int k, int b, int a) {
    return s.rv_M[(size_t)s.rv_rowdone[a] * k + s.rv_pivrow[b]];
}

// rows of structural positions: B^-1[P[b], R[a]] = B11^-1[b][a]
__global__ void k_scatter_struct(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const size_t total = (size_t)k * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / k), a = (int)(e % k);
        s.binv[(size_t)s.rv_struct_pos[b] * s.p.ld + s.rv_rows[a]] = b11inv(s, k, b, a);
    }
}

// rows of slack positions: B^-1[p, s] = 1 and B^-1[p, R[a]] = -sum_b A[s, J[b]] B11^-1[b][a]
// (an (m-k) x k x k FP64 product, 64x64 output tiles, 4x4 per thread).
constexpr int kTM = 64, kTN = 64, kTK = 16;
__global__ void __launch_bounds__(256) k_slack_rows(DevState s, int k, int nslack) {
    if (s.ctrl->err != kErrNone) return;
    __shared__ double As[kTK][kTM + 1];
    __shared__ double Bs[kTK][kTN + 1];
    const int row0 = blockIdx.y * kTM, col0 = blockIdx.x * kTN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    const int ld = s.p.ld, n = s.p.n;
    for (int b0 = 0; b0 < k; b0 += kTK) {
        for (int e = threadIdx.x; e < kTM * kTK; e += blockDim.x) {
            const int rr = e % kTM, bb = e / kTM;
            const int gr = row0 + rr, gb = b0 + bb;
            double v = 0.0;
            if (gr < nslack && gb < k) {
                const int srow = s.basis[s.rv_slack_pos[gr]] - n;
                const int j = s.basis[s.rv_struct_pos[gb]];
                v = s.A_cm[(size_t)j * ld + srow];
            }
            As[bb][rr] = v;
        }
        for (int e = threadIdx.x; e < kTN * kTK; e += blockDim.x) {
            const int cc = e % kTN, bb = e / kTN;
            const int gc = col0 + cc, gb = b0 + bb;
            Bs[bb][cc] = (gc < k && gb < k) ? b11inv(s, k, gb, gc) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < kTK; ++bb) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[bb][ty * 4 + i];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) bv[jj] = Bs[bb][tx * 4 + jj];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(av[i], bv[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gr = row0 + ty * 4 + i;
        if (gr >= nslack) continue;
        const int p = s.rv_slack_pos[gr];
        double* out = s.binv + (size_t)p * ld;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gc = col0 + tx * 4 + jj;
            if (gc < k) out[s.rv_rows[gc]] = -acc[i][jj];
        }
    }
}

__global__ void k_slack_unit(DevState s, int nslack) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslack; i += gridDim.x * blockDim.x) {
        const int p = s.rv_slack_pos[i];
        s.binv[(size_t)p * s.p.ld + (s.basis[p] - s.p.n)] = 1.0;
    }
}

// bbar = B^-1 b (warp per row)
__global__ void k_bbar(DevState s) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int half = s.p.ld >> 1;
    const double2* b2 = reinterpret_cast<const double2*>(s.b);
    for (int i = gw; i < s.p.m; i += nw) {
        const double2* row = reinterpret_cast<const double2*>(s.binv + (size_t)i * s.p.ld);
        double a0 = 0.0, a1 = 0.0;
        for (int k = lane; k < half; k += 32) {
            const double2 v = row[k], w = b2[k];
            a0 = fma(v.x, w.x, a0);
            a1 = fma(v.y, w.y, a1);
        }
        double t = a0 + a1;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s.bbar[i] = t;
    }
}

// y[R[a]] = sum_b c_{J[b]} B11^-1[b][a]; y = 0 on rows with a basic slack
__global__ void k_duals(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const int m = s.p.m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.p.ld; i += gridDim.x * blockDim.x) {
        if (i >= m || s.rv_row_index[i] < 0) { s.y[i] = 0.0; continue; }
        const int a = s.rv_row_index[i];
        double acc = 0.0;
        for (int b = 0; b < k; ++b) {
            const int j = s.basis[s.rv_struct_pos[b]];
            acc = fma(s.c[j], b11inv(s, k, b, a), acc);
        }
        s.y[i] = acc;
    }
}

// objective, feasibility of the rebuilt basis, status for the next iteration
__global__ void __launch_bounds__(1024) k_reinv_close(DevState s, int check_feasible) {
    __shared__ double sz[32];
    __shared__ int sbad[32];
    const int m = s.p.m, n = s.p.n;
    double z = 0.0;
    int bad = 0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int var = s.basis[p];
        const double v = s.bbar[p];
        if (var < n) z = fma(s.c[var], v, z);
        if (v < -1e-9 * s.p.b_scale) bad = 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        z += __shfl_xor_sync(0xffffffffu, z, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) { sz[threadIdx.x >> 5] = z; sbad[threadIdx.x >> 5] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += sz[w]; b |= sbad[w]; }
        Ctrl* C = s.ctrl;
        C->z = t;
        C->n_reinv++;
        C->nsb = C->k_struct;
        C->pending = 0;
        C->ticket_price = C->ticket_update = C->ticket_pivot = 0;
        if (check_feasible && b && C->err == kErrNone) C->err = kErrInfeasibleStart;
        C->status = (C->it >= s.p.max_iters) ? kIterLimit : kRunning;
    }
}

}  // namespace

void launch_reinv_classify(const DevState& s, cudaStream_t st) {
    k_classify<<<1, kClassifyThreads, 0, st>>>(s);
}

void launch_reinv_gather(const DevState& s, int k, cudaStream_t st) {
    if (k <= 0) return;
    const size_t total = (size_t)k * k;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_gather<<<blocks, 256, 0, st>>>(s, k);
}

void launch_reinv_gj(const DevState& s, int k, const Geometry& g, cudaStream_t st) {
    if (k <= 0) return;
    k_gj_search0<<<1, kStepThreads, 0, st>>>(s, k);
    int blocks = k < 2 * g.sms ? k : 2 * g.sms;
    for (int j = 0; j < k; ++j) k_gj_step<<<blocks, kStepThreads, 0, st>>>(s, k, j);
    k_pivinv<<<(k + 255) / 256, 256, 0, st>>>(s, k);
}

void launch_reinv_assemble(const DevState& s, int k, const Geometry& g, cudaStream_t st) {
    const size_t total = (size_t)s.p.m * s.p.ld;
    k_zero<<<g.sms * 8, 256, 0, st>>>(s.binv, total);
    const int nslack = s.p.m - k;
    if (k > 0) {
        const size_t kk = (size_t)k * k;
        int blocks = (int)((kk + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_scatter_struct<<<blocks, 256, 0, st>>>(s, k);
        if (nslack > 0) {
            dim3 grid((k + kTN - 1) / kTN, (nslack + kTM - 1) / kTM);
            k_slack_rows<<<grid, 256, 0, st>>>(s, k, nslack);
        }
    }
    if (nslack > 0) k_slack_unit<<<(nslack + 255) / 256, 256, 0, st>>>(s, nslack);
}

void launch_reinv_finish(const DevState& s, int k, const Geometry& g, cudaStream_t st, int check_feasible) {
    k_bbar<<<g.sms * 4, 256, 0, st>>>(s);
    k_duals<<<(s.p.ld + 255) / 256, 256, 0, st>>>(s, k);
    k_reinv_close<<<1, 1024, 0, st>>>(s, check_feasible);
}

}  // namespace lpgb
