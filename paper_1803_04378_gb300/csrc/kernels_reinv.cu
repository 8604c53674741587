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

#include <cooperative_groups.h>

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
        int tot;
        const int e1 = block_excl_scan(fs, &tot);
        if (fs) s.rv_struct_pos[ks + e1] = p;
        if (p < m) s.rv_b_of_pos[p] = fs ? ks + e1 : -1;
        ks += tot;
        // rows (index p used as a row here): slack basic -> S list, else R list
        const int fl = (p < m && s.pos[n + p] >= 0) ? 1 : 0;
        const int e2 = block_excl_scan(fl, &tot);
        if (fl) s.rv_slack_pos[kl + e2] = p;
        if (p < m) s.rv_g_of_row[p] = fl ? kl + e2 : -1;
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

// Whole Gauss-Jordan elimination of B11 (k <= kClusterMaxK) in one cluster of
// kCS CTAs.  CTA r keeps the columns t = r, r+kCS, ... in shared memory.  At
// step j every CTA applies the pivot (p_j, j) to its columns; the owner of
// column j+1 first updates that column, searches its pivot among rows not yet
// used and writes the column and the pivot row into every CTA's shared memory
// (double-buffered), so one hardware cluster barrier per step is the only
// synchronisation.  Writes B11 in the same column-major form as the
// per-step kernels, and the pivot rows.
constexpr int kCS = 16;
constexpr int kClusterMaxK = 512;
constexpr int kClusterThreads = 256;

__device__ int cl_search(const double* col, const int* rowdone, int k, double* sv, int* si) {
    double best = -1.0;
    int bi = -1;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        if (rowdone[a]) continue;
        const double v = fabs(col[a]);
        if (v > best) { best = v; bi = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (ov > best || (ov == best && (bi < 0 || oi < bi)))) { best = ov; bi = oi; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sv[w] = best; si[w] = bi; }
    __syncthreads();
    double b = -1.0;
    int p = -1;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
        if (si[i] >= 0 && (sv[i] > b || (sv[i] == b && si[i] < p))) { b = sv[i]; p = si[i]; }
    return b > 0.0 ? p : -1;
}

__global__ void __launch_bounds__(kClusterThreads) k_gj_cluster(DevState s, int k) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int cpc = (k + kCS - 1) / kCS;
    extern __shared__ double sm[];
    double* cols = sm;                     // cpc columns of k
    double* fbuf = cols + (size_t)cpc * k; // 2 x k pivot columns
    double* gcol = fbuf + 2 * (size_t)k;   // cpc multipliers
    int* pbuf = reinterpret_cast<int*>(gcol + cpc);  // [2] pivot rows
    int* rowdone = pbuf + 2;               // k
    __shared__ double sv[32];
    __shared__ int si[32];
    const int ld = s.p.ld;
    for (int c = 0; c < cpc; ++c) {
        const int t = rank + c * kCS;
        if (t >= k) break;
        const int jcol = s.basis[s.rv_struct_pos[t]];
        for (int a = threadIdx.x; a < k; a += blockDim.x) cols[(size_t)c * k + a] = s.A_cm[(size_t)jcol * ld + s.rv_rows[a]];
    }
    for (int a = threadIdx.x; a < k; a += blockDim.x) rowdone[a] = 0;
    __syncthreads();
    auto broadcast = [&](const double* col, int p, int buf) {
        for (int r = 0; r < kCS; ++r) {
            double* dst = cl.map_shared_rank(fbuf + (size_t)buf * k, r);
            for (int a = threadIdx.x; a < k; a += blockDim.x) dst[a] = col[a];
            if (threadIdx.x == 0) *cl.map_shared_rank(pbuf + buf, r) = p;
        }
    };
    if (rank == 0) {
        const int p0 = cl_search(cols, rowdone, k, sv, si);
        broadcast(cols, p0, 0);
    }
    cl.sync();
    int fail = 0;
    for (int j = 0; j < k; ++j) {
        const int buf = j & 1;
        const int p = pbuf[buf];
        if (p < 0) { fail = 1; break; }
        const double* f = fbuf + (size_t)buf * k;
        const double pv = f[p];
        if (threadIdx.x == 0) rowdone[p] = 1;
        if (rank == 0 && threadIdx.x == 0) s.rv_pivrow[j] = p;
        // multipliers of the local columns (row p / pivot), read before any write
        for (int c = threadIdx.x; c < cpc; c += blockDim.x) {
            const int t = rank + c * kCS;
            gcol[c] = (t < k && t != j) ? cols[(size_t)c * k + p] / pv : 0.0;
        }
        __syncthreads();
        const int nxt = j + 1;
        const int own_next = (nxt < k && rank == nxt % kCS) ? nxt / kCS : -1;
        auto upd = [&](int c) {
            const int t = rank + c * kCS;
            double* col = cols + (size_t)c * k;
            if (t == j) {
                for (int a = threadIdx.x; a < k; a += blockDim.x) col[a] = (a == p) ? 1.0 / pv : -f[a] / pv;
            } else {
                const double g = gcol[c];
                for (int a = threadIdx.x; a < k; a += blockDim.x) col[a] = (a == p) ? g : fma(-f[a], g, col[a]);
            }
        };
        if (own_next >= 0) {
            upd(own_next);
            __syncthreads();
            const int pn = cl_search(cols + (size_t)own_next * k, rowdone, k, sv, si);
            broadcast(cols + (size_t)own_next * k, pn, nxt & 1);
        }
        for (int c = 0; c < cpc; ++c) {
            if (c == own_next || rank + c * kCS >= k) continue;
            upd(c);
        }
        cl.sync();
    }
    if (fail && rank == 0 && threadIdx.x == 0) s.ctrl->err = kErrSingular;
    // columns back to global (column-major), as the assembly kernels expect
    for (int c = 0; c < cpc; ++c) {
        const int t = rank + c * kCS;
        if (t >= k) break;
        for (int a = threadIdx.x; a < k; a += blockDim.x) s.rv_M[(size_t)t * k + a] = cols[(size_t)c * k + a];
    }
}

size_t gj_cluster_smem(int k) {
    const int cpc = (k + kCS - 1) / kCS;
    return ((size_t)cpc * k + 2 * (size_t)k + cpc) * sizeof(double) + (2 + (size_t)k) * sizeof(int);
}

// pinv[pivrow[t]] = t (stored over rv_rowdone, no longer needed)
__global__ void k_pivinv(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        const int p = s.rv_pivrow[t];
        if (p >= 0 && p < k) s.rv_rowdone[p] = t;
    }
}

// J[b], c_J[b] and the dense B11^-1 (row b, column a) = M[pinv[a]*k + pivrow[b]]
__global__ void k_b11i(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const size_t total = (size_t)k * k;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / k), a = (int)(e % k);
        s.rv_W[e] = s.rv_M[(size_t)s.rv_rowdone[a] * k + s.rv_pivrow[b]];
    }
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += gridDim.x * blockDim.x) {
        const int j = s.basis[s.rv_struct_pos[b]];
        s.rv_J[b] = j;
        s.rv_cJ[b] = s.c[j];
    }
}

// C (nslack x k, after B11^-1 in rv_W) = -A[S, J] B11^-1; S rows in increasing
// order so that a tile's gathers from a column of A are close together.
constexpr int kGM = 64, kGN = 64, kGK = 16;
__global__ void __launch_bounds__(256) k_slack_gemm(DevState s, int k, int nslack) {
    if (s.ctrl->err != kErrNone) return;
    __shared__ double As[kGK][kGM + 1];
    __shared__ double Bs[kGK][kGN + 1];
    const double* B11i = s.rv_W;
    double* Cs = s.rv_W + (size_t)k * k;
    const int row0 = blockIdx.y * kGM, col0 = blockIdx.x * kGN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
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
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gc = col0 + tx * 4 + jj;
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
// slack of row s: b[s] + sum_a C[g][a] b[R[a]] (warp per basis position)
__global__ void k_bbar_struct(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
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

// y[R[a]] = sum_b c_J[b] B11^-1[b][a]; y = 0 on rows with a basic slack
__global__ void k_duals_struct(DevState s, int k) {
    if (s.ctrl->err != kErrNone) return;
    const int m = s.p.m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.p.ld; i += gridDim.x * blockDim.x) {
        const int a = i < m ? s.rv_row_index[i] : -1;
        double acc = 0.0;
        if (a >= 0) {
            for (int b = 0; b < k; ++b) acc = fma(s.rv_cJ[b], s.rv_W[(size_t)b * k + a], acc);
        }
        s.y[i] = acc;
        s.y32[i] = (float)acc;
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

void launch_reinv_gj(const DevState& s, int k, const Geometry& g, cudaStream_t st) {
    if (k <= 0) return;
    if (k <= kClusterMaxK) {
        const size_t smem = gj_cluster_smem(k);
        static bool configured = false;
        if (!configured) {
            cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gj_cluster_smem(kClusterMaxK));
            configured = true;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kCS, 1, 1);
        cfg.blockDim = dim3(kClusterThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kCS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_gj_cluster, s, k) == cudaSuccess) {
            k_pivinv<<<(k + 255) / 256, 256, 0, st>>>(s, k);
            return;
        }
        (void)cudaGetLastError();  // cluster launch unavailable: per-step kernels below
    }
    {
        const size_t total = (size_t)k * k;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_gather<<<blocks, 256, 0, st>>>(s, k);
    }
    k_gj_search0<<<1, kStepThreads, 0, st>>>(s, k);
    int blocks = k < 2 * g.sms ? k : 2 * g.sms;
    for (int j = 0; j < k; ++j) k_gj_step<<<blocks, kStepThreads, 0, st>>>(s, k, j);
    k_pivinv<<<(k + 255) / 256, 256, 0, st>>>(s, k);
}

void launch_reinv_assemble(const DevState& s, int k, const Geometry& g, cudaStream_t st) {
    const int nslack = s.p.m - k;
    if (k > 0) {
        const size_t kk = (size_t)k * k;
        int blocks = (int)((kk + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_b11i<<<blocks, 256, 0, st>>>(s, k);
        if (nslack > 0) {
            dim3 grid((k + kGN - 1) / kGN, (nslack + kGM - 1) / kGM);
            k_slack_gemm<<<grid, 256, 0, st>>>(s, k, nslack);
        }
    }
    k_assemble_rows<<<g.sms * 4, 256, 0, st>>>(s, k);
}

void launch_reinv_finish(const DevState& s, int k, const Geometry& g, cudaStream_t st, int check_feasible) {
    k_bbar_struct<<<g.sms * 2, 256, 0, st>>>(s, k);
    k_duals_struct<<<(s.p.ld + 255) / 256, 256, 0, st>>>(s, k);
    k_reinv_close<<<1, 1024, 0, st>>>(s, check_feasible);
}

}  // namespace lpgb
