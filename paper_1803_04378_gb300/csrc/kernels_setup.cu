// kernels_setup.cu -- problem upload: transpose of the row-major A (the
// paper's d_A[i*n+j] layout, Section 3.2) into the padded column-major layout
// the iteration kernels stream, input validation, and warm-start basis load.
#include "lpgb_internal.cuh"

namespace lpgb {

namespace {

constexpr int kT = 32;

// A_cm[j*ld + i] = A_rm[i*n + j] for i < m; rows m..ld-1 of every column = 0.
__global__ void k_transpose_pad(const double* __restrict__ A, int m, int n, int ld,
                                double* __restrict__ out) {
    __shared__ double tile[kT][kT + 1];
    const int i0 = blockIdx.y * kT, j0 = blockIdx.x * kT;
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < m && j < n) ? A[(size_t)i * n + j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        if (j < n && i < ld) out[(size_t)j * ld + i] = tile[threadIdx.x][r];
    }
}

// flag bit 1: non-finite A; bit 2: non-finite or negative b; bit 4: non-finite c
__global__ void k_validate(const double* A_cm, const double* b, const double* c, int m, int n, int ld,
                           int32_t* flag) {
    int f = 0;
    const size_t total = (size_t)n * ld;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(A_cm[e])) f |= 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if (!isfinite(b[i])) f |= 2;
        if (b[i] < 0.0) f |= 8;  // not an error: the solve starts with Phase I
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (!isfinite(c[j])) f |= 4;
    if (f) atomicOr(flag, f);
}

// basis[] was uploaded; derive pos[], clear tabu and the control block.
__global__ void k_load_basis(DevState s) {
    const int m = s.p.m, n = s.p.n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int j = tid; j < n + m; j += stride) {
        s.pos[j] = -1;
        s.tabu_until[j] = 0;
    }
    for (int i = tid; i < s.p.ld; i += stride) {
        s.rho[i] = 0.0;
        s.y32[i] = 0.f;
        s.alpha[i] = 0.0;
        s.alpha[s.p.ld + i] = 0.0;
    }
}

__global__ void k_load_basis_pos(DevState s) {
    const int m = s.p.m;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m; p += gridDim.x * blockDim.x)
        s.pos[s.basis[p]] = p;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl c = {};
        c.status = kRunning;
        c.q = -1;
        c.r = -1;
        *s.ctrl = c;
    }
}

}  // namespace

void launch_transpose_pad(const double* A_rm, int m, int n, int ld, double* A_cm, cudaStream_t st) {
    dim3 block(kT, 8);
    dim3 grid((n + kT - 1) / kT, (ld + kT - 1) / kT);
    k_transpose_pad<<<grid, block, 0, st>>>(A_rm, m, n, ld, A_cm);
}

void launch_validate(const double* A_cm, const double* b, const double* c, int m, int n, int ld,
                     int32_t* flag, cudaStream_t st) {
    k_validate<<<1024, 256, 0, st>>>(A_cm, b, c, m, n, ld, flag);
}

// Phase I problem (Section 3.4): [A | -e] row-major, e_i = 1 where b_i < 0,
// and the objective -x0 on the artificial column n.
__global__ void k_build_aux(const double* __restrict__ A_cm, int ld, int m, int n, const double* __restrict__ b,
                            double* __restrict__ A_aux, double* __restrict__ c_aux) {
    const size_t total = (size_t)m * (n + 1);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / (n + 1)), j = (int)(e % (n + 1));
        A_aux[e] = j < n ? A_cm[(size_t)j * ld + i] : (b[i] < 0.0 ? -1.0 : 0.0);
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += gridDim.x * blockDim.x)
        c_aux[j] = j < n ? 0.0 : -1.0;
}

void launch_build_aux(const double* A_cm, int ld, int m, int n, const double* b, double* A_aux, double* c_aux,
                      cudaStream_t st) {
    k_build_aux<<<1024, 256, 0, st>>>(A_cm, ld, m, n, b, A_aux, c_aux);
}

void launch_load_basis(const DevState& s, cudaStream_t st) {
    k_load_basis<<<256, 256, 0, st>>>(s);
    k_load_basis_pos<<<64, 256, 0, st>>>(s);
}

}  // namespace lpgb

namespace lpgb {
namespace {

// Warm-start repair (one block): if some basic value is below -tol, pick the
// most negative position p and, among nonbasic slacks s, the most negative
// B^-1[p][s]; stage the pivot (q = n+s, r = p) for k_pivot / k_update.
// tol = Ctrl::repair_tol.  Ctrl::repair becomes 2 when no value is negative,
// 3 when no slack can fix p, 4 when p exists but the iteration count has
// reached Ctrl::repair_limit.  Nothing is staged (q = -1, so k_pivot and
// k_update do nothing) when the repair has ended or the solve is not running
// (a reinversion is due): repair steps run in batches (a captured graph) and
// the host reads the outcome once per batch.
__global__ void __launch_bounds__(1024) k_repair_pick(DevState s) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int p_sh;
    __shared__ int go_sh, limit_sh;
    __shared__ double tol_sh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        go_sh = C->repair == 1 && C->status == kRunning;
        tol_sh = C->repair_tol;
        limit_sh = C->repair_limit;
        C->q = -1;
    }
    __syncthreads();
    if (!go_sh) return;
    const double tol = tol_sh;
    const int limit_it = limit_sh;
    // most negative basic value (ties: smallest position)
    double v = 0.0;
    int pi = -1;
    for (int p = threadIdx.x; p < P.m; p += blockDim.x) {
        const double bv = s.bbar[p];
        if (bv < -tol && (pi < 0 || bv < v)) { v = bv; pi = p; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, pi, o);
        if (oi >= 0 && (pi < 0 || ov < v || (ov == v && oi < pi))) { v = ov; pi = oi; }
    }
    if (lane == 0) { sv[w] = v; si[w] = pi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bvv = 0.0;
        int bp = -1;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            if (si[i] >= 0 && (bp < 0 || sv[i] < bvv || (sv[i] == bvv && si[i] < bp))) { bvv = sv[i]; bp = si[i]; }
        if (bp < 0) C->repair = 2;
        else if (C->it >= limit_it) { C->repair = 4; bp = -1; }
        p_sh = bp;
    }
    __syncthreads();
    const int p = p_sh;
    if (p < 0) return;
    // entering slack: most negative B^-1[p][s] over nonbasic slacks s
    const double* row = s.binv + (size_t)p * P.ld;
    double best = 0.0;
    int bs = -1;
    for (int r = threadIdx.x; r < P.m; r += blockDim.x) {
        if (s.pos[P.n + r] >= 0) continue;
        const double e = row[r];
        if (e < 0.0 && (bs < 0 || e < best)) { best = e; bs = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bs, o);
        if (oi >= 0 && (bs < 0 || ov < best || (ov == best && oi < bs))) { best = ov; bs = oi; }
    }
    __syncthreads();
    if (lane == 0) { sv[w] = best; si[w] = bs; }
    __syncthreads();
    __shared__ int s_sh;
    __shared__ double e_sh;
    if (threadIdx.x == 0) {
        double be = 0.0;
        int b2 = -1;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            if (si[i] >= 0 && (b2 < 0 || sv[i] < be || (sv[i] == be && si[i] < b2))) { be = sv[i]; b2 = si[i]; }
        s_sh = b2;
        e_sh = be;
        if (b2 < 0) C->repair = 3;
    }
    __syncthreads();
    const int sl = s_sh;
    if (sl < 0) return;
    // alpha = column sl of B^-1 into the current alpha buffer
    double* al = s.alpha + (size_t)C->abuf * P.ld;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) al[i] = s.binv[(size_t)i * P.ld + sl];
    if (threadIdx.x == 0) {
        C->q = P.n + sl;
        C->r = p;
        C->dq = -s.y[sl];
        C->theta = s.bbar[p] / e_sh;
        C->tcount = 1;
        C->status = kRunning;
        C->flags = 0;
    }
}

// after the repair pivot's bookkeeping: no FTRAN of a next column
__global__ void k_repair_clear(DevState s) { s.ctrl->q = -1; }

__global__ void k_repair_begin(DevState s, double tol, int limit_it) {
    Ctrl* C = s.ctrl;
    C->repair = 1;
    C->repair_tol = tol;
    C->repair_limit = limit_it;
}

// ---- warm-start crash from the slack basis ---------------------------------------
// The proposed structurals enter one by one, in the order given, each by an
// ordinary pivot of the method: FTRAN of the column and the ratio test of
// Step 6 (k_update), so the basis stays primal feasible.  A candidate is
// passed over when it is basic already, when no alpha_i exceeds tol_piv, or
// when the ratio test would make a structural leave (a crash only replaces
// slacks).  Ctrl::crash: 1 running, 2 done; Ctrl::crash_t: the next list
// position.  Every kernel does nothing unless a crash is running and the
// solve is running (a reinversion may fall due between crash pivots).

__global__ void k_crash_begin(DevState s, int count) {
    Ctrl* C = s.ctrl;
    C->crash = count > 0 ? 1 : 2;
    C->crash_t = 0;
    C->crash_n = count;
    C->q = -1;
}

// next candidate into q with d_q = c_q - y^T a_q (one block); q = -1 and
// crash = 2 once the list is exhausted
__global__ void __launch_bounds__(256) k_crash_next(DevState s) {
    Ctrl* C = s.ctrl;
    const Params& P = s.p;
    __shared__ int q_sh;
    __shared__ double part[8];
    if (threadIdx.x == 0) {
        int q = -1;
        if (C->crash == 1 && C->status == kRunning) {
            int t = C->crash_t;
            while (t < C->crash_n && s.pos[s.crash_list[t]] >= 0) ++t;
            if (t < C->crash_n) {
                q = s.crash_list[t];
                C->crash_t = t + 1;
            } else {
                C->crash = 2;
                C->crash_t = t;
                C->q = -1;
            }
        }
        q_sh = q;
    }
    __syncthreads();
    const int q = q_sh;
    if (q < 0) return;
    const double* col = s.A_cm + (size_t)q * P.ld;
    double acc = 0.0;
    for (int i = threadIdx.x; i < P.m; i += blockDim.x) acc = fma(s.y[i], col[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        C->q = q;
        C->dq = s.c[q] - t;
        C->flags = 0;
    }
}

// after k_update's FTRAN and ratio test: pass the candidate over (q = -1)
// when its column has no alpha_i > tol_piv (k_update then reported the
// problem unbounded along it) or a structural would leave
__global__ void k_crash_check(DevState s) {
    Ctrl* C = s.ctrl;
    if (C->crash != 1 || C->q < 0) return;
    if (C->status == kUnbounded) {
        C->status = kRunning;
        C->q = -1;
        return;
    }
    if (C->status != kRunning) return;
    const int r = C->r;
    if (r < 0 || r >= s.p.m || s.basis[r] < s.p.n) C->q = -1;
}

}  // namespace

void launch_crash_begin(const DevState& s, int count, cudaStream_t st) { k_crash_begin<<<1, 1, 0, st>>>(s, count); }

// `steps` crash steps: the next candidate, the pending update with the
// candidate's FTRAN and ratio test, the check, the pivot's bookkeeping
void launch_crash_steps(const DevState& s, const Geometry& g, int steps, cudaStream_t st) {
    for (int t = 0; t < steps; ++t) {
        k_crash_next<<<1, 256, 0, st>>>(s);
        launch_update(s, g, st);
        k_crash_check<<<1, 1, 0, st>>>(s);
        launch_pivot(s, g, st);
    }
}

void launch_repair_begin(const DevState& s, double tol, int limit_it, cudaStream_t st) {
    k_repair_begin<<<1, 1, 0, st>>>(s, tol, limit_it);
}

// `steps` repair pivots (pick, the pivot's bookkeeping, no next column, the
// B^-1 update) enqueued back to back; the steps after the repair ends, a
// reinversion falls due or the iteration count reaches the limit do nothing.
void launch_repair_steps(const DevState& s, const Geometry& g, int steps, cudaStream_t st) {
    for (int t = 0; t < steps; ++t) {
        k_repair_pick<<<1, 1024, 0, st>>>(s);
        launch_pivot(s, g, st);
        k_repair_clear<<<1, 1, 0, st>>>(s);
        launch_update(s, g, st);
    }
}

}  // namespace lpgb
