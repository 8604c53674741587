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
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        if (!isfinite(b[i]) || b[i] < 0.0) f |= 2;
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

void launch_load_basis(const DevState& s, cudaStream_t st) {
    k_load_basis<<<256, 256, 0, st>>>(s);
    k_load_basis_pos<<<64, 256, 0, st>>>(s);
}

}  // namespace lpgb
