// kernels_sparse.cu -- compressed sparse column copy of A for the sparse FP64
// PRICE (price_mode 2; the S20/S60 classes of the paper's dense test set have
// 20% and 60% zero entries).
//
// Step 3 PRICE computes d_j = c_j - y^T a_j; with a_j stored as its nonzeros
// (row index, value) in increasing row order, the dot product runs over the
// nonzeros only: the FMAs and the bytes both scale with the density, while
// the dense B^-1 and everything else in the iteration stay as they are.
//
// The copy is built on the device from the column-major A (no host round
// trip of A): one warp per column counts, a block scan turns the counts into
// column pointers, one warp per column writes its nonzeros in row order.
#include "lpgb_internal.cuh"

namespace lpgb {

namespace {

__global__ void k_csc_count(const double* __restrict__ A_cm, int m, int n, int ld, int32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nwarps) {
        const double* col = A_cm + (size_t)j * ld;
        int c = 0;
        for (int i = lane; i < m; i += 32) c += col[i] != 0.0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[j] = c;
    }
}

// exclusive scan of n counts into ptr[0..n] (one block)
__global__ void __launch_bounds__(1024) k_csc_scan(const int32_t* __restrict__ cnt, int n, int64_t* __restrict__ ptr) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t base_sh;
    if (threadIdx.x == 0) base_sh = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int j = c0 + threadIdx.x;
        int64_t v = j < n ? cnt[j] : 0;
        int64_t x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        int64_t before = base_sh;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (j < n) ptr[j] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base_sh = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) ptr[n] = base_sh;
}

__global__ void k_csc_fill(const double* __restrict__ A_cm, int m, int n, int ld, const int64_t* __restrict__ ptr,
                           int32_t* __restrict__ row, double* __restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nwarps) {
        const double* col = A_cm + (size_t)j * ld;
        int64_t at = ptr[j];
        for (int i0 = 0; i0 < m; i0 += 32) {
            const int i = i0 + lane;
            const double a = i < m ? col[i] : 0.0;
            const unsigned bal = __ballot_sync(0xffffffffu, a != 0.0);
            if (a != 0.0) {
                const int64_t e = at + __popc(bal & ((1u << lane) - 1u));
                row[e] = i;
                val[e] = a;
            }
            at += __popc(bal);
        }
    }
}

}  // namespace

void launch_csc_count(const double* A_cm, int m, int n, int ld, int32_t* cnt, int64_t* ptr, cudaStream_t st) {
    k_csc_count<<<1024, 256, 0, st>>>(A_cm, m, n, ld, cnt);
    k_csc_scan<<<1, 1024, 0, st>>>(cnt, n, ptr);
}

void launch_csc_fill(const double* A_cm, int m, int n, int ld, const int64_t* ptr, int32_t* row, double* val,
                     cudaStream_t st) {
    k_csc_fill<<<1024, 256, 0, st>>>(A_cm, m, n, ld, ptr, row, val);
}

}  // namespace lpgb
