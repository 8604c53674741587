// family.cu -- LP families for the learned warm start (lp_family_* in include/lpgb.h).
//
// A family is a base LP (A0, b0, c0) whose instances multiply every entry of
// A, b and c by an independent N(1, sigma^2) draw.  Training instances are
// drawn here on the GPU so that tens of thousands of them never cross PCIe:
// draw e of an instance is a normal from the Box-Muller transform of the
// uniforms u_{2p}, u_{2p+1} (p = e / 2; cos for even e, sin for odd e), and the
// uniforms are SplitMix64 in counter mode (Steele, Lea & Flood 2014) under the
// instance's key -- the same definition as the host-side generator, so an
// instance drawn here matches the host's up to the last bits of log/cos/sin.
//
// Features of an instance (what the network sees), standardised to about
// N(0, 1): (b_i/b0_i - 1)/sigma, (c_j/c0_j - 1)/sigma, and the row and column
// means of A/A0 over the nonzero entries of A0, minus 1, times
// sqrt(count)/sigma.
#include "../../include/lpgb.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t key, uint64_t k) {
    uint64_t z = key + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(uint64_t key, uint64_t k) {
    return (double)(sm64(key, k) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double normal_draw(uint64_t key, uint64_t e) {
    const uint64_t p = e >> 1;
    const double u1 = 1.0 - u01(key, 2 * p);
    const double u2 = u01(key, 2 * p + 1);
    const double r = sqrt(-2.0 * log(u1));
    const double ang = 6.283185307179586 * u2;
    return (e & 1) ? r * sin(ang) : r * cos(ang);
}

__global__ void k_perturb(int m, int n, const double* __restrict__ A0, const double* __restrict__ b0,
                          const double* __restrict__ c0, uint64_t key, double sigma, double* __restrict__ A,
                          double* __restrict__ b, double* __restrict__ c) {
    const uint64_t mn = (uint64_t)m * n;
    const uint64_t total = mn + m + n;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const double f = 1.0 + sigma * normal_draw(key, e);
        if (e < mn) A[e] = A0[e] * f;
        else if (e < mn + m) b[e - mn] = b0[e - mn] * f;
        else c[e - mn - m] = c0[e - mn - m] * f;
    }
}

// row features: one block per row
__global__ void k_feat_rows(int m, int n, const double* __restrict__ A0, const double* __restrict__ A,
                            double sigma, float* __restrict__ out) {
    const int i = blockIdx.x;
    double s = 0.0;
    int cnt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double a0 = A0[(size_t)i * n + j];
        if (a0 != 0.0) { s += A[(size_t)i * n + j] / a0; cnt++; }
    }
    __shared__ double ss[32];
    __shared__ int sc[32];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) { ss[threadIdx.x >> 5] = s; sc[threadIdx.x >> 5] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int ct = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t += ss[w]; ct += sc[w]; }
        out[i] = ct ? (float)((t / ct - 1.0) * sqrt((double)ct) / sigma) : 0.f;
    }
}

// column features, b and c ratios: a thread per column (coalesced over rows)
__global__ void k_feat_cols(int m, int n, const double* __restrict__ A0, const double* __restrict__ A,
                            const double* __restrict__ b0, const double* __restrict__ b,
                            const double* __restrict__ c0, const double* __restrict__ c, double sigma,
                            float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double s = 0.0;
        int cnt = 0;
        for (int i = 0; i < m; ++i) {
            const double a0 = A0[(size_t)i * n + j];
            if (a0 != 0.0) { s += A[(size_t)i * n + j] / a0; cnt++; }
        }
        out[2 * m + n + j] = cnt ? (float)((s / cnt - 1.0) * sqrt((double)cnt) / sigma) : 0.f;
        out[m + j] = c0[j] != 0.0 ? (float)((c[j] / c0[j] - 1.0) / sigma) : 0.f;
    }
    if (j < m) out[j] = b0[j] != 0.0 ? (float)((b[j] / b0[j] - 1.0) / sigma) : 0.f;
}

// ---- the proposed basis from the network's scores ------------------------------
// Structural j is proposed when its score z_j exceeds the threshold; the
// proposed structurals in the order (z_j descending, j ascending), at most m of
// them, are J_0, J_1, ...  Slack rows in the order (z_{n+i} ascending, i ascending) give up their
// positions: the t-th of them holds J_t.  Orders are computed as ranks (the
// number of elements that come first), which needs no sort and is exact for
// ties.  Scores are read through shared-memory tiles.

constexpr int kTile = 1024;

// rank of every proposed structural; J[rank] = j for rank < m; work[m] counts them
__global__ void __launch_bounds__(256) k_rank_structurals(int m, int n, const float* __restrict__ z,
                                                          float thr, int32_t* __restrict__ work) {
    __shared__ float zt[kTile];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const float zj = j < n ? z[j] : 0.f;
    const bool cand = j < n && zj > thr;
    int rank = 0;
    for (int t0 = 0; t0 < n; t0 += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile && t0 + k < n; k += blockDim.x) zt[k] = z[t0 + k];
        __syncthreads();
        const int tn = n - t0 < kTile ? n - t0 : kTile;
        if (cand)
            for (int k = 0; k < tn; ++k) {
                const float v = zt[k];
                rank += (v > zj || (v == zj && t0 + k < j)) ? 1 : 0;  // v >= zj > thr: proposed too
            }
    }
    if (cand) {
        if (rank < m) work[rank] = j;
        atomicAdd(work + m, 1);
    }
}

// basis[i]: J_t when slack row i is the t-th to give up its position (t < k =
// min(m, count)), else the slack n + i
__global__ void __launch_bounds__(256) k_place_structurals(int m, int n, const float* __restrict__ z,
                                                           const int32_t* __restrict__ work,
                                                           int32_t* __restrict__ basis) {
    __shared__ float zt[kTile];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float zi = i < m ? z[n + i] : 0.f;
    int rank = 0;
    for (int t0 = 0; t0 < m; t0 += kTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kTile && t0 + k < m; k += blockDim.x) zt[k] = z[n + t0 + k];
        __syncthreads();
        const int tn = m - t0 < kTile ? m - t0 : kTile;
        if (i < m)
            for (int k = 0; k < tn; ++k) {
                const float v = zt[k];
                rank += (v < zi || (v == zi && t0 + k < i)) ? 1 : 0;
            }
    }
    if (i < m) {
        const int cnt = work[m];
        const int kk = cnt < m ? cnt : m;
        basis[i] = rank < kk ? work[rank] : n + i;
    }
}

}  // namespace

extern "C" {

int lp_family_propose(int32_t m, int32_t n, const float* scores, float threshold, int32_t* basis, int32_t* work,
                      void* cuda_stream) {
    if (m < 1 || n < 1 || !scores || !basis || !work || !(threshold == threshold)) return LP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(work + m, 0, sizeof(int32_t), st) != cudaSuccess) return LP_ERR_CUDA;
    k_rank_structurals<<<(n + 255) / 256, 256, 0, st>>>(m, n, scores, threshold, work);
    k_place_structurals<<<(m + 255) / 256, 256, 0, st>>>(m, n, scores, work, basis);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int lp_family_perturb(int32_t m, int32_t n, const double* A0, const double* b0, const double* c0, uint64_t key,
                      double sigma, double* A, double* b, double* c, void* cuda_stream) {
    if (m < 1 || n < 1 || !A0 || !b0 || !c0 || !A || !b || !c || !(sigma >= 0)) return LP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_perturb<<<1024, 256, 0, st>>>(m, n, A0, b0, c0, key, sigma, A, b, c);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int lp_family_features(int32_t m, int32_t n, const double* A0, const double* b0, const double* c0,
                       const double* A, const double* b, const double* c, double sigma, float* features,
                       void* cuda_stream) {
    if (m < 1 || n < 1 || !A0 || !b0 || !c0 || !A || !b || !c || !features || !(sigma > 0))
        return LP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_feat_rows<<<m, 256, 0, st>>>(m, n, A0, A, sigma, features + m + n);
    const int cols = n > m ? n : m;
    k_feat_cols<<<(cols + 255) / 256, 256, 0, st>>>(m, n, A0, A, b0, b, c0, c, sigma, features);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

}  // extern "C"
