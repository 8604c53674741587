// mlp.cu -- the learned warm start's network (lp_mlp_* in include/lpgb.h).
//
// A 3-layer perceptron  in -> H -> H -> out  with ReLU, trained with the
// binary cross-entropy on logits against the 0/1 "basic at the optimum"
// labels of a family of LPs, and Adam.  Weights are used in FP16 with FP32
// accumulation on the tensor cores (mma.sync m16n8k16); FP32 master weights
// and Adam moments are kept for the update.
//
// Loss (per batch of B samples):  L = (1/B) sum_b sum_o [softplus(z_bo) - t_bo z_bo]
// so dL/dz = (sigmoid(z) - t) / B, small enough and large enough for FP16.
//
// Layout: activations row-major [B x features]; W_l row-major [in_l x out_l];
// parameters packed W1, b1, W2, b2, W3, b3.
#include "../../include/lpgb.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32;
constexpr int kGemmThreads = 128;

__device__ __forceinline__ uint32_t pack2(__half lo, __half hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

// C[M x N] (fp32) = op(A)[M x K] * op(B)[K x N], fp16 operands.
//   transA = 0: A is [M x K] row-major (lda >= K); 1: A is [K x M] (lda >= M)
//   transB = 0: B is [K x N] row-major (ldb >= N); 1: B is [N x K] (ldb >= K)
__global__ void __launch_bounds__(kGemmThreads) k_gemm_f16(int M, int N, int K, const __half* __restrict__ A,
                                                           int lda, int transA, const __half* __restrict__ B,
                                                           int ldb, int transB, float* __restrict__ C, int ldc) {
    __shared__ __half As[kBM][kBK + 8];  // [m][k]
    __shared__ __half Bs[kBN][kBK + 8];  // [n][k]
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kBK) {
        for (int e = threadIdx.x; e < kBM * kBK; e += kGemmThreads) {
            const int mm = transA ? e % kBM : e / kBK;
            const int kk = transA ? e / kBM : e % kBK;
            const int gm = m0 + mm, gk = k0 + kk;
            __half v = __float2half(0.f);
            if (gm < M && gk < K) v = transA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[mm][kk] = v;
        }
        for (int e = threadIdx.x; e < kBN * kBK; e += kGemmThreads) {
            const int nn = transB ? e / kBK : e % kBN;
            const int kk = transB ? e % kBK : e / kBN;
            const int gn = n0 + nn, gk = k0 + kk;
            __half v = __float2half(0.f);
            if (gn < N && gk < K) v = transB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[nn][kk] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = pack2(As[r][ks + 2 * t], As[r][ks + 2 * t + 1]);
                af[i][1] = pack2(As[r + 8][ks + 2 * t], As[r + 8][ks + 2 * t + 1]);
                af[i][2] = pack2(As[r][ks + 2 * t + 8], As[r][ks + 2 * t + 9]);
                af[i][3] = pack2(As[r + 8][ks + 2 * t + 8], As[r + 8][ks + 2 * t + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cidx = wn + 8 * j + g;
                bf[j][0] = pack2(Bs[cidx][ks + 2 * t], Bs[cidx][ks + 2 * t + 1]);
                bf[j][1] = pack2(Bs[cidx][ks + 2 * t + 8], Bs[cidx][ks + 2 * t + 9]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]),
                          "r"(bf[j][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = m0 + wm + 16 * i + g + (h >= 2 ? 8 : 0);
                const int cc = n0 + wn + 8 * j + 2 * t + (h & 1);
                if (r < M && cc < N) C[(size_t)r * ldc + cc] = acc[i][j][h];
            }
}

__global__ void k_f32_to_f16(const float* __restrict__ x, __half* __restrict__ y, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = __float2half_rn(x[e]);
}

// z += bias (per column); a = relu(z) in fp16 (relu = 0: a = z)
__global__ void k_bias_act(float* __restrict__ z, const float* __restrict__ bias, int rows, int cols, int relu,
                           __half* __restrict__ a) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float v = z[e] + bias[e % cols];
        z[e] = v;
        if (a) a[e] = __float2half_rn(relu ? fmaxf(v, 0.f) : v);
    }
}

// dz = (sigmoid(z) - t) / B in fp16; loss partial sums (softplus(z) - t z) / B
__global__ void k_bce(const float* __restrict__ z, const float* __restrict__ t, int rows, int cols,
                      __half* __restrict__ dz, float* __restrict__ loss) {
    const size_t n = (size_t)rows * cols;
    const float inv = 1.f / (float)rows;
    float l = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float v = z[e], tt = t[e];
        const float sp = v > 0.f ? v + log1pf(expf(-v)) : log1pf(expf(v));
        l += (sp - tt * v) * inv;
        const float sg = 1.f / (1.f + expf(-v));
        dz[e] = __float2half_rn((sg - tt) * inv);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dz = da * (z > 0), fp16
__global__ void k_relu_back(const float* __restrict__ da, const float* __restrict__ z, size_t n,
                            __half* __restrict__ dz) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        dz[e] = __float2half_rn(z[e] > 0.f ? da[e] : 0.f);
}

// db[c] = sum_r dz[r][c]
__global__ void k_colsum(const __half* __restrict__ dz, int rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += __half2float(dz[(size_t)r * cols + c]);
    db[c] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, __half* __restrict__ p16) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gg;
        const float v = b2 * m2[e] + (1.f - b2) * gg * gg;
        m1[e] = a;
        m2[e] = v;
        const float pn = p[e] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        p[e] = pn;
        p16[e] = __float2half_rn(pn);
    }
}

}  // namespace

struct lp_mlp {
    int in = 0, hid = 0, out = 0, maxb = 0;
    size_t np = 0;
    size_t off[6] = {};  // W1 b1 W2 b2 W3 b3 offsets into the packed vectors
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // packed fp32
    __half* p16 = nullptr;                                           // packed fp16 copy
    __half* x16 = nullptr;                                           // [maxb x in]
    float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;               // pre-activations
    __half *a1 = nullptr, *a2 = nullptr;                             // activations
    __half *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    float *da2 = nullptr, *da1 = nullptr;
    float* loss = nullptr;
    int64_t steps = 0;
};

namespace {

int mfail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA; }

#define MCK(x)                                   \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return mfail(e_); \
    } while (0)

template <typename T>
int malloc_t(lp_mlp* h, T** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return mfail(e);
    h->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return LP_OK;
}

void gemm(const lp_mlp* h, int M, int N, int K, const __half* A, int lda, int ta, const __half* B, int ldb, int tb,
          float* C, int ldc) {
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    k_gemm_f16<<<grid, kGemmThreads, 0, h->stream>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc);
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

// forward pass for a batch already converted to x16; logits in z3
void forward(lp_mlp* h, int B) {
    const __half *W1 = h->p16 + h->off[0], *W2 = h->p16 + h->off[2], *W3 = h->p16 + h->off[4];
    const float *b1 = h->p + h->off[1], *b2 = h->p + h->off[3], *b3 = h->p + h->off[5];
    gemm(h, B, h->hid, h->in, h->x16, h->in, 0, W1, h->hid, 0, h->z1, h->hid);
    k_bias_act<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->z1, b1, B, h->hid, 1, h->a1);
    gemm(h, B, h->hid, h->hid, h->a1, h->hid, 0, W2, h->hid, 0, h->z2, h->hid);
    k_bias_act<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->z2, b2, B, h->hid, 1, h->a2);
    gemm(h, B, h->out, h->hid, h->a2, h->hid, 0, W3, h->out, 0, h->z3, h->out);
    k_bias_act<<<blocks_for((size_t)B * h->out), 256, 0, h->stream>>>(h->z3, b3, B, h->out, 0, nullptr);
}

// loss and gradients into h->g for targets t (fp32, device, [B x out])
int backward(lp_mlp* h, int B, const float* t) {
    MCK(cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream));
    k_bce<<<blocks_for((size_t)B * h->out), 256, 0, h->stream>>>(h->z3, t, B, h->out, h->dz3, h->loss);
    const __half *W2 = h->p16 + h->off[2], *W3 = h->p16 + h->off[4];
    float *gW1 = h->g + h->off[0], *gb1 = h->g + h->off[1], *gW2 = h->g + h->off[2];
    float *gb2 = h->g + h->off[3], *gW3 = h->g + h->off[4], *gb3 = h->g + h->off[5];
    // layer 3
    gemm(h, h->hid, h->out, B, h->a2, h->hid, 1, h->dz3, h->out, 0, gW3, h->out);
    k_colsum<<<(h->out + 255) / 256, 256, 0, h->stream>>>(h->dz3, B, h->out, gb3);
    gemm(h, B, h->hid, h->out, h->dz3, h->out, 0, W3, h->out, 1, h->da2, h->hid);
    k_relu_back<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->da2, h->z2, (size_t)B * h->hid, h->dz2);
    // layer 2
    gemm(h, h->hid, h->hid, B, h->a1, h->hid, 1, h->dz2, h->hid, 0, gW2, h->hid);
    k_colsum<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dz2, B, h->hid, gb2);
    gemm(h, B, h->hid, h->hid, h->dz2, h->hid, 0, W2, h->hid, 1, h->da1, h->hid);
    k_relu_back<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->da1, h->z1, (size_t)B * h->hid, h->dz1);
    // layer 1
    gemm(h, h->in, h->hid, B, h->x16, h->in, 1, h->dz1, h->hid, 0, gW1, h->hid);
    k_colsum<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dz1, B, h->hid, gb1);
    MCK(cudaGetLastError());
    return LP_OK;
}

int load_x(lp_mlp* h, const float* X, int B) {
    if (B < 1 || B > h->maxb || !X) return LP_ERR_INVALID_ARG;
    const size_t n = (size_t)B * h->in;
    k_f32_to_f16<<<blocks_for(n), 256, 0, h->stream>>>(X, h->x16, n);
    MCK(cudaGetLastError());
    return LP_OK;
}

}  // namespace

extern "C" {

int lp_mlp_create(lp_mlp** out, int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch,
                  void* cuda_stream) {
    if (!out || in_dim < 1 || hidden < 1 || out_dim < 1 || max_batch < 1) return LP_ERR_INVALID_ARG;
    *out = nullptr;
    lp_mlp* h = new (std::nothrow) lp_mlp();
    if (!h) return LP_ERR_OOM;
    h->in = in_dim; h->hid = hidden; h->out = out_dim; h->maxb = max_batch;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t sz[6] = {(size_t)in_dim * hidden, (size_t)hidden, (size_t)hidden * hidden, (size_t)hidden,
                          (size_t)hidden * out_dim, (size_t)out_dim};
    size_t o = 0;
    for (int i = 0; i < 6; ++i) { h->off[i] = o; o += sz[i]; }
    h->np = o;
    const size_t B = max_batch;
    int rc = LP_OK;
    if ((rc = malloc_t(h, &h->p, o)) || (rc = malloc_t(h, &h->g, o)) || (rc = malloc_t(h, &h->m1, o)) ||
        (rc = malloc_t(h, &h->m2, o)) || (rc = malloc_t(h, &h->p16, o)) ||
        (rc = malloc_t(h, &h->x16, B * in_dim)) || (rc = malloc_t(h, &h->z1, B * hidden)) ||
        (rc = malloc_t(h, &h->z2, B * hidden)) || (rc = malloc_t(h, &h->z3, B * out_dim)) ||
        (rc = malloc_t(h, &h->a1, B * hidden)) || (rc = malloc_t(h, &h->a2, B * hidden)) ||
        (rc = malloc_t(h, &h->dz3, B * out_dim)) || (rc = malloc_t(h, &h->dz2, B * hidden)) ||
        (rc = malloc_t(h, &h->dz1, B * hidden)) || (rc = malloc_t(h, &h->da2, B * hidden)) ||
        (rc = malloc_t(h, &h->da1, B * hidden)) || (rc = malloc_t(h, &h->loss, 1))) {
        lp_mlp_destroy(h);
        return rc;
    }
    if (cudaMemsetAsync(h->p, 0, o * sizeof(float), h->stream) || cudaMemsetAsync(h->m1, 0, o * sizeof(float), h->stream) ||
        cudaMemsetAsync(h->m2, 0, o * sizeof(float), h->stream) || cudaMemsetAsync(h->p16, 0, o * sizeof(__half), h->stream)) {
        lp_mlp_destroy(h);
        return LP_ERR_CUDA;
    }
    *out = h;
    return LP_OK;
}

int64_t lp_mlp_num_params(const lp_mlp* h) { return h ? (int64_t)h->np : -1; }

int lp_mlp_set_params(lp_mlp* h, const float* params) {
    if (!h || !params) return LP_ERR_INVALID_ARG;
    MCK(cudaMemcpyAsync(h->p, params, h->np * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    k_f32_to_f16<<<blocks_for(h->np), 256, 0, h->stream>>>(h->p, h->p16, h->np);
    MCK(cudaMemsetAsync(h->m1, 0, h->np * sizeof(float), h->stream));
    MCK(cudaMemsetAsync(h->m2, 0, h->np * sizeof(float), h->stream));
    h->steps = 0;
    MCK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_mlp_get_params(const lp_mlp* h, float* params) {
    if (!h || !params) return LP_ERR_INVALID_ARG;
    MCK(cudaMemcpyAsync(params, h->p, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_mlp_forward(lp_mlp* h, const float* X, int32_t batch, float* logits) {
    if (!h || !logits) return LP_ERR_INVALID_ARG;
    int rc = load_x(h, X, batch);
    if (rc != LP_OK) return rc;
    forward(h, batch);
    MCK(cudaMemcpyAsync(logits, h->z3, (size_t)batch * h->out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    MCK(cudaGetLastError());
    return LP_OK;
}

int lp_mlp_gradients(lp_mlp* h, const float* X, const float* T, int32_t batch, float* grads, float* loss) {
    if (!h || !T) return LP_ERR_INVALID_ARG;
    int rc = load_x(h, X, batch);
    if (rc != LP_OK) return rc;
    forward(h, batch);
    if ((rc = backward(h, batch, T)) != LP_OK) return rc;
    if (grads) MCK(cudaMemcpyAsync(grads, h->g, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (loss) MCK(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return LP_OK;
}

int lp_mlp_train_step(lp_mlp* h, const float* X, const float* T, int32_t batch, float lr, float* loss) {
    if (!h || !T || !(lr > 0.f)) return LP_ERR_INVALID_ARG;
    int rc = load_x(h, X, batch);
    if (rc != LP_OK) return rc;
    forward(h, batch);
    if ((rc = backward(h, batch, T)) != LP_OK) return rc;
    h->steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)h->steps), c2 = 1.f - powf(b2, (float)h->steps);
    k_adam<<<blocks_for(h->np), 256, 0, h->stream>>>(h->p, h->g, h->m1, h->m2, h->np, lr, b1, b2, 1e-8f, c1, c2,
                                                     h->p16);
    MCK(cudaGetLastError());
    if (loss) {
        MCK(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        MCK(cudaStreamSynchronize(h->stream));
    }
    return LP_OK;
}

void lp_mlp_destroy(lp_mlp* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    delete h;
}

}  // extern "C"
