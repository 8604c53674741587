// mlp.cu -- the learned warm start's network (lp_mlp_* in include/lpgb.h).
//
// A 3-layer perceptron  in -> H -> H -> out  with ReLU, trained with the
// binary cross-entropy on logits against the 0/1 "basic at the optimum"
// labels of a family of LPs, and Adam.  Weights are used in FP16 with FP32
// accumulation on the tensor cores (tcgen05.mma through tc_gemm: TMA-staged
// tiles, accumulators in TMEM); FP32 master weights and Adam moments are kept
// for the update.
//
// Loss (per batch of B samples):  L = (1/B) sum_b sum_o [softplus(z_bo) - t_bo z_bo]
// so dL/dz = (sigmoid(z) - t) / B, small enough and large enough for FP16.
//
// Every product is D = X Y^T with both operands K-major (tc_gemm), so each
// FP16 operand is kept in the layout its GEMM reads: activations row-major
// [B x features] and, for the weight gradients, transposed [features x B];
// the weights as W^T (forward) and W (the input gradients of the backward
// pass).  FP16 rows are padded to a multiple of 8 elements (16-byte TMA
// strides); FP32 results keep the logical widths.  Parameters are packed
// W1, b1, W2, b2, W3, b3 with W_l row-major [in_l x out_l].
#include "../../include/lpgb.h"
#include "lpgb_internal.cuh"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace lpgb {
cudaError_t tc_gemm(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K, bool bf16,
                    int32_t* err, cudaStream_t st);
}

namespace {

inline int pad8(int v) { return (v + 7) & ~7; }

// X (rows x cols, FP32) -> x16 (row stride ld) and xT (cols x rows, row stride ldt), FP16
__global__ void k_input16(const float* __restrict__ X, int rows, int cols, __half* __restrict__ x16, int ld,
                          __half* __restrict__ xT, int ldt) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const __half h = __float2half_rn(X[e]);
        x16[(size_t)r * ld + c] = h;
        xT[(size_t)c * ldt + r] = h;
    }
}

// z += bias (per column); a = relu(z) (relu = 0: a = z) in FP16, row-major
// (row stride lda) and transposed (row stride ldt)
__global__ void k_bias_act(float* __restrict__ z, const float* __restrict__ bias, int rows, int cols, int relu,
                           __half* __restrict__ a, int lda, __half* __restrict__ aT, int ldt) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const float v = z[e] + bias[c];
        z[e] = v;
        if (a) {
            const __half h = __float2half_rn(relu ? fmaxf(v, 0.f) : v);
            a[(size_t)r * lda + c] = h;
            aT[(size_t)c * ldt + r] = h;
        }
    }
}

// dz = (sigmoid(z) - t) / B in FP16 (row-major and transposed); loss partial sums (softplus(z) - t z) / B
__global__ void k_bce(const float* __restrict__ z, const float* __restrict__ t, int rows, int cols,
                      __half* __restrict__ dz, int ld, __half* __restrict__ dzT, int ldt, float* __restrict__ loss) {
    const size_t n = (size_t)rows * cols;
    const float inv = 1.f / (float)rows;
    float l = 0.f;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const float v = z[e], tt = t[e];
        const float sp = v > 0.f ? v + log1pf(expf(-v)) : log1pf(expf(v));
        l += (sp - tt * v) * inv;
        const float sg = 1.f / (1.f + expf(-v));
        const __half h = __float2half_rn((sg - tt) * inv);
        dz[(size_t)r * ld + c] = h;
        dzT[(size_t)c * ldt + r] = h;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dz = da * (z > 0), FP16 (row-major and transposed)
__global__ void k_relu_back(const float* __restrict__ da, const float* __restrict__ z, int rows, int cols,
                            __half* __restrict__ dz, int ld, __half* __restrict__ dzT, int ldt) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const __half h = __float2half_rn(z[e] > 0.f ? da[e] : 0.f);
        dz[(size_t)r * ld + c] = h;
        dzT[(size_t)c * ldt + r] = h;
    }
}

// db[c] = sum_r dz[r][c] (row stride ld)
__global__ void k_colsum(const __half* __restrict__ dz, int ld, int rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += __half2float(dz[(size_t)r * ld + c]);
    db[c] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * gg;
        const float v = b2 * m2[e] + (1.f - b2) * gg * gg;
        m1[e] = a;
        m2[e] = v;
        p[e] = p[e] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// FP16 copies of W (rows x cols, FP32 row-major): W itself (row stride ldn)
// and W^T (cols x rows, row stride ldt)
__global__ void k_weight16(const float* __restrict__ W, int rows, int cols, __half* __restrict__ Wn, int ldn,
                           __half* __restrict__ WT, int ldt) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const __half h = __float2half_rn(W[e]);
        if (Wn) Wn[(size_t)r * ldn + c] = h;
        WT[(size_t)c * ldt + r] = h;
    }
}

}  // namespace

struct lp_mlp {
    int in = 0, hid = 0, out = 0, maxb = 0;
    int in_p = 0, hid_p = 0, out_p = 0, b_p = 0;  // FP16 row strides (multiples of 8)
    size_t np = 0;
    size_t off[6] = {};  // W1 b1 W2 b2 W3 b3 offsets into the packed vectors
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // packed fp32
    __half *w1t = nullptr, *w2t = nullptr, *w3t = nullptr;           // W^T: [hid x in], [hid x hid], [out x hid]
    __half *w2n = nullptr, *w3n = nullptr;                           // W:   [hid x hid], [hid x out]
    __half *x16 = nullptr, *xT = nullptr;                            // [maxb x in], [in x maxb]
    float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;               // pre-activations
    __half *a1 = nullptr, *a2 = nullptr, *a1T = nullptr, *a2T = nullptr;
    __half *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    __half *dz3T = nullptr, *dz2T = nullptr, *dz1T = nullptr;
    float *da2 = nullptr, *da1 = nullptr;
    float* loss = nullptr;
    int32_t* err = nullptr;  // bounded-wait flag of the tensor-core GEMMs
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

// D (M x N, FP32, row stride ldd) = X (M x K, FP16, row stride ldx) * Y (N x K, FP16, row stride ldy)^T
int gemm(const lp_mlp* h, int M, int N, int K, const __half* X, int ldx, const __half* Y, int ldy, float* D,
         int ldd) {
    MCK(lpgb::tc_gemm(X, ldx, Y, ldy, D, ldd, M, N, K, false, h->err, h->stream));
    return LP_OK;
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

// FP16 copies of the weights from the FP32 masters
int refresh_weights(lp_mlp* h) {
    const float *W1 = h->p + h->off[0], *W2 = h->p + h->off[2], *W3 = h->p + h->off[4];
    k_weight16<<<blocks_for((size_t)h->in * h->hid), 256, 0, h->stream>>>(W1, h->in, h->hid, nullptr, 0, h->w1t, h->in_p);
    k_weight16<<<blocks_for((size_t)h->hid * h->hid), 256, 0, h->stream>>>(W2, h->hid, h->hid, h->w2n, h->hid_p, h->w2t,
                                                                            h->hid_p);
    k_weight16<<<blocks_for((size_t)h->hid * h->out), 256, 0, h->stream>>>(W3, h->hid, h->out, h->w3n, h->out_p, h->w3t,
                                                                            h->hid_p);
    MCK(cudaGetLastError());
    return LP_OK;
}

// forward pass for a batch already converted to x16 / xT; logits in z3
int forward(lp_mlp* h, int B) {
    const float *b1 = h->p + h->off[1], *b2 = h->p + h->off[3], *b3 = h->p + h->off[5];
    int rc;
    if ((rc = gemm(h, B, h->hid, h->in, h->x16, h->in_p, h->w1t, h->in_p, h->z1, h->hid))) return rc;
    k_bias_act<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->z1, b1, B, h->hid, 1, h->a1, h->hid_p, h->a1T,
                                                                      h->b_p);
    if ((rc = gemm(h, B, h->hid, h->hid, h->a1, h->hid_p, h->w2t, h->hid_p, h->z2, h->hid))) return rc;
    k_bias_act<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->z2, b2, B, h->hid, 1, h->a2, h->hid_p, h->a2T,
                                                                      h->b_p);
    if ((rc = gemm(h, B, h->out, h->hid, h->a2, h->hid_p, h->w3t, h->hid_p, h->z3, h->out))) return rc;
    k_bias_act<<<blocks_for((size_t)B * h->out), 256, 0, h->stream>>>(h->z3, b3, B, h->out, 0, nullptr, 0, nullptr, 0);
    MCK(cudaGetLastError());
    return LP_OK;
}

// loss and gradients into h->g for targets t (fp32, device, [B x out])
int backward(lp_mlp* h, int B, const float* t) {
    MCK(cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream));
    k_bce<<<blocks_for((size_t)B * h->out), 256, 0, h->stream>>>(h->z3, t, B, h->out, h->dz3, h->out_p, h->dz3T, h->b_p,
                                                                 h->loss);
    float *gW1 = h->g + h->off[0], *gb1 = h->g + h->off[1], *gW2 = h->g + h->off[2];
    float *gb2 = h->g + h->off[3], *gW3 = h->g + h->off[4], *gb3 = h->g + h->off[5];
    int rc;
    // layer 3: gW3 = a2^T dz3, da2 = dz3 W3^T
    if ((rc = gemm(h, h->hid, h->out, B, h->a2T, h->b_p, h->dz3T, h->b_p, gW3, h->out))) return rc;
    k_colsum<<<(h->out + 255) / 256, 256, 0, h->stream>>>(h->dz3, h->out_p, B, h->out, gb3);
    if ((rc = gemm(h, B, h->hid, h->out, h->dz3, h->out_p, h->w3n, h->out_p, h->da2, h->hid))) return rc;
    k_relu_back<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->da2, h->z2, B, h->hid, h->dz2, h->hid_p,
                                                                       h->dz2T, h->b_p);
    // layer 2: gW2 = a1^T dz2, da1 = dz2 W2^T
    if ((rc = gemm(h, h->hid, h->hid, B, h->a1T, h->b_p, h->dz2T, h->b_p, gW2, h->hid))) return rc;
    k_colsum<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dz2, h->hid_p, B, h->hid, gb2);
    if ((rc = gemm(h, B, h->hid, h->hid, h->dz2, h->hid_p, h->w2n, h->hid_p, h->da1, h->hid))) return rc;
    k_relu_back<<<blocks_for((size_t)B * h->hid), 256, 0, h->stream>>>(h->da1, h->z1, B, h->hid, h->dz1, h->hid_p,
                                                                       h->dz1T, h->b_p);
    // layer 1: gW1 = x^T dz1
    if ((rc = gemm(h, h->in, h->hid, B, h->xT, h->b_p, h->dz1T, h->b_p, gW1, h->hid))) return rc;
    k_colsum<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dz1, h->hid_p, B, h->hid, gb1);
    MCK(cudaGetLastError());
    return LP_OK;
}

int load_x(lp_mlp* h, const float* X, int B) {
    if (B < 1 || B > h->maxb || !X) return LP_ERR_INVALID_ARG;
    k_input16<<<blocks_for((size_t)B * h->in), 256, 0, h->stream>>>(X, B, h->in, h->x16, h->in_p, h->xT, h->b_p);
    MCK(cudaGetLastError());
    return LP_OK;
}

// the GEMMs' bounded waits: LP_ERR_TIMEOUT if one gave up
int check_err(lp_mlp* h) {
    int32_t e = 0;
    MCK(cudaMemcpyAsync(&e, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return e ? LP_ERR_TIMEOUT : LP_OK;
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
    h->in_p = pad8(in_dim); h->hid_p = pad8(hidden); h->out_p = pad8(out_dim); h->b_p = pad8(max_batch);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t sz[6] = {(size_t)in_dim * hidden, (size_t)hidden, (size_t)hidden * hidden, (size_t)hidden,
                          (size_t)hidden * out_dim, (size_t)out_dim};
    size_t o = 0;
    for (int i = 0; i < 6; ++i) { h->off[i] = o; o += sz[i]; }
    h->np = o;
    const size_t B = max_batch, I = in_dim, H = hidden, O = out_dim;
    int rc = LP_OK;
    if ((rc = malloc_t(h, &h->p, o)) || (rc = malloc_t(h, &h->g, o)) || (rc = malloc_t(h, &h->m1, o)) ||
        (rc = malloc_t(h, &h->m2, o)) || (rc = malloc_t(h, &h->w1t, H * h->in_p)) ||
        (rc = malloc_t(h, &h->w2t, H * h->hid_p)) || (rc = malloc_t(h, &h->w3t, O * h->hid_p)) ||
        (rc = malloc_t(h, &h->w2n, H * h->hid_p)) || (rc = malloc_t(h, &h->w3n, H * h->out_p)) ||
        (rc = malloc_t(h, &h->x16, B * h->in_p)) || (rc = malloc_t(h, &h->xT, I * h->b_p)) ||
        (rc = malloc_t(h, &h->z1, B * H)) || (rc = malloc_t(h, &h->z2, B * H)) || (rc = malloc_t(h, &h->z3, B * O)) ||
        (rc = malloc_t(h, &h->a1, B * h->hid_p)) || (rc = malloc_t(h, &h->a2, B * h->hid_p)) ||
        (rc = malloc_t(h, &h->a1T, H * h->b_p)) || (rc = malloc_t(h, &h->a2T, H * h->b_p)) ||
        (rc = malloc_t(h, &h->dz3, B * h->out_p)) || (rc = malloc_t(h, &h->dz2, B * h->hid_p)) ||
        (rc = malloc_t(h, &h->dz1, B * h->hid_p)) || (rc = malloc_t(h, &h->dz3T, O * h->b_p)) ||
        (rc = malloc_t(h, &h->dz2T, H * h->b_p)) || (rc = malloc_t(h, &h->dz1T, H * h->b_p)) ||
        (rc = malloc_t(h, &h->da2, B * H)) || (rc = malloc_t(h, &h->da1, B * H)) ||
        (rc = malloc_t(h, &h->loss, 1)) || (rc = malloc_t(h, &h->err, 1))) {
        lp_mlp_destroy(h);
        return rc;
    }
    if (cudaMemsetAsync(h->p, 0, o * sizeof(float), h->stream) || cudaMemsetAsync(h->m1, 0, o * sizeof(float), h->stream) ||
        cudaMemsetAsync(h->m2, 0, o * sizeof(float), h->stream) || cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream) ||
        refresh_weights(h) != LP_OK) {
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
    int rc = refresh_weights(h);
    if (rc != LP_OK) return rc;
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
    if ((rc = forward(h, batch)) != LP_OK) return rc;
    MCK(cudaMemcpyAsync(logits, h->z3, (size_t)batch * h->out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    MCK(cudaGetLastError());
    return LP_OK;
}

int lp_mlp_gradients(lp_mlp* h, const float* X, const float* T, int32_t batch, float* grads, float* loss) {
    if (!h || !T) return LP_ERR_INVALID_ARG;
    int rc = load_x(h, X, batch);
    if (rc != LP_OK) return rc;
    if ((rc = forward(h, batch)) != LP_OK) return rc;
    if ((rc = backward(h, batch, T)) != LP_OK) return rc;
    if (grads) MCK(cudaMemcpyAsync(grads, h->g, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (loss) MCK(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return check_err(h);
}

int lp_mlp_train_step(lp_mlp* h, const float* X, const float* T, int32_t batch, float lr, float* loss) {
    if (!h || !T || !(lr > 0.f)) return LP_ERR_INVALID_ARG;
    int rc = load_x(h, X, batch);
    if (rc != LP_OK) return rc;
    if ((rc = forward(h, batch)) != LP_OK) return rc;
    if ((rc = backward(h, batch, T)) != LP_OK) return rc;
    h->steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)h->steps), c2 = 1.f - powf(b2, (float)h->steps);
    k_adam<<<blocks_for(h->np), 256, 0, h->stream>>>(h->p, h->g, h->m1, h->m2, h->np, lr, b1, b2, 1e-8f, c1, c2);
    MCK(cudaGetLastError());
    if ((rc = refresh_weights(h)) != LP_OK) return rc;
    if (loss) {
        MCK(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        return check_err(h);
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
