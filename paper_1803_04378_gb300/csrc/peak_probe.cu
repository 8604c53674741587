// peak_probe.cu -- standalone throughput probe of the GPU (not part of the
// solver library): FP64 FMA, FP64 mma.sync m8n8k4, FP32 FMA, HBM read and
// copy bandwidth, and a PRICE-shaped FP64 GEMV (warp per column, y in shared
// memory).  These figures set the FP64 roofline the benchmark reports.  Every
// access stays inside its buffer.
#include <cstdio>
#include <cuda_runtime.h>
#include <cstdint>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void dfma_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void ffma_kernel(float* out, int iters, float a, float b) {
    float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dmma_kernel(double* out, int iters) {
    double a = 1.0 + threadIdx.x * 1e-3, b = 0.5;
    double c0 = 0, c1 = 0, d0 = 0, d1 = 0, e0 = 0, e1 = 0, f0 = 0, f1 = 0;
    for (int i = 0; i < iters; ++i) {
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(e0), "+d"(e1) : "d"(a), "d"(b));
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(f0), "+d"(f1) : "d"(a), "d"(b));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + d0 + d1 + e0 + e1 + f0 + f1;
}

__global__ void read_kernel(const double2* __restrict__ in, size_t n2, double* out) {
    double s = 0;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        double2 v = __ldcs(in + i);
        s += v.x + v.y;
    }
    if (s == 12345.678) out[0] = s;
}

__global__ void copy_kernel(const double2* __restrict__ in, double2* __restrict__ o, size_t n2) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) __stcs(o + i, __ldcs(in + i));
}

// GEMV-like streaming: per element one DFMA against a smem vector (mimics PRICE)
__global__ void gemv_col_kernel(const double* __restrict__ A, int m, int ncol, const double* __restrict__ y, double* out) {
    extern __shared__ double ys[];
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[i] = y[i];
    __syncthreads();
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < ncol; j += nw) {
        const double2* col = reinterpret_cast<const double2*>(A + (size_t)j * m);
        double s0 = 0, s1 = 0;
        #pragma unroll 8
        for (int k = lane; k < m / 2; k += 32) {
            double2 a = __ldcs(col + k);
            double2 yy = reinterpret_cast<const double2*>(ys)[k];
            s0 = fma(a.x, yy.x, s0); s1 = fma(a.y, yy.y, s1);
        }
        double s = s0 + s1;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
        if (lane == 0) out[j] = s;
    }
}

int main() {
    int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
    int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    printf("device %s SMs %d smem/block optin %zu L2 %d clock(kHz) %d cc %d.%d\n", p.name, p.multiProcessorCount, p.sharedMemPerBlockOptin, p.l2CacheSize, clk, p.major, p.minor);
    int sms = p.multiProcessorCount;
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    double* dout; CK(cudaMalloc(&dout, sizeof(double) * sms * 16 * 1024));
    float* fout; CK(cudaMalloc(&fout, sizeof(float) * sms * 16 * 1024));
    // DFMA
    for (int bpsm : {4, 8, 16}) {
        int iters = 4096; int blocks = sms * bpsm, threads = 256;
        dfma_kernel<<<blocks, threads>>>(dout, iters, 0.999, 1e-3);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0); dfma_kernel<<<blocks, threads>>>(dout, iters, 0.999, 1e-3); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        double fl = 2.0 * 8 * iters * (double)blocks * threads;
        printf("DFMA blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, fl / ms / 1e9);
    }
    for (int bpsm : {8}) {
        int iters = 65536; int blocks = sms * bpsm, threads = 256;
        ffma_kernel<<<blocks, threads>>>(fout, iters, 0.999f, 1e-3f);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0); ffma_kernel<<<blocks, threads>>>(fout, iters, 0.999f, 1e-3f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        double fl = 2.0 * 8 * iters * (double)blocks * threads;
        printf("FFMA blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, fl / ms / 1e9);
    }
    for (int bpsm : {4, 8}) {
        int iters = 2048; int blocks = sms * bpsm, threads = 256;
        dmma_kernel<<<blocks, threads>>>(dout, iters);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0); dmma_kernel<<<blocks, threads>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
        float ms; cudaEventElapsedTime(&ms, e0, e1);
        double fl = 2.0 * 8 * 8 * 4 * 4.0 * iters * (double)blocks * (threads / 32);
        printf("DMMA blocks/SM %d: %.3f ms  %.3f TFLOP/s\n", bpsm, ms, fl / ms / 1e9);
    }
    // HBM
    size_t bytes = (size_t)2 << 30; size_t n2 = bytes / 16;
    double2 *a, *b; CK(cudaMalloc(&a, bytes)); CK(cudaMalloc(&b, bytes));
    CK(cudaMemset(a, 0, bytes)); CK(cudaMemset(b, 0, bytes));
    for (int bpsm : {4, 8, 16}) {
        int blocks = sms * bpsm;
        read_kernel<<<blocks, 256>>>(a, n2, dout); CK(cudaDeviceSynchronize());
        float best = 1e9;
        for (int r = 0; r < 5; ++r) { cudaEventRecord(e0); read_kernel<<<blocks, 256>>>(a, n2, dout); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms; }
        printf("read  blocks/SM %d: %.3f ms  %.1f GB/s\n", bpsm, best, bytes / best / 1e6);
        best = 1e9;
        for (int r = 0; r < 5; ++r) { cudaEventRecord(e0); copy_kernel<<<blocks, 256>>>(a, b, n2); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms; }
        printf("copy  blocks/SM %d: %.3f ms  %.1f GB/s\n", bpsm, best, 2 * bytes / best / 1e6);
    }
    // GEMV-like PRICE shape: m=4096, ncol=8192 (268 MB) -- repeated over 2 GB buffer windows
    {
        int m = 4096, ncol = 8192; size_t sz = (size_t)m * ncol * 8;
        double* y; CK(cudaMalloc(&y, m * 8)); CK(cudaMemset(y, 0, m * 8));
        double* o; CK(cudaMalloc(&o, ncol * 8));
        cudaFuncSetAttribute(gemv_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m * 8);
        for (int bpsm : {2, 4, 6}) {
            int blocks = sms * bpsm;
            float best = 1e9;
            for (int r = 0; r < 6; ++r) {
                const double* Ap = reinterpret_cast<const double*>(a) + (size_t)(r % 7) * (sz / 8);
                cudaEventRecord(e0); gemv_col_kernel<<<blocks, 512, m * 8>>>(Ap, m, ncol, y, o); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
                float ms; cudaEventElapsedTime(&ms, e0, e1); if (r > 0 && ms < best) best = ms;
            }
            printf("gemv_col m=4096 n=8192 blocks/SM %d (512 thr): %.3f ms  %.1f GB/s\n", bpsm, best, sz / best / 1e6);
        }
    }
    CK(cudaGetLastError());
    printf("done\n");
    return 0;
}
