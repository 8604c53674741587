// price_static.cu -- reduced costs and Dantzig's entering choice without any
// allocation (lp_price_static in include/lpgb.h).
//
// Some callers cannot allocate device memory: code running inside a CUDA
// graph they capture themselves, allocator-free embedded runtimes, or hosts
// whose memory budget is fixed up front.  This entry point takes only the
// caller's buffers.  The one piece of scratch the kernel needs -- a partial
// best candidate per block plus the last-block ticket -- lives in a
// file-scope __device__ array, so every GPU that loads the library holds it
// (about 17 KB) until the process exits.
//
// Host code must not hand the array's name to a kernel: in host code the name
// is only a host-side stand-in.  The device address is fetched once per
// device context with cudaGetSymbolAddress (with that device current) and
// passed in; a call that finds a different context on its device than the
// one the address was fetched in (after cudaDeviceReset, say) fetches it again.
#include "../../include/lpgb.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <mutex>

namespace {

constexpr int kThreads = 512;
constexpr int kMaxBlocks = 1024;   // partial slots in the static scratch
constexpr int kMaxDevices = 64;

struct Best {
    double d;
    int32_t j;
    int32_t pad;
};

struct Scratch {
    Best part[kMaxBlocks];
    int32_t ticket;  // must be zero when a launch starts
    int32_t pad[63];
};

static __device__ __align__(256) Scratch g_price_scratch;

struct DeviceSetup {
    bool ready = false;
    unsigned long long ctx_id = 0;  // the context the address below belongs to
    Scratch* scratch = nullptr;     // device address of g_price_scratch
    int sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

__device__ __forceinline__ bool better(double da, int ja, double db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide best (d, j); valid in thread 0.
__device__ void block_best(double& d, int& j) {
    __shared__ double sd[32];
    __shared__ int sj[32];
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, d, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(od, oj, d, j)) { d = od; j = oj; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sd[w] = d; sj[w] = j; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (better(sd[i], sj[i], d, j)) { d = sd[i]; j = sj[i]; }
    }
}

// d_j = c_j - y^T a_j for nonbasic j (d_{n+i} = -y_i for slacks); the block
// that finishes last writes the largest d_j > tol_d (exact ties to the
// smallest j) to q_out / dq_out, or q_out = -1 when none exceeds tol_d.
__global__ void __launch_bounds__(kThreads) k_price_static(int m, int n, const double* __restrict__ A, int lda,
                                                           const double* __restrict__ c,
                                                           const double* __restrict__ y,
                                                           const int32_t* __restrict__ pos, double tol_d,
                                                           int32_t* q_out, double* dq_out, Scratch* sc) {
    extern __shared__ __align__(16) double ysh[];  // read as double2 below
    const int me = (m + 1) & ~1;
    for (int k = threadIdx.x; k < me; k += blockDim.x) ysh[k] = k < m ? y[k] : 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = m >> 1;
    const double2* y2 = reinterpret_cast<const double2*>(ysh);
    double best_d = -DBL_MAX;
    int best_j = -1;
    const int G = gridDim.x;
    const int owned = (n - (int)blockIdx.x + G - 1) / G;
    for (int l = warp; l < owned; l += nw) {
        const int j = blockIdx.x + G * l;
        if (pos[j] >= 0) continue;
        const double* colp = A + (size_t)j * lda;
        const double2* col = reinterpret_cast<const double2*>(colp);
        double a0 = 0.0, a1 = 0.0;
#pragma unroll 4
        for (int k = lane; k < half; k += 32) {
            const double2 u = __ldg(col + k), w = y2[k];
            a0 = fma(u.x, w.x, a0);
            a1 = fma(u.y, w.y, a1);
        }
        if ((m & 1) && lane == 0) a0 = fma(__ldg(colp + m - 1), ysh[m - 1], a0);
        const double d = c[j] - warp_sum(a0 + a1);
        if (better(d, j, best_d, best_j)) { best_d = d; best_j = j; }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int j = n + i;
        if (pos[j] >= 0) continue;
        const double d = -ysh[i];
        if (better(d, j, best_d, best_j)) { best_d = d; best_j = j; }
    }
    block_best(best_d, best_j);
    __shared__ int last;
    if (threadIdx.x == 0) {
        sc->part[blockIdx.x].d = best_d;
        sc->part[blockIdx.x].j = best_j;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1) == G - 1;
    }
    __syncthreads();
    if (!last) return;
    double d = -DBL_MAX;
    int j = -1;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        const double od = __ldcg(&sc->part[b].d);
        const int oj = __ldcg(&sc->part[b].j);
        if (better(od, oj, d, j)) { d = od; j = oj; }
    }
    block_best(d, j);
    if (threadIdx.x == 0) {
        *q_out = (j >= 0 && d > tol_d) ? j : -1;
        *dq_out = j >= 0 ? d : 0.0;
        sc->ticket = 0;
    }
}

// Identity of the calling thread's current context (driver entry points
// looked up through the runtime, so the library needs no libcuda at link
// time).  Host-only queries: they enqueue nothing and allocate nothing.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

int current_ctx_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return LP_ERR_CUDA;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return LP_ERR_CUDA;
    if (get_id(ctx, id) != CUDA_SUCCESS) return LP_ERR_CUDA;
    return LP_OK;
}

// Once per device context, with that device current: the scratch's device
// address, the shared-memory opt-in and the SM count.
int setup_device(int dev, DeviceSetup** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    unsigned long long ctx_id = 0;
    if (current_ctx_id(&ctx_id) != LP_OK) return LP_ERR_CUDA;
    if (s.ready && s.ctx_id != ctx_id) s.ready = false;  // a new context: the old address is void
    if (!s.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_price_scratch) != cudaSuccess || ptr == nullptr) return LP_ERR_CUDA;
        if (cudaFuncSetAttribute(k_price_static, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(LP_PRICE_STATIC_MAX_M * sizeof(double))) != cudaSuccess)
            return LP_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return LP_ERR_CUDA;
        s.scratch = static_cast<Scratch*>(ptr);
        s.sms = sms;
        s.ctx_id = ctx_id;
        s.ready = true;
    }
    *out = &s;
    return LP_OK;
}

}  // namespace

extern "C" int lp_price_static(int32_t m, int32_t n, const double* A_colmajor, int32_t lda, const double* c,
                               const double* y, const int32_t* pos, double tol_d, int32_t* q_out,
                               double* dq_out, void* cuda_stream) {
    if (m < 1 || n < 1 || m > LP_PRICE_STATIC_MAX_M || (int64_t)n + m > ((int64_t)1 << 30)) return LP_ERR_INVALID_ARG;
    if (lda < m || (lda & 1)) return LP_ERR_INVALID_ARG;
    if (!A_colmajor || !c || !y || !pos || !q_out || !dq_out) return LP_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(A_colmajor) & 15) != 0 || !(tol_d >= 0)) return LP_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LP_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LP_ERR_INVALID_ARG;
    DeviceSetup* s = nullptr;
    int rc = setup_device(dev, &s);
    if (rc != LP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int blocks = 2 * s->sms;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    if (blocks > n) blocks = n;
    if (cudaMemsetAsync(&s->scratch->ticket, 0, sizeof(int32_t), st) != cudaSuccess) return LP_ERR_CUDA;
    const size_t smem = (size_t)((m + 1) & ~1) * sizeof(double);
    k_price_static<<<blocks, kThreads, smem, st>>>(m, n, A_colmajor, lda, c, y, pos, tol_d, q_out, dq_out,
                                                   s->scratch);
    if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
    return LP_OK;
}
