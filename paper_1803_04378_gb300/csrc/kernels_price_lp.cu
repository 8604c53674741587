// kernels_price_lp.cu -- mixed-precision PRICE (price_mode 1).
//
// Step 3 PRICE streams all of A every iteration, and on GB300 the FP64 pipe
// (about 2 FMA/clock/SM) caps an FP64 GEMV near 70% of HBM bandwidth.  This
// mode screens the columns with a BF16 copy of A (2 bytes/element, 4x fewer
// bytes) and FP32 FMAs on the CUDA cores -- a matrix-vector product has no
// reuse for tensor cores to exploit, so plain FMAs at HBM speed are the right
// unit -- then re-prices the top k candidates exactly in FP64 and enters the
// best of them.  Whenever no exactly re-priced candidate improves (or the
// Bland safety net is on) the full FP64 PRICE runs, so optimality is always
// certified in FP64 and the final objective equals the FP64 method's.  The
// entering choice can differ from Dantzig's FP64 argmax when the argmax is
// not among a block's screened best.
//
//   k_price_lp   BF16 screen: approximate d~_j over nonbasic, non-tabu
//                structural columns; each block re-prices its best `topk`
//                (1 or 2) columns exactly in FP64 and offers the best exact
//                candidate, slacks (d = -y_i, exact) included.  The last block
//                enters the best exact candidate, or asks for the full PRICE.
//                The candidates re-priced are therefore the union of every
//                block's screened best (2 x grid columns), a superset of the
//                global top-k except where one block holds more than two of
//                them.
#include "lpgb_internal.cuh"

#include <cfloat>

namespace lpgb {

namespace {

constexpr int kLpThreads = 512;

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (d desc, j asc); j < 0 sorts last
__device__ __forceinline__ bool cand_before(float da, int ja, float db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

__device__ __forceinline__ bool dbl_before(double da, int ja, double db, int jb) {
    if (ja < 0) return false;
    if (jb < 0) return true;
    return da > db || (da == db && ja < jb);
}

__device__ __forceinline__ void top2_offer(float d, int j, float& d0, int& j0, float& d1, int& j1) {
    if (cand_before(d, j, d0, j0)) {
        d1 = d0; j1 = j0; d0 = d; j0 = j;
    } else if (cand_before(d, j, d1, j1)) {
        d1 = d; j1 = j;
    }
}

__global__ void k_to_bf16(const double* __restrict__ src, uint16_t* __restrict__ dst, size_t count) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn((float)src[e]);
        dst[e] = *reinterpret_cast<const uint16_t*>(&h);
    }
}

__global__ void __launch_bounds__(kLpThreads, 2) k_price_lp(DevState s) {
    pdl_enter();
    Ctrl* C = s.ctrl;
    if (C->status != kRunning || C->bland) return;
    const Params& P = s.p;
    extern __shared__ double y64[];                 // ld doubles (exact re-price)
    float* ysf = reinterpret_cast<float*>(y64 + P.ld);  // ld floats (screen)
    for (int k = threadIdx.x; k < P.ld; k += blockDim.x) {
        y64[k] = s.y[k];
        ysf[k] = s.y32[k];
    }
    __syncthreads();
    const int it = C->it;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int vecs = P.ld >> 3;  // 8 BF16 values per 16-byte load
    const float4* y4 = reinterpret_cast<const float4*>(ysf);
    float d0 = -FLT_MAX, d1 = -FLT_MAX;
    int j0 = -1, j1 = -1;
    const int G = gridDim.x;
    const int owned = (P.n - (int)blockIdx.x + G - 1) / G;
    for (int l = warp; l < owned; l += nw) {
        const int j = blockIdx.x + G * l;
        if (s.pos[j] >= 0 || s.tabu_until[j] > it) continue;
        const uint4* col = reinterpret_cast<const uint4*>(s.A_lp + (size_t)j * P.ld);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
        for (int k = lane; k < vecs; k += 32) {
            const uint4 u = __ldcs(col + k);
            const float4 ya = y4[2 * k], yb = y4[2 * k + 1];
            a0 = fmaf(bf16_lo(u.x), ya.x, a0);
            a1 = fmaf(bf16_hi(u.x), ya.y, a1);
            a2 = fmaf(bf16_lo(u.y), ya.z, a2);
            a3 = fmaf(bf16_hi(u.y), ya.w, a3);
            a0 = fmaf(bf16_lo(u.z), yb.x, a0);
            a1 = fmaf(bf16_hi(u.z), yb.y, a1);
            a2 = fmaf(bf16_lo(u.w), yb.z, a2);
            a3 = fmaf(bf16_hi(u.w), yb.w, a3);
        }
        const float d = (float)s.c[j] - warp_sum_f((a0 + a1) + (a2 + a3));
        top2_offer(d, j, d0, j0, d1, j1);
    }
    // exact slack candidates
    double ds = -DBL_MAX;
    int js = -1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.m; i += gridDim.x * blockDim.x) {
        const int j = P.n + i;
        if (s.pos[j] >= 0 || s.tabu_until[j] > it) continue;
        const double d = -y64[i];
        if (dbl_before(d, j, ds, js)) { ds = d; js = j; }
    }
    // block top-2 of the screen and best slack
    __shared__ float sd0[32], sd1[32];
    __shared__ int sj0[32], sj1[32], sjs[32], cand2[2];
    __shared__ double sds[32], exact[2];
    for (int o = 16; o > 0; o >>= 1) {
        const double ods = __shfl_xor_sync(0xffffffffu, ds, o);
        const int ojs = __shfl_xor_sync(0xffffffffu, js, o);
        if (dbl_before(ods, ojs, ds, js)) { ds = ods; js = ojs; }
    }
    if (lane == 0) { sd0[warp] = d0; sj0[warp] = j0; sd1[warp] = d1; sj1[warp] = j1; sds[warp] = ds; sjs[warp] = js; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float b0 = -FLT_MAX, b1 = -FLT_MAX;
        int c0 = -1, c1 = -1;
        double bs = -DBL_MAX;
        int cs = -1;
        for (int w = 0; w < nw; ++w) {
            top2_offer(sd0[w], sj0[w], b0, c0, b1, c1);
            top2_offer(sd1[w], sj1[w], b0, c0, b1, c1);
            if (dbl_before(sds[w], sjs[w], bs, cs)) { bs = sds[w]; cs = sjs[w]; }
        }
        cand2[0] = c0;
        cand2[1] = P.topk >= 2 ? c1 : -1;
        sds[0] = bs;
        sjs[0] = cs;
    }
    __syncthreads();
    // exact FP64 re-price of the block's two candidates: half of the warps
    // per column, each warp one segment; segments summed in a fixed order
    __shared__ double epart[32];
    {
        const int wpc = nw >> 1;               // warps per candidate
        const int which = warp / wpc, seg = warp % wpc;
        const int j = which < 2 ? cand2[which] : -1;
        double a0 = 0.0, a1 = 0.0;
        if (j >= 0) {
            const int h2 = P.ld >> 1, segl = (h2 + wpc - 1) / wpc;
            const int k0 = seg * segl, k1 = min(h2, k0 + segl);
            const double2* col = reinterpret_cast<const double2*>(s.A_cm + (size_t)j * P.ld);
            const double2* yy = reinterpret_cast<const double2*>(y64);
#pragma unroll 4
            for (int k = k0 + lane; k < k1; k += 32) {
                const double2 u = __ldg(col + k), w = yy[k];
                a0 = fma(u.x, w.x, a0);
                a1 = fma(u.y, w.y, a1);
            }
        }
        const double t = warp_sum(a0 + a1);
        if (lane == 0) epart[warp] = t;
        __syncthreads();
        if (threadIdx.x < 2) {
            const int jj = cand2[threadIdx.x];
            double e = -DBL_MAX;
            if (jj >= 0) {
                double sum = 0.0;
                for (int w = 0; w < wpc; ++w) sum += epart[threadIdx.x * wpc + w];
                e = s.c[jj] - sum;
            }
            exact[threadIdx.x] = e;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bd = sds[0];
        int bj = sjs[0];
        for (int t = 0; t < 2; ++t)
            if (cand2[t] >= 0 && dbl_before(exact[t], cand2[t], bd, bj)) { bd = exact[t]; bj = cand2[t]; }
        LpCand pc;
        pc.d0 = 0.f; pc.j0 = 0; pc.d1 = 0.f; pc.j1 = 0;
        pc.ds = bd; pc.js = bj; pc.pad_ = (cand2[0] >= 0) + (cand2[1] >= 0);
        s.lp_part[blockIdx.x] = pc;
    }
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&C->ticket_lp, 1) == G - 1;
    }
    __syncthreads();
    if (!last) return;
    // last block: best exact candidate over the blocks
    double bd = -DBL_MAX;
    int bj = -1, nrep = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) {
        const double od = __ldcg(&s.lp_part[b].ds);
        const int oj = __ldcg(&s.lp_part[b].js);
        nrep += __ldcg(&s.lp_part[b].pad_);
        if (dbl_before(od, oj, bd, bj)) { bd = od; bj = oj; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        nrep += __shfl_xor_sync(0xffffffffu, nrep, o);
        if (dbl_before(od, oj, bd, bj)) { bd = od; bj = oj; }
    }
    __syncthreads();
    if (lane == 0) { sds[warp] = bd; sjs[warp] = bj; sj0[warp] = nrep; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double fd = -DBL_MAX;
        int fj = -1, tot = 0;
        for (int w = 0; w < nw; ++w) {
            tot += sj0[w];
            if (dbl_before(sds[w], sjs[w], fd, fj)) { fd = sds[w]; fj = sjs[w]; }
        }
        C->ticket_lp = 0;
        C->bytes_price += 2.0 * P.m * (double)(P.n - C->nsb) + 8.0 * P.m * (double)tot;
        C->n_lp++;
        if (fj >= 0 && fd > P.tol_d) {
            C->q = fj;
            C->dq = fd;
            C->need_full = 0;
        } else {
            C->need_full = 1;
        }
        __threadfence();
    }
}

}  // namespace

void launch_to_bf16(const double* src, uint16_t* dst, size_t count, cudaStream_t st) {
    k_to_bf16<<<2048, 256, 0, st>>>(src, dst, count);
}

void launch_price_lp(const DevState& s, const Geometry& g, cudaStream_t st, bool pdl) {
    launch_k(k_price_lp, dim3(g.price_lp_blocks), dim3(kLpThreads), (size_t)s.p.ld * (sizeof(float) + sizeof(double)),
             st, pdl, s);
}

int occupancy_price_lp(int ld) {
    const size_t smem = (size_t)ld * (sizeof(float) + sizeof(double));
    cudaFuncSetAttribute(k_price_lp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_price_lp, kLpThreads, smem);
    return nb;
}

}  // namespace lpgb
