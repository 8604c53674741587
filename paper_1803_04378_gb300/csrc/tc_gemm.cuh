// tc_gemm.cuh -- the tensor-core GEMM mainloop (tcgen05) shared by the plain
// GEMM (tc_gemm.cu) and the sliced FP64 products (ozaki.cu).
//
// A is M x K and B is N x K, both row-major (K contiguous, "K-major") with
// 16-bit elements (FP16 or BF16).  One CTA computes a 128 x BN tile of A B^T:
//   warp 0 (one lane)  TMA producer: 128 x 64 tiles of A and BN x 64 tiles of B
//                      into a ring of shared-memory stages (128-byte swizzle),
//                      each stage completing on its "full" mbarrier;
//   warp 1 (one lane)  MMA issuer: four tcgen05.mma (K = 16 each) per stage into
//                      one FP32 accumulator in TMEM; tcgen05.commit frees the
//                      stage ("empty" mbarrier) once its MMAs have read it, and
//                      signals the epilogue after the last stage;
//   warps 2-5          epilogue: tcgen05.ld of the accumulator, 32 columns at a
//                      time (warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e.
//                      rows of the tile), handed to the epilogue functor.
// Tiles past the edge of A or B are zero-filled by the TMA unit, so ragged M,
// N and K need no special code.  Every mbarrier wait is bounded: on timeout
// the kernel records kErrTimeout in *err and leaves.
#pragma once
#include "tc_common.cuh"
#include "lpgb_internal.cuh"

namespace lpgb {

namespace tcg {

constexpr int kTM = 128;      // tile rows (MMA M)
constexpr int kTK = 64;       // elements of K per stage (one 128-byte swizzle row)
constexpr int kGemmThreads = 192;

template <int BN, int kStages>
struct GemmSmem {
    static constexpr int kA = kTM * kTK * 2;
    static constexpr int kB = BN * kTK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kBars = 256;
    static constexpr size_t kBytes = 1024 + (size_t)kStages * kStage + kBars;
};

// Epi: a functor called by every lane of an epilogue warp (warp-collective)
// with the tile row of the lane (0..127, the TMEM lane), the tile's first row
// and column in the output, the first of the 32 columns, and their values.
// kStages shared-memory stages; kMinBlocks CTAs share an SM (their TMEM
// allocations, BN columns each, must fit the SM's 512).
template <int BN, int kStages, int kMinBlocks, bool kBF16, class Epi>
__global__ void __launch_bounds__(kGemmThreads, kMinBlocks)
    k_tc_gemm(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, Epi epi, int K,
              int32_t* err) {
    static_assert(kMinBlocks * BN <= 512, "TMEM columns of the co-resident CTAs");
    using L = GemmSmem<BN, kStages>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * L::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;
    uint32_t* tholder = reinterpret_cast<uint32_t*>(tfull + 1);
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;
    const int nk = (K + kTK - 1) / kTK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(tfull, 1);
        tc::fence_barrier_init();
        fail = 0;
    }
    if (warp == 1) tc::tmem_alloc(tholder, BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tholder;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&ma);
            tc::tma_prefetch_desc(&mb);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages, use = kb / kStages;
                if (kb >= kStages && !tc::mbar_wait(&empty[s], (use - 1) & 1)) {
                    fail = 1;
                    break;
                }
                uint8_t* sa = smem + s * L::kStage;
                tc::mbar_arrive_expect_tx(&full[s], L::kStage);
                tc::tma_load_2d(sa, &ma, &full[s], kb * kTK, m0);
                tc::tma_load_2d(sa + L::kA, &mb, &full[s], kb * kTK, n0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_f16(kTM, BN, kBF16);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (!tc::mbar_wait(&full[s], (kb / kStages) & 1)) {
                    fail = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint8_t* sa = smem + s * L::kStage;
                const uint64_t ad = tc::sdesc_k128(tc::smem_u32(sa));
                const uint64_t bd = tc::sdesc_k128(tc::smem_u32(sa + L::kA));
#pragma unroll
                for (int kk = 0; kk < kTK / 16; ++kk)
                    tc::mma_f16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(tfull);
        }
    } else {
        if (!tc::mbar_wait(tfull, 0)) {
            fail = 1;
        } else {
            tc::tc_fence_after();
            const int lg = warp & 3;  // TMEM lane group of this warp
            const int trow = lg * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0, v);
                epi(trow, m0, n0, c0, v);
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, BN);
    }
    if (threadIdx.x == 0 && fail && err) atomicExch(err, kErrTimeout);
}

// Persistent form of k_tc_gemm for products of many tiles: each CTA takes the
// tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (the tile's column block
// varies fastest, so CTAs working at once share the A tile in L2).  The TMEM
// holds two accumulators: the MMA issuer fills accumulator i & 1 for the
// CTA's i-th tile while the epilogue warps drain the other, and the
// shared-memory ring runs on across tiles, so the epilogue of one tile, the
// loads of the next and the setup of the CTA overlap.  Barriers:
//   full[s] / empty[s]  the stage ring (TMA -> MMA -> TMA), as in k_tc_gemm;
//   tfull[a]            MMA -> epilogue: accumulator a holds a finished tile;
//   tempty[a]           epilogue -> MMA: accumulator a was read (one arrival
//                       per epilogue warp).
// kEpiWarps epilogue warps (2 .. kEpiWarps + 1): the kEpiWarps / 4 warps of a
// TMEM lane quarter take alternate 32-column chunks, so that several warps per
// scheduler hide the latency of the epilogue's dependent integer chains and
// shuffles; kCtas CTAs share an SM (their TMEM, 2 BN columns each, must fit
// the SM's 512).
// Every wait is bounded.  On a timeout the kernel records kErrTimeout, the
// producer waits (bounded) for the loads it issued, the MMA issuer for its
// MMAs, and the TMEM is freed.
template <int kEpiWarps>
constexpr int gemm_p_threads() { return 64 + 32 * kEpiWarps; }

template <int BN, int kStages, int kEpiWarps, int kCtas, bool kBF16, class Epi>
__global__ void __launch_bounds__(gemm_p_threads<kEpiWarps>(), kCtas)
    k_tc_gemm_p(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, Epi epi, int M,
                int N, int K, int32_t* err) {
    static_assert(kCtas * 2 * BN <= 512, "two accumulators for each co-resident CTA");
    static_assert(kEpiWarps % 4 == 0 && kEpiWarps >= 4, "whole TMEM lane quarters");
    constexpr int kEpiPerQuarter = kEpiWarps / 4;
    pdl_enter();  // the operands' slices come from the previous launch
    using L = GemmSmem<BN, kStages>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * L::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;  // 2
    uint64_t* tempty = tfull + 2;       // 2
    uint64_t* mdone = tempty + 2;       // 1: every MMA of the CTA has completed
    uint32_t* tholder = reinterpret_cast<uint32_t*>(mdone + 1);
    __shared__ volatile int fail;  // read by the other roles' loops: an early way out after a timeout
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K + kTK - 1) / kTK;
    const int ntn = (N + BN - 1) / BN, ntiles = ntn * ((M + kTM - 1) / kTM);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], kEpiWarps);
        }
        tc::mbar_init(mdone, 1);
        tc::fence_barrier_init();
        fail = 0;
    }
    if (warp == 1) tc::tmem_alloc(tholder, 2 * BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tholder;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&ma);
            tc::tma_prefetch_desc(&mb);
            int g = 0;  // stage-ring position, across the CTA's tiles
            for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x) {
                const int m0 = (t / ntn) * kTM, n0 = (t % ntn) * BN;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % kStages, use = g / kStages;
                    if (g >= kStages && !tc::mbar_wait(&empty[s], (use - 1) & 1)) {
                        fail = 1;
                        break;
                    }
                    uint8_t* sa = smem + s * L::kStage;
                    tc::mbar_arrive_expect_tx(&full[s], L::kStage);
                    tc::tma_load_2d(sa, &ma, &full[s], kb * kTK, m0);
                    tc::tma_load_2d(sa + L::kA, &mb, &full[s], kb * kTK, n0);
                }
            }
            if (fail) {
                // the loads in flight land before the CTA leaves
                for (int h = g - kStages; h < g; ++h)
                    if (h >= 0) (void)tc::mbar_wait(&full[h % kStages], (h / kStages) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_f16(kTM, BN, kBF16);
            int g = 0, i = 0;
            for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x, ++i) {
                const int a = i & 1;
                if (i >= 2 && !tc::mbar_wait(&tempty[a], ((i >> 1) - 1) & 1)) {
                    fail = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(a * BN);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % kStages;
                    if (!tc::mbar_wait(&full[s], (g / kStages) & 1)) {
                        fail = 1;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint8_t* sa = smem + s * L::kStage;
                    const uint64_t ad = tc::sdesc_k128(tc::smem_u32(sa));
                    const uint64_t bd = tc::sdesc_k128(tc::smem_u32(sa + L::kA));
#pragma unroll
                    for (int kk = 0; kk < kTK / 16; ++kk)
                        tc::mma_f16(acc, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
                    tc::mma_commit(&empty[s]);
                }
                if (fail) break;
                tc::mma_commit(&tfull[a]);
            }
            // every MMA issued by this CTA has completed before the TMEM is freed
            tc::mma_commit(mdone);
            if (!tc::mbar_wait(mdone, 0)) fail = 1;
        }
    } else {
        const int lg = warp & 3;  // TMEM lane group of this warp
        const int trow = lg * 32 + lane;
        const int cfirst = 32 * ((warp - 2) >> 2);  // the quarter's warps take chunks cfirst, + 32 kEpiPerQuarter, ...
        int i = 0;
        for (int t = blockIdx.x; t < ntiles && !fail; t += gridDim.x, ++i) {
            const int a = i & 1;
            if (!tc::mbar_wait(&tfull[a], (i >> 1) & 1)) {
                fail = 1;
                break;
            }
            tc::tc_fence_after();
            const int m0 = (t / ntn) * kTM, n0 = (t % ntn) * BN;
#pragma unroll 1
            for (int c0 = cfirst; c0 < BN; c0 += 32 * kEpiPerQuarter) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(a * BN + c0), v);
                epi(trow, m0, n0, c0, v);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[a]);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 2 * BN);
    }
    if (threadIdx.x == 0 && fail && err) atomicExch(err, kErrTimeout);
}

// Grid of the persistent form: kCtas CTAs per SM, at most one per tile; a
// programmatic dependent launch (the kernel waits before it reads its operands).
template <int BN, int kStages, int kEpiWarps, int kCtas, bool kBF16, class Epi>
cudaError_t launch_tc_gemm_p(const CUtensorMap& ma, const CUtensorMap& mb, const Epi& epi, int M, int N, int K,
                             int32_t* err, cudaStream_t st) {
    using L = GemmSmem<BN, kStages>;
    static_assert(L::kBars >= (2 * kStages + 5) * 8 + 4, "barrier area");
    static_assert(kCtas * (L::kBytes + 1024) <= 232448, "shared memory of the co-resident CTAs");
    static cudaError_t attr_rc = cudaFuncSetAttribute(k_tc_gemm_p<BN, kStages, kEpiWarps, kCtas, kBF16, Epi>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
    if (attr_rc != cudaSuccess) return attr_rc;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int tiles = ((N + BN - 1) / BN) * ((M + kTM - 1) / kTM);
    const int grid = tiles < kCtas * sms ? tiles : kCtas * sms;
    return launch_k(k_tc_gemm_p<BN, kStages, kEpiWarps, kCtas, kBF16, Epi>, dim3(grid),
                    dim3(gemm_p_threads<kEpiWarps>()), L::kBytes, st, true, ma, mb, epi, M, N, K, err);
}

// Tensor maps of the two operands and the launch (grid = N/BN x M/128 tiles).
template <int BN, int kStages, int kMinBlocks, bool kBF16, class Epi>
cudaError_t launch_tc_gemm(const CUtensorMap& ma, const CUtensorMap& mb, const Epi& epi, int M, int N, int K,
                           int32_t* err, cudaStream_t st) {
    using L = GemmSmem<BN, kStages>;
    static cudaError_t attr_rc = cudaFuncSetAttribute(k_tc_gemm<BN, kStages, kMinBlocks, kBF16, Epi>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kBytes);
    if (attr_rc != cudaSuccess) return attr_rc;
    const dim3 grid((N + BN - 1) / BN, (M + kTM - 1) / kTM);
    k_tc_gemm<BN, kStages, kMinBlocks, kBF16, Epi><<<grid, kGemmThreads, L::kBytes, st>>>(ma, mb, epi, K, err);
    return cudaGetLastError();
}

}  // namespace tcg
}  // namespace lpgb
