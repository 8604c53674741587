// tc_gemm.cu -- D = A B^T on the 5th-generation tensor cores (tcgen05).
//
// A is M x K and B is N x K, both row-major (K contiguous, "K-major") with
// 16-bit elements (FP16 or BF16); D is M x N, FP32, row-major.  One CTA
// computes a 128 x BN tile of D:
//   warp 0 (one lane)  TMA producer: 128 x 64 tiles of A and BN x 64 tiles of B
//                      into a ring of shared-memory stages (128-byte swizzle),
//                      each stage completing on its "full" mbarrier;
//   warp 1 (one lane)  MMA issuer: four tcgen05.mma (K = 16 each) per stage into
//                      one FP32 accumulator in TMEM; tcgen05.commit frees the
//                      stage ("empty" mbarrier) once its MMAs have read it, and
//                      signals the epilogue after the last stage;
//   warps 2-5          epilogue: tcgen05.ld of the accumulator (warp w reads
//                      TMEM lanes 32 (w % 4) .. + 31, i.e. rows of the tile)
//                      and the stores to D.
// Tiles past the edge of A or B are zero-filled by the TMA unit, so ragged M,
// N and K need no special code; stores are masked.  Every mbarrier wait is
// bounded: on timeout the kernel records kErrTimeout in *err and leaves.
#include "tc_common.cuh"
#include "lpgb_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

namespace lpgb {

namespace {

constexpr int kTM = 128;      // tile rows (MMA M)
constexpr int kTK = 64;       // elements of K per stage (one 128-byte swizzle row)
constexpr int kStages = 4;
constexpr int kGemmThreads = 192;

template <int BN>
struct GemmSmem {
    static constexpr int kA = kTM * kTK * 2;
    static constexpr int kB = BN * kTK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kBars = 256;
    static constexpr size_t kBytes = 1024 + (size_t)kStages * kStage + kBars;
};

template <int BN, bool kBF16>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb, float* __restrict__ D,
              int ldd, int M, int N, int K, int32_t* err) {
    using L = GemmSmem<BN>;
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
            const int row = m0 + lg * 32 + lane;
            float* drow = D + (size_t)row * ldd;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0, v);
                if (row < M) {
                    const int cb = n0 + c0;
                    if (cb + 32 <= N && (ldd & 3) == 0) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            *reinterpret_cast<float4*>(drow + cb + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (cb + i < N) drow[cb + i] = v[i];
                    }
                }
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

template <int BN, bool kBF16>
cudaError_t launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, float* D, int ldd, int M, int N, int K,
                        int32_t* err, cudaStream_t st) {
    using L = GemmSmem<BN>;
    static std::once_flag once;
    static cudaError_t attr_rc = cudaSuccess;
    std::call_once(once, [] {
        attr_rc = cudaFuncSetAttribute(k_tc_gemm<BN, kBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::kBytes);
    });
    if (attr_rc != cudaSuccess) return attr_rc;
    const dim3 grid((N + BN - 1) / BN, (M + kTM - 1) / kTM);
    k_tc_gemm<BN, kBF16><<<grid, kGemmThreads, L::kBytes, st>>>(ma, mb, D, ldd, M, N, K, err);
    return cudaGetLastError();
}

}  // namespace

bool tc_make_map_16bit(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows < 1 || cols < 1 || ld < cols || (ld % 8) != 0 || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
              const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// D (M x N, FP32, row stride ldd) = A (M x K, row stride lda) * B (N x K, row
// stride ldb)^T; 16-bit operands, lda and ldb multiples of 8, bases 16-byte
// aligned.  Returns cudaErrorInvalidValue for shapes or pointers the tensor
// maps cannot describe.
cudaError_t tc_gemm(const void* A, int lda, const void* B, int ldb, float* D, int ldd, int M, int N, int K, bool bf16,
                    int32_t* err, cudaStream_t st) {
    if (M < 1 || N < 1 || K < 1 || ldd < N) return cudaErrorInvalidValue;
    constexpr int BN = 128;
    CUtensorMap ma, mb;
    if (!tc_make_map_16bit(&ma, A, M, K, lda, kTM, bf16) || !tc_make_map_16bit(&mb, B, N, K, ldb, BN, bf16))
        return cudaErrorInvalidValue;
    return bf16 ? launch_gemm<BN, true>(ma, mb, D, ldd, M, N, K, err, st)
                : launch_gemm<BN, false>(ma, mb, D, ldd, M, N, K, err, st);
}

}  // namespace lpgb

// Test and library entry point (declared in include/lpgb.h).
namespace {
__device__ int32_t g_tc_gemm_err;
}

extern "C" int lp_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B, int32_t ldb,
                          float* D, int32_t ldd, int32_t bf16, void* cuda_stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !D || lda < K || ldb < K || ldd < N || (lda % 8) || (ldb % 8))
        return -1;  // LP_ERR_INVALID_ARG
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int32_t* err = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_tc_gemm_err) != cudaSuccess) return -2;
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), st) != cudaSuccess) return -2;
    const cudaError_t e = lpgb::tc_gemm(A, lda, B, ldb, D, ldd, M, N, K, bf16 != 0, err, st);
    if (e == cudaErrorInvalidValue) return -1;
    if (e != cudaSuccess) return -2;  // LP_ERR_CUDA
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -2;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -2;
    return h ? -5 : 0;  // LP_ERR_TIMEOUT : LP_OK
}
