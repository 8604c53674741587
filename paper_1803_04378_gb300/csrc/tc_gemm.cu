// tc_gemm.cu -- D = A B^T on the 5th-generation tensor cores (tcgen05); the
// mainloop is in tc_gemm.cuh, this file adds the FP32 store epilogue, the
// tensor maps and the C entry point.
#include "tc_gemm.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

namespace lpgb {

namespace {

// D[row][col] = accumulator, masked to M x N.
struct StoreF32 {
    float* D;
    int ldd, M, N;
    __device__ void operator()(int trow, int m0, int n0, int c0, const float (&v)[32]) const {
        const int row = m0 + trow;
        if (row >= M) return;
        float* drow = D + (size_t)row * ldd;
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
};

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

}  // namespace

bool tc_make_map_16bit(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows < 1 || cols < 1 || ld < cols || (ld % 8) != 0 || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)tcg::kTK, (cuuint32_t)box_rows};
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
    if (!tc_make_map_16bit(&ma, A, M, K, lda, tcg::kTM, bf16) || !tc_make_map_16bit(&mb, B, N, K, ldb, BN, bf16))
        return cudaErrorInvalidValue;
    const StoreF32 epi{D, ldd, M, N};
    return bf16 ? tcg::launch_tc_gemm<BN, 4, 1, true>(ma, mb, epi, M, N, K, err, st)
                : tcg::launch_tc_gemm<BN, 4, 1, false>(ma, mb, epi, M, N, K, err, st);
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
