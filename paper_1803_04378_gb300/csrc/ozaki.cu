// ozaki.cu -- FP64 matrix products on the BF16 tensor cores, from exact
// 7-bit slices of the operands (the error-free splitting of Ozaki, Ogita,
// Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applicability",
// Numer. Algorithms 59, 2012), used for the slack rows of the reinversion,
// C = -A[S, J] B11^-1 (kernels_reinv.cu).  On this chip FP64 FMAs run at
// 1/58 of the FP32 rate and FP64 tensor instructions at the FMA rate, while
// BF16 tensor instructions run three orders of magnitude faster.
//
// Splitting.  Row i of X (M x K) gets the exponent e_i with max_l |X_il| <
// 2^e_i; then X_il = 2^e_i sum_{p<8} d_p(X_il) 2^{-7(p+1)} + r_il with integer
// digits |d_p| <= 127 (sign-magnitude, taken from the bits of the double:
// no FP64 instruction) and |r_il| < 2^{e_i - 56}.  Column c of Y (K x N)
// likewise with exponents f_c.  A digit is exact in BF16.
//
// Products.  S_pq[i][c] = sum_l d_p(X_il) d_q(Y_lc) has |terms| < 2^14, so for
// K <= 1024 every partial sum is an integer below 2^24 and the tensor cores'
// FP32 accumulation is exact (checked bit for bit by the GPU tests of
// lp_tc_gemm).  One GEMM computes all 64 digit pairs: the A operand stacks
// the slices of X with row 8 i + p, the B operand those of Y with row 8 c + q.
//
// Combination (GEMM epilogue).  X Y = 2^{e_i + f_c} sum_{p,q} S_pq 2^{-7(p+q+2)},
// all 64 pairs, added as 64-bit integers in fixed point with 51 fraction bits
// relative to 2^{e_i + f_c}: the lane holding digit p of row i pairs adjacent
// q exactly in 32 bits, sums them into two exact 64-bit partials, and shifts
// each once to the common point (rounding to nearest); the 8 lanes that hold
// p = 0..7 of one row combine by a reduce-scatter of shuffles, and each sum
// is converted to FP64 once.  Relative to 2^{e_i + f_c}, the error is below K 2^-55 (the
// remainders r) and 2^-48 (the 16 roundings of the shifts), plus the final
// rounding to FP64: of the order of an FP64 product's own rounding (bound
// K 2^-53 sum_l |X_il||Y_lc|) unless a row or column mixes entries of very
// different size.
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <climits>

namespace lpgb {
namespace {

constexpr int kSlices = 8;   // 7-bit digits per operand (56 bits)
constexpr int kOzBN = 256;     // GEMM tile columns; two TMEM accumulators of them per CTA (all 512)
constexpr int kOzStages = 4;   // shared-memory stages of 48 KB (one persistent CTA per SM)
constexpr int kOzEpiWarps = 16;
constexpr int kOzCtas = 1;
constexpr int kFrac = 51;    // fraction bits of the fixed-point combination
constexpr int kNoDigits = INT_MIN / 4;  // exponent of an all-zero row or column

// binary exponent E of x = 1.f 2^E; zero and subnormals (below 2^-1022) give kNoDigits
__device__ __forceinline__ int dexp(double x) {
    const int ef = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
    return ef == 0 ? kNoDigits : ef - 1023;
}

// the 8 signed 7-bit digits of x / 2^e (|x| < 2^e), as BF16
__device__ __forceinline__ void digits(double x, int e, __nv_bfloat16 (&d)[kSlices]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    unsigned long long fix = 0;  // |x| 2^{56 - e}, truncated
    if (ef != 0 && e != kNoDigits) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = (ef - 1023) + 4 - e;  // <= 3
        if (sh >= 0) fix = mant << sh;
        else if (sh > -64) fix = mant >> (-sh);
    }
    const bool neg = (b >> 63) != 0;
#pragma unroll
    for (int p = 0; p < kSlices; ++p) {
        const int dg = (int)((fix >> (49 - 7 * p)) & 127u);
        d[p] = __float2bfloat16_rn((float)(neg ? -dg : dg));
    }
}

// X rows of the slack-row product: X[i][l] = A[S_i, J_l] (A column-major)
struct SrcAsj {
    const double* A;
    const int32_t* J;
    const int32_t* S;
    int ld;
    __device__ double operator()(int i, int l) const { return A[(size_t)J[l] * ld + S[i]]; }
};
// Y columns: Y[l][c] = W[l * k + c] (row-major k x k)
struct SrcRowMajor {
    const double* W;
    int k;
    __device__ double operator()(int c, int l) const { return W[(size_t)l * k + c]; }
};
// X rows of a row-major k x k matrix: X[i][l] = W[i * k + l]
struct SrcRowsOf {
    const double* W;
    int k;
    __device__ double operator()(int i, int l) const { return W[(size_t)i * k + l]; }
};
// X rows of a column-major k x k matrix: X[i][l] = W[l * k + i]
struct SrcColsOf {
    const double* W;
    int k;
    __device__ double operator()(int i, int l) const { return W[(size_t)l * k + i]; }
};

// exp[o] = 1 + max_l E(src(o, l)) over l < K (kNoDigits when all zero);
// 32 outer indices per block (consecutive, for coalescing) x 8 inner groups.
template <class Src>
__device__ void oz_exp_block(Src src, int nout, int K, int32_t* exps, int bx, int (*red)[33]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int o = bx * 32 + tx;
    int e = kNoDigits;
    if (o < nout)
        for (int l = ty; l < K; l += 8) e = max(e, dexp(src(o, l)));
    red[ty][tx] = e;
    __syncthreads();
    if (ty == 0 && o < nout) {
        int m = red[0][tx];
#pragma unroll
        for (int t = 1; t < 8; ++t) m = max(m, red[t][tx]);
        exps[o] = m == kNoDigits ? kNoDigits : m + 1;
    }
}

// out[(8 o + p) * ldk + l] = digit p of src(o, l) / 2^exp[o]; 32 x 32 tiles
// read along o and written along l through shared memory.
template <class Src>
__device__ void oz_slice_block(Src src, int nout, int K, const int32_t* exps, __nv_bfloat16* out, int ldk, int bx,
                               int by, __nv_bfloat16 (*t)[32][34]) {
    const int o0 = bx * 32, l0 = by * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int o = o0 + tx;
    const int e = o < nout ? exps[o] : kNoDigits;
    for (int ll = ty; ll < 32; ll += 8) {
        const int l = l0 + ll;
        __nv_bfloat16 d[kSlices];
        digits((o < nout && l < K) ? src(o, l) : 0.0, e, d);
#pragma unroll
        for (int p = 0; p < kSlices; ++p) t[p][tx][ll] = d[p];
    }
    __syncthreads();
    // each warp writes rows (o, p) with l along the lanes
    for (int r = ty; r < 32 * kSlices; r += 8) {
        const int oo = r / kSlices, p = r % kSlices;
        const int orow = o0 + oo, l = l0 + tx;
        if (orow < nout && l < K) out[(size_t)(kSlices * orow + p) * ldk + l] = t[p][oo][tx];
    }
}

// The exponents of both operands in one launch: blocks 0 .. ceil(M/32)-1 take
// the rows of X, the others the columns of Y.
template <class SX, class SY>
__global__ void __launch_bounds__(256) k_oz_exp(SX sx, int M, SY sy, int N, int K, int32_t* ex, int32_t* ey,
                                                const int32_t* err) {
    pdl_enter();
    if (*err != kErrNone) return;
    __shared__ int red[8][33];
    const int bxm = (M + 31) / 32;
    if ((int)blockIdx.x < bxm) oz_exp_block(sx, M, K, ex, blockIdx.x, red);
    else oz_exp_block(sy, N, K, ey, blockIdx.x - bxm, red);
}

// The slices of both operands in one launch (grid: outer tiles of X then of
// Y, by 32-element chunks of K).
template <class SX, class SY>
__global__ void __launch_bounds__(256) k_oz_slice(SX sx, int M, SY sy, int N, int K, const int32_t* ex,
                                                  const int32_t* ey, __nv_bfloat16* xs, __nv_bfloat16* ys, int ldk,
                                                  const int32_t* err) {
    pdl_enter();
    if (*err != kErrNone) return;
    __shared__ __nv_bfloat16 t[kSlices][32][34];  // [p][o][l]
    const int bxm = (M + 31) / 32;
    if ((int)blockIdx.x < bxm) oz_slice_block(sx, M, K, ex, xs, ldk, blockIdx.x, blockIdx.y, t);
    else oz_slice_block(sy, N, K, ey, ys, ldk, blockIdx.x - bxm, blockIdx.y, t);
}

// GEMM epilogue: combines the 64 digit pairs of each output (see the file
// comment) and writes sign * (X Y)[i][c] into out (row stride ldo); integer
// instructions only.
struct OzEpi {
    double* out;
    int ldo, M, N;
    const int32_t* ex;
    const int32_t* ey;
    int negate;
    __device__ void operator()(int trow, int m0, int n0, int c0, const float (&v)[32]) const {
        const int grow = m0 + trow;
        const int i = grow >> 3, p = grow & 7;
        const int cb = (n0 + c0) >> 3;  // n0 + c0 is a multiple of 32
        // This lane holds S_pq, q = 0..7, of 4 outputs.  In units of 2^-kFrac
        // its share is 2^{-7p} sum_q S_pq 2^{kFrac - 14 - 7q}; adjacent digits
        // pair exactly in 32 bits (w = 128 S_pq + S_p,q+1, |w| < 2^31 for
        // K <= 1024), and two exact 64-bit sums of two pairs each, a1 (q < 4)
        // and a2 (q >= 4), give the share as a1 2^{16 - 7p} + a2 2^{-12 - 7p}.
        static_assert(kFrac == 51, "the pair weights below are for 51 fraction bits");
        // The 8 lanes of a row reduce-scatter their 4 sums: lanes 2 cc and
        // 2 cc + 1 end with output cb + cc (exact integer adds, so the order
        // does not change the result); the even lane converts and stores it.
        const int c = cb + (p >> 1);
        const bool mine_out = (p & 1) == 0 && i < M && c < N;
        const int ei = mine_out ? __ldg(ex + i) : kNoDigits, fc = mine_out ? __ldg(ey + c) : kNoDigits;
        const int s1 = 7 * p, s2 = 12 + 7 * p;
        const long long r1 = p ? 1ll << (s1 - 1) : 0ll, r2 = 1ll << (s2 - 1);  // round to nearest
        long long t[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            int w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                w[j] = __float2int_rz(v[cc * 8 + 2 * j]) * 128 + __float2int_rz(v[cc * 8 + 2 * j + 1]);
            const long long a1 = (long long)w[0] * 16384 + w[1], a2 = (long long)w[2] * 16384 + w[3];
            t[cc] = ((a1 * 65536 + r1) >> s1) + ((a2 + r2) >> s2);
        }
        const bool hi2 = (p & 4) != 0, hi1 = (p & 2) != 0;
        long long u[2];  // outputs 2 hi2 + j, summed over lanes p and p ^ 4
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const long long give = hi2 ? t[j] : t[2 + j];
            u[j] = (hi2 ? t[2 + j] : t[j]) + __shfl_xor_sync(0xffffffffu, give, 4);
        }
        long long mine = (hi1 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, hi1 ? u[0] : u[1], 2);
        mine += __shfl_xor_sync(0xffffffffu, mine, 1);
        if (mine_out) {
            double val = 0.0;
            if (mine != 0 && ei != kNoDigits && fc != kNoDigits) val = ll_scaled(negate ? -mine : mine, ei + fc - kFrac);
            out[(size_t)i * ldo + c] = val;
        }
    }
};

}  // namespace

bool oz_fits(int k) { return k >= 1 && k <= 1024; }

size_t oz_scratch_x_elems(int m) {
    // 8 max(m - k, k) ldk over 1 <= k <= min(m, 1024), ldk = k rounded up to 8
    // (the slack rows, m - k of them, or the k rows of a refinement product)
    size_t best = 0;
    const int kmax = m < 1024 ? m : 1024;
    for (int k = 1; k <= kmax; ++k) {
        const int rows = m - k > k ? m - k : k;
        const size_t v = (size_t)kSlices * (size_t)rows * (size_t)((k + 7) & ~7);
        if (v > best) best = v;
    }
    return best;
}
size_t oz_scratch_y_elems(int m) {
    const int kmax = m < 1024 ? m : 1024;
    return (size_t)kSlices * kmax * (size_t)((kmax + 7) & ~7);
}

namespace {

// out (M x N, row stride ldo) = sign (X Y), X = sx (M x K), Y = sy (K x N),
// K <= 1024: exponents, slices of both operands, then one stacked GEMM whose
// epilogue combines the digit pairs.
template <class SX, class SY>
cudaError_t oz_product(SX sx, SY sy, int M, int N, int K, double* out, int ldo, int negate, __nv_bfloat16* xs,
                       __nv_bfloat16* ys, int32_t* ex, int32_t* ey, int32_t* err, cudaStream_t st) {
    if (!oz_fits(K) || M < 1 || N < 1) return cudaErrorInvalidValue;
    const int ldk = (K + 7) & ~7;
    const int bx = (M + 31) / 32 + (N + 31) / 32;
    const int32_t* cerr = err;
    launch_k(k_oz_exp<SX, SY>, dim3(bx), dim3(256), 0, st, true, sx, M, sy, N, K, ex, ey, cerr);
    const int32_t* cex = ex;
    const int32_t* cey = ey;
    launch_k(k_oz_slice<SX, SY>, dim3(bx, (K + 31) / 32), dim3(256), 0, st, true, sx, M, sy, N, K, cex, cey, xs, ys,
             ldk, cerr);
    CUtensorMap ma, mb;
    constexpr int BN = kOzBN;
    if (!tc_make_map_16bit(&ma, xs, kSlices * M, K, ldk, tcg::kTM, true) ||
        !tc_make_map_16bit(&mb, ys, kSlices * N, K, ldk, BN, true))
        return cudaErrorInvalidValue;
    const OzEpi epi{out, ldo, M, N, ex, ey, negate};
    return tcg::launch_tc_gemm_p<BN, kOzStages, kOzEpiWarps, kOzCtas, true>(ma, mb, epi, kSlices * M, kSlices * N, K,
                                                                           err, st);
}

}  // namespace

// C (nslack x k, row stride k) = -A[S, J] W, W = B11^-1 row-major k x k.
// xs / ys: BF16 slice scratch (oz_scratch_*_elems), ex / ey: nslack and k ints.
cudaError_t oz_slack_product(const double* A_cm, int ld, const int32_t* J, const int32_t* S, const double* W,
                             int k, int nslack, double* C, __nv_bfloat16* xs, __nv_bfloat16* ys, int32_t* ex,
                             int32_t* ey, int32_t* err, cudaStream_t st) {
    return oz_product(SrcAsj{A_cm, J, S, ld}, SrcRowMajor{W, k}, nslack, k, k, C, k, 1, xs, ys, ex, ey, err, st);
}

// The two products of a Newton-Schulz refinement step (kernels_reinv.cu), k x k:
// P = -(B11 Y0) with B11 column-major and Y0 row-major, and P = Y0 R with both
// row-major; P row-major.
cudaError_t oz_refine_residual_product(const double* B11_cm, const double* Y0, int k, double* P,
                                       __nv_bfloat16* xs, __nv_bfloat16* ys, int32_t* ex, int32_t* ey,
                                       int32_t* err, cudaStream_t st) {
    return oz_product(SrcColsOf{B11_cm, k}, SrcRowMajor{Y0, k}, k, k, k, P, k, 1, xs, ys, ex, ey, err, st);
}

cudaError_t oz_refine_update_product(const double* Y0, const double* R, int k, double* P, __nv_bfloat16* xs,
                                     __nv_bfloat16* ys, int32_t* ex, int32_t* ey, int32_t* err, cudaStream_t st) {
    return oz_product(SrcRowsOf{Y0, k}, SrcRowMajor{R, k}, k, k, k, P, k, 0, xs, ys, ex, ey, err, st);
}

}  // namespace lpgb
