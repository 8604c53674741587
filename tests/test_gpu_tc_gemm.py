"""The tensor-core GEMM (lp_tc_gemm: tcgen05.mma with TMA-staged tiles)
against FP64 products computed on the host.

* Integer-valued operands in [-127, 127] (the digit range of the 7-bit
  slices that the reinversion's FP64 products are built from): every product
  is exact in FP32 and every partial sum stays below 2^24 for K <= 1024, so
  the tensor cores must return the exact integer result, bit for bit, in FP16
  and BF16.  This is the premise of the sliced FP64 products.
* Random normal operands: within the FP32-accumulation bound of the exact
  product of the 16-bit operands.
* Ragged M, N and K (zero fill at the tile edges, masked stores) and row
  strides larger than K.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(M, N, K, bf16, A, B, ld_pad=0):
    import torch
    from paper_1803_04378_gb300 import lpgb
    dt = torch.bfloat16 if bf16 else torch.float16
    lda = ((K + 7) // 8) * 8 + ld_pad
    At = torch.zeros((M, lda), dtype=dt, device="cuda")
    Bt = torch.zeros((N, lda), dtype=dt, device="cuda")
    At[:, K:] = float("nan") if ld_pad else 0.0   # padding the GEMM must not read
    Bt[:, K:] = float("nan") if ld_pad else 0.0
    At[:, :K] = torch.from_numpy(A).to(dt).cuda()
    Bt[:, :K] = torch.from_numpy(B).to(dt).cuda()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    rc = lpgb.tc_gemm(At[:, :K], Bt[:, :K], D, bf16)
    assert rc == lpgb.LP_OK, rc
    torch.cuda.synchronize()
    return D.cpu().numpy(), At[:, :K].double().cpu().numpy(), Bt[:, :K].double().cpu().numpy()


@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (3752, 344, 344), (200, 150, 1000), (1, 1, 8), (130, 260, 1024)])
def test_integer_products_are_exact(M, N, K, bf16):
    rng = np.random.default_rng(M + 7 * N + K)
    A = rng.integers(-127, 128, size=(M, K)).astype(np.float64)
    B = rng.integers(-127, 128, size=(N, K)).astype(np.float64)
    # a few rows at the extremes, where the partial sums are largest
    A[0, :] = 127.0
    B[0, :] = 127.0
    if N > 1:
        B[1, :] = -127.0
    D, _, _ = _run(M, N, K, bf16, A, B)
    ref = A @ B.T
    assert np.max(np.abs(ref)) < 2.0 ** 24
    assert np.array_equal(D.astype(np.float64), ref)


@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("M,N,K,pad", [(256, 512, 6144, 0), (24, 48, 70, 8), (333, 257, 200, 16)])
def test_random_products(M, N, K, pad, bf16):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    D, A16, B16 = _run(M, N, K, bf16, A, B, ld_pad=pad)
    ref = A16 @ B16.T
    bound = 2.0 ** -22 * K * (np.abs(A16) @ np.abs(B16).T) + 1e-30
    assert np.all(np.abs(D - ref) <= bound)


def test_rejects_bad_strides():
    import torch
    from paper_1803_04378_gb300 import lpgb
    A = torch.zeros((16, 12), dtype=torch.float16, device="cuda")  # row stride 12: not a multiple of 8
    B = torch.zeros((16, 16), dtype=torch.float16, device="cuda")
    D = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    assert lpgb.tc_gemm(A, B[:, :12], D, False) == lpgb.LP_ERR_INVALID_ARG
