"""The fixed-point combination of the sliced FP64 product's epilogue, checked
on the CPU against exact rational arithmetic (no GPU).

The tensor cores leave, for each output, the 64 exact integer sums S_pq of
digit products (|S_pq| <= K 127^2, K <= 1024).  The product is
2^{e+f} sum_{p,q} S_pq 2^{-7(p+q+2)}.  The epilogue combines it in 64-bit
fixed point with 51 fraction bits relative to 2^{e+f}:

* the lane holding digit p pairs adjacent q into one 32-bit integer,
  w = 128 S_pq + S_p,q+1;
* it forms two exact 64-bit partials, a1 = 2^14 w0 + w1 and a2 = 2^14 w2 + w3;
* it shifts each once to the common point, rounding to nearest (half up):
  a1 2^{16 - 7p} and a2 2^{-12 - 7p};
* the 8 lanes of a row reduce-scatter their 4 outputs' sums.

The claims pinned here:
* no intermediate leaves its integer type at the extreme digit values;
* the result is within 8 units of 2^-51 of the exact value (the 16
  roundings, 2^-48 relative to 2^{e+f});
* the reduce-scatter leaves each output's total on lanes 2 cc and 2 cc + 1.

The arithmetic is restated here from that description in plain Python
integers; the CUDA epilogue is checked against FP64 products by the GPU tests
(test_gpu_reinv_tc.py, test_gpu_tc_gemm.py).
"""
from fractions import Fraction

import numpy as np

KFRAC = 51
SMAX = 1024 * 127 * 127  # the largest |S_pq| for K <= 1024
I32 = 2 ** 31
I64 = 2 ** 63


def lane_share(p, S):
    """Lane p's 64-bit fixed-point share of one output, from its S_pq, q = 0..7."""
    w = [S[2 * j] * 128 + S[2 * j + 1] for j in range(4)]
    assert all(-I32 <= x < I32 for x in w), "a digit pair leaves 32 bits"
    a1 = w[0] * 16384 + w[1]
    a2 = w[2] * 16384 + w[3]
    s1, s2 = 7 * p, 12 + 7 * p
    r1 = (1 << (s1 - 1)) if p else 0
    r2 = 1 << (s2 - 1)
    for v in (a1 * 65536 + r1, a2 + r2):
        assert -I64 <= v < I64, "a partial leaves 64 bits"
    return ((a1 * 65536 + r1) >> s1) + ((a2 + r2) >> s2)  # Python >> is the arithmetic shift


def exact_units(S):
    """The exact value in units of 2^-51 relative to 2^{e+f}."""
    return sum(Fraction(S[p][q]) * Fraction(2) ** (KFRAC - 14 - 7 * (p + q)) for p in range(8) for q in range(8))


def test_extremes_fit_and_error_bound():
    rng = np.random.default_rng(7)
    cases = [[[SMAX] * 8 for _ in range(8)], [[-SMAX] * 8 for _ in range(8)],
             [[SMAX if (p + q) % 2 else -SMAX for q in range(8)] for p in range(8)],
             [[0] * 8 for _ in range(8)], [[1] * 8 for _ in range(8)], [[-1] * 8 for _ in range(8)]]
    for _ in range(3000):
        lim = int(rng.choice([SMAX, 1000, 2 ** 20, 3]))
        cases.append([[int(rng.integers(-lim, lim + 1)) for _ in range(8)] for _ in range(8)])
    worst = Fraction(0)
    for S in cases:
        t = sum(lane_share(p, S[p]) for p in range(8))
        assert -I64 <= t < I64
        worst = max(worst, abs(t - exact_units(S)))
    assert worst <= 8, float(worst)


def test_reduce_scatter_leaves_each_output_on_its_lanes():
    rng = np.random.default_rng(8)
    for _ in range(200):
        t = [[int(v) for v in rng.integers(-2 ** 60, 2 ** 60, 4)] for _ in range(8)]  # t[p][cc]
        # step 1 (partner p ^ 4): keep outputs 2 hi2 + j, give the other two
        u = []
        for p in range(8):
            hi2, q = bool(p & 4), p ^ 4
            give_q = [t[q][j] if bool(q & 4) else t[q][2 + j] for j in range(2)]
            u.append([(t[p][2 + j] if hi2 else t[p][j]) + give_q[j] for j in range(2)])
        # step 2 (partner p ^ 2): keep output 2 hi2 + hi1
        mine = []
        for p in range(8):
            hi1, q = bool(p & 2), p ^ 2
            mine.append((u[p][1] if hi1 else u[p][0]) + (u[q][0] if bool(q & 2) else u[q][1]))
        # step 3 (partner p ^ 1)
        fin = [mine[p] + mine[p ^ 1] for p in range(8)]
        for p in range(8):
            assert fin[p] == sum(t[q][p >> 1] for q in range(8))
