"""The reinversion's products on the tensor cores (exact 7-bit slices of the
FP64 operands, combined in 64-bit fixed point) -- the slack-row product
-A[S, J] B11^-1 and the two Newton-Schulz refinement products B11 Y0 and
Y0 R -- against the same products in FP64 FMAs and against the oracle.

* B^-1 of a basis with k structural columns: with the tensor cores and
  without, within 1e-12 of the largest entry of each other, and both within
  1e-9 of the oracle's Gauss-Jordan inverse with B B^-1 = I to 1e-9.
* Operands whose rows and columns are scaled over 3 orders of magnitude:
  the slices of a row keep 56 bits relative to the row's largest entry, so
  the product loses precision with the spread of a row or column (here to
  within 1e-10 of the largest entry of FP64's result) but stays within the
  solver's 1e-9 of the oracle.
* Whole solves with reinversions every 16 pivots: the oracle follows every
  pivot, the objective equals that of FP64 products to 1e-12, and on the real
  family (no ties) the pivots are those of FP64 products.
* A refined reinversion (the updated inverse refined by one Newton-Schulz
  step): B^-1, bbar and y with the tensor cores and without within 1e-12 of
  the largest entry of each other, and within 1e-9 of the oracle's.
* k > 1024 (beyond the exact FP32 accumulation of the digit products) falls
  back to FP64 products.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import follow_check

pytestmark = pytest.mark.gpu


def _basis_with_k_structurals(m, n, k, seed, spread=0.0):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.0, 1.0, (m, n))
    A[rng.uniform(size=(m, n)) < 0.1] = 0.0
    if spread:
        A *= 10.0 ** rng.uniform(-spread, spread, (m, 1))   # rows of different scale
        A *= 10.0 ** rng.uniform(-spread, spread, (1, n))   # columns of different scale
    J = rng.choice(n, k, replace=False)
    R = np.sort(rng.choice(m, k, replace=False))
    xJ = rng.uniform(1.0, 2.0, k)
    s = rng.uniform(1.0, 2.0, m)
    s[R] = 0.0
    b = A[:, J] @ xJ + s
    c = rng.uniform(0.0, 1.0, n)
    basis = np.arange(n, n + m, dtype=np.int32)
    basis[R] = J
    return A, b, c, basis


def _state(A, b, c, basis, tc):
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, max_iters=0, reinvert_tc=tc) as lp:
        lp.set_basis(basis)
        res = lp.solve()
        binv, bbar = lp.state()
        y = lp.solution()[1]
    return res, binv, bbar, y


@pytest.mark.parametrize("m,n,k,spread,tol", [(300, 500, 1, 0.0, 1e-12), (300, 500, 37, 0.0, 1e-12),
                                              (700, 900, 600, 0.0, 1e-12), (1200, 1500, 1024, 0.0, 1e-12),
                                              (400, 600, 150, 1.5, 1e-10)])
def test_slack_rows_on_tensor_cores_match_fp64(m, n, k, spread, tol):
    A, b, c, basis = _basis_with_k_structurals(m, n, k, 7 + k, spread)
    r1, binv1, bbar1, y1 = _state(A, b, c, basis, 1)
    r0, binv0, bbar0, y0 = _state(A, b, c, basis, 0)
    assert r1.reinversions == 1 and r1.tc_reinversions == 1
    assert r0.reinversions == 1 and r0.tc_reinversions == 0
    scale = max(1.0, np.max(np.abs(binv0)))
    assert np.max(np.abs(binv1 - binv0)) <= tol * scale
    # bbar = B^-1 b sums terms of size |B^-1| |b| that cancel to bbar: that is its error scale
    assert np.max(np.abs(bbar1 - bbar0)) <= tol * max(1.0, np.max(np.abs(binv0) @ np.abs(b)))
    assert np.array_equal(y1, y0)  # y comes from B11^-1 alone
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=0), start_basis=basis, want_binv=True)
    rs = max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(binv1 - ref.binv)) <= 1e-9 * rs
    B = np.hstack([A, np.eye(m)])[:, basis]
    assert np.max(np.abs(binv1 @ B - np.eye(m))) <= 1e-9 * rs


@pytest.mark.parametrize("kind,m,n,seed", [("real", 300, 600, 5), ("int", 200, 200, 0), ("degenerate", 150, 300, 4)])
def test_solves_with_tensor_core_reinversions(kind, m, n, seed):
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    runs = []
    for tc in (1, 0):
        with lpgb.LP(A, b, c, reinvert_every=16, reinvert_tc=tc, trace_cap=1 << 16) as lp:
            res = lp.solve()
            x, y, z = lp.solution()
            runs.append((res, lp.trace(), z))
    (r1, t1, z1), (r0, t0, z0) = runs
    assert r1.status == r0.status == lpgb.LP_OPTIMAL
    assert r1.reinversions >= 1 and r1.tc_reinversions >= 1 and r0.tc_reinversions == 0
    assert r1.refined_reinversions >= 1 and r0.refined_reinversions >= 1
    if kind == "real":
        # no ties: the last-bit differences of the two products cannot change a choice
        assert np.array_equal(t1["q"], t0["q"]) and np.array_equal(t1["r"], t0["r"])
    assert z1 == pytest.approx(z0, rel=1e-12, abs=1e-12)
    follow_check(A, b, c, r1, t1, oracle.Options(reinvert_every=16))


@pytest.mark.parametrize("kind,m,n,seed,K", [("real", 600, 1000, 7, 80), ("real", 1100, 1600, 8, 192)])
def test_refined_reinversion_on_tensor_cores(kind, m, n, seed, K):
    """State right after the refined reinversion at pivot K (reinversions every
    K/2 pivots), with and without the tensor cores, against the oracle
    following the same pivots."""
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    out = []
    for tc in (1, 0):
        with lpgb.LP(A, b, c, reinvert_every=K // 2, reinvert_tc=tc, max_iters=K, trace_cap=K) as lp:
            res = lp.solve()
            binv, bbar = lp.state()
            y = lp.solution()[1]
            tr = lp.trace()
        assert res.iterations == K and res.refined_reinversions == 2, (res.iterations, res.refined_reinversions)
        out.append((binv, bbar, y, tr))
    (B1, b1, y1, t1), (B0, b0, y0, t0) = out
    assert np.array_equal(t1["q"], t0["q"]) and np.array_equal(t1["r"], t0["r"])
    for u, v in ((B1, B0), (b1, b0), (y1, y0)):
        assert np.max(np.abs(u - v)) <= 1e-12 * max(1.0, np.max(np.abs(v)))
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=K, reinvert_every=K // 2),
                       follow=(t1["q"], t1["r"]), follow_status=lpgb.LP_ITER_LIMIT, want_binv=True)
    assert ref.mismatch_at < 0
    assert np.max(np.abs(B1 - ref.binv)) <= 1e-9 * max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(b1 - ref.bbar)) <= 1e-9 * max(1.0, np.max(np.abs(ref.bbar)))


def test_more_than_1024_structurals_use_fp64_products():
    A, b, c, basis = _basis_with_k_structurals(1100, 1300, 1050, 3)
    r1, binv1, _, _ = _state(A, b, c, basis, 1)
    assert r1.reinversions == 1 and r1.tc_reinversions == 0
