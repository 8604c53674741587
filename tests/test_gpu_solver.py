"""CUDA solver vs the oracle, through the C ABI (needs a GB300).

Bars (from the method's tolerances): identical pivot sequence wherever ties
are separated by more than 1e-12 (checked by the oracle's follow mode), optimal
objective within 1e-9 relative, primal/dual residuals <= 1e-9.  Element-wise
state (B^-1, bbar) within 1e-9 of the largest entry: FP64 with different
summation orders over at most 64 rank-1 updates stays far below that.
"""
import json
import os

import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate, follow_check, gpu_solve

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb  # noqa: F401


CASES = [
    ("int", 200, 200, 0),      # the 200x200 dense integer workload
    ("int", 37, 61, 5),
    ("real", 256, 512, 1),
    ("real", 300, 200, 3),     # n < m
    ("real", 129, 257, 4),     # ragged against the 64-wide row padding
    ("degenerate", 64, 128, 2),
    ("degenerate", 128, 256, 2),
]


@pytest.mark.parametrize("kind,m,n,seed", CASES)
def test_pivot_sequence_and_objective(kind, m, n, seed):
    A, b, c = lpgen.make(kind, m, n, seed)
    lp, res, x, y, z, tr = gpu_solve(A, b, c)
    assert res.status == 1
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr)
    lp.close()


def test_klee_minty_pivot_count():
    for d in (3, 6, 9):
        A = np.zeros((d, d)); b = np.zeros(d); c = np.zeros(d)
        for i in range(d):
            for j in range(i):
                A[i, j] = 2 * 10.0 ** (i - j)
            A[i, i] = 1.0
            b[i] = 100.0 ** i
            c[i] = 10.0 ** (d - 1 - i)
        lp, res, x, y, z, tr = gpu_solve(A, b, c)
        assert res.status == 1 and res.iterations == 2 ** d - 1
        assert z == pytest.approx(100.0 ** (d - 1), rel=1e-12)
        lp.close()


def test_beale_terminates():
    g = json.load(open(os.path.join(GOLD, "beale_1955.json")))
    A, b, c = np.array(g["A"]), np.array(g["b"]), np.array(g["c"])
    lp, res, x, y, z, tr = gpu_solve(A, b, c)
    assert res.status == 1 and z == pytest.approx(g["optimum"], abs=1e-15)
    assert np.allclose(x, g["x_opt"], atol=1e-15)
    follow_check(A, b, c, res, tr)
    lp.close()


@pytest.mark.parametrize("K,reinv", [(1, 64), (17, 64), (63, 64), (64, 64), (100, 64), (40, 0)])
def test_state_elementwise(K, reinv):
    A, b, c = lpgen.dense_real_lp(150, 260, 21)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, max_iters=K, reinvert_every=reinv)
    assert res.status == 3 and res.iterations == K
    o = oracle.Options(max_iters=K, reinvert_every=reinv)
    follow_check(A, b, c, res, tr, o)
    ref = oracle.solve(A, b, c, o, want_binv=True)
    binv, bbar = lp.state()
    assert np.array_equal(lp.basis(), ref.basis)
    scale = max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(binv - ref.binv)) <= 1e-9 * scale
    assert np.max(np.abs(bbar - ref.bbar)) <= 1e-9 * max(1.0, np.max(np.abs(ref.bbar)))
    assert np.max(np.abs(y - ref.y)) <= 1e-9 * max(1.0, np.max(np.abs(ref.y)))
    assert z == pytest.approx(ref.objective, rel=1e-12)
    lp.close()


def test_warm_start_reinversion_elementwise():
    A, b, c = lpgen.dense_real_lp(180, 300, 22)
    ref_full = oracle.solve(A, b, c)
    # a feasible intermediate basis from the oracle's own path
    mid = oracle.solve(A, b, c, oracle.Options(max_iters=ref_full.iterations // 2))
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, max_iters=0) as lp:
        lp.set_basis(mid.basis)
        res = lp.solve()
        assert res.status == 3 and res.reinversions == 1
        binv, bbar = lp.state()
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=0), start_basis=mid.basis, want_binv=True)
    assert np.max(np.abs(binv - ref.binv)) <= 1e-9 * max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(bbar - ref.bbar)) <= 1e-9 * max(1.0, np.max(np.abs(ref.bbar)))
    # and a warm solve from the optimal basis takes no pivots
    with lpgb.LP(A, b, c) as lp:
        lp.set_basis(ref_full.basis)
        res = lp.solve()
        _, _, z = lp.solution()
        assert res.status == 1 and res.iterations == 0
        assert z == pytest.approx(ref_full.objective, rel=1e-12)


def _basis_with_k_structurals(m, n, k, seed):
    """A feasible basis with exactly k structural columns: J (k columns) sit at
    the positions of k rows R whose slacks are nonbasic; b = A[:, J] x_J + s
    with x_J > 0 and s > 0 off R, so that bbar = (x_J, s) >= 0."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.0, 1.0, (m, n))
    A[rng.uniform(size=(m, n)) < 0.1] = 0.0
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


@pytest.mark.parametrize("m,n,k", [(40, 60, 5), (80, 100, 32), (80, 100, 33), (150, 200, 64),
                                   (150, 200, 65), (700, 900, 600)])
def test_reinversion_panels(m, n, k):
    """Fresh B^-1 of a basis with k structurals against the oracle's Gauss-Jordan
    inverse of the whole basis matrix: covers CTAs that own no rows (k < 16),
    panel edges (32/33, 64/65) and more rows per CTA than a warp (k = 600)."""
    A, b, c, basis = _basis_with_k_structurals(m, n, k, 40 + k)
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, max_iters=0) as lp:
        lp.set_basis(basis)
        res = lp.solve()
        assert res.status == 3 and res.reinversions == 1
        binv, bbar = lp.state()
        y = lp.solution()[1]
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=0), start_basis=basis, want_binv=True)
    scale = max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(binv - ref.binv)) <= 1e-9 * scale
    assert np.max(np.abs(bbar - ref.bbar)) <= 1e-9 * max(1.0, np.max(np.abs(ref.bbar)))
    assert np.max(np.abs(y - ref.y)) <= 1e-9 * max(1.0, np.max(np.abs(ref.y)))
    B = np.hstack([A, np.eye(m)])[:, basis]
    assert np.max(np.abs(binv @ B - np.eye(m))) <= 1e-9 * scale


@pytest.mark.parametrize("kind,m,n,seed,K", [("real", 256, 512, 1, 0), ("degenerate", 128, 256, 2, 0),
                                          ("int", 200, 200, 0, 0), ("real", 300, 200, 3, 100)])
def test_persistent_engine_matches_graph_engine(kind, m, n, seed, K):
    """The persistent cooperative kernel and the captured three-kernel graphs
    run the same arithmetic in the same order: identical pivots and
    bit-identical B^-1, bbar, x, y (K > 0 stops at an iteration limit that is
    not a multiple of the pivots per launch)."""
    A, b, c = lpgen.make(kind, m, n, seed)
    from paper_1803_04378_gb300 import lpgb
    runs = []
    for engine in (0, 1):
        extra = {"max_iters": K} if K else {}
        with lpgb.LP(A, b, c, engine=engine, trace_cap=1 << 14, **extra) as lp:
            res = lp.solve()
            tr = lp.trace()
            binv, bbar = lp.state()
            x, y, z = lp.solution()
            runs.append((res, tr, binv, bbar, x, y, z))
    (r0, t0, B0, bb0, x0, y0, z0), (r1, t1, B1, bb1, x1, y1, z1) = runs
    assert r0.persistent == 1 and r1.persistent == 0
    assert r0.status == r1.status and r0.iterations == r1.iterations
    assert r0.reinversions == r1.reinversions and r0.tabu_pushes == r1.tabu_pushes
    assert np.array_equal(t0["q"], t1["q"]) and np.array_equal(t0["r"], t1["r"])
    assert np.array_equal(B0, B1) and np.array_equal(bb0, bb1)
    assert np.array_equal(x0, x1) and np.array_equal(y0, y1) and z0 == z1


def test_grid_barrier_wait_is_bounded():
    """The persistent engine's grid barrier gives up after its spin limit: a
    barrier that cannot complete (it expects one CTA more than the grid has)
    returns LP_ERR_TIMEOUT within seconds, and the context stays usable."""
    import time
    from paper_1803_04378_gb300 import lpgb
    t0 = time.time()
    assert lpgb.selftest_barrier_timeout(4) == lpgb.LP_ERR_TIMEOUT
    assert time.time() - t0 < 60
    A, b, c = lpgen.dense_int_lp(20, 30, 0)
    with lpgb.LP(A, b, c) as lp:
        assert lp.solve().status == 1


def test_reinvert_every_pivot_same_path():
    A, b, c = lpgen.dense_real_lp(120, 200, 12)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, reinvert_every=1)
    assert res.status == 1 and res.reinversions == res.iterations
    follow_check(A, b, c, res, tr, oracle.Options(reinvert_every=1))
    lp.close()


def test_edge_shapes():
    rng = np.random.default_rng(5)
    for (m, n) in [(1, 1), (1, 7), (7, 1), (63, 64), (64, 63), (65, 65)]:
        A = rng.random((m, n)) + 0.05
        b = rng.random(m) * 3
        c = rng.random(n)
        lp, res, x, y, z, tr = gpu_solve(A, b, c)
        ref = oracle.solve(A, b, c)
        assert res.status == 1 and z == pytest.approx(ref.objective, rel=1e-12, abs=1e-15)
        follow_check(A, b, c, res, tr)
        lp.close()


def test_trivial_and_unbounded():
    # c <= 0: the slack basis is optimal
    A = np.ones((3, 4)); b = np.ones(3); c = -np.ones(4)
    lp, res, x, y, z, tr = gpu_solve(A, b, c)
    assert res.status == 1 and res.iterations == 0 and z == 0.0
    lp.close()
    # column 1 has no positive entry: unbounded
    A = np.array([[1.0, -1.0], [2.0, 0.0]]); b = np.array([1.0, 2.0]); c = np.array([1.0, 1.0])
    lp, res, x, y, z, tr = gpu_solve(A, b, c)
    ref = oracle.solve(A, b, c)
    assert res.status == 2 and ref.status == oracle.UNBOUNDED
    follow_check(A, b, c, res, tr)
    lp.close()


def test_pinned_host_inputs():
    """A in pinned host memory is read in place by the upload's transpose
    and validated on the device: the same solve as from pageable memory, and
    a NaN or an infinity anywhere in it (also in a large A, past the host's
    threaded check size) is rejected with LP_ERR_INVALID_ARG."""
    import torch
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("real", 300, 500, 3)
    Ap = torch.empty(A.shape, dtype=torch.float64, pin_memory=True)
    Ap.numpy()[:] = A
    with lpgb.LP(Ap.numpy(), b, c) as lp0, lpgb.LP(A, b, c) as lp1:
        r0, r1 = lp0.solve(), lp1.solve()
        assert r0.status == r1.status == 1 and r0.iterations == r1.iterations
        assert lp0.solution()[2] == lp1.solution()[2]
    for bad in (float("nan"), float("inf"), -float("inf")):
        Ap.numpy()[123, 456] = bad
        with pytest.raises(lpgb.LPError) as e:
            lpgb.LP(Ap.numpy(), b, c)
        assert e.value.code == lpgb.LP_ERR_INVALID_ARG
        Ap.numpy()[123, 456] = A[123, 456]
    # lp_update_problem takes the same path: a pinned A' on a handle built from
    # another problem solves as a fresh handle on A', and a NaN in it is refused
    A2, b2, c2 = lpgen.make("real", 300, 500, 4)
    Ap.numpy()[:] = A2
    with lpgb.LP(A, b, c) as lpu, lpgb.LP(A2, b2, c2) as lpf:
        lpu.update_problem(Ap.numpy(), b2, c2)
        ru, rf = lpu.solve(), lpf.solve()
        assert ru.status == rf.status == 1 and ru.iterations == rf.iterations
        assert lpu.solution()[2] == lpf.solution()[2]
        Ap.numpy()[7, 9] = float("nan")
        with pytest.raises(lpgb.LPError) as e:
            lpu.update_problem(Ap.numpy(), b2, c2)
        assert e.value.code == lpgb.LP_ERR_INVALID_ARG
    Ap.numpy()[:] = A
    m, n = 1100, 4000  # 4.4 M entries
    Ab = torch.ones((m, n), dtype=torch.float64, pin_memory=True)
    Ab.numpy()[m - 1, n - 1] = float("nan")
    with pytest.raises(lpgb.LPError) as e:
        lpgb.LP(Ab.numpy(), np.ones(m), np.ones(n))
    assert e.value.code == lpgb.LP_ERR_INVALID_ARG
    An = np.ones((m, n))
    An[m - 1, n - 1] = float("inf")  # pageable: the host's threaded check
    with pytest.raises(lpgb.LPError) as e:
        lpgb.LP(An, np.ones(m), np.ones(n))
    assert e.value.code == lpgb.LP_ERR_INVALID_ARG


def test_invalid_arguments():
    from paper_1803_04378_gb300 import lpgb
    A = np.ones((2, 2))
    with pytest.raises(lpgb.LPError) as e:
        lpgb.LP(A, np.array([1.0, np.inf]), np.ones(2))
    assert e.value.code == lpgb.LP_ERR_INVALID_ARG
    with pytest.raises(lpgb.LPError):
        lpgb.LP(np.array([[1.0, np.nan], [1.0, 1.0]]), np.ones(2), np.ones(2))
    with lpgb.LP(A, np.ones(2), np.ones(2)) as lp:
        with pytest.raises(lpgb.LPError) as e:
            lp.set_basis(np.array([0, 0], np.int32))
        assert e.value.code == lpgb.LP_ERR_INVALID_ARG
        with pytest.raises(lpgb.LPError) as e:
            lp.solution()
        assert e.value.code == lpgb.LP_ERR_STATE


def test_device_inputs_match_host_inputs():
    import torch
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_real_lp(200, 330, 9)
    with lpgb.LP(A, b, c) as lp:
        r1 = lp.solve()
        z1 = lp.solution()[2]
    At, bt, ct = (torch.from_numpy(v).cuda() for v in (A, b, c))
    with lpgb.LP(At, bt, ct) as lp:
        r2 = lp.solve()
        z2 = lp.solution()[2]
    assert r1.iterations == r2.iterations and z1 == z2


def test_reset_repeats_identically():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_real_lp(256, 400, 10)
    with lpgb.LP(A, b, c, trace_cap=10000) as lp:
        r1 = lp.solve(); t1 = lp.trace(); z1 = lp.solution()[2]
        lp.reset()
        r2 = lp.solve(); t2 = lp.trace(); z2 = lp.solution()[2]
    assert r1.iterations == r2.iterations and z1 == z2
    assert np.array_equal(t1["q"], t2["q"]) and np.array_equal(t1["r"], t2["r"])


@pytest.mark.parametrize("kind,m,n,seed", CASES)
def test_bf16_price_mode(kind, m, n, seed):
    """price_mode 1: BF16 screen + FP64 re-price of the top k.  The entering
    choice may differ from Dantzig's FP64 argmax (pivot-sequence parity is not
    claimed), so every pivot is checked as a valid simplex pivot -- an
    improving eligible column and the ratio-test row -- and the optimum must
    match the FP64 oracle to 1e-9."""
    A, b, c = lpgen.make(kind, m, n, seed)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, price_mode=1, topk=16)
    ref = oracle.solve(A, b, c)
    assert res.status == 1
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr, oracle.Options(follow_relaxed=1))
    lp.close()


def test_bf16_price_mode_small_topk_and_klee_minty():
    for d in (4, 7):
        A = np.zeros((d, d)); b = np.zeros(d); c = np.zeros(d)
        for i in range(d):
            for j in range(i):
                A[i, j] = 2 * 10.0 ** (i - j)
            A[i, i] = 1.0
            b[i] = 100.0 ** i
            c[i] = 10.0 ** (d - 1 - i)
        lp, res, x, y, z, tr = gpu_solve(A, b, c, price_mode=1, topk=1)
        assert res.status == 1 and z == pytest.approx(100.0 ** (d - 1), rel=1e-12)
        follow_check(A, b, c, res, tr, oracle.Options(follow_relaxed=1))
        lp.close()


def test_update_problem_equals_fresh_handle():
    from paper_1803_04378_gb300 import lpgb
    P1 = lpgen.dense_real_lp(220, 350, 41)
    P2 = lpgen.perturbed_lp(P1, 7)
    with lpgb.LP(*P2, trace_cap=5000) as fresh:
        rf = fresh.solve(); zf = fresh.solution()[2]; tf = fresh.trace()
    with lpgb.LP(*P1, trace_cap=5000) as lp:
        lp.solve()
        lp.update_problem(*P2)
        r2 = lp.solve(); z2 = lp.solution()[2]; t2 = lp.trace()
    assert r2.iterations == rf.iterations and z2 == zf
    assert np.array_equal(t2["q"], tf["q"]) and np.array_equal(t2["r"], tf["r"])


def test_guided_priority_warm_start():
    """lp_set_priority: the optimal basis of a perturbed neighbour, listed as
    priorities, cuts the pivots; every pivot is still a valid simplex pivot and
    the optimum is the oracle's."""
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(300, 600, 42)
    inst = lpgen.perturbed_lp(base, 11)
    ref_base = oracle.solve(*base)
    ref = oracle.solve(*inst)
    A, b, c = inst
    hint = [int(v) for v in ref_base.basis if v < A.shape[1]]
    with lpgb.LP(A, b, c, trace_cap=20000) as lp:
        cold = lp.solve()
        lp.reset()
        lp.set_priority(hint)
        guided = lp.solve()
        x, y, z = lp.solution()
        tr = lp.trace()
    assert guided.status == 1 and abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert_certificate(A, b, c, x, y)
    assert np.any(tr["flags"] & lpgb.LP_TF_GUIDED)
    follow_check(A, b, c, guided, tr, oracle.Options(follow_relaxed=1))
    # direct start from the neighbour's optimal basis, repaired where infeasible
    with lpgb.LP(A, b, c) as lp:
        lp.set_basis_repair(ref_base.basis, 300)
        warm = lp.solve()
        x, y, z = lp.solution()
    assert warm.status == 1 and warm.warm_fallback == 0
    assert abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert_certificate(A, b, c, x, y)
    assert warm.iterations < cold.iterations
    # a useless priority list (every column, in index order) still ends optimal
    with lpgb.LP(A, b, c) as lp:
        lp.set_priority(np.arange(A.shape[1] + A.shape[0]))
        r = lp.solve()
        assert r.status == 1 and abs(lp.solution()[2] - ref.objective) <= 1e-9 * abs(ref.objective)
    with lpgb.LP(A, b, c, price_mode=1) as lp:
        with pytest.raises(lpgb.LPError) as e:
            lp.set_priority(hint)
        assert e.value.code == lpgb.LP_ERR_STATE
