"""The slack-structured persistent engine (LP_ENGINE_STRUCTURED) against the
oracle and against the dense persistent engine (needs a GB300).

The structured engine computes the method's quantities over the rows whose
slack is nonbasic only; every term it skips is an exact zero of the dense
computation (y on rows with a basic slack, the unit columns of B^-1), so the
bars are the dense engine's: identical pivot sequence where ties are separated
by more than 1e-12 (oracle follow mode), objective within 1e-9 relative,
certificates within 1e-9.  Against the dense engine the sums differ only in
the order of their nonzero terms: same pivots on these data, objectives and
duals within rounding.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate, follow_check, gpu_solve

pytestmark = pytest.mark.gpu

S = 2  # LP_ENGINE_STRUCTURED


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
    ("degenerate", 128, 256, 2),  # slacks re-enter the basis
]


@pytest.mark.parametrize("kind,m,n,seed", CASES)
def test_pivot_sequence_and_objective(kind, m, n, seed):
    A, b, c = lpgen.make(kind, m, n, seed)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, engine=S)
    assert res.persistent == 2
    assert res.status == 1
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr)
    lp.close()


@pytest.mark.parametrize("kind,m,n,seed,K,G", [
    ("real", 256, 512, 1, 0, 64), ("int", 200, 200, 0, 0, 64), ("degenerate", 128, 256, 2, 0, 64),
    ("real", 300, 200, 3, 100, 64), ("real", 160, 300, 6, 0, 1), ("degenerate", 96, 160, 7, 0, 5),
    ("real", 200, 330, 8, 77, 3), ("real", 300, 500, 9, 64, 64), ("real", 300, 500, 9, 128, 64),
    ("int", 200, 200, 0, 129, 64)])
def test_matches_dense_engine(kind, m, n, seed, K, G):
    """Same pivots, counters and final state as the dense persistent engine
    (K > 0 stops at an iteration limit, also one that falls on a periodic
    reinversion, which the structured engine queues with its next launch; G
    pivots per launch: the state crosses launch boundaries in every phase of
    the slot moves)."""
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    runs = []
    for engine in (0, S):
        extra = {"max_iters": K} if K else {}
        with lpgb.LP(A, b, c, engine=engine, graph_iters=G, trace_cap=1 << 14, **extra) as lp:
            res = lp.solve()
            tr = lp.trace()
            binv, bbar = lp.state()
            x, y, z = lp.solution()
            runs.append((res, tr, binv, bbar, x, y, z))
    (r0, t0, B0, bb0, x0, y0, z0), (r1, t1, B1, bb1, x1, y1, z1) = runs
    assert r0.persistent == 1 and r1.persistent == 2
    assert r0.status == r1.status and r0.iterations == r1.iterations
    assert r0.reinversions == r1.reinversions and r0.tabu_pushes == r1.tabu_pushes
    assert r0.degenerate == r1.degenerate and r0.bland_fallbacks == r1.bland_fallbacks
    assert np.array_equal(t0["q"], t1["q"]) and np.array_equal(t0["r"], t1["r"])
    assert np.array_equal(t0["flags"], t1["flags"])
    scale = max(1.0, np.max(np.abs(bb0)))
    assert np.max(np.abs(bb0 - bb1)) <= 1e-9 * scale
    # B^-1 read back from the structured state: live columns, and exact unit
    # columns wherever the dense engine's are exact units
    assert np.max(np.abs(B0 - B1)) <= 1e-9 * max(1.0, np.max(np.abs(B0)))
    unit = np.all((B0 == 0.0) | (B0 == 1.0), axis=0) & (np.sum(B0 == 1.0, axis=0) == 1)
    assert np.array_equal(B0[:, unit], B1[:, unit])
    assert abs(z0 - z1) <= 1e-12 * max(1.0, abs(z0))
    assert np.max(np.abs(x0 - x1)) <= 1e-9 * max(1.0, np.max(np.abs(x0)))
    assert np.max(np.abs(y0 - y1)) <= 1e-9 * max(1.0, np.max(np.abs(y0)))


def test_klee_minty_and_beale():
    import json
    import os
    for d in (3, 6, 9):
        A = np.zeros((d, d)); b = np.zeros(d); c = np.zeros(d)
        for i in range(d):
            for j in range(i):
                A[i, j] = 2 * 10.0 ** (i - j)
            A[i, i] = 1.0
            b[i] = 100.0 ** i
            c[i] = 10.0 ** (d - 1 - i)
        lp, res, x, y, z, tr = gpu_solve(A, b, c, engine=S)
        assert res.status == 1 and res.iterations == 2 ** d - 1
        assert z == pytest.approx(100.0 ** (d - 1), rel=1e-12)
        lp.close()
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "beale_1955.json")))
    A, b, c = np.array(g["A"]), np.array(g["b"]), np.array(g["c"])
    lp, res, x, y, z, tr = gpu_solve(A, b, c, engine=S)
    assert res.status == 1 and z == pytest.approx(g["optimum"], abs=1e-15)
    follow_check(A, b, c, res, tr)
    lp.close()


def test_edge_shapes_and_outcomes():
    from paper_1803_04378_gb300 import lpgb
    for (m, n, seed) in [(1, 1, 0), (1, 7, 1), (7, 1, 2), (65, 3, 3), (3, 130, 4)]:
        A, b, c = lpgen.dense_int_lp(m, n, seed)
        lp, res, x, y, z, tr = gpu_solve(A, b, c, engine=S)
        ref = oracle.solve(A, b, c)
        assert res.status == 1 and abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
        assert_certificate(A, b, c, x, y)
        lp.close()
    # c <= 0: optimal at the slack basis, no pivot
    with lpgb.LP(np.ones((3, 4)), np.ones(3), -np.ones(4), engine=S) as lp:
        res = lp.solve()
        assert res.status == 1 and res.iterations == 0 and lp.solution()[2] == 0.0
    # unbounded: a column with no positive entry
    with lpgb.LP(np.array([[1.0, -1.0], [2.0, 0.0]]), np.ones(2), np.array([0.0, 1.0]), engine=S) as lp:
        assert lp.solve().status == lpgb.LP_UNBOUNDED


def test_reset_and_update_problem():
    """The slot map survives a reset (the next solve starts from the slack
    basis on the permuted rows) and follows a new A."""
    from paper_1803_04378_gb300 import lpgb
    P1 = lpgen.dense_real_lp(220, 350, 41)
    P2 = lpgen.perturbed_lp(P1, 7)
    with lpgb.LP(*P2, engine=S, trace_cap=5000) as fresh:
        rf = fresh.solve(); zf = fresh.solution()[2]; tf = fresh.trace()
    with lpgb.LP(*P1, engine=S, trace_cap=5000) as lp:
        r1 = lp.solve(); z1 = lp.solution()[2]; t1 = lp.trace()
        lp.reset()
        r1b = lp.solve(); z1b = lp.solution()[2]; t1b = lp.trace()
        lp.update_problem(*P2)
        r2 = lp.solve(); z2 = lp.solution()[2]; t2 = lp.trace()
    assert r1.iterations == r1b.iterations and z1 == z1b
    assert np.array_equal(t1["q"], t1b["q"]) and np.array_equal(t1["r"], t1b["r"])
    assert r2.iterations == rf.iterations and z2 == zf
    assert np.array_equal(t2["q"], tf["q"]) and np.array_equal(t2["r"], tf["r"])


def test_warm_starts():
    """lp_set_basis (dense reinversion, then the structured entry rebuilds the
    slot map), lp_set_basis_repair (dense repair pivots first) and lp_set_priority."""
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(300, 600, 42)
    inst = lpgen.perturbed_lp(base, 11)
    ref_base = oracle.solve(*base)
    ref = oracle.solve(*inst)
    A, b, c = inst
    with lpgb.LP(*base, engine=S) as lp:
        lp.set_basis(ref_base.basis)
        res = lp.solve()
        assert res.status == 1 and res.iterations == 0
        assert abs(lp.solution()[2] - ref_base.objective) <= 1e-9 * abs(ref_base.objective)
    with lpgb.LP(A, b, c, engine=S) as lp:
        cold = lp.solve()
        lp.set_basis_repair(ref_base.basis, 300)
        warm = lp.solve()
        x, y, z = lp.solution()
    assert warm.status == 1 and warm.warm_fallback == 0 and warm.iterations < cold.iterations
    assert abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert_certificate(A, b, c, x, y)
    hint = [int(v) for v in ref_base.basis if v < A.shape[1]]
    with lpgb.LP(A, b, c, engine=S, trace_cap=20000) as lp:
        lp.set_priority(hint)
        guided = lp.solve()
        x, y, z = lp.solution()
        tr = lp.trace()
    assert guided.status == 1 and abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert np.any(tr["flags"] & lpgb.LP_TF_GUIDED)
    follow_check(A, b, c, guided, tr, oracle.Options(follow_relaxed=1))


@pytest.mark.parametrize("m,n,seed", [(20, 30, 1), (200, 300, 4), (301, 257, 5)])
def test_two_phase(m, n, seed):
    """Phase I on the structured engine; the exchange of an artificial left
    basic at zero reads B^-1 from the structured state."""
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.general_lp(m, n, seed)
    ref = oracle.solve_two_phase(A, b, c)
    with lpgb.LP(A, b, c, engine=S, trace_cap=1 << 14) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
        tr = lp.trace()
    assert res.status == lpgb.LP_OPTIMAL and res.phase1_iterations == ref.phase1.iterations
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    chk = oracle.solve(A, b, c, start_basis=ref.start_basis, follow=(tr["q"], tr["r"]))
    assert chk.mismatch_at < 0 and chk.status == oracle.OPTIMAL, chk.mismatch_at
    A = np.array([[-1.0], [-1.0], [3.0], [1.0]])
    b = np.array([0.0, -1.0, 3.0, 10.0])
    with lpgb.LP(A, b, np.array([1.0]), engine=S) as lp:
        res = lp.solve()
        assert res.status == lpgb.LP_OPTIMAL and res.phase1_exchanged == 1
        assert lp.solution()[2] == pytest.approx(1.0)


def test_device_inputs():
    import torch
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_real_lp(180, 260, 12)
    with lpgb.LP(A, b, c, engine=S) as lp:
        r1 = lp.solve(); z1 = lp.solution()[2]
    At, bt, ct = (torch.from_numpy(v).cuda() for v in (A, b, c))
    with lpgb.LP(At, bt, ct, engine=S) as lp:
        r2 = lp.solve(); z2 = lp.solution()[2]
    assert r1.iterations == r2.iterations and z1 == z2


def test_screen_fallbacks():
    """The FP32 screen of PRICE steps aside where its bound does not hold: an
    entry of A beyond 2^40 switches it off for the problem (the full FP64
    PRICE runs), and the pivots stay the method's."""
    A, b, c = lpgen.dense_real_lp(150, 240, 21)
    A[3, 7] = 3.0e13          # beyond 2^40: no FP32 screen for this problem
    b[3] = 5.0e13
    lp, res, x, y, z, tr = gpu_solve(A, b, c, engine=S)
    assert res.status == 1 and res.persistent == 2
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr)
    lp.close()
    # tiny entries (below 2^-100) also switch it off
    A2, b2, c2 = lpgen.dense_real_lp(120, 200, 22)
    A2[5, 9] = 1e-40
    lp, res, x, y, z, tr = gpu_solve(A2, b2, c2, engine=S)
    ref = oracle.solve(A2, b2, c2)
    assert res.status == 1 and abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    follow_check(A2, b2, c2, res, tr)
    lp.close()
