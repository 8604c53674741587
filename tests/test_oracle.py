"""Pins for the CPU oracle against facts fixed by the mathematics and the
textbooks, independent of the oracle's own code (no GPU needed).

What each pin catches:
* brute force / HiGHS / closed forms -- any wrong objective (a dropped term in
  PRICE, a wrong sign in the y or z update, a wrong ratio test);
* Klee-Minty pivot counts -- any deviation from Dantzig's largest-d_j entering
  rule or from the ratio test (the count 2^d - 1 needs every pivot exact);
* Beale's cycle -- the textbook tie-breaks, the tabu/Bland safety nets;
* fresh-inverse comparison -- the Step 8 update of B^-1, bbar, y and z;
* duality certificates -- primal and dual feasibility at every optimum;
* follow mode -- acceptance of tie-equivalent choices and rejection of others.
"""
import json
import os

import numpy as np
import pytest

import lpgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_tiny(rng, m, n, kind):
    if kind == "pos":
        A = rng.integers(1, 10, size=(m, n)).astype(float)
        b = rng.integers(1, 30, size=m).astype(float)
        c = rng.integers(1, 10, size=n).astype(float)
    elif kind == "mixed":
        A = rng.integers(-3, 8, size=(m, n)).astype(float)
        A[:, rng.integers(0, n)] = np.abs(A[:, rng.integers(0, n)]) + 1
        b = rng.integers(0, 20, size=m).astype(float)
        c = rng.integers(-2, 8, size=n).astype(float)
        # keep it bounded: every column has a positive entry
        for j in range(n):
            if np.all(A[:, j] <= 0):
                A[rng.integers(0, m), j] = 1.0
    else:  # real
        A = rng.random((m, n))
        b = rng.random(m) * 5
        c = rng.random(n)
    return A, b, c


@pytest.mark.parametrize("kind", ["pos", "mixed", "real"])
def test_brute_force_tiny(kind):
    rng = np.random.default_rng(123)
    checked = 0
    for trial in range(40):
        m = int(rng.integers(1, 5))
        n = int(rng.integers(1, 5))
        A, b, c = _rand_tiny(rng, m, n, kind)
        z_bf, x_bf = oracle.brute_force(A, b, c)
        s = oracle.solve(A, b, c)
        if s.status == oracle.UNBOUNDED:
            # an unbounded ray must exist: d >= 0, A d <= 0, c.d > 0 (checked by LP below)
            from scipy.optimize import linprog
            r = linprog(-c, A_ub=A, b_ub=b, method="highs")
            assert r.status == 3
            continue
        assert s.status == oracle.OPTIMAL
        assert z_bf is not None
        assert abs(s.objective - z_bf) <= 1e-9 * max(1.0, abs(z_bf))
        cert = oracle.certificate(A, b, c, s.x, s.y)
        assert cert["primal"] <= 1e-9 and cert["dual"] <= 1e-9 and cert["gap"] <= 1e-9
        checked += 1
    assert checked >= 20


def test_closed_form_single_row():
    # m = 1: max c.x s.t. a.x <= b  ->  z* = b * max_j c_j / a_j  (a, c > 0)
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = int(rng.integers(1, 30))
        a = rng.random(n) + 0.1
        c = rng.random(n)
        b = float(rng.random() * 10)
        s = oracle.solve(a[None, :], np.array([b]), c)
        assert s.status == oracle.OPTIMAL
        assert abs(s.objective - b * np.max(c / a)) <= 1e-12 * max(1, b)


def test_closed_form_diagonal():
    # diagonal A: x_i = b_i / a_ii for every c_i > 0, z* = sum c_i b_i / a_ii
    rng = np.random.default_rng(8)
    n = 50
    a = rng.random(n) + 0.5
    b = rng.random(n) * 3
    c = rng.random(n) - 0.3
    s = oracle.solve(np.diag(a), b, c)
    want = float(np.sum(np.where(c > 0, c * b / a, 0.0)))
    assert s.status == oracle.OPTIMAL
    assert abs(s.objective - want) <= 1e-12 * max(1, want)
    assert s.iterations == int(np.sum(c > 1e-9))


def _klee_minty(d):
    A = np.zeros((d, d))
    b = np.zeros(d)
    c = np.zeros(d)
    for i in range(d):
        for j in range(i):
            A[i, j] = 2 * 10.0 ** (i - j)
        A[i, i] = 1.0
        b[i] = 100.0 ** i
        c[i] = 10.0 ** (d - 1 - i)
    return A, b, c


def test_klee_minty_dantzig_pivot_count():
    spec = json.load(open(os.path.join(GOLD, "klee_minty.json")))
    for d in spec["dims"]:
        A, b, c = _klee_minty(d)
        s = oracle.solve(A, b, c)
        assert s.status == oracle.OPTIMAL
        assert s.iterations == 2 ** d - 1, d
        assert s.objective == pytest.approx(100.0 ** (d - 1), rel=1e-12)


def _beale():
    g = json.load(open(os.path.join(GOLD, "beale_1955.json")))
    return np.array(g["A"]), np.array(g["b"]), np.array(g["c"]), g


def test_beale_cycles_under_textbook_rule():
    A, b, c, g = _beale()
    o = oracle.Options(tabu_tenure=0, bland_after=0, ratio_rule=1, max_iters=60)
    s = oracle.solve(A, b, c, o, trace_cap=60)
    assert s.status == oracle.ITER_LIMIT
    assert s.objective == 0.0
    q, r = s.trace["q"], s.trace["r"]
    p = g["cycle_period"]
    assert np.array_equal(q[:p], q[p:2 * p]) and np.array_equal(r[:p], r[p:2 * p])
    # the basis after one period is the slack basis again
    assert sorted(s.basis.tolist()) == [4, 5, 6]


def test_beale_terminates_with_method_rules():
    A, b, c, g = _beale()
    for o in [oracle.Options(),                                    # tabu + largest pivot + Bland net
              oracle.Options(ratio_rule=1, tabu_tenure=0, bland_after=3),  # Bland net alone
              oracle.Options(tabu_tenure=7, bland_after=0)]:        # tabu + largest pivot
        s = oracle.solve(A, b, c, o)
        assert s.status == oracle.OPTIMAL
        assert s.objective == pytest.approx(g["optimum"], abs=1e-15)
        assert np.allclose(s.x, g["x_opt"], atol=1e-15)


def test_tabu_tenure_respected():
    # whenever the tabu rule fires at iteration t on leaving variable v, v does
    # not enter during iterations t+1 .. t+tenure unless the step is flagged
    # as aspiration or Bland
    A, b, c = lpgen.degenerate_lp(128, 256, 2)
    o = oracle.Options(bland_after=0)
    s = oracle.solve(A, b, c, o, trace_cap=100000)
    assert s.status == oracle.OPTIMAL
    m, n = A.shape
    basis = list(range(n, n + m))
    until = {}
    tr = s.trace
    fired = 0
    for t in range(len(tr["q"])):
        q, r, f = int(tr["q"][t]), int(tr["r"][t]), int(tr["flags"][t])
        if q in until and t < until[q]:
            assert f & (oracle.TF_ASPIRATION | oracle.TF_BLAND), (t, q)
        leave = basis[r]
        if f & oracle.TF_TABU_PUSH:
            until[leave] = t + 1 + o.tabu_tenure
            fired += 1
            assert f & (oracle.TF_DEGENERATE | oracle.TF_TIE_SET)
        basis[r] = q
    assert fired > 10
    assert sorted(basis) == sorted(s.basis.tolist())


def test_degenerate_family_needs_anti_cycling():
    # the degenerate family has x = 0 as its only feasible point; every pivot
    # is degenerate and the method must still prove optimality
    A, b, c = lpgen.degenerate_lp(256, 512, 2)
    s = oracle.solve(A, b, c, oracle.Options(max_iters=100000))
    assert s.status == oracle.OPTIMAL and s.objective == 0.0
    assert s.degenerate == s.iterations and s.bland_fallbacks >= 1
    cert = oracle.certificate(A, b, c, s.x, s.y)
    assert cert["dual"] <= 1e-9 and cert["primal"] <= 1e-12


def test_update_matches_fresh_inverse():
    # after K pivots with no reinversion, the updated B^-1, bbar, y, z equal
    # the quantities computed from scratch with LAPACK from the same basis
    A, b, c = lpgen.dense_real_lp(60, 110, 11)
    for K in (1, 7, 40):
        s = oracle.solve(A, b, c, oracle.Options(max_iters=K, reinvert_every=0), want_binv=True)
        assert s.status == oracle.ITER_LIMIT and s.iterations == K
        B = oracle.basis_matrix(A, s.basis)
        Binv = np.linalg.inv(B)
        assert np.max(np.abs(s.binv - Binv)) <= 1e-10 * max(1, np.max(np.abs(Binv)))
        assert np.allclose(s.bbar, Binv @ b, rtol=1e-10, atol=1e-10)
        cB = np.concatenate([c, np.zeros(60)])[s.basis]
        assert np.allclose(s.y, cB @ Binv, rtol=1e-10, atol=1e-12)
        assert s.objective == pytest.approx(float(cB @ (Binv @ b)), rel=1e-12)
        # reduced costs of basic variables vanish
        d = oracle.reduced_costs(A, c, s.y)
        assert np.max(np.abs(d[s.basis])) <= 1e-10


def test_reinversion_does_not_change_nondegenerate_path():
    A, b, c = lpgen.dense_real_lp(120, 200, 12)
    runs = [oracle.solve(A, b, c, oracle.Options(reinvert_every=k), trace_cap=5000) for k in (0, 1, 64)]
    for s in runs:
        assert s.status == oracle.OPTIMAL
    for s in runs[1:]:
        assert np.array_equal(s.trace["q"], runs[0].trace["q"])
        assert np.array_equal(s.trace["r"], runs[0].trace["r"])
        assert s.objective == pytest.approx(runs[0].objective, rel=1e-12)
    assert runs[1].reinversions == runs[1].iterations


def test_gj_inverse_against_lapack():
    rng = np.random.default_rng(3)
    for k in (1, 2, 5, 33):
        M = rng.standard_normal((k, k))
        if k > 1:
            M[0, 0] = 0.0  # forces a row exchange
        inv = oracle.gj_inverse(M)
        assert np.allclose(inv, np.linalg.inv(M), rtol=1e-9, atol=1e-11)
    S = np.ones((3, 3))
    with pytest.raises(np.linalg.LinAlgError):
        oracle.gj_inverse(S)


def test_start_basis_reinverts():
    A, b, c = lpgen.dense_real_lp(80, 150, 13)
    s = oracle.solve(A, b, c)
    warm = oracle.solve(A, b, c, start_basis=s.basis)
    assert warm.status == oracle.OPTIMAL and warm.iterations == 0
    assert warm.objective == pytest.approx(s.objective, rel=1e-12)


def test_highs_crosscheck():
    from scipy.optimize import linprog
    cases = [lpgen.dense_int_lp(200, 200, 0), lpgen.dense_real_lp(300, 600, 1),
             lpgen.degenerate_lp(96, 192, 2)]
    for A, b, c in cases:
        s = oracle.solve(A, b, c)
        r = linprog(-c, A_ub=A, b_ub=b, method="highs")
        assert s.status == oracle.OPTIMAL and r.status == 0
        assert abs(s.objective - (-r.fun)) <= 1e-9 * max(1.0, abs(r.fun))
        cert = oracle.certificate(A, b, c, s.x, s.y)
        assert max(cert["primal"], cert["dual"], cert["gap"], cert["cs"]) <= 1e-9


def test_follow_mode_self_and_planted_mistake():
    A, b, c = lpgen.dense_real_lp(100, 180, 14)
    s = oracle.solve(A, b, c, trace_cap=10000)
    q = np.append(s.trace["q"], -1)
    r = np.append(s.trace["r"], -1)
    f = oracle.solve(A, b, c, follow=(q, r))
    assert f.status == oracle.OPTIMAL and f.adopted == 0 and f.mismatch_at == -1
    # plant a clearly worse entering choice at iteration 5
    q2 = q.copy()
    d_best = s.trace["dq"][5]
    cand = [j for j in range(180) if j != q[5]]
    q2[5] = cand[0]
    g = oracle.solve(A, b, c, follow=(q2, r))
    assert g.status == oracle.MISMATCH and g.mismatch_at == 5 and g.mismatch_kind == 1
    assert d_best > 0
    # plant a wrong leaving row
    r2 = r.copy()
    r2[3] = (r[3] + 1) % 100
    h = oracle.solve(A, b, c, follow=(q, r2))
    assert h.status == oracle.MISMATCH and h.mismatch_at == 3 and h.mismatch_kind == 2


def test_follow_mode_accepts_exact_ties():
    # two identical columns: choosing the higher index is a tie and is accepted
    A = np.array([[1.0, 1.0, 2.0], [3.0, 3.0, 1.0]])
    b = np.array([4.0, 6.0])
    c = np.array([2.0, 2.0, 1.0])
    s = oracle.solve(A, b, c, trace_cap=10)
    assert s.trace["q"][0] == 0
    q = np.append(s.trace["q"], -1)
    r = np.append(s.trace["r"], -1)
    q[0] = 1
    f = oracle.solve(A, b, c, follow=(q, r))
    assert f.status == oracle.OPTIMAL and f.adopted >= 1
    assert f.objective == pytest.approx(s.objective, rel=1e-15)


def test_follow_relaxed_accepts_any_improving_column_only():
    A, b, c = lpgen.dense_real_lp(100, 180, 14)
    s = oracle.solve(A, b, c, trace_cap=10000)
    q = np.append(s.trace["q"], -1)
    r = np.append(s.trace["r"], -1)
    # at pivot 0, y = 0 so d = c: take the second-best column, which improves
    # but is not Dantzig's choice
    order = np.argsort(-c, kind="stable")
    assert order[0] == q[0]
    q2 = q[:1].copy()
    q2[0] = order[1]
    strict = oracle.solve(A, b, c, oracle.Options(max_iters=1), follow=(q2, r[:1]))
    assert strict.status == oracle.MISMATCH and strict.mismatch_kind == 1
    # relaxed: accepted as an entering choice; the leaving row must still be
    # the ratio-test row, which does not depend on c -- take it from a run
    # whose costs make order[1] Dantzig's choice
    c_alt = c.copy()
    c_alt[order[1]] = c[order[0]] + 1.0
    r_alt = oracle.solve(A, b, c_alt, oracle.Options(max_iters=1), trace_cap=1).trace["r"]
    probe = oracle.solve(A, b, c, oracle.Options(max_iters=1, follow_relaxed=1),
                         follow=(q2, r_alt), follow_status=oracle.ITER_LIMIT)
    assert probe.mismatch_at < 0 and probe.adopted >= 1
    wrong_r = np.array([(r_alt[0] + 1) % 100], np.int32)
    probe2 = oracle.solve(A, b, c, oracle.Options(max_iters=1, follow_relaxed=1),
                          follow=(q2, wrong_r), follow_status=oracle.ITER_LIMIT)
    assert probe2.status == oracle.MISMATCH and probe2.mismatch_kind == 2
    # a column with d <= 0 is rejected even when relaxed
    c3 = c.copy()
    c3[5] = -1.0
    s3 = oracle.solve(A, b, c3, trace_cap=2)
    q3 = np.array([5], np.int32)
    bad = oracle.solve(A, b, c3, oracle.Options(max_iters=1, follow_relaxed=1),
                       follow=(q3, np.array([0], np.int32)))
    assert bad.status == oracle.MISMATCH and bad.mismatch_kind == 1


def test_certificate_flags_infeasible_and_suboptimal_points():
    """Negative pins of ``certificate``: it must flag a primal-infeasible x, a
    dual-infeasible y (a violated A^T y >= c, or a negative y_i) and a
    feasible but suboptimal pair, each by the residual that names it."""
    A, b, c = lpgen.dense_real_lp(40, 70, 21)
    s = oracle.solve(A, b, c)
    assert s.status == oracle.OPTIMAL
    ok = oracle.certificate(A, b, c, s.x, s.y)
    assert ok["primal"] <= 1e-12 and ok["dual"] <= 1e-12 and ok["gap"] <= 1e-12
    # primal: push a basic x_j past its row's bound (A x <= b violated)
    j = int(np.argmax(s.x))
    x_bad = s.x.copy()
    x_bad[j] += 2.0 * np.max(b) / max(1e-3, float(np.min(A[A[:, j] > 0, j])))
    assert oracle.certificate(A, b, c, x_bad, s.y)["primal"] > 1e-3
    x_neg = s.x.copy()
    x_neg[j] = -1.0
    assert oracle.certificate(A, b, c, x_neg, s.y)["primal"] >= 1.0 / max(1.0, np.max(b))
    # dual: y = 0 leaves A^T y >= c violated by max c
    d0 = oracle.certificate(A, b, c, s.x, np.zeros_like(s.y))
    assert d0["dual"] >= 0.99 * np.max(c) / max(1.0, np.max(c))
    y_neg = s.y.copy()
    i = int(np.argmax(s.y))
    y_neg[i] = -0.5
    assert oracle.certificate(A, b, c, s.x, y_neg)["dual"] >= 0.5 / max(1.0, np.max(c))
    # gap: x = 0 is feasible but not optimal against the optimal y
    g = oracle.certificate(A, b, c, np.zeros_like(s.x), s.y)
    assert g["primal"] == 0.0 and g["dual"] <= 1e-12 and g["gap"] > 1.0
