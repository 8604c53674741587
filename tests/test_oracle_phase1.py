"""Phase I of the oracle (two-phase method with one artificial variable,
Section 3.4 "Finding the initial feasible solution") against brute-force
vertex enumeration, closed forms and an independent HiGHS solve."""
import numpy as np
import pytest

import lpgen
import oracle


def _random_instances(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        m, n = int(rng.integers(2, 6)), int(rng.integers(1, 5))
        A = rng.integers(-4, 6, (m, n)).astype(float)
        b = rng.integers(-4, 8, m).astype(float)
        if b.min() >= 0:
            continue
        c = rng.integers(1, 6, n).astype(float)
        # a bounding row keeps every objective finite
        out.append((np.vstack([A, np.ones((1, n))]), np.concatenate([b, [12.0]]), c))
    return out


def test_two_phase_matches_brute_force():
    feasible = infeasible = 0
    for A, b, c in _random_instances(60, 7):
        r = oracle.solve_two_phase(A, b, c)
        z, _ = oracle.brute_force(A, b, c)
        if z is None:
            assert r.status == oracle.INFEASIBLE
            infeasible += 1
        else:
            assert r.status == oracle.OPTIMAL
            assert abs(r.objective - z) <= 1e-9 * max(1.0, abs(z))
            cert = oracle.certificate(A, b, c, r.x, r.y)
            assert cert["primal"] <= 1e-9 and cert["dual"] <= 1e-9 and cert["gap"] <= 1e-9
            feasible += 1
    assert feasible >= 20 and infeasible >= 3


def test_general_lp_family_is_feasible_and_needs_phase_one():
    for (m, n, s) in [(5, 4, 1), (8, 6, 2), (6, 7, 3)]:
        A, b, c = lpgen.general_lp(m, n, s)
        assert np.min(b) < 0
        r = oracle.solve_two_phase(A, b, c)
        z, _ = oracle.brute_force(A, b, c)
        assert r.status == oracle.OPTIMAL and abs(r.objective - z) <= 1e-9 * max(1.0, abs(z))


def test_infeasible_systems():
    # x1 <= -1 with x >= 0
    r = oracle.solve_two_phase(np.array([[1.0, 0.0]]), np.array([-1.0]), np.array([1.0, 1.0]))
    assert r.status == oracle.INFEASIBLE
    # x1 + x2 <= 1 and x1 + x2 >= 2
    r = oracle.solve_two_phase(np.array([[1.0, 1.0], [-1.0, -1.0]]), np.array([1.0, -2.0]), np.array([1.0, 1.0]))
    assert r.status == oracle.INFEASIBLE
    assert r.phase1.objective == pytest.approx(-1.0, abs=1e-12)  # the smallest x0 is the gap 2 - 1


def test_auxiliary_start_is_feasible_in_closed_form():
    A, b, c = lpgen.general_lp(30, 20, 5)
    A_aux, c_aux, start = oracle.auxiliary_problem(A, b)
    m, n = A.shape
    xb = np.linalg.solve(oracle.basis_matrix(A_aux, start), b)
    istar = int(np.argmin(b))
    assert xb[istar] == pytest.approx(-b[istar])  # x0 = -min b
    neg = b < 0
    assert np.allclose(xb[~neg], b[~neg]) and np.all(xb >= -1e-12)
    others = neg.copy()
    others[istar] = False
    assert np.allclose(xb[others], b[others] - b[istar])


def test_artificial_left_basic_at_zero_is_exchanged():
    # -x1 <= 0, -x1 <= -1, 3 x1 <= 3, x1 <= 10: the only feasible point is x1 = 1
    A = np.array([[-1.0], [-1.0], [3.0], [1.0]])
    b = np.array([0.0, -1.0, 3.0, 10.0])
    r = oracle.solve_two_phase(A, b, np.array([1.0]))
    assert r.exchanged and r.status == oracle.OPTIMAL
    assert r.objective == pytest.approx(1.0) and r.x[0] == pytest.approx(1.0)
    B = oracle.basis_matrix(A, r.start_basis)
    assert abs(np.linalg.det(B)) > 1e-12
    assert np.all(np.linalg.solve(B, b) >= -1e-12)


def test_nonnegative_b_is_the_plain_method():
    A, b, c = lpgen.dense_int_lp(30, 40, 3)
    r = oracle.solve_two_phase(A, b, c)
    s = oracle.solve(A, b, c)
    assert r.phase1 is None and r.status == s.status and r.objective == s.objective
    assert np.array_equal(r.basis, s.basis)


def test_two_phase_against_highs():
    linprog = pytest.importorskip("scipy.optimize").linprog
    for (m, n, s) in [(40, 60, 11), (80, 50, 12)]:
        A, b, c = lpgen.general_lp(m, n, s)
        r = oracle.solve_two_phase(A, b, c)
        h = linprog(-c, A_ub=A, b_ub=b, bounds=[(0, None)] * n, method="highs")
        assert h.status == 0 and r.status == oracle.OPTIMAL
        assert abs(r.objective - (-h.fun)) <= 1e-9 * max(1.0, abs(h.fun))
