"""Pins for the oracle's lexicographic ratio rule (the textbook anti-cycling
rule the tabu rule of Sections 2.2 and 3.4 is compared with; no GPU).

* Beale's example cycles under Dantzig's rule with the smallest-index
  tie-break and must terminate at its optimum under the lexicographic rule
  (the rule provably never cycles).
* At the slack basis B^-1 = I, so a tied row i compares as e_i / alpha_i: at
  the first tied column c the row i = c has 1/alpha_c > 0 and every other
  tied row 0 -- the lexicographic choice is the tied row with the largest
  index.  A hand-built LP fixes this (column order and sign of the rule).
* Klee-Minty has no ties: the rule must not change Dantzig's 2^d - 1 pivots.
* Objectives equal brute-force vertex enumeration on small degenerate LPs.
* On the degenerate family every pivot is degenerate; the rule needs neither
  the tabu list nor the Bland safety net.
"""
import json
import os

import numpy as np
import pytest

import lpgen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_beale_terminates_lexicographic():
    g = json.load(open(os.path.join(GOLD, "beale_1955.json")))
    A, b, c = np.array(g["A"]), np.array(g["b"]), np.array(g["c"])
    cyc = oracle.solve(A, b, c, oracle.Options(tabu_tenure=0, bland_after=0, ratio_rule=1, max_iters=60))
    assert cyc.status == oracle.ITER_LIMIT
    s = oracle.solve(A, b, c, oracle.lexicographic_options())
    assert s.status == oracle.OPTIMAL and s.bland_fallbacks == 0 and s.tabu_pushes == 0
    assert s.objective == pytest.approx(g["optimum"], abs=1e-15)
    assert np.allclose(s.x, g["x_opt"], atol=1e-15)


def test_slack_basis_tie_takes_the_last_tied_row():
    # rows 0 and 2 tie at ratio 0 (b = 0) for the entering x0; row 1 has a
    # larger ratio.  Lexicographic: row 2.  Largest pivot: row 0 (alpha 3 > 1).
    A = np.array([[3.0, 1.0], [1.0, 0.0], [1.0, 1.0]])
    b = np.array([0.0, 5.0, 0.0])
    c = np.array([1.0, 0.0])
    lex = oracle.solve(A, b, c, oracle.lexicographic_options(), trace_cap=10)
    big = oracle.solve(A, b, c, oracle.Options(tabu_tenure=0, bland_after=0), trace_cap=10)
    assert lex.trace["q"][0] == 0 and big.trace["q"][0] == 0
    assert lex.trace["r"][0] == 2
    assert big.trace["r"][0] == 0
    assert lex.status == big.status == oracle.OPTIMAL and lex.objective == big.objective == 0.0


def test_klee_minty_unchanged():
    for d in (3, 6, 9):
        A = np.zeros((d, d)); b = np.zeros(d); c = np.zeros(d)
        for i in range(d):
            for j in range(i):
                A[i, j] = 2 * 10.0 ** (i - j)
            A[i, i] = 1.0
            b[i] = 100.0 ** i
            c[i] = 10.0 ** (d - 1 - i)
        s = oracle.solve(A, b, c, oracle.lexicographic_options())
        assert s.status == oracle.OPTIMAL and s.iterations == 2 ** d - 1


def test_brute_force_on_degenerate_tiny():
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(60):
        m = int(rng.integers(2, 5))
        n = int(rng.integers(2, 5))
        A = rng.integers(-2, 6, size=(m, n)).astype(float)
        for j in range(n):
            if np.all(A[:, j] <= 0):
                A[rng.integers(0, m), j] = 1.0
        b = rng.integers(0, 3, size=m).astype(float)  # many zero rows: ties at ratio 0
        c = rng.integers(-1, 5, size=n).astype(float)
        s = oracle.solve(A, b, c, oracle.lexicographic_options())
        if s.status != oracle.OPTIMAL:
            continue
        z_bf, _ = oracle.brute_force(A, b, c)
        assert s.objective == pytest.approx(z_bf, abs=1e-9)
        checked += 1
    assert checked > 40


@pytest.mark.parametrize("m,n,seed", [(128, 256, 2), (256, 512, 2), (96, 200, 11)])
def test_degenerate_family_without_safety_nets(m, n, seed):
    A, b, c = lpgen.degenerate_lp(m, n, seed)
    s = oracle.solve(A, b, c, oracle.lexicographic_options(max_iters=200000))
    assert s.status == oracle.OPTIMAL and s.objective == 0.0
    assert s.bland_fallbacks == 0 and s.tabu_pushes == 0
    assert s.degenerate == s.iterations
    cert = oracle.certificate(A, b, c, s.x, s.y)
    assert cert["dual"] <= 1e-9 and cert["primal"] <= 1e-12


def test_follow_mode_under_the_rule():
    A, b, c = lpgen.degenerate_lp(64, 128, 2)
    o = oracle.lexicographic_options()
    s = oracle.solve(A, b, c, o, trace_cap=100000)
    chk = oracle.solve(A, b, c, o, follow=(s.trace["q"], s.trace["r"]))
    assert chk.mismatch_at < 0 and chk.iterations == s.iterations
    # a planted wrong leaving row among the tied ones is rejected
    t = next(i for i, f in enumerate(s.trace["flags"]) if f & oracle.TF_TIE_SET)
    r_bad = s.trace["r"].copy()
    A2 = A  # same problem
    q = s.trace["q"]
    for cand in range(A.shape[0]):
        if cand == r_bad[t]:
            continue
        r_bad[t] = cand
        chk = oracle.solve(A2, b, c, o, follow=(q, r_bad))
        if chk.mismatch_at == t:
            break
    assert chk.mismatch_at == t
