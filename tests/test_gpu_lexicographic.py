"""The lexicographic anti-cycling rule on the GPU (LP_ANTICYCLING_LEXICOGRAPHIC)
against the oracle's lexicographic mode, pivot by pivot (needs a GB300).

The tie set, its size and the leaving row are checked by the oracle's follow
mode; a different leaving row is accepted only where the two rows are
lexicographically equal within the follow tolerance in the oracle's own
arithmetic.  Neither the tabu list nor the safety net may fire.
"""
import json
import os

import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate, follow_check, gpu_solve

pytestmark = pytest.mark.gpu

LEX = 1  # LP_ANTICYCLING_LEXICOGRAPHIC


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb  # noqa: F401


@pytest.mark.parametrize("kind,m,n,seed", [("degenerate", 64, 128, 2), ("degenerate", 128, 256, 3),
                                          ("degenerate", 200, 300, 5), ("int", 37, 61, 5),
                                          ("int", 200, 200, 0), ("real", 129, 257, 4)])
def test_pivots_match_oracle(kind, m, n, seed):
    A, b, c = lpgen.make(kind, m, n, seed)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, anticycling=LEX)
    assert res.status == 1 and res.persistent == 0
    assert res.tabu_pushes == 0 and res.bland_fallbacks == 0
    ref = oracle.solve(A, b, c, oracle.lexicographic_options())
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr, oracle.lexicographic_options())
    lp.close()


def test_beale_and_slack_basis_tie():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "beale_1955.json")))
    A, b, c = np.array(g["A"]), np.array(g["b"]), np.array(g["c"])
    lp, res, x, y, z, tr = gpu_solve(A, b, c, anticycling=LEX)
    assert res.status == 1 and z == pytest.approx(g["optimum"], abs=1e-15)
    lp.close()
    # rows 0 and 2 tie at ratio 0: the lexicographic choice is row 2
    A = np.array([[3.0, 1.0], [1.0, 0.0], [1.0, 1.0]])
    b = np.array([0.0, 5.0, 0.0])
    lp, res, x, y, z, tr = gpu_solve(A, b, np.array([1.0, 0.0]), anticycling=LEX)
    assert tr["q"][0] == 0 and tr["r"][0] == 2
    lp.close()


def test_two_phase_lexicographic():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.general_lp(120, 160, 6)
    ref = oracle.solve_two_phase(A, b, c, oracle.lexicographic_options())
    with lpgb.LP(A, b, c, anticycling=LEX) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
    assert res.status == lpgb.LP_OPTIMAL and res.phase1_iterations == ref.phase1.iterations
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
