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


ENGINES = {"structured": (2, 2), "graph": (1, 0)}  # lp_options.engine, lp_result.persistent


@pytest.mark.parametrize("engine", ["structured", "graph"])
@pytest.mark.parametrize("kind,m,n,seed", [("degenerate", 64, 128, 2), ("degenerate", 128, 256, 3),
                                          ("degenerate", 200, 300, 5), ("int", 37, 61, 5),
                                          ("int", 200, 200, 0), ("real", 129, 257, 4),
                                          ("degenerate", 700, 900, 6)])
def test_pivots_match_oracle(kind, m, n, seed, engine):
    A, b, c = lpgen.make(kind, m, n, seed)
    eng, persistent = ENGINES[engine]
    lp, res, x, y, z, tr = gpu_solve(A, b, c, anticycling=LEX, engine=eng, reinvert_every=32)
    assert res.status == 1 and res.persistent == persistent and res.engine_reason == 0
    assert res.tabu_pushes == 0 and res.bland_fallbacks == 0
    opts = oracle.lexicographic_options()
    opts.reinvert_every = 32
    ref = oracle.solve(A, b, c, opts)
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr, opts)
    lp.close()


def test_structured_engine_equals_graph_engine_on_the_degenerate_workload():
    """2048 x 4096, integer A in -5..10, 30% of b_i = 0: every pivot is
    degenerate.  Both engines make the same pivots under the lexicographic
    rule; the oracle follows the structured engine's first 96 of them."""
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("degenerate", 2048, 4096, 2)
    out = {}
    for engine in ("structured", "graph"):
        eng, persistent = ENGINES[engine]
        lp, res, x, y, z, tr = gpu_solve(A, b, c, anticycling=LEX, engine=eng)
        assert res.status == lpgb.LP_OPTIMAL and res.persistent == persistent
        assert res.tabu_pushes == 0 and res.bland_fallbacks == 0
        out[engine] = (res, tr, z)
        lp.close()
    rs, ts, zs = out["structured"]
    rg, tg, zg = out["graph"]
    assert rs.iterations == rg.iterations and np.array_equal(ts["q"], tg["q"]) and np.array_equal(ts["r"], tg["r"])
    assert abs(zs) <= 1e-9 and abs(zg) <= 1e-9
    K = 96
    chk = oracle.solve(A, b, c, oracle.lexicographic_options(max_iters=K), follow=(ts["q"][:K], ts["r"][:K]),
                       follow_status=lpgb.LP_ITER_LIMIT, threads=0)
    assert chk.mismatch_at < 0 and chk.iterations == min(K, rs.iterations), (chk.mismatch_at, chk.iterations)


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
