"""Case 2 of Section 3 (Figure 4): the explicit inverse exceeds the device
memory granted to it (lp_options.tableau_budget_mb) and streams through the
device in blocks of consecutive rows every pivot.

The blocks run the per-row arithmetic of the captured-graph engine's UPDATE,
and PRICE, the ratio test and the pivot bookkeeping are its kernels, so the
out-of-core solve must equal the captured-graph solve bit for bit: the same
pivot sequence, x, y, objective and B^-1 (read back after a stop at an
iteration limit inside a reinversion period, which checks that the block left
on the device goes back to host memory).  The oracle follows the out-of-core
pivots one by one.  Budgets give 3 to 10 blocks, some with a ragged last block,
reinversions every 8 or 16 pivots, a Phase I solve; a budget that holds the
inverse keeps it resident.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import follow_check

pytestmark = pytest.mark.gpu


def _mb(m):
    """The inverse's size in MB at row stride ld (m rounded up to 64)."""
    ld = (m + 63) // 64 * 64
    return 8.0 * m * ld / 1e6


def _run(A, b, c, **opts):
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, trace_cap=1 << 16, **opts) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
        binv, bbar = lp.state()
        tr = lp.trace()
    return res, x, y, z, binv, bbar, tr


@pytest.mark.parametrize("kind,m,n,seed,frac,reinv", [
    ("real", 300, 500, 11, 0.4, 64),      # 10 blocks of 30 rows
    ("int", 200, 200, 0, 0.5, 8),         # 8 blocks, a reinversion every 8 pivots
    ("degenerate", 150, 300, 4, 0.9, 16), # 5 blocks, the last of 18 rows; ties, tabu, the Bland net
    ("real", 257, 300, 12, 1.5, 16),      # 3 blocks of 96 rows, the last of 65
])
def test_out_of_core_equals_resident_solve(kind, m, n, seed, frac, reinv):
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make(kind, m, n, seed)
    budget = frac * _mb(m) / 2.0 if frac < 1.0 else _mb(m) * 0.75
    ro, xo, yo, zo, Bo, bo, to = _run(A, b, c, tableau_budget_mb=budget, reinvert_every=reinv)
    rg, xg, yg, zg, Bg, bg, tg = _run(A, b, c, engine=lpgb.LP_ENGINE_GRAPH, reinvert_every=reinv)
    assert ro.engine_reason == lpgb.LP_ENGINE_REASON_OUT_OF_CORE and ro.persistent == 0
    assert ro.ooc_blocks >= 2 and ro.ooc_block_rows * (ro.ooc_blocks - 1) < m <= ro.ooc_block_rows * ro.ooc_blocks
    assert ro.ooc_bytes > 0 and rg.ooc_blocks == 0
    assert ro.status == rg.status == lpgb.LP_OPTIMAL
    assert ro.iterations == rg.iterations and ro.reinversions == rg.reinversions
    assert np.array_equal(to["q"], tg["q"]) and np.array_equal(to["r"], tg["r"])
    assert zo == zg and np.array_equal(xo, xg) and np.array_equal(yo, yg)
    assert np.array_equal(Bo, Bg) and np.array_equal(bo, bg)
    follow_check(A, b, c, ro, to, oracle.Options(reinvert_every=reinv))


def test_out_of_core_stop_inside_a_period_reads_back_the_inverse():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("real", 240, 400, 13)
    budget = _mb(240) / 5.0
    ro, xo, yo, zo, Bo, bo, to = _run(A, b, c, tableau_budget_mb=budget, reinvert_every=16, max_iters=37)
    rg, xg, yg, zg, Bg, bg, tg = _run(A, b, c, engine=lpgb.LP_ENGINE_GRAPH, reinvert_every=16, max_iters=37)
    assert ro.status == rg.status == lpgb.LP_ITER_LIMIT and ro.iterations == 37
    assert ro.ooc_blocks >= 2
    assert np.array_equal(Bo, Bg) and np.array_equal(bo, bg) and np.array_equal(yo, yg)
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=37, reinvert_every=16), want_binv=True)
    assert np.array_equal(lpgb_basis(A, b, c, budget), ref.basis)
    assert np.max(np.abs(Bo - ref.binv)) <= 1e-9 * max(1.0, np.max(np.abs(ref.binv)))


def lpgb_basis(A, b, c, budget):
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, tableau_budget_mb=budget, reinvert_every=16, max_iters=37) as lp:
        lp.solve()
        return lp.basis()


def test_out_of_core_phase1():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.general_lp(120, 160, 5)
    assert np.min(b) < 0
    ro, xo, yo, zo, _, _, _ = _run(A, b, c, tableau_budget_mb=_mb(120) / 3.0)
    rg, xg, yg, zg, _, _, _ = _run(A, b, c, engine=lpgb.LP_ENGINE_GRAPH)
    assert ro.status == rg.status == lpgb.LP_OPTIMAL and ro.ooc_blocks >= 2
    assert zo == zg and ro.phase1_iterations == rg.phase1_iterations
    ref = oracle.solve_two_phase(A, b, c)
    assert zo == pytest.approx(ref.objective, rel=1e-9)


def test_budget_that_fits_keeps_the_inverse_resident_and_lexicographic_is_refused():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("real", 100, 150, 2)
    with lpgb.LP(A, b, c, tableau_budget_mb=2 * _mb(100)) as lp:
        r = lp.solve()
    assert r.ooc_blocks == 0 and r.engine_reason == lpgb.LP_ENGINE_REASON_NONE
    with pytest.raises(Exception):
        lpgb.LP(A, b, c, tableau_budget_mb=_mb(100) / 4.0, anticycling=lpgb.LP_ANTICYCLING_LEXICOGRAPHIC)
