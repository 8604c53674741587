"""Sparse FP64 PRICE (price_mode 2: a compressed sparse column copy of A built
on the device) against the oracle and against the dense PRICE (needs a
GB300).  The dot products run over the nonzeros only; every pivot is
checked in follow mode, the objective to 1e-9 and the duality certificate.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate, follow_check, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb  # noqa: F401


@pytest.mark.parametrize("kind,m,n,seed", [("s20", 256, 512, 1), ("s60", 256, 512, 2), ("s60", 300, 200, 3),
                                          ("s20", 129, 257, 4), ("int", 200, 200, 0), ("degenerate", 128, 256, 2)])
@pytest.mark.parametrize("engine", [0, 1])
def test_pivots_match_oracle(kind, m, n, seed, engine):
    A, b, c = lpgen.make(kind, m, n, seed)
    lp, res, x, y, z, tr = gpu_solve(A, b, c, price_mode=2, engine=engine)
    assert res.status == 1 and res.persistent == (1 if engine == 0 else 0)
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    follow_check(A, b, c, res, tr)
    lp.close()


def test_empty_columns_and_rows_and_default_engine():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("s60", 150, 220, 9)
    A[:, 5] = 0.0       # an empty column (never enters: d_5 = c_5 > 0 would make the LP unbounded)
    c[5] = -1.0
    A[7, :] = 0.0       # an empty row
    ref = oracle.solve(A, b, c)
    with lpgb.LP(A, b, c, price_mode=2) as lp:   # the default engine falls back to the dense persistent one
        res = lp.solve()
        x, y, z = lp.solution()
    assert res.status == 1 and res.persistent == 1
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)


def test_same_pivots_as_dense_price_and_update_problem():
    from paper_1803_04378_gb300 import lpgb
    P1 = lpgen.make("s60", 240, 400, 5)
    P2 = lpgen.make("s20", 240, 400, 6)
    runs = []
    for pm in (0, 2):
        with lpgb.LP(*P1, price_mode=pm, engine=0, trace_cap=10000) as lp:
            r1 = lp.solve(); z1 = lp.solution()[2]; t1 = lp.trace()
            lp.update_problem(*P2)   # the sparse copy is rebuilt for the new A
            r2 = lp.solve(); z2 = lp.solution()[2]; t2 = lp.trace()
        runs.append((r1, z1, t1, r2, z2, t2))
    (a1, az1, at1, a2, az2, at2), (b1, bz1, bt1, b2, bz2, bt2) = runs
    assert a1.iterations == b1.iterations and np.array_equal(at1["q"], bt1["q"])
    assert a2.iterations == b2.iterations and np.array_equal(at2["q"], bt2["q"])
    assert abs(az1 - bz1) <= 1e-12 * abs(az1) and abs(az2 - bz2) <= 1e-12 * abs(az2)
    ref = oracle.solve(*P2)
    assert abs(bz2 - ref.objective) <= 1e-9 * abs(ref.objective)
