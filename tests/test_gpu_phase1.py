"""Phase I on the GPU (b with negative entries; Section 3.4, the two-phase
method with one artificial variable) against the oracle's two-phase solve."""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb  # noqa: F401


@pytest.mark.parametrize("m,n,seed", [(20, 30, 1), (60, 80, 2), (200, 300, 4), (301, 257, 5)])
def test_two_phase_matches_oracle(m, n, seed):
    A, b, c = lpgen.general_lp(m, n, seed)
    assert np.min(b) < 0
    ref = oracle.solve_two_phase(A, b, c)
    assert ref.status == oracle.OPTIMAL
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, trace_cap=1 << 14) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
        tr = lp.trace()
    assert res.status == lpgb.LP_OPTIMAL
    assert res.phase1_iterations == ref.phase1.iterations
    assert bool(res.phase1_exchanged) == ref.exchanged
    assert abs(z - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective))
    assert_certificate(A, b, c, x, y)
    # Phase II, pivot by pivot, from the oracle's own Phase II start
    chk = oracle.solve(A, b, c, start_basis=ref.start_basis, follow=(tr["q"], tr["r"]))
    assert chk.mismatch_at < 0 and chk.status == oracle.OPTIMAL, chk.mismatch_at


def test_infeasible_lp_is_reported():
    from paper_1803_04378_gb300 import lpgb
    for A, b in [(np.array([[1.0, 0.0]]), np.array([-1.0])),
                 (np.array([[1.0, 1.0], [-1.0, -1.0]]), np.array([1.0, -2.0]))]:
        with lpgb.LP(A, b, np.ones(2)) as lp:
            res = lp.solve()
            assert res.status == lpgb.LP_INFEASIBLE and res.phase1_iterations >= 0
            with pytest.raises(lpgb.LPError) as e:
                lp.solution()
            assert e.value.code == lpgb.LP_ERR_STATE


def test_artificial_basic_at_zero_is_exchanged():
    # -x1 <= 0, -x1 <= -1, 3 x1 <= 3, x1 <= 10: the only feasible point is x1 = 1
    A = np.array([[-1.0], [-1.0], [3.0], [1.0]])
    b = np.array([0.0, -1.0, 3.0, 10.0])
    c = np.array([1.0])
    ref = oracle.solve_two_phase(A, b, c)
    assert ref.exchanged
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
    assert res.status == lpgb.LP_OPTIMAL and res.phase1_exchanged == 1
    assert z == pytest.approx(1.0) and x[0] == pytest.approx(1.0)


def test_engines_and_device_inputs_agree():
    import torch
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.general_lp(150, 200, 8)
    out = []
    for engine, dev in ((0, False), (1, False), (0, True)):
        args = (A, b, c) if not dev else tuple(torch.from_numpy(v).cuda() for v in (A, b, c))
        with lpgb.LP(*args, engine=engine) as lp:
            res = lp.solve()
            out.append((res.status, res.phase1_iterations, res.iterations, lp.solution()[2]))
    assert out[0] == out[1] == out[2]


def test_reset_repeats_phase_one():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.general_lp(80, 60, 9)
    with lpgb.LP(A, b, c) as lp:
        r1 = lp.solve()
        z1 = lp.solution()[2]
        lp.reset()
        r2 = lp.solve()
        z2 = lp.solution()[2]
    assert r1.phase1_iterations == r2.phase1_iterations > 0
    assert r1.iterations == r2.iterations and z1 == z2
