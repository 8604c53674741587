"""Reinversion by refinement (lp_options.reinvert_refine): one Newton-Schulz
step Y + Y (I - B11 Y) of the updated inverse in place of a fresh Gauss-Jordan
elimination of B11 (needs a GB300).

* On every engine, every periodic reinversion of a well-conditioned solve is
  refined: the stored inverse must be that of the current basis (the engines
  apply the last pivot's update before they stop for the reinversion), else
  its residual is large and the elimination runs instead.
* The refined solve makes the same pivots, reaches the same optimum and keeps
  the same counters as the one with eliminations; the oracle follows it pivot
  by pivot.
* B^-1 right after a refined reinversion agrees with the oracle's fresh
  inverse of the same basis element by element, and B^-1 B = I.
* With set_basis (no updated inverse to refine) the elimination runs.
* refine_tol = 0: every residual is computed and rejected, and the
  elimination that follows gives a run identical, bit for bit, to one without
  refinement (the fallback path leaves nothing behind).
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


@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("kind,m,n,seed,every", [("real", 300, 500, 31, 16), ("int", 200, 300, 7, 8)])
def test_periodic_reinversions_refined(engine, kind, m, n, seed, every):
    A, b, c = lpgen.make(kind, m, n, seed)
    lp1, r1, x1, y1, z1, t1 = gpu_solve(A, b, c, engine=engine, reinvert_every=every)
    lp0, r0, x0, y0, z0, t0 = gpu_solve(A, b, c, engine=engine, reinvert_every=every, reinvert_refine=0)
    assert r1.status == r0.status == 1
    assert r1.reinversions >= 3 and r1.refined_reinversions == r1.reinversions
    assert r0.refined_reinversions == 0
    assert r1.iterations == r0.iterations and r1.reinversions == r0.reinversions
    assert np.array_equal(t1["q"], t0["q"]) and np.array_equal(t1["r"], t0["r"])
    assert abs(z1 - z0) <= 1e-12 * max(1.0, abs(z0))
    assert np.max(np.abs(x1 - x0)) <= 1e-9 * max(1.0, np.max(np.abs(x0)))
    assert_certificate(A, b, c, x1, y1)
    follow_check(A, b, c, r1, t1, oracle.Options(reinvert_every=every))
    lp1.close()
    lp0.close()


@pytest.mark.parametrize("engine", [0, 2])
def test_refined_inverse_elementwise(engine):
    """Stop right after the reinversion at pivot 48 (iteration limit 48 with a
    period of 16): B^-1 is the refined one."""
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_real_lp(260, 400, 9)
    m = A.shape[0]
    with lpgb.LP(A, b, c, engine=engine, reinvert_every=16, max_iters=48) as lp:
        res = lp.solve()
        assert res.status == lpgb.LP_ITER_LIMIT and res.iterations == 48
        assert res.reinversions == 3 and res.refined_reinversions == 3
        binv, bbar = lp.state()
        basis = lp.basis()
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=0), start_basis=basis, want_binv=True)
    scale = max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(binv - ref.binv)) <= 1e-10 * scale
    assert np.max(np.abs(bbar - ref.bbar)) <= 1e-10 * max(1.0, np.max(np.abs(ref.bbar)))
    B = np.hstack([A, np.eye(m)])[:, basis]
    assert np.max(np.abs(binv @ B - np.eye(m))) <= 1e-10 * scale


def test_set_basis_eliminates():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_real_lp(180, 300, 22)
    ref_full = oracle.solve(A, b, c)
    mid = oracle.solve(A, b, c, oracle.Options(max_iters=ref_full.iterations // 2))
    with lpgb.LP(A, b, c, max_iters=0) as lp:
        lp.set_basis(mid.basis)
        res = lp.solve()
        assert res.reinversions == 1 and res.refined_reinversions == 0


@pytest.mark.parametrize("engine", [0, 1, 2])
def test_rejected_refinement_falls_back(engine):
    A, b, c = lpgen.dense_real_lp(300, 500, 31)
    lp1, r1, x1, y1, z1, t1 = gpu_solve(A, b, c, engine=engine, reinvert_every=16, refine_tol=0.0)
    lp0, r0, x0, y0, z0, t0 = gpu_solve(A, b, c, engine=engine, reinvert_every=16, reinvert_refine=0)
    assert r1.status == r0.status == 1 and r1.reinversions >= 3
    assert r1.refined_reinversions == 0 and r1.refine_residual_max > 0.0
    assert r0.refine_residual_max == 0.0
    assert np.array_equal(t1["q"], t0["q"]) and np.array_equal(t1["r"], t0["r"])
    assert z1 == z0 and np.array_equal(x1, x0) and np.array_equal(y1, y0)
    lp1.close()
    lp0.close()


def test_option_validated():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.dense_int_lp(20, 30, 0)
    with pytest.raises(lpgb.LPError):
        lpgb.LP(A, b, c, reinvert_refine=2)
    with pytest.raises(lpgb.LPError):
        lpgb.LP(A, b, c, refine_tol=1e-6)
    with pytest.raises(lpgb.LPError):
        lpgb.LP(A, b, c, refine_tol=-1.0)
