"""Edge values on the default engine (needs a GB300).

* Scaling b by 2^16 scales x, bbar, every ratio of the ratio test and z by
  exactly 2^16 and leaves y, d and alpha unchanged: every operation on
  them is exact under a power-of-two scale.  On the dense real family no
  ratio is near a tie or the degeneracy tolerance, so the pivots must be the
  same as the unscaled problem's and x, z exactly 2^16 times its values.  (A
  scale of A, by contrast, is not exact: the slack columns stay the identity,
  so the slacks' reduced costs scale against the structurals' and the
  absolute optimality tolerance sees different values.)
* A column whose entries are subnormal: its FTRAN partial sums are subnormal
  and take the FP64 warp sum instead of the fixed-point one, and its largest
  alpha stays below tol_piv, so the method stops unbounded along it.  The
  oracle, in plain FP64, must agree pivot by pivot.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import follow_check, gpu_solve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,seed", [(300, 500, 21), (1000, 1800, 22)])
def test_power_of_two_scale_of_b_is_exact(m, n, seed):
    A, b, c = lpgen.make("real", m, n, seed)
    s = 2.0 ** 16
    lp0, r0, x0, y0, z0, t0 = gpu_solve(A, b, c)
    lp1, r1, x1, y1, z1, t1 = gpu_solve(A, b * s, c)
    assert r0.status == r1.status == 1
    assert r0.persistent == r1.persistent == 2 and r0.reinversions >= 2
    assert np.array_equal(t0["q"], t1["q"]) and np.array_equal(t0["r"], t1["r"])
    assert z1 == z0 * s and np.array_equal(x1, x0 * s)
    assert np.array_equal(y1, y0)
    lp0.close()
    lp1.close()


def test_subnormal_column_is_unbounded_like_the_oracle():
    m, n = 64, 96
    A, b, c = lpgen.make("real", m, n, 23)
    A = A.copy()
    c = c.copy()
    A[:, 7] = 4.0e-310 * (1.0 + np.arange(m) / m)  # subnormal entries
    c[7] = 50.0                                    # the largest reduced cost at the slack basis
    lp, res, x, y, z, tr = gpu_solve(A, b, c)
    ref = oracle.solve(A, b, c)
    assert ref.status == oracle.UNBOUNDED
    assert res.status == 2  # LP_UNBOUNDED
    follow_check(A, b, c, res, tr)
    lp.close()
