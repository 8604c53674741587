"""The OpenMP build of the oracle (used to write the full-size golden files
and for the all-cores CPU figure) against the serial build: every output
element is summed by one thread in the serial order, so the pivot sequences,
margins, solutions and inverses must be identical bit for bit."""
import numpy as np
import pytest

import lpgen
import oracle


@pytest.mark.parametrize("kind,m,n,seed,iters", [
    ("real", 260, 470, 3, 10**6),        # several reinversions, to optimality
    ("degenerate", 150, 300, 4, 10**6),  # ties, tabu pushes, Bland net
    ("int", 200, 200, 0, 10**6),
])
def test_openmp_build_is_bit_identical(kind, m, n, seed, iters):
    A, b, c = lpgen.make(kind, m, n, seed)
    opts = oracle.Options(max_iters=iters, reinvert_every=16)
    s1 = oracle.solve(A, b, c, opts, trace_cap=1 << 20, want_binv=True, threads=1)
    s4 = oracle.solve(A, b, c, opts, trace_cap=1 << 20, want_binv=True, threads=4)
    assert oracle.threads_used(4) == 4 and oracle.threads_used(1) == 1
    assert s1.status == s4.status and s1.iterations == s4.iterations
    assert s1.reinversions == s4.reinversions and s1.reinversions >= 1
    assert s1.objective == s4.objective
    for key in ("q", "r", "flags", "theta", "dq", "margin_q", "margin_r"):
        assert np.array_equal(s1.trace[key], s4.trace[key]), key
    for a, b_ in ((s1.x, s4.x), (s1.y, s4.y), (s1.bbar, s4.bbar), (s1.binv, s4.binv)):
        assert np.array_equal(a, b_)
    # the parallel PRICE and Gauss-Jordan on their own
    y = np.random.default_rng(seed).random(m)
    assert np.array_equal(oracle.reduced_costs(A, c, y), oracle.reduced_costs(A, c, y, threads=4))
    B = oracle.basis_matrix(A, s1.basis)
    assert np.array_equal(oracle.gj_inverse(B), oracle.gj_inverse(B, threads=4))
