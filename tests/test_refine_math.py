"""The premises of a reinversion by refinement, checked on the CPU with the
oracle's own updated inverses (no GPU).

After K rank-1 updates from the slack basis (no reinversion), with P the
basis positions of the structural columns J and R the rows whose slack is
nonbasic (both in increasing order):

* the block formula: B^-1[P, R] inverts B11 = A[R, J] and B^-1 is rebuilt from
  it as rows P = [B11^-1 on R | 0] and, for the slack of row s, the row
  [-A[s, J] B11^-1 on R | e_s] -- checked against LAPACK's inverse of the
  whole basis matrix;
* the updated block Y0 = B^-1[P, R] has ||I - B11 Y0||_inf far below the
  2^-26 at which the solver refines, on each of the method's workload
  families and for K up to 192 updates (three reinversion periods);
* one Newton-Schulz step Y0 + Y0 (I - B11 Y0) agrees with LAPACK's inverse of
  B11 to the rounding of the products, and its residual is at least as small
  as that of the updated block.
"""
import numpy as np
import pytest

import lpgen
import oracle

TOL_REFINE = 2.0 ** -26


def _blocks(A, basis):
    m, n = A.shape
    P = np.array([p for p in range(m) if basis[p] < n], dtype=np.int64)
    J = basis[P].astype(np.int64)
    in_basis = np.zeros(n + m, dtype=bool)
    in_basis[basis] = True
    R = np.array([i for i in range(m) if not in_basis[n + i]], dtype=np.int64)
    return P, J, R


def _updated(A, b, c, K):
    s = oracle.solve(A, b, c, oracle.Options(reinvert_every=0, max_iters=K), want_binv=True)
    assert s.iterations == K
    return s.basis.astype(np.int64), s.binv


@pytest.mark.parametrize("kind,m,n,seed,K", [("real", 300, 500, 3, 64), ("real", 300, 500, 3, 192),
                                             ("int", 400, 600, 5, 64), ("degenerate", 128, 256, 2, 192)])
def test_refinement_premises(kind, m, n, seed, K):
    A, b, c = lpgen.make(kind, m, n, seed)
    basis, binv = _updated(A, b, c, K)
    P, J, R = _blocks(A, basis)
    k = len(P)
    assert k == len(R) and k > 0
    B11 = A[np.ix_(R, J)]
    Y0 = binv[np.ix_(P, R)]
    E0 = np.eye(k) - B11 @ Y0
    r0 = np.max(np.sum(np.abs(E0), axis=1))
    assert r0 <= 1e-3 * TOL_REFINE  # the updates leave the block close to B11^-1
    Y1 = Y0 + Y0 @ E0
    fresh = np.linalg.inv(B11)
    scale = max(1.0, np.max(np.abs(fresh)))
    assert np.max(np.abs(Y1 - fresh)) <= 1e-12 * scale
    r1 = np.max(np.sum(np.abs(np.eye(k) - B11 @ Y1), axis=1))
    assert r1 <= max(r0, 1e-13)

    # the block formula rebuilds all of B^-1 from Y1
    B = np.hstack([A, np.eye(m)])[:, basis]
    full = np.zeros((m, m))
    full[np.ix_(P, R)] = Y1
    for p in range(m):
        v = basis[p]
        if v >= n:
            s_row = v - n
            full[p, R] = -A[s_row, J] @ Y1
            full[p, s_row] = 1.0
    ref = np.linalg.inv(B)
    assert np.max(np.abs(full - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(full @ B - np.eye(m))) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_planted_block_error_is_detected():
    """A wrong block (one entry off by 1e-6) shows in the residual above the
    refinement threshold, so it would be eliminated afresh instead."""
    A, b, c = lpgen.make("real", 240, 400, 4)
    basis, binv = _updated(A, b, c, 64)
    P, J, R = _blocks(A, basis)
    B11 = A[np.ix_(R, J)]
    Y0 = binv[np.ix_(P, R)].copy()
    Y0[0, 0] += 1e-6 * max(1.0, abs(Y0[0, 0]))
    r0 = np.max(np.sum(np.abs(np.eye(len(P)) - B11 @ Y0), axis=1))
    assert r0 > TOL_REFINE
