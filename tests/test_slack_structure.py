"""The slack structure of the explicit inverse, on the CPU (no GPU).

The default engine relies on two facts about Step 8's update of the explicit
B^-1 in IEEE FP64 (rho = B^-1[r,:] / alpha_r, B^-1[i,:] -= alpha_i rho,
y += d_q rho):
  * the column of B^-1 that belongs to a row with a basic slack stays exactly
    the unit vector of that slack's basis position, and
  * y stays exactly zero on those rows,
so that PRICE, FTRAN and UPDATE restricted to the rows whose slack is
nonbasic (slot-ordered, with the moves of the structured engine) reproduce
the dense quantities.  Both are checked pivot by pivot on small LPs of the
three workload families, with the dense and the compact state run in
lockstep.
"""
import numpy as np
import pytest

import lpgen


def _lockstep(A, b, c, max_pivots=400):
    m, n = A.shape
    # dense state
    B = np.eye(m)
    y = np.zeros(m)
    bbar = b.astype(float).copy()
    basis = np.arange(n, n + m)
    pos = -np.ones(n + m, int)
    pos[n:] = np.arange(m)
    # compact state: slots (rows of nonbasic slacks first), live columns
    slot_row = np.arange(m)
    k = 0
    Bp = np.zeros((m, m))
    yp = np.zeros(m)
    events = {"join": 0, "ent": 0}

    def col(j):
        if j < n:
            return A[:, j]
        e = np.zeros(m)
        e[j - n] = 1.0
        return e

    pivots = 0
    while pivots < max_pivots:
        d = np.full(n + m, -np.inf)
        for j in range(n + m):
            if pos[j] < 0:
                d[j] = (c[j] if j < n else 0.0) - y @ col(j)
        # compact PRICE: structural columns over the live rows, slacks of the live rows
        rows = slot_row[:k]
        for j in range(n):
            if pos[j] < 0:
                assert d[j] == pytest.approx(c[j] - yp[:k] @ A[rows, j], rel=1e-12, abs=1e-9)
        for t in range(k):
            assert d[n + rows[t]] == -yp[t]
        q = int(np.argmax(d))
        if d[q] <= 1e-9:
            return pivots, events
        alpha = B @ col(q)
        # compact FTRAN: live columns plus the unit columns of the basic slacks
        if q < n:
            a2 = Bp[:, :k] @ A[rows, q]
            for i in range(m):
                if basis[i] >= n:
                    a2[i] += A[basis[i] - n, q]
        else:
            a2 = Bp[:, list(rows).index(q - n)].copy()
        assert np.allclose(alpha, a2, rtol=1e-12, atol=1e-9)
        ok = alpha > 1e-9
        if not ok.any():
            return pivots, events
        th = np.where(ok, bbar / np.where(ok, alpha, 1.0), np.inf)
        r = int(np.argmin(th))
        ar, dq, theta, leave = alpha[r], d[q], th[r], basis[r]
        # dense Step 8
        rho = B[r] / ar
        for i in range(m):
            if i != r:
                B[i] = B[i] - alpha[i] * rho
        B[r] = rho
        y = y + dq * rho
        bbar = bbar - theta * alpha
        bbar[r] = theta
        pos[leave] = -1
        basis[r] = q
        pos[q] = r
        # compact update: the leaving slack's row joins at slot k (its old
        # column is e_r, rho = 1); the entering slack's column is dropped
        live = list(slot_row[:k])
        newcols = {}
        for t, row in enumerate(live):
            rn = Bp[r, t] / ar
            newcols[row] = (np.where(np.arange(m) == r, rn, Bp[:, t] - alpha * rn), yp[t] + dq * rn)
        if leave >= n:
            events["join"] += 1
            rn = 1.0 / ar
            newcols[leave - n] = (np.where(np.arange(m) == r, rn, 0.0 - alpha * rn), 0.0 + dq * rn)
        if q >= n:
            events["ent"] += 1
            del newcols[q - n]
        R = [i for i in range(m) if pos[n + i] < 0]
        assert sorted(newcols) == R
        k = len(R)
        slot_row = np.array(R + [i for i in range(m) if pos[n + i] >= 0])
        for t, row in enumerate(R):
            Bp[:, t], yp[t] = newcols[row]
        # the facts: exact unit columns and exact zeros of y on the rows of basic slacks
        for s in range(m):
            if pos[n + s] >= 0:
                e = np.zeros(m)
                e[pos[n + s]] = 1.0
                assert np.array_equal(B[:, s], e)
                assert y[s] == 0.0
        assert np.allclose(Bp[:, :k], B[:, R], rtol=1e-12, atol=1e-9)
        assert np.allclose(yp[:k], y[R], rtol=1e-12, atol=1e-12)
        pivots += 1
    return pivots, events


@pytest.mark.parametrize("kind,m,n,seed", [("real", 30, 50, 1), ("int", 25, 40, 2), ("degenerate", 32, 48, 3),
                                          ("degenerate", 40, 70, 5), ("int", 40, 30, 7)])
def test_dense_update_keeps_slack_structure(kind, m, n, seed):
    A, b, c = lpgen.make(kind, m, n, seed)
    pivots, events = _lockstep(A, b, c)
    assert pivots > 0 and events["join"] > 0


def test_slack_reentry_is_exercised():
    # integer and degenerate families make slacks re-enter the basis
    total = 0
    for seed in (2, 3, 5, 7):
        A, b, c = lpgen.make("degenerate", 32, 48, seed)
        total += _lockstep(A, b, c)[1]["ent"]
    assert total > 0
