"""The structural-block form of B^-1 on the CPU (no GPU): only W = B^-1[P, R]
is kept (P: basis positions of the structural columns J, R: rows whose slack
is nonbasic, both in insertion order), and every quantity of an iteration
comes from W and A:

    alpha_P = W a_q[R],  alpha_S = a_q[S] - A[S, J] alpha_P
    rho_R   = W[r, :]                 (a structural column leaves)
            = -A[s, J] W              (the slack of row s leaves)

and W follows each pivot by one of four exchanges (structural or slack
entering, structural or slack leaving), growing or shrinking by one row and
column when a slack leaves or enters.  The oracle's pivot sequences are
replayed twice, once with a dense B^-1 and once with W alone; alpha, rho and
W must agree with the dense replay at every pivot, and all four exchanges
must occur.
"""
import numpy as np
import pytest

import lpgen
import oracle


def _replay(A, b, c, q_seq, r_seq):
    m, n = A.shape
    basis = list(range(n, n + m))
    Binv = np.eye(m)
    P, R = [], []          # W rows: positions of structural basics; W columns: rows of nonbasic slacks
    W = np.zeros((0, 0))
    cases = {"struct-struct": 0, "struct-for-slack": 0, "slack-for-struct": 0, "slack-slack": 0}
    worst = 0.0
    for q, r in zip(q_seq, r_seq):
        if q < 0:
            break
        aq = A[:, q] if q < n else np.eye(m)[:, q - n]
        alpha = Binv @ aq
        S = [i for i in range(m) if i not in R]
        J = [basis[p] for p in P]
        # alpha from W and A
        alpha_P = W @ aq[R] if P else np.zeros(0)
        alpha_w = np.zeros(m)
        alpha_w[P] = alpha_P
        if S:
            ex = A[np.ix_(S, J)] @ alpha_P if P else np.zeros(len(S))
            # a basic slack of row s sits at the position that holds it
            for t, s_row in enumerate(S):
                pos = basis.index(n + s_row)
                alpha_w[pos] = aq[s_row] - ex[t]
        worst = max(worst, np.max(np.abs(alpha_w - alpha)) / max(1.0, np.max(np.abs(alpha))))
        ar = alpha[r]
        leave = basis[r]
        # rho on the R columns from W and A
        if leave < n:
            rho_R = W[P.index(r), :].copy()
        else:
            s_out = leave - n
            rho_R = -A[s_out, J] @ W if P else np.zeros(0)
        worst = max(worst, np.max(np.abs(rho_R - Binv[r, R]), initial=0.0) / max(1.0, np.max(np.abs(Binv[r]))))
        # W after the exchange
        if q < n and leave < n:
            cases["struct-struct"] += 1
            i = P.index(r)
            W = W - np.outer(alpha_P, rho_R) / ar
            W[i, :] = rho_R / ar
        elif q < n:  # the slack of row s_out leaves: position r joins P, row s_out joins R
            cases["struct-for-slack"] += 1
            s_out = leave - n
            k = len(P)
            W2 = np.zeros((k + 1, k + 1))
            W2[:k, :k] = W - np.outer(alpha_P, rho_R) / ar
            W2[:k, k] = -alpha_P / ar
            W2[k, :k] = rho_R / ar
            W2[k, k] = 1.0 / ar
            W = W2
            P.append(r)
            R.append(s_out)
        else:
            s_in = q - n
            a_in = R.index(s_in)
            Wn = W - np.outer(alpha_P, rho_R) / ar
            keep_c = [a for a in range(len(R)) if a != a_in]
            if leave < n:  # slack enters for a structural column: position r leaves P
                cases["slack-for-struct"] += 1
                i = P.index(r)
                keep_r = [x for x in range(len(P)) if x != i]
                W = Wn[np.ix_(keep_r, keep_c)]
                del P[i]
                del R[a_in]
            else:  # slack for slack: row s_in leaves R, row s_out joins it
                cases["slack-slack"] += 1
                s_out = leave - n
                W = np.hstack([Wn[:, keep_c], (-alpha_P / ar)[:, None]])
                del R[a_in]
                R.append(s_out)
        # the dense update (Step 8) and the basis exchange
        rho = Binv[r, :] / ar
        Binv = Binv - np.outer(alpha, rho)
        Binv[r, :] = rho
        basis[r] = q
        if P:
            worst = max(worst, np.max(np.abs(W - Binv[np.ix_(P, R)])) / max(1.0, np.max(np.abs(Binv))))
        assert sorted(P) == [p for p in range(m) if basis[p] < n]
        assert sorted(R) == [i for i in range(m) if (n + i) not in basis]
    return cases, worst


CASES = [("real", 120, 200, 3), ("degenerate", 48, 96, 5), ("int", 100, 160, 1)]


@pytest.mark.parametrize("kind,m,n,seed", CASES)
def test_structural_block_follows_the_dense_inverse(kind, m, n, seed):
    A, b, c = lpgen.make(kind, m, n, seed)
    s = oracle.solve(A, b, c, trace_cap=100000)
    assert s.status == oracle.OPTIMAL
    cases, worst = _replay(A, b, c, s.trace["q"], s.trace["r"])
    assert worst <= 1e-10, worst
    assert cases["struct-for-slack"] > 0


def test_all_four_exchanges_occur():
    """Slacks re-enter the basis on these paths, so each of the four exchange
    types is exercised (the real and degenerate replays have all four)."""
    seen = {}
    for kind, m, n, seed in CASES:
        A, b, c = lpgen.make(kind, m, n, seed)
        s = oracle.solve(A, b, c, trace_cap=100000)
        cases, _ = _replay(A, b, c, s.trace["q"], s.trace["r"])
        for key, v in cases.items():
            seen[key] = seen.get(key, 0) + v
    assert all(v > 0 for v in seen.values()), seen
