"""The warm-start repair of lp_set_basis_repair and the crash of
lp_set_crash, pivot by pivot.

The repair rule written out plainly in numpy (FP64, B^-1 from a fresh
inverse every pivot): while some basic value is below -1e-9 max(1, max|b|),
the most negative position p leaves (ties: the smallest position) and the
nonbasic slack s with the most negative B^-1[p][s] enters (ties: the
smallest s).  The device runs the repair in batches of pivots whose outcome
the host reads once per batch; the sequence, the count, the cap (a proposal
still infeasible after max_repairs falls back to the slack basis) and the
reinversions falling inside a batch must not change any of it.
"""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate

pytestmark = pytest.mark.gpu


def repair_reference(A, b, basis, cap):
    m, n = A.shape
    AI = np.hstack([A, np.eye(m)])
    basis = np.array(basis, dtype=np.int64)
    tol = 1e-9 * max(1.0, float(np.max(np.abs(b))))
    seq = []
    while True:
        Binv = np.linalg.inv(AI[:, basis])
        bbar = Binv @ b
        neg = np.nonzero(bbar < -tol)[0]
        if len(neg) == 0:
            return seq, "feasible"
        if len(seq) >= cap:
            return seq, "cap"
        p = int(neg[np.argmin(bbar[neg])])
        inb = set(basis.tolist())
        nb = np.array([s for s in range(m) if n + s not in inb])
        row = Binv[p, nb]
        k = int(np.argmin(row))
        if row[k] >= 0.0:
            return seq, "stuck"
        seq.append((n + int(nb[k]), p))
        basis[p] = n + int(nb[k])


def _proposal(A, b, c, seed):
    """The neighbour's optimal basis with a few structurals swapped: an
    infeasible proposal that needs tens of repair pivots."""
    m, n = A.shape
    base_basis = oracle.solve(A, b, c).basis.copy()
    rng = np.random.default_rng(seed)
    spos = np.nonzero(base_basis < n)[0]
    nonb = np.setdiff1d(np.arange(n), base_basis)
    pos = rng.choice(spos, min(6, len(spos)), replace=False)
    base_basis[pos] = rng.choice(nonb, len(pos), replace=False)
    return base_basis


@pytest.mark.parametrize("m,n,seed,reinv", [(120, 200, 1, 8), (257, 300, 2, 64), (96, 192, 3, 5)])
def test_repair_sequence_matches_rule(m, n, seed, reinv):
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(m, n, 40 + seed)
    A, b, c = lpgen.perturbed_lp(base, seed)
    prop = _proposal(*base, seed)
    seq, outcome = repair_reference(A, b, prop, m)
    assert outcome == "feasible" and len(seq) > 0
    with lpgb.LP(A, b, c, trace_cap=1 << 14, reinvert_every=reinv) as lp:
        lp.set_basis_repair(prop, m)
        res = lp.solve()
        tr = lp.trace()
        x, y, z = lp.solution()
    assert res.warm_fallback == 0 and res.warm_repairs == len(seq), (res.warm_repairs, len(seq))
    got = list(zip(tr["q"][:len(seq)].tolist(), tr["r"][:len(seq)].tolist()))
    assert got == seq
    assert res.status == lpgb.LP_OPTIMAL
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert_certificate(A, b, c, x, y)


def test_repair_cap_falls_back_and_exact_cap_succeeds():
    from paper_1803_04378_gb300 import lpgb
    m, n = 150, 260
    base = lpgen.dense_real_lp(m, n, 47)
    A, b, c = lpgen.perturbed_lp(base, 9)
    prop = _proposal(*base, 9)
    seq, outcome = repair_reference(A, b, prop, m)
    need = len(seq)
    assert outcome == "feasible" and need >= 2
    with lpgb.LP(A, b, c, trace_cap=1 << 14, reinvert_every=16) as lp:
        cold = lp.solve()
        zc = lp.solution()[2]
        for cap, fallback in ((need - 1, 1), (need, 0), (0, 1), (need + 40, 0)):
            lp.reset()
            lp.set_basis_repair(prop, cap)
            r = lp.solve()
            assert r.warm_fallback == fallback, (cap, r.warm_fallback)
            assert r.status == lpgb.LP_OPTIMAL and abs(lp.solution()[2] - zc) <= 1e-9 * abs(zc)
            if fallback:
                # the repair pivots are dropped with the proposal: the cold path from the slack basis
                assert r.iterations == cold.iterations
            else:
                assert r.warm_repairs == need


def crash_reference(A, b, order):
    """The crash written out plainly: from the slack basis, each listed
    structural that is not basic enters by the ratio test of Step 6 (alpha_i >
    1e-9; the tie set within 1e-12 relative of the smallest ratio; the largest
    alpha, then the smallest basic index), unless its column has no alpha_i
    > 1e-9 or a structural would leave."""
    m, n = A.shape
    AI = np.hstack([A, np.eye(m)])
    basis = np.arange(n, n + m)
    seq = []
    for j in order:
        if j in set(basis.tolist()):
            continue
        Binv = np.linalg.inv(AI[:, basis])
        bbar = Binv @ b
        al = Binv @ AI[:, j]
        R = np.nonzero(al > 1e-9)[0]
        if len(R) == 0:
            continue
        th = bbar[R] / al[R]
        tmin = th.min()
        T = R[th <= tmin + 1e-12 * max(1.0, abs(tmin))]
        r = sorted(T.tolist(), key=lambda i: (-al[i], basis[i]))[0]
        if basis[r] < n:
            continue
        seq.append((int(j), int(r)))
        basis[r] = j
    return seq


@pytest.mark.parametrize("m,n,seed,reinv", [(200, 300, 5, 64), (150, 260, 6, 5), (257, 400, 7, 16)])
def test_crash_sequence_matches_rule(m, n, seed, reinv):
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(m, n, 60 + seed)
    A, b, c = lpgen.perturbed_lp(base, seed)
    ref_base = oracle.solve(*base)
    rng = np.random.default_rng(seed)
    S = [int(v) for v in ref_base.basis if v < n]
    extra = [int(v) for v in rng.choice(np.setdiff1d(np.arange(n), S), len(S) // 2, replace=False)]
    order = [int(v) for v in rng.permutation(S + extra)]
    seq = crash_reference(A, b, order)
    assert len(seq) > 0
    with lpgb.LP(A, b, c, trace_cap=1 << 14, reinvert_every=reinv) as lp:
        cold = lp.solve()
        lp.reset()
        lp.set_crash(order)
        res = lp.solve()
        tr = lp.trace()
        x, y, z = lp.solution()
    assert res.warm_repairs == len(seq), (res.warm_repairs, len(seq))
    got = list(zip(tr["q"][:len(seq)].tolist(), tr["r"][:len(seq)].tolist()))
    assert got == seq
    assert res.status == lpgb.LP_OPTIMAL
    ref = oracle.solve(A, b, c)
    assert abs(z - ref.objective) <= 1e-9 * abs(ref.objective)
    assert_certificate(A, b, c, x, y)
    # the crash consumed the list: the next solve is cold again
    with lpgb.LP(A, b, c, reinvert_every=reinv) as lp:
        lp.set_crash(order)
        lp.solve()
        lp.reset()
        r2 = lp.solve()
    assert r2.warm_repairs == 0 and r2.iterations == cold.iterations


def test_crash_arguments():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("real", 20, 30, 1)
    with lpgb.LP(A, b, c) as lp:
        for bad in ([3, 3], [30], [-1], list(range(21))):
            with pytest.raises(lpgb.LPError):
                lp.set_crash(bad)
        lp.set_crash([])
        assert lp.solve().warm_repairs == 0
    A, b, c = lpgen.general_lp(30, 40, 2)
    with lpgb.LP(A, b, c) as lp:
        with pytest.raises(lpgb.LPError) as e:
            lp.set_crash([1, 2])
        assert e.value.code == lpgb.LP_ERR_STATE
