"""Parity at the full sizes of the two large workloads, on the default engine.

The expected values come from the oracle's own full solves, stored by
``tests/golden/make_fullsize.py`` (a script that calls only the oracle and the
input generator): the status, the pivot and reinversion counts, the rule
counters, the objective, and the whole pivot sequence with the oracle's
separation margin of every choice.

* dense_real_4096x8192 (A_ij ~ U[0,1) with 10% zeros, seed 1) and
  degenerate_2048x4096 (integer A, 30% of b_i = 0, seed 2, tabu tenure 7):
  the GPU's pivot sequence must equal the oracle's.  The two may part only at
  a pivot where the oracle's own choice was not separated by more than the
  1e-12 tie tolerance (Section 2.2's ties; the method then takes either row or
  column), and after such a point only the optimum is compared.  The
  objective must agree to 1e-9 relative and the GPU's x and y must pass the
  optimality certificate to 1e-9.
* The first 192 pivots of the 4096 x 8192 solve (three refined reinversions,
  after pivots 64, 128 and 192) are checked pivot by pivot in follow mode, and
  B^-1, bbar and y after 130 pivots element by element against the oracle
  (within 1e-9 of the largest entry: both sides are FP64 and differ only in
  summation order and in refinement against elimination).
"""
import json
import os

import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TIE = 1e-12


def _golden(name):
    with open(os.path.join(GOLD, f"{name}.json")) as f:
        meta = json.load(f)
    tr = np.load(os.path.join(GOLD, f"{name}_trace.npz"))
    return meta, {k: tr[k] for k in tr.files}


def first_divergence(gq, gr, q, r):
    """First pivot at which two (q, r) sequences differ, or -1."""
    n = min(len(gq), len(q))
    diff = np.nonzero((gq[:n] != q[:n]) | (gr[:n] != r[:n]))[0]
    if len(diff):
        return int(diff[0])
    return -1 if len(gq) == len(q) else n


@pytest.mark.parametrize("name", ["dense_real_4096x8192", "degenerate_2048x4096"])
def test_full_solve_matches_oracle_golden(name):
    from paper_1803_04378_gb300 import lpgb
    meta, g = _golden(name)
    A, b, c = lpgen.make(meta["kind"], meta["m"], meta["n"], meta["seed"])
    with lpgb.LP(A, b, c, trace_cap=meta["iterations"] + 4096) as lp:
        res = lp.solve()
        x, y, z = lp.solution()
        tr = lp.trace()
    # the default engine ran, with nothing forcing another one
    assert res.persistent == 2 and res.engine_reason == 0, (res.persistent, res.engine_reason)
    assert res.status_name == meta["status"] == "optimal"
    t = first_divergence(g["q"], g["r"], tr["q"], tr["r"])
    print(f"{name}: {res.iterations} pivots (oracle {meta['iterations']}), first divergence {t}")
    if t < 0:
        assert res.iterations == meta["iterations"]
        assert res.reinversions == meta["reinversions"]
        assert res.degenerate == meta["degenerate"]
        assert res.tabu_pushes == meta["tabu_pushes"]
        assert res.bland_fallbacks == meta["bland_fallbacks"]
    else:
        # the paths part only where the oracle's choice was itself a tie
        assert t < len(g["q"]) and t < len(tr["q"]), (t, len(g["q"]), len(tr["q"]))
        if g["q"][t] != tr["q"][t]:
            assert g["margin_q"][t] <= TIE, (t, g["margin_q"][t])
        else:
            assert g["margin_r"][t] <= TIE, (t, g["margin_r"][t])
    rel = abs(z - meta["objective"]) / max(1.0, abs(meta["objective"]))
    assert rel <= 1e-9, (z, meta["objective"], rel)
    cert = oracle.certificate(A, b, c, x, y)
    assert max(cert["primal"], cert["dual"], cert["gap"]) <= 1e-9, cert


def test_golden_separation_covers_every_divergence():
    """Sanity of the golden files themselves: a trace agrees with itself, and
    a planted change at a separated pivot is reported there."""
    meta, g = _golden("dense_real_4096x8192")
    q, r = g["q"].copy(), g["r"].copy()
    assert first_divergence(g["q"], g["r"], q, r) == -1
    sep = int(np.nonzero(g["margin_q"] > 1e-6)[0][3])
    q[sep] = q[sep] + 1
    assert first_divergence(g["q"], g["r"], q, r) == sep
    assert len(g["q"]) == meta["iterations"] and meta["status"] == "optimal"


def test_first_192_pivots_follow_mode_and_state_at_130():
    from paper_1803_04378_gb300 import lpgb
    A, b, c = lpgen.make("real", 4096, 8192, 1)
    with lpgb.LP(A, b, c, max_iters=192, trace_cap=192) as lp:
        res = lp.solve()
        tr = lp.trace()
    assert res.persistent == 2 and res.iterations == 192
    assert res.reinversions == 3 and res.refined_reinversions == 3, (res.reinversions, res.refined_reinversions)
    chk = oracle.solve(A, b, c, oracle.Options(max_iters=192),
                       follow=(np.append(tr["q"], -1), np.append(tr["r"], -1)),
                       follow_status=res.status, threads=0)
    assert chk.mismatch_at < 0, (chk.mismatch_at, chk.mismatch_kind)
    assert chk.iterations == 192 and chk.reinversions == 3
    # the state two pivots after the refined reinversion at pivot 128
    K = 130
    with lpgb.LP(A, b, c, max_iters=K) as lp:
        resk = lp.solve()
        binv, bbar = lp.state()
        _, y, z = lp.solution()
        basis = lp.basis()
    assert resk.iterations == K
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=K), follow=(tr["q"][:K], tr["r"][:K]),
                       follow_status=lpgb.LP_ITER_LIMIT, want_binv=True, threads=0)
    assert ref.mismatch_at < 0 and ref.iterations == K
    assert np.array_equal(basis, ref.basis)
    assert np.max(np.abs(binv - ref.binv)) <= 1e-9 * max(1.0, np.max(np.abs(ref.binv)))
    assert np.max(np.abs(bbar - ref.bbar)) <= 1e-9 * max(1.0, np.max(np.abs(ref.bbar)))
    assert np.max(np.abs(y - ref.y)) <= 1e-9 * max(1.0, np.max(np.abs(ref.y)))
    assert z == pytest.approx(ref.objective, rel=1e-12)
