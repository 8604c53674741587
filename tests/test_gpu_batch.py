"""Batched persistent solver (lp_batch_*) against the oracle, LP by LP.

Bars: the same as the single-LP solver -- with the FP64 PRICE (price_mode 0)
every pivot is verified against the oracle (follow mode, ties within 1e-12);
with the BF16-screened PRICE (price_mode 1, the batch default) every pivot is
verified as a valid simplex pivot; objectives within 1e-9 relative and
duality certificates within 1e-9 in both modes.
"""
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


def _mixed_batch():
    """Every size bucket, both LP families of the batch workload and a few
    degenerate LPs (tabu, Bland net) and real ones long enough to reinvert."""
    probs = []
    ms, ns = lpgen.batch_sizes(24, seed=3)
    for k in range(24):
        probs.append(lpgen.batch_lp(k, int(ms[k]), int(ns[k])))
    probs.append(lpgen.degenerate_lp(64, 128, 2))
    probs.append(lpgen.degenerate_lp(48, 96, 7))
    probs.append(lpgen.dense_real_lp(200, 400, 5))   # > 64 pivots: reinversion inside the CTA
    probs.append(lpgen.dense_real_lp(250, 500, 6))
    probs.append(lpgen.dense_real_lp(17, 17, 8))
    probs.append(lpgen.dense_int_lp(1, 3, 9))
    return probs


@pytest.mark.parametrize("price_mode", [0, 1])
def test_batch_matches_oracle(price_mode):
    from paper_1803_04378_gb300 import lpgb
    probs = _mixed_batch()
    with lpgb.Batch(probs, price_mode=price_mode, trace_cap=4096, max_iters=200000) as bt:
        summary = bt.solve()
        st, it, obj, xs, ys = bt.results()
        assert summary["solved"] == len(probs) and summary["failed"] == 0
        for k, (A, b, c) in enumerate(probs):
            ref = oracle.solve(A, b, c)
            assert st[k] == 1 and ref.status == oracle.OPTIMAL
            assert abs(obj[k] - ref.objective) <= 1e-9 * max(1.0, abs(ref.objective)), k
            assert_certificate(A, b, c, xs[k], ys[k])
            tr = bt.trace(k)
            assert len(tr["q"]) == it[k]
            o = oracle.Options(follow_relaxed=1 if price_mode == 1 else 0)
            chk = oracle.solve(A, b, c, o, follow=(np.append(tr["q"], -1), np.append(tr["r"], -1)))
            assert chk.mismatch_at < 0 and chk.status == oracle.OPTIMAL, (k, chk.mismatch_at)
            assert chk.iterations == it[k]
    assert max(it) > 64  # at least one LP reinverted inside its CTA


def test_batch_tuning_changes_nothing_but_speed():
    from paper_1803_04378_gb300 import lpgb
    probs = _mixed_batch()
    with lpgb.Batch(probs) as bt:
        bt.solve()
        _, it0, obj0, _, _ = bt.results()
        table = bt.tune(trials=1)
        assert set(table[0::2]) <= {128, 256, 512} and set(table[1::2]) <= {0, 1}
        assert table[5] == 0 and table[7] == 0  # B^-1 of m > 128 does not fit in shared memory
        bt.solve()
        _, it1, obj1, _, _ = bt.results()
        # same pivots; the objective may differ in the last bits because the
        # block size sets the summation order of z after a reinversion
        assert np.array_equal(it0, it1) and np.allclose(obj0, obj1, rtol=1e-12, atol=0)
        for t in ([128, 1, 128, 1, 128, 0, 128, 0], [512, 0, 512, 0, 512, 0, 512, 0]):
            bt.set_tuning(np.array(t, np.int32))
            bt.solve()
            _, it2, obj2, _, _ = bt.results()
            assert np.array_equal(it0, it2) and np.allclose(obj0, obj2, rtol=1e-12, atol=0)
        with pytest.raises(lpgb.LPError):
            bt.set_tuning(np.array([256, 1, 256, 1, 256, 1, 256, 1], np.int32))


def test_batch_unbounded_and_invalid():
    from paper_1803_04378_gb300 import lpgb
    unb = (np.array([[1.0, -1.0], [2.0, 0.0]]), np.array([1.0, 2.0]), np.array([1.0, 1.0]))
    ok = lpgen.dense_int_lp(20, 30, 1)
    with lpgb.Batch([unb, ok], price_mode=0) as bt:
        s = bt.solve()
        st, it, obj, xs, ys = bt.results()
        assert st[0] == 2 and st[1] == 1 and s["unbounded"] == 1
    with pytest.raises(lpgb.LPError):
        lpgb.Batch([(np.ones((300, 300)), np.ones(300), np.ones(300))])
    with pytest.raises(lpgb.LPError):
        lpgb.Batch([(np.ones((2, 2)), np.array([1.0, -1.0]), np.ones(2))])
