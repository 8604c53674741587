"""lp_price_static (the allocation-free PRICE) against the solver's own PRICE.

Some callers cannot allocate device memory -- for example code that runs
inside a CUDA graph it is capturing itself, or a runtime whose device memory
is fixed up front.  lp_price_static serves them: it keeps its scratch in a
static device array and allocates nothing.  The existing entry point that
performs the same PRICE and Dantzig choice is the solver itself (lp_create +
lp_solve, which records every pivot's entering variable and reduced cost in
lp_get_trace).  This test stops a solve after K pivots, hands its duals and
basis to lp_price_static, and checks the answer against the entering variable
and reduced cost that the solver records at pivot K, and against the CPU
oracle's reduced costs at the same duals.  The reference solves run without
the tabu list (tenure 0), so their entering choice is the plain Dantzig
argmax that lp_price_static computes.  The calls come one after another,
because the static scratch keeps the previous call's contents.
"""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu


def _solver_state(A, b, c, K):
    from paper_1803_04378_gb300 import lpgb
    with lpgb.LP(A, b, c, max_iters=K, tabu_tenure=0) as lp:
        res = lp.solve()
        _, y, _ = lp.solution()
        basis = lp.basis()
    with lpgb.LP(A, b, c, max_iters=K + 1, trace_cap=K + 1, tabu_tenure=0) as lp:
        lp.solve()
        tr = lp.trace()
    return res, y, basis, tr


def _oracle_choice(A, c, y, pos, tol_d=1e-9):
    """Dantzig's choice from the oracle's reduced costs at the same duals
    (largest d_j > tol_d over nonbasic j, exact ties to the smallest j)."""
    d = oracle.reduced_costs(A, c, y)
    d = np.where(pos < 0, d, -np.inf)
    j = int(np.argmax(d))
    return (j if d[j] > tol_d else -1), float(d[j])


def test_price_static_matches_solver_pricing():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb

    m, n = 300, 500
    A, b, c = lpgen.dense_real_lp(m, n, 31)
    lda = m + 2  # even; the padding holds NaN, which the kernel must never read
    Acm = torch.full((n, lda), float("nan"), dtype=torch.float64, device="cuda")
    Acm[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    ct = torch.from_numpy(c).cuda()
    q_out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    dq_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    for K in (5, 23):  # two calls in a row
        res, y, basis, tr = _solver_state(A, b, c, K)
        assert res.iterations == K and len(tr["q"]) == K + 1
        assert tr["flags"][K] & (lpgb.LP_TF_ASPIRATION | lpgb.LP_TF_BLAND) == 0
        pos = np.full(n + m, -1, np.int32)
        pos[basis] = np.arange(m, dtype=np.int32)
        yt = torch.from_numpy(y).cuda()
        post = torch.from_numpy(pos).cuda()
        rc = lpgb.price_static(m, n, Acm, lda, ct, yt, post, 1e-9, q_out, dq_out, stream)
        assert rc == lpgb.LP_OK
        torch.cuda.synchronize()
        assert int(q_out.item()) == int(tr["q"][K])
        want = float(tr["dq"][K])
        assert abs(float(dq_out.item()) - want) <= 1e-12 * max(1.0, abs(want))
        # the oracle at the same y: the same column, d_q to 1e-12 (summation order only)
        oq, od = _oracle_choice(A, c, y, pos)
        assert int(q_out.item()) == oq
        assert abs(float(dq_out.item()) - od) <= 1e-12 * max(1.0, abs(od))

    # at the optimal basis there is no entering variable
    with lpgb.LP(A, b, c) as lp:
        res = lp.solve()
        _, y, _ = lp.solution()
        basis = lp.basis()
    assert res.status == lpgb.LP_OPTIMAL
    pos = np.full(n + m, -1, np.int32)
    pos[basis] = np.arange(m, dtype=np.int32)
    rc = lpgb.price_static(m, n, Acm, lda, ct, torch.from_numpy(y).cuda(), torch.from_numpy(pos).cuda(),
                           1e-9, q_out, dq_out, stream)
    assert rc == lpgb.LP_OK
    torch.cuda.synchronize()
    assert int(q_out.item()) == -1
    assert float(dq_out.item()) <= 1e-9


def test_price_static_rejects_sizes_beyond_its_limit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_04378_gb300 import lpgb
    big = lpgb.LP_PRICE_STATIC_MAX_M + 1
    # rejected before any pointer is used
    assert lpgb.price_static(big, 10, None, big + 1, None, None, None, 1e-9, None, None) == lpgb.LP_ERR_INVALID_ARG
    assert lpgb.price_static(8, 10, None, 9, None, None, None, 1e-9, None, None) == lpgb.LP_ERR_INVALID_ARG
