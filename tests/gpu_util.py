"""Helpers shared by the GPU tests: run the CUDA solver and check it against
the oracle (pivot sequence in follow mode, objective, certificates)."""
import numpy as np

import oracle


def gpu_solve(A, b, c, **opts):
    from paper_1803_04378_gb300 import lpgb
    opts.setdefault("trace_cap", 1 << 20)
    opts.setdefault("max_iters", 2_000_000)
    lp = lpgb.LP(A, b, c, **opts)
    res = lp.solve()
    x, y, z = lp.solution()
    tr = lp.trace()
    return lp, res, x, y, z, tr


def follow_check(A, b, c, res, tr, opts=None):
    """The oracle re-runs the method and checks the GPU's pivots one by one;
    a different choice is accepted only where the oracle's own values tie
    within 1e-12.  Returns the oracle's Solution."""
    q = np.append(tr["q"], -1)
    r = np.append(tr["r"], -1)
    chk = oracle.solve(A, b, c, opts, follow=(q, r), follow_status=res.status)
    assert chk.mismatch_at < 0, f"pivot mismatch at iteration {chk.mismatch_at} (kind {chk.mismatch_kind})"
    assert chk.status == res.status, (chk.status, res.status)
    assert chk.iterations == res.iterations, (chk.iterations, res.iterations)
    return chk


def assert_certificate(A, b, c, x, y, tol=1e-9):
    cert = oracle.certificate(A, b, c, x, y)
    assert cert["primal"] <= tol and cert["dual"] <= tol and cert["gap"] <= tol, cert
    return cert
