"""Learned warm start on the GPU: family generator, features, the network's
kernels against the numpy reference, training, and what the trained network
gains over the cold method on held-out instances."""
import numpy as np
import pytest

import lpgen
import oracle
from gpu_util import assert_certificate
from oracle import mlp as mlp_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_family_perturb_matches_host_generator():
    import torch
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(37, 53, 4)
    A0, b0, c0 = (torch.from_numpy(v).cuda() for v in base)
    A, b, c = torch.empty_like(A0), torch.empty_like(b0), torch.empty_like(c0)
    for seed in (5, 99):
        lpgb.family_perturb(A0, b0, c0, lpgen.stream_key(seed, lpgen.TAG_NOISE), 0.05, A, b, c)
        torch.cuda.synchronize()
        Ah, bh, ch = lpgen.perturbed_lp(base, seed)
        for g, h in ((A, Ah), (b, bh), (c, ch)):
            assert np.allclose(g.cpu().numpy(), h, rtol=1e-13, atol=0)


def test_family_draw_then_solve_sees_the_whole_instance():
    """A device draw is followed at once by the solve (the solver reads the
    tensors on its own stream): the result must be that of the instance
    itself, copied to the host after the draw finished."""
    import torch
    from paper_1803_04378_gb300 import lpgb, warmstart
    base = lpgen.dense_real_lp(512, 1024, 4)
    fam = warmstart.Family(base)
    for seed in (3, 4, 5):
        fam.draw(seed)
        res, basis = fam.solve(None)
        z = fam.lp.solution()[2]
        torch.cuda.synchronize()
        A, b, c = fam.A.cpu().numpy(), fam.b.cpu().numpy(), fam.c.cpu().numpy()
        with lpgb.LP(A, b, c) as lp:
            ref = lp.solve()
            zr = lp.solution()[2]
            br = lp.basis()
        assert res.iterations == ref.iterations and z == zr, (seed, res.iterations, ref.iterations, z, zr)
        assert np.array_equal(basis, br)
    fam.close()


def test_family_features_definition():
    import torch
    from paper_1803_04378_gb300 import lpgb
    base = lpgen.dense_real_lp(30, 45, 4)
    A0, b0, c0 = base
    A, b, c = lpgen.perturbed_lp(base, 3)
    t = [torch.from_numpy(v).cuda() for v in (A0, b0, c0, A, b, c)]
    out = torch.empty(2 * (30 + 45), dtype=torch.float32, device="cuda")
    lpgb.family_features(*t, 0.05, out)
    torch.cuda.synchronize()
    f = out.cpu().numpy()
    nz = A0 != 0
    R = np.where(nz, A / np.where(nz, A0, 1.0), 0.0)
    rows = (R.sum(1) / nz.sum(1) - 1) * np.sqrt(nz.sum(1)) / 0.05
    cols = (R.sum(0) / nz.sum(0) - 1) * np.sqrt(nz.sum(0)) / 0.05
    want = np.concatenate([(b / b0 - 1) / 0.05, (c / c0 - 1) / 0.05, rows, cols])
    assert np.allclose(f, want, rtol=1e-5, atol=1e-5)


def test_mlp_gradients_match_reference():
    """Kernel gradients vs the numpy reference evaluated with the same FP16
    rounding points; ragged sizes against the 64x64 GEMM tiles."""
    import torch
    from paper_1803_04378_gb300 import lpgb
    rng = np.random.default_rng(1)
    i, h, o, B = 70, 48, 40, 24
    net = lpgb.MLP(i, h, o, B)
    p = (rng.standard_normal(net.num_params) * 0.2).astype(np.float32)
    net.set_params(p)
    X = rng.standard_normal((B, i)).astype(np.float32)
    T = (rng.random((B, o)) < 0.35).astype(np.float32)
    g, loss = net.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    loss_ref, g_ref = mlp_ref.loss_and_grads(p.astype(np.float64), X, T, i, h, o, fp16_points=True)
    assert abs(loss - loss_ref) <= 1e-4 * abs(loss_ref)
    assert np.max(np.abs(g - g_ref)) <= 5e-3 * np.max(np.abs(g_ref))
    # and the full-precision gradients are close as well (FP16 storage error only)
    _, g64 = mlp_ref.loss_and_grads(p.astype(np.float64), X, T, i, h, o)
    assert np.max(np.abs(g - g64)) <= 5e-2 * np.max(np.abs(g64))
    # forward logits
    logits = torch.empty((B, o), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(X).cuda(), logits)
    torch.cuda.synchronize()
    z_ref = mlp_ref.forward(p.astype(np.float64), X, i, h, o, fp16_points=True)["z3"]
    assert np.max(np.abs(logits.cpu().numpy() - z_ref)) <= 1e-3 * max(1.0, np.max(np.abs(z_ref)))
    net.close()


def test_mlp_training_reduces_loss():
    import torch
    from paper_1803_04378_gb300 import lpgb, warmstart
    rng = np.random.default_rng(2)
    N, i, o = 2048, 64, 32
    W = rng.standard_normal((i, o))
    X = rng.standard_normal((N, i)).astype(np.float32)
    Y = (X @ W > 0).astype(np.float32)
    net, losses = warmstart.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), hidden=128,
                                  epochs=8, batch=128, lr=3e-3)
    assert losses[-1] < 0.35 * losses[0]
    net.close()


def test_propose_kernel_matches_definition():
    """lp_family_propose against the plain rule: ties in the scores, more
    positive structurals than m, none at all, and sizes over several
    1024-score tiles with ragged ends."""
    import torch
    from paper_1803_04378_gb300 import lpgb
    from proposal_ref import basis_from_scores
    rng = np.random.default_rng(7)
    cases = [(5, 4, None, 0.0), (2, 5, "all", 0.0), (7, 9, "none", 0.0), (300, 600, None, 0.0),
             (1300, 2500, None, 0.0), (1024, 2048, "ties", 0.0), (64, 3000, "many", 0.0),
             (300, 600, None, 1.25), (1024, 2048, "ties", -0.5)]
    for m, n, kind, thr in cases:
        z = rng.standard_normal(n + m).astype(np.float32)
        if kind == "all":
            z[:] = 1.0
        elif kind == "none":
            z[:n] = -np.abs(z[:n])
        elif kind == "ties":
            z = np.round(z * 2) / 2          # many equal scores on both sides
        elif kind == "many":
            z[:n] = np.abs(z[:n]) + 0.1      # 3000 proposed structurals for 64 rows
        zt = torch.from_numpy(z).cuda()
        basis = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        work = torch.full((m + 1,), -1, dtype=torch.int32, device="cuda")
        lpgb.family_propose(zt, m, n, basis, work, thr)
        torch.cuda.synchronize()
        want_basis, want_J = basis_from_scores(z, m, n, thr)
        got_basis, got_work = basis.cpu().numpy(), work.cpu().numpy()
        assert got_work[m] == int(np.sum(z[:n] > np.float32(thr))), (m, n, kind)
        k = min(int(got_work[m]), m)
        assert got_work[:k].tolist() == want_J, (m, n, kind)
        assert np.array_equal(got_basis, want_basis), (m, n, kind)
        assert len(set(got_basis.tolist())) == m


def test_learned_warm_start_gains_on_heldout():
    """Train on solver-generated pairs of a 256 x 512 family (labels: cold
    optimal bases), then compare cold and warm solves of held-out instances:
    every warm solve reaches the cold optimum (and the oracle's, checked on
    two of them) in fewer pivots on the whole."""
    from paper_1803_04378_gb300 import warmstart
    m, n = 256, 512
    base = lpgen.dense_real_lp(m, n, 4)
    fam = warmstart.Family(base)
    X, Y, piv = warmstart.generate_labels(fam, range(1, 1001))
    net, losses = warmstart.train(X, Y, hidden=512, epochs=20, batch=128, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    held = [lpgen.perturbed_lp(base, 10_000_000 + k) for k in range(24)]
    modes = ("repair", "guided")
    rows = warmstart.evaluate(fam, net, held, modes)
    s = warmstart.summarize(rows, modes)
    print(s)
    for mode in modes:
        assert s[mode]["optimal"] and s[mode]["max_rel_objective_gap"] <= 1e-9, (mode, s[mode])
    assert s["repair"]["pivot_ratio"] < 0.8, s
    for k in (0, 7):
        A, b, c = held[k]
        ref = oracle.solve(A, b, c)
        assert abs(rows[k]["repair"]["z"] - ref.objective) <= 1e-9 * abs(ref.objective)
    fam.close()
    net.close()
