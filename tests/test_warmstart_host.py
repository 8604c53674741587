"""Host-side logic of the learned warm start (no GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_basis_from_scores_places_structurals_on_low_slack_rows():
    from proposal_ref import basis_from_scores
    m, n = 5, 4
    # structural scores: 2 and 0 positive (2 best); slack scores: rows 3 and 1 lowest
    z = np.array([0.5, -1.0, 2.0, -0.2,  0.3, -4.0, 1.0, -5.0, 0.1])
    basis, J = basis_from_scores(z, m, n)
    assert J == [2, 0]
    assert basis.tolist() == [n + 0, 0, n + 2, 2, n + 4]
    assert len(set(basis.tolist())) == m


def test_basis_from_scores_caps_at_m_and_handles_none():
    from proposal_ref import basis_from_scores
    m, n = 2, 5
    basis, J = basis_from_scores(np.ones(n + m), m, n)
    assert len(J) == 2 and sorted(basis.tolist()) == sorted(J)
    basis, J = basis_from_scores(-np.ones(n + m), m, n)
    assert J == [] and basis.tolist() == [n, n + 1]


def test_init_params_shapes():
    from paper_1803_04378_gb300.warmstart import init_params
    shapes = [(6, 4), (4,), (4, 4), (4,), (4, 3), (3,)]
    p = init_params(shapes, seed=1)
    assert p.dtype == np.float32 and p.size == 24 + 4 + 16 + 4 + 12 + 3
    assert np.all(p[24:28] == 0) and np.max(np.abs(p[:24])) <= np.sqrt(6 / 6)
