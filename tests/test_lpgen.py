"""Seeded generators: determinism, ranges and the structure of each family."""
import numpy as np

import lpgen


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of Vigna's reference splitmix64.c
    z = lpgen.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_offsets():
    a = lpgen.uniform(12345, 1000)
    b = lpgen.uniform(12345, 1000)
    assert np.array_equal(a, b)
    assert np.array_equal(lpgen.uniform(12345, 10, start=500), a[500:510])
    assert np.all((a >= 0) & (a < 1))


def test_dense_int_family():
    A, b, c = lpgen.dense_int_lp(200, 200, 0)
    assert A.shape == (200, 200) and b.shape == (200,) and c.shape == (200,)
    assert A.min() >= 1 and A.max() <= 100 and np.all(A == np.round(A))
    assert b.min() >= 1000 and b.max() <= 10000
    assert c.min() >= 1 and c.max() <= 100 and np.all(c == np.round(c))
    assert len(np.unique(A)) == 100


def test_dense_real_family():
    A, b, c = lpgen.dense_real_lp(256, 512, 1)
    frac0 = np.mean(A == 0)
    assert 0.08 < frac0 < 0.12
    assert b.min() >= 512 / 4 and b.max() <= 512 / 2
    assert np.all((c >= 0) & (c < 1))
    # bounded: every column has a positive sum, so y = t*1 is dual feasible
    assert np.all(A.sum(axis=0) > 0)


def test_degenerate_family():
    m, n = 2048, 4096
    A, b, c = lpgen.degenerate_lp(m, n, 2)
    assert int(np.sum(b == 0)) == int(np.floor(0.3 * m))
    assert A.min() == -5 and A.max() == 10
    assert c.min() >= 1 and c.max() <= 20
    assert np.all(A.sum(axis=0) > 0)


def test_batch_sizes():
    ms, ns = lpgen.batch_sizes(4096)
    assert ms.min() >= 16 and ms.max() <= 256
    assert np.all(ns >= ms) and np.all(ns <= 2 * ms)
    A, b, c = lpgen.batch_lp(5, int(ms[5]), int(ns[5]))
    assert A.shape == (ms[5], ns[5])


def test_perturbed_family():
    base = lpgen.dense_real_lp(64, 128, 4)
    A, b, c = lpgen.perturbed_lp(base, 99)
    ratio = A[base[0] != 0] / base[0][base[0] != 0]
    assert abs(np.mean(ratio) - 1) < 0.01 and abs(np.std(ratio) - 0.05) < 0.01
    A2, _, _ = lpgen.perturbed_lp(base, 99)
    assert np.array_equal(A, A2)


def test_sparse_classes():
    # the S20 / S60 classes: the dense real family with 20% / 60% zeros
    for kind, frac in (("s20", 0.2), ("s60", 0.6)):
        A, b, c = lpgen.make(kind, 300, 500, 3)
        zeros = float(np.mean(A == 0.0))
        assert abs(zeros - frac) < 0.01, (kind, zeros)
        A10, b10, c10 = lpgen.dense_real_lp(300, 500, 3)
        keep = A != 0.0
        assert np.all(A[keep] == A10[keep])  # same values, a larger zero mask over the same draws
        assert np.array_equal(b, b10) and np.array_equal(c, c10)
