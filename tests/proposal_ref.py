"""The proposal rule of the learned warm start, written out plainly (the
reference the device kernel lp_family_propose is compared with): structurals
with score > threshold, best first (ties: lower index), at most m of them, take the
positions of the slack rows of lowest score (ties: lower row), the t-th
structural the t-th row; every other row keeps its slack."""
import numpy as np


def basis_from_scores(z, m: int, n: int, threshold: float = 0.0):
    z = np.asarray(z, dtype=np.float32)
    zs = z[:n]
    order = np.argsort(-zs, kind="stable")
    J = [int(j) for j in order if zs[j] > np.float32(threshold)][:m]
    rows = np.argsort(z[n:n + m], kind="stable")[:len(J)]
    basis = np.arange(n, n + m, dtype=np.int32)
    for j, r in zip(J, rows):
        basis[r] = j
    return basis, J
