"""Seeded synthetic LP generators shared by the CPU oracle, the tests and the bench.

This module holds no simplex arithmetic: it only draws numbers.  Both the CUDA
path and the oracle receive byte-identical inputs from it.

Random numbers come from SplitMix64 used as a counter-based generator
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): draw k of a stream with key K is ``mix(K + (k+1)*GAMMA)`` where
``mix`` is the SplitMix64 finaliser.  Every named stream (matrix values, zero
mask, right-hand side, costs, ...) gets its own key, derived from the seed and a
fixed tag, so the fill order of one stream never shifts another.

Uniform reals are ``(z >> 11) * 2**-53`` on [0, 1).  Uniform integers on
[lo, hi] are ``lo + floor(u * (hi - lo + 1))``: for the ranges used here
(at most 100 values) the bias against a rejection sampler is below 1e-13 and is
ignored.  Normal draws use the Box-Muller transform on two uniforms.

Workloads are shaped like the paper's dense random problems (Section 4,
Appendix A: dense A, m:n between 1:1.6 and 1:1.9, sizes up to 3500x5500); the
paper publishes neither its generator nor its seeds, so these stand in for its
random set.  All problems are ``max c^T x  s.t.  A x <= b, x >= 0`` with
``b >= 0`` (Section 2.1 standard form after adding slacks).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags (fixed; changing one changes every generated workload).
TAG_A = 1
TAG_A_MASK = 2
TAG_B = 3
TAG_C = 4
TAG_B_ZERO_ROWS = 5
TAG_SIZES = 6
TAG_NOISE = 7
TAG_XSTAR = 8
TAG_NEG_ROWS = 9


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(key: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream with ``key``."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        return _mix(z)


def stream_key(seed: int, tag: int) -> int:
    """Key of the named stream ``tag`` under ``seed`` (one SplitMix64 draw)."""
    return int(splitmix64(seed, 1, start=tag)[0])


def uniform(key: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform float64 on [0, 1) with 53 random bits."""
    z = splitmix64(key, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def randint(key: int, count: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Uniform integers on [lo, hi] inclusive, returned as float64."""
    u = uniform(key, count, start)
    return lo + np.floor(u * float(hi - lo + 1))


def normal(key: int, count: int) -> np.ndarray:
    """Standard normal draws by Box-Muller (two uniforms per pair)."""
    pairs = (count + 1) // 2
    u = uniform(key, 2 * pairs)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# --------------------------------------------------------------------------
# LP families
# --------------------------------------------------------------------------

def dense_int_lp(m: int, n: int, seed: int):
    """Dense integer LP: A_ij in {1..100}, b_i ~ U[1000, 10000], c_j in {1..100}.

    Feasible (b >= 0 so x = 0 is feasible) and bounded (A > 0 elementwise).
    Returns (A row-major m x n, b, c) as float64 arrays.
    """
    A = randint(stream_key(seed, TAG_A), m * n, 1, 100).reshape(m, n)
    b = 1000.0 + 9000.0 * uniform(stream_key(seed, TAG_B), m)
    c = randint(stream_key(seed, TAG_C), n, 1, 100)
    return A, b, c


def dense_real_lp(m: int, n: int, seed: int, zero_frac: float = 0.1):
    """Dense real LP: A_ij ~ U[0,1) with a fraction ``zero_frac`` zeroed at
    random, b_i ~ U[n/4, n/2], c_j ~ U[0,1)."""
    A = uniform(stream_key(seed, TAG_A), m * n).reshape(m, n)
    if zero_frac > 0:
        mask = uniform(stream_key(seed, TAG_A_MASK), m * n).reshape(m, n) < zero_frac
        A[mask] = 0.0
    b = n / 4.0 + (n / 4.0) * uniform(stream_key(seed, TAG_B), m)
    c = uniform(stream_key(seed, TAG_C), n)
    return A, b, c


def degenerate_lp(m: int, n: int, seed: int, zero_row_frac: float = 0.3):
    """Degenerate dense LP: A_ij in {-5..10}; exactly floor(zero_row_frac*m)
    rows get b_i = 0 (chosen by a partial Fisher-Yates shuffle), the rest
    b_i ~ U[1, 100]; c_j in {1..20}."""
    A = randint(stream_key(seed, TAG_A), m * n, -5, 10).reshape(m, n)
    b = 1.0 + 99.0 * uniform(stream_key(seed, TAG_B), m)
    z = int(np.floor(zero_row_frac * m))
    u = uniform(stream_key(seed, TAG_B_ZERO_ROWS), z)
    perm = list(range(m))
    for i in range(z):
        j = i + int(np.floor(u[i] * (m - i)))
        perm[i], perm[j] = perm[j], perm[i]
    b[np.array(perm[:z], dtype=np.int64)] = 0.0
    c = randint(stream_key(seed, TAG_C), n, 1, 20)
    return A, b, c


def general_lp(m: int, n: int, seed: int, neg_row_frac: float = 0.3):
    """Dense LP with some negative b_i (needs Phase I), feasible and bounded by
    construction.  Rows are dealt "negative" with probability neg_row_frac:
    their A_ij are in {-10..2}, the other rows' in {-2..10}.  A point
    x* ~ U[0, 1)^n gives b = A x* + s with s ~ U[0, 1), so x* is feasible and
    the mostly negative rows get b_i < 0.  The last row is all ones with
    b = sum x* + n, which bounds every objective.  c_j in {1..20}."""
    if m < 2:
        raise ValueError("general_lp needs m >= 2")
    neg = uniform(stream_key(seed, TAG_NEG_ROWS), m) < neg_row_frac
    lo = np.where(neg, -10, -2)[:, None]
    hi = np.where(neg, 2, 10)[:, None]
    u = uniform(stream_key(seed, TAG_A), m * n).reshape(m, n)
    A = np.floor(lo + u * (hi - lo + 1)).astype(np.float64)
    A = np.minimum(A, hi)
    xs = uniform(stream_key(seed, TAG_XSTAR), n)
    A[m - 1, :] = 1.0
    b = A @ xs + uniform(stream_key(seed, TAG_B), m)
    b[m - 1] = float(np.sum(xs)) + n
    c = randint(stream_key(seed, TAG_C), n, 1, 20)
    return A, b, c


def batch_sizes(count: int, seed: int = 3, m_lo: int = 16, m_hi: int = 256):
    """Sizes of a batch: m_k uniform integer in [m_lo, m_hi], n_k in [m_k, 2 m_k]."""
    key = stream_key(seed, TAG_SIZES)
    u = uniform(key, 2 * count)
    ms = (m_lo + np.floor(u[0::2] * (m_hi - m_lo + 1))).astype(np.int64)
    ns = (ms + np.floor(u[1::2] * (ms + 1))).astype(np.int64)
    return ms, ns


def batch_instance_seed(k: int, seed: int = 3) -> int:
    return seed * (1 << 32) + k


def batch_lp(k: int, m: int, n: int, seed: int = 3):
    """Instance k of a batch, generated as a dense integer LP."""
    return dense_int_lp(m, n, batch_instance_seed(k, seed))


def perturbed_lp(base, instance_seed: int, sigma: float = 0.05):
    """Multiplies every entry of (A, b, c) by an independent N(1, sigma^2) draw."""
    A0, b0, c0 = base
    m, n = A0.shape
    g = normal(stream_key(instance_seed, TAG_NOISE), m * n + m + n)
    f = 1.0 + sigma * g
    A = A0 * f[: m * n].reshape(m, n)
    b = b0 * f[m * n: m * n + m]
    c = c0 * f[m * n + m:]
    return A, b, c


# Named workloads: dense integer 200x200 (seed 0); dense real 4096x8192 with
# 10% zeros (seed 1); degenerate 2048x4096 (seed 2); a batch of 4096 small
# LPs (seed 3); a perturbed 1024x2048 family for the learned warm start (seed 4).
WORKLOADS = {
    "dense_int_200x200": dict(kind="int", m=200, n=200, seed=0),
    "dense_real_4096x8192": dict(kind="real", m=4096, n=8192, seed=1),
    "degenerate_2048x4096": dict(kind="degenerate", m=2048, n=4096, seed=2),
    # the paper's sparser dense classes (its S20/S60 problems have 20% and 60% zeros)
    "s20_4096x8192": dict(kind="s20", m=4096, n=8192, seed=1),
    "s60_4096x8192": dict(kind="s60", m=4096, n=8192, seed=1),
    "batch_4096_small": dict(kind="batch", count=4096, seed=3),
    "warm_family_1024x2048": dict(kind="warm", m=1024, n=2048, seed=4),
}


def make(kind: str, m: int, n: int, seed: int):
    if kind == "int":
        return dense_int_lp(m, n, seed)
    if kind == "real":
        return dense_real_lp(m, n, seed)
    if kind == "general":
        return general_lp(m, n, seed)
    if kind == "degenerate":
        return degenerate_lp(m, n, seed)
    if kind == "warm":
        return dense_real_lp(m, n, seed)
    if kind == "s20":
        return dense_real_lp(m, n, seed, zero_frac=0.2)
    if kind == "s60":
        return dense_real_lp(m, n, seed, zero_frac=0.6)
    raise ValueError(f"unknown LP kind {kind!r}")
