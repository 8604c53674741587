"""CPU oracle for the dense revised simplex method (Sections 2.1-2.2, 3.1, 3.4).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the solver package never imports
it.  It shares no code with the CUDA path.

* ``solve``            -- plain FP64 revised simplex in C (``simplex_oracle.c``),
                          with the tabu entering rule and optional follow mode.
* ``gj_inverse``       -- Gauss-Jordan inverse with partial pivoting (C).
* ``reduced_costs``    -- d = c - A^T y and d_slack = -y (C).
* ``brute_force``      -- vertex enumeration for tiny LPs (numpy).
* ``certificate``      -- primal/dual feasibility and duality-gap residuals.
* ``solve_two_phase``  -- Phase I with one artificial variable for b with
                          negative entries (Section 3.4, "Finding the initial
                          feasible solution"), then ``solve`` as Phase II.

Every floating-point function here is FP64.  Parity status: every function is
pinned by tests in ``tests/test_oracle.py`` (brute force, closed forms,
Klee-Minty pivot counts, Beale's cycling example, duality certificates and an
independent HiGHS solve).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OPTIMAL, UNBOUNDED, ITER_LIMIT, SINGULAR, MISMATCH = 1, 2, 3, 4, 5
INFEASIBLE = 7  # two-phase only: the auxiliary optimum is below -tol (no feasible x)
STATUS_NAMES = {0: "running", 1: "optimal", 2: "unbounded", 3: "iter_limit",
                4: "singular", 5: "mismatch", 6: "nomem"}
TF_DEGENERATE, TF_TABU_PUSH, TF_ASPIRATION, TF_BLAND = 1, 2, 4, 8
TF_ADOPT_Q, TF_ADOPT_R, TF_TIE_SET = 16, 32, 64


def build(force: bool = False, openmp: bool = False) -> str:
    """Compiles the oracle with gcc (no FP contraction, same bits on x86/Arm).
    ``openmp`` builds the parallel variant (same source, -fopenmp), whose
    results are bit-identical to the serial build."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_OMP_PATH if openmp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class _Opts(ctypes.Structure):
    _fields_ = [("reinvert_every", ctypes.c_int32), ("tabu_tenure", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("bland_after", ctypes.c_int32),
                ("ratio_rule", ctypes.c_int32), ("follow_relaxed", ctypes.c_int32),
                ("tol_d", ctypes.c_double), ("tol_piv", ctypes.c_double),
                ("tol_tie", ctypes.c_double), ("tie_cmp", ctypes.c_double)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("reinversions", ctypes.c_int32), ("degenerate", ctypes.c_int32),
                ("tabu_pushes", ctypes.c_int32), ("bland_fallbacks", ctypes.c_int32),
                ("aspirations", ctypes.c_int32), ("adopted", ctypes.c_int32),
                ("mismatch_at", ctypes.c_int32), ("mismatch_kind", ctypes.c_int32),
                ("objective", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [("q", ctypes.c_void_p), ("r", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("dq", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("margin_q", ctypes.c_void_p), ("margin_r", ctypes.c_void_p),
                ("cap", ctypes.c_int32)]


def _load(threads: int = 1):
    """The serial library, or the OpenMP one when ``threads`` != 1 (0 = every
    host core)."""
    global _lib, _lib_omp
    with _lock:
        if threads != 1:
            if _lib_omp is None:
                _lib_omp = _bind(ctypes.CDLL(build(openmp=True)))
            _lib_omp.oracle_threads(threads if threads > 0 else (os.cpu_count() or 1))
            return _lib_omp
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def threads_used(threads: int) -> int:
    """Threads the library selected by ``threads`` runs with."""
    return int(_load(threads).oracle_threads(0))


def _bind(lib):
    """Declares the exported functions' signatures."""
    vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.oracle_solve.restype = i32
    lib.oracle_solve.argtypes = [i32, i32, vp, vp, vp, ctypes.POINTER(_Opts), vp,
                                 vp, vp, i32, i32, ctypes.POINTER(_Trace),
                                 vp, vp, vp, vp, vp, ctypes.POINTER(_Result)]
    lib.oracle_gj_inverse.restype = i32
    lib.oracle_gj_inverse.argtypes = [i32, vp, vp]
    lib.oracle_reduced_costs.restype = None
    lib.oracle_reduced_costs.argtypes = [i32, i32, vp, vp, vp, vp]
    lib.oracle_threads.restype = i32
    lib.oracle_threads.argtypes = [i32]
    return lib


def _p(a):
    return None if a is None else a.ctypes.data


RATIO_LARGEST_ALPHA, RATIO_SMALLEST_INDEX, RATIO_LEXICOGRAPHIC = 0, 1, 2


@dataclass
class Options:
    """Solver options; the defaults are the method's settings: reinversion
    every 64 iterations, tabu tenure 7, Bland fallback after 50 consecutive
    degenerate pivots, tolerances 1e-9 / 1e-9 / 1e-12.  ratio_rule: the
    leaving row among the ratio-test tie set (RATIO_*)."""
    reinvert_every: int = 64
    tabu_tenure: int = 7
    max_iters: int = 1_000_000
    bland_after: int = 50
    ratio_rule: int = 0
    follow_relaxed: int = 0
    tol_d: float = 1e-9
    tol_piv: float = 1e-9
    tol_tie: float = 1e-12
    tie_cmp: float = 1e-12


def lexicographic_options(**kw) -> "Options":
    """The lexicographic anti-cycling rule in place of the tabu rule: the
    leaving row is the lexicographically smallest row of B^-1 / alpha_i in the
    tie set; no tabu list and no Bland safety net."""
    kw.setdefault("ratio_rule", RATIO_LEXICOGRAPHIC)
    kw.setdefault("tabu_tenure", 0)
    kw.setdefault("bland_after", 0)
    return Options(**kw)


@dataclass
class Solution:
    status: int
    iterations: int
    objective: float
    x: np.ndarray
    y: np.ndarray
    basis: np.ndarray
    bbar: np.ndarray
    binv: np.ndarray | None
    reinversions: int = 0
    degenerate: int = 0
    tabu_pushes: int = 0
    bland_fallbacks: int = 0
    aspirations: int = 0
    adopted: int = 0
    mismatch_at: int = -1
    mismatch_kind: int = 0
    trace: dict = field(default_factory=dict)

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


def solve(A, b, c, opts: Options | None = None, start_basis=None, follow=None,
          follow_status: int = OPTIMAL, want_binv: bool = False, trace_cap: int = 0,
          threads: int = 1) -> Solution:
    """Runs the oracle on ``max c^T x, A x <= b, x >= 0``.

    ``follow=(q_seq, r_seq)`` checks another solver's pivot sequence pivot by
    pivot (see the C file); ``q_seq[t] = -1`` marks where it stopped.
    ``threads`` != 1 runs the OpenMP build (0 = every host core); its results
    are bit-identical to the serial build.
    """
    lib = _load(threads)
    o = opts or Options()
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m, n = A.shape
    assert b.shape == (m,) and c.shape == (n,)
    copts = _Opts(o.reinvert_every, o.tabu_tenure, o.max_iters, o.bland_after, o.ratio_rule, o.follow_relaxed,
                  o.tol_d, o.tol_piv, o.tol_tie, o.tie_cmp)
    sb = None if start_basis is None else np.ascontiguousarray(start_basis, dtype=np.int32)
    fq = fr = None
    flen = 0
    if follow is not None:
        fq = np.ascontiguousarray(follow[0], dtype=np.int32)
        fr = np.ascontiguousarray(follow[1], dtype=np.int32)
        flen = len(fq)
    tr = None
    arrays = {}
    if trace_cap > 0:
        arrays = dict(q=np.full(trace_cap, -1, np.int32), r=np.full(trace_cap, -1, np.int32),
                      theta=np.zeros(trace_cap), dq=np.zeros(trace_cap),
                      flags=np.zeros(trace_cap, np.int32), margin_q=np.zeros(trace_cap),
                      margin_r=np.zeros(trace_cap))
        tr = _Trace(*(arrays[k].ctypes.data for k in ("q", "r", "theta", "dq", "flags",
                                                      "margin_q", "margin_r")), trace_cap)
    x = np.zeros(n)
    y = np.zeros(m)
    basis = np.zeros(m, np.int32)
    bbar = np.zeros(m)
    binv = np.zeros((m, m)) if want_binv else None
    res = _Result()
    lib.oracle_solve(m, n, _p(A), _p(b), _p(c), ctypes.byref(copts), _p(sb), _p(fq), _p(fr),
                     flen, follow_status, ctypes.byref(tr) if tr is not None else None,
                     _p(x), _p(y), _p(basis), _p(binv), _p(bbar), ctypes.byref(res))
    if arrays:
        k = min(res.iterations, trace_cap)
        arrays = {key: v[:k].copy() for key, v in arrays.items()}
    return Solution(res.status, res.iterations, res.objective, x, y, basis, bbar, binv,
                    res.reinversions, res.degenerate, res.tabu_pushes, res.bland_fallbacks,
                    res.aspirations, res.adopted, res.mismatch_at, res.mismatch_kind, arrays)


def gj_inverse(M, threads: int = 1) -> np.ndarray:
    """Gauss-Jordan inverse with partial pivoting (raises on a zero pivot column)."""
    lib = _load(threads)
    M = np.ascontiguousarray(M, dtype=np.float64)
    k = M.shape[0]
    out = np.zeros_like(M)
    rc = lib.oracle_gj_inverse(k, _p(M), _p(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return out


def reduced_costs(A, c, y, threads: int = 1) -> np.ndarray:
    """d_j = c_j - y^T a_j for j < n and d_{n+i} = -y_i."""
    lib = _load(threads)
    A = np.ascontiguousarray(A, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m, n = A.shape
    d = np.zeros(n + m)
    lib.oracle_reduced_costs(m, n, _p(A), _p(c), _p(y), _p(d))
    return d


def basis_matrix(A, basis) -> np.ndarray:
    """B = [A | I][:, basis]."""
    m, n = A.shape
    full = np.hstack([A, np.eye(m)])
    return full[:, np.asarray(basis)]


def brute_force(A, b, c, tol: float = 1e-9):
    """Optimum of max c^T x, Ax <= b, x >= 0 by enumerating every basis of
    [A | I] (tiny problems only).  Uses numpy's LAPACK solve per basis, an
    independent route from the simplex iterations.  Returns (z, x) or
    (None, None) if no feasible basis exists."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    full = np.hstack([A, np.eye(m)])
    cf = np.concatenate([c, np.zeros(m)])
    best, bx = None, None
    for cols in itertools.combinations(range(n + m), m):
        B = full[:, cols]
        if abs(np.linalg.det(B)) < 1e-12:
            continue
        xb = np.linalg.solve(B, b)
        if np.min(xb) < -tol:
            continue
        zz = float(cf[list(cols)] @ xb)
        if best is None or zz > best:
            best = zz
            bx = np.zeros(n + m)
            bx[list(cols)] = xb
    return (best, None if bx is None else bx[:n])


def certificate(A, b, c, x, y) -> dict:
    """Residuals of an optimality certificate for max c^T x, Ax <= b, x >= 0
    with dual min b^T y, A^T y >= c, y >= 0 (all relative to max(1, scale))."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    s = b - A @ x
    primal = max(float(np.max(-s, initial=0.0)), float(np.max(-x, initial=0.0)))
    dual_slack = A.T @ y - c
    dual = max(float(np.max(-dual_slack, initial=0.0)), float(np.max(-y, initial=0.0)))
    pz, dz = float(c @ x), float(b @ y)
    gap = abs(pz - dz) / max(1.0, abs(pz))
    # complementary slackness: x_j * (A^T y - c)_j and y_i * s_i
    cs = max(float(np.max(np.abs(x * dual_slack), initial=0.0)),
             float(np.max(np.abs(y * s), initial=0.0)))
    scale_b = max(1.0, float(np.max(np.abs(b), initial=0.0)))
    scale_c = max(1.0, float(np.max(np.abs(c), initial=0.0)))
    return dict(primal=primal / scale_b, dual=dual / scale_c, gap=gap,
                cs=cs / max(1.0, abs(pz)), primal_obj=pz, dual_obj=dz)


@dataclass
class TwoPhaseSolution:
    status: int
    objective: float
    x: np.ndarray | None
    y: np.ndarray | None
    basis: np.ndarray | None
    phase1: Solution | None     # the auxiliary problem's solve (None when b >= 0)
    phase2: Solution | None
    exchanged: bool = False     # the artificial was basic at zero and swapped for a slack
    start_basis: np.ndarray | None = None  # Phase II start (original variable numbering)


def auxiliary_problem(A, b):
    """Phase I problem for max c^T x, Ax <= b, x >= 0 with some b_i < 0
    (Section 3.4 asks for artificial variables and the two-phase method; this
    uses the textbook single artificial x0): maximize -x0 subject to
    A x - x0 e <= b, x, x0 >= 0, where e_i = 1 on the rows with b_i < 0.
    x0 is structural column n; the slacks become n+1 .. n+m.  Returns
    (A_aux, c_aux, start_basis): the start basis is the slack basis with x0 in
    the row of the most negative b_i (the smallest such row on ties), which is
    feasible: x0 = -min b and slack_i = b_i - min b >= 0 on the negative rows."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    e = (b < 0).astype(np.float64)
    A_aux = np.hstack([A, -e[:, None]])
    c_aux = np.zeros(n + 1)
    c_aux[n] = -1.0
    istar = int(np.argmin(b))
    start = np.arange(n + 1, n + 1 + m, dtype=np.int32)
    start[istar] = n
    return A_aux, c_aux, start


def phase2_start(basis_aux, binv_row_of_x0, n: int):
    """Phase II start from the auxiliary optimum (original numbering: the aux
    slack n+1+i is the slack n+i).  If x0 is still basic (at value zero), it is
    exchanged for the nonbasic slack s with the largest |B^-1[p][s]| (p = x0's
    row; ties to the smallest s): that entry is the pivot of bringing slack s
    into row p, so the new basis is nonsingular.  Returns (basis, exchanged)."""
    basis = np.array(basis_aux, dtype=np.int64)
    m = len(basis)
    exchanged = False
    where = np.nonzero(basis == n)[0]
    if len(where):
        p = int(where[0])
        in_basis = set(int(v) for v in basis)
        best, s = -1.0, -1
        for i in range(m):
            if n + 1 + i in in_basis:
                continue
            v = abs(float(binv_row_of_x0[i]))
            if v > best:
                best, s = v, i
        if s < 0 or best <= 1e-12:
            raise np.linalg.LinAlgError("artificial cannot leave the basis")
        basis[p] = n + 1 + s
        exchanged = True
    return np.array([v if v < n else v - 1 for v in basis], dtype=np.int32), exchanged


def solve_two_phase(A, b, c, opts: Options | None = None) -> TwoPhaseSolution:
    """max c^T x, Ax <= b, x >= 0 for any b: with b >= 0 this is ``solve``;
    otherwise Phase I maximises -x0 over the auxiliary problem from its
    feasible start basis, reports INFEASIBLE when the optimum is below
    -1e-9 max(1, max|b|), and Phase II runs the method on the original problem
    from the final auxiliary basis.  Both phases use the same rules (Dantzig,
    tabu, reinversion every 64 pivots, Bland net)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    m, n = A.shape
    if np.min(b) >= 0:
        s = solve(A, b, c, opts)
        return TwoPhaseSolution(s.status, s.objective, s.x, s.y, s.basis, None, s)
    A_aux, c_aux, start = auxiliary_problem(A, b)
    p1 = solve(A_aux, b, c_aux, opts, start_basis=start, want_binv=True)
    if p1.status != OPTIMAL:
        return TwoPhaseSolution(p1.status, float("nan"), None, None, None, p1, None)
    if p1.objective < -1e-9 * max(1.0, float(np.max(np.abs(b)))):
        return TwoPhaseSolution(INFEASIBLE, float("nan"), None, None, None, p1, None)
    where = np.nonzero(p1.basis == n)[0]
    row = p1.binv[int(where[0])] if len(where) else None
    start2, exchanged = phase2_start(p1.basis, row, n)
    p2 = solve(A, b, c, opts, start_basis=start2)
    return TwoPhaseSolution(p2.status, p2.objective, p2.x, p2.y, p2.basis, p1, p2, exchanged, start2)
