"""Thin ctypes binding of the C ABI in ``include/lpgb.h``.

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Importing this module loads ``_build/liblpgb.so`` and raises if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblpgb.so")

LP_OK = 0
LP_ERR_INVALID_ARG = -1
LP_ERR_CUDA = -2
LP_ERR_OOM = -3
LP_ERR_SINGULAR = -4
LP_ERR_TIMEOUT = -5
LP_ERR_STATE = -6
LP_ERR_DEVICE = -7

LP_RUNNING, LP_OPTIMAL, LP_UNBOUNDED, LP_ITER_LIMIT, LP_INFEASIBLE = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "running", 1: "optimal", 2: "unbounded", 3: "iter_limit", 4: "infeasible"}
LP_TF_DEGENERATE, LP_TF_TABU_PUSH, LP_TF_ASPIRATION, LP_TF_BLAND, LP_TF_TIE_SET = 1, 2, 4, 8, 64
LP_TF_GUIDED = 128
LP_ENGINE_DENSE, LP_ENGINE_GRAPH, LP_ENGINE_STRUCTURED = 0, 1, 2
(LP_ENGINE_REASON_NONE, LP_ENGINE_REASON_PRICE_MODE, LP_ENGINE_REASON_LEXICOGRAPHIC, LP_ENGINE_REASON_NO_COOPERATIVE,
 LP_ENGINE_REASON_SIZE, LP_ENGINE_REASON_OCCUPANCY, LP_ENGINE_REASON_OUT_OF_CORE) = range(7)
ENGINE_REASONS = {0: "none", 1: "price_mode", 2: "lexicographic", 3: "no_cooperative", 4: "size",
                  5: "occupancy", 6: "out_of_core"}
LP_ANTICYCLING_TABU, LP_ANTICYCLING_LEXICOGRAPHIC = 0, 1


class lp_options(ctypes.Structure):
    _fields_ = [("reinvert_every", ctypes.c_int32), ("tabu_tenure", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("bland_after", ctypes.c_int32),
                ("price_mode", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("trace_cap", ctypes.c_int32), ("graph_iters", ctypes.c_int32),
                ("kernel_timing", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("anticycling", ctypes.c_int32), ("reinvert_refine", ctypes.c_int32),
                ("reinvert_tc", ctypes.c_int32),
                ("tol_d", ctypes.c_double), ("tol_piv", ctypes.c_double),
                ("tol_tie", ctypes.c_double), ("refine_tol", ctypes.c_double),
                ("tableau_budget_mb", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p)]


class lp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("reinversions", ctypes.c_int32), ("degenerate", ctypes.c_int32),
                ("tabu_pushes", ctypes.c_int32), ("bland_fallbacks", ctypes.c_int32),
                ("aspirations", ctypes.c_int32), ("tc_reinversions", ctypes.c_int32),
                ("objective", ctypes.c_double), ("seconds", ctypes.c_double),
                ("reinvert_seconds", ctypes.c_double), ("bytes_moved", ctypes.c_double),
                ("price_seconds", ctypes.c_double), ("update_seconds", ctypes.c_double),
                ("price_bytes", ctypes.c_double), ("update_bytes", ctypes.c_double),
                ("price_launches", ctypes.c_int32), ("update_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("warm_repairs", ctypes.c_int32),
                ("warm_fallback", ctypes.c_int32), ("screen_passes", ctypes.c_int32),
                ("full_passes", ctypes.c_int32), ("reinvert_gj_seconds", ctypes.c_double),
                ("reinvert_assemble_seconds", ctypes.c_double), ("chain_seconds", ctypes.c_double),
                ("chain_bytes", ctypes.c_double), ("chain_launches", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("phase1_iterations", ctypes.c_int32),
                ("phase1_exchanged", ctypes.c_int32), ("refined_reinversions", ctypes.c_int32),
                ("engine_reason", ctypes.c_int32), ("refine_residual_max", ctypes.c_double),
                ("ooc_blocks", ctypes.c_int32), ("ooc_block_rows", ctypes.c_int32),
                ("ooc_bytes", ctypes.c_double)]


class lp_batch_result(ctypes.Structure):
    _fields_ = [("solved", ctypes.c_int32), ("unbounded", ctypes.c_int32),
                ("iter_limit", ctypes.c_int32), ("failed", ctypes.c_int32),
                ("iterations", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("fp64_flops", ctypes.c_double)]


class LPError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {_lib.lp_strerror(code).decode()} ({code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"solver library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
    lib.lp_default_options.argtypes = [P(lp_options)]
    lib.lp_selftest_barrier_timeout.argtypes = [i32, vp]
    lib.lp_selftest_barrier_timeout.restype = ctypes.c_int
    lib.lp_default_options.restype = None
    lib.lp_create.argtypes = [P(vp), i32, i32, vp, vp, vp, i32, P(lp_options)]
    lib.lp_create.restype = ctypes.c_int
    lib.lp_set_basis.argtypes = [vp, vp]
    lib.lp_set_basis.restype = ctypes.c_int
    lib.lp_reset.argtypes = [vp]
    lib.lp_reset.restype = ctypes.c_int
    lib.lp_solve.argtypes = [vp, P(lp_result)]
    lib.lp_solve.restype = ctypes.c_int
    lib.lp_get_solution.argtypes = [vp, vp, vp, vp]
    lib.lp_get_solution.restype = ctypes.c_int
    lib.lp_get_basis.argtypes = [vp, vp]
    lib.lp_get_basis.restype = ctypes.c_int
    lib.lp_get_state.argtypes = [vp, vp, vp]
    lib.lp_get_state.restype = ctypes.c_int
    lib.lp_get_trace.argtypes = [vp, vp, vp, vp, vp, vp, i32, P(i32)]
    lib.lp_get_trace.restype = ctypes.c_int
    lib.lp_destroy.argtypes = [vp]
    lib.lp_destroy.restype = None
    lib.lp_strerror.argtypes = [ctypes.c_int]
    lib.lp_strerror.restype = ctypes.c_char_p
    lib.lp_price_static.argtypes = [i32, i32, vp, i32, vp, vp, vp, ctypes.c_double, vp, vp, vp]
    lib.lp_price_static.restype = ctypes.c_int
    lib.lp_tc_gemm.argtypes = [i32, i32, i32, vp, i32, vp, i32, vp, i32, i32, vp]
    lib.lp_tc_gemm.restype = ctypes.c_int
    lib.lp_set_basis_repair.argtypes = [vp, vp, i32]
    lib.lp_set_basis_repair.restype = ctypes.c_int
    lib.lp_set_crash.argtypes = [vp, vp, i32]
    lib.lp_set_crash.restype = ctypes.c_int
    lib.lp_update_problem.argtypes = [vp, vp, vp, vp, i32]
    lib.lp_update_problem.restype = ctypes.c_int
    lib.lp_set_priority.argtypes = [vp, vp, i32]
    lib.lp_set_priority.restype = ctypes.c_int
    lib.lp_mlp_create.argtypes = [P(vp), i32, i32, i32, i32, vp]
    lib.lp_mlp_create.restype = ctypes.c_int
    lib.lp_mlp_num_params.argtypes = [vp]
    lib.lp_mlp_num_params.restype = ctypes.c_int64
    lib.lp_mlp_set_params.argtypes = [vp, vp]
    lib.lp_mlp_set_params.restype = ctypes.c_int
    lib.lp_mlp_get_params.argtypes = [vp, vp]
    lib.lp_mlp_get_params.restype = ctypes.c_int
    lib.lp_mlp_forward.argtypes = [vp, vp, i32, vp]
    lib.lp_mlp_forward.restype = ctypes.c_int
    lib.lp_mlp_gradients.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.lp_mlp_gradients.restype = ctypes.c_int
    lib.lp_mlp_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp]
    lib.lp_mlp_train_step.restype = ctypes.c_int
    lib.lp_mlp_destroy.argtypes = [vp]
    lib.lp_mlp_destroy.restype = None
    lib.lp_family_perturb.argtypes = [i32, i32, vp, vp, vp, ctypes.c_uint64, ctypes.c_double, vp, vp, vp, vp]
    lib.lp_family_perturb.restype = ctypes.c_int
    lib.lp_family_features.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp]
    lib.lp_family_features.restype = ctypes.c_int
    lib.lp_family_propose.argtypes = [i32, i32, vp, ctypes.c_float, vp, vp, vp]
    lib.lp_family_propose.restype = ctypes.c_int
    lib.lp_batch_create.argtypes = [P(vp), i32, vp, vp, vp, vp, vp, i32, P(lp_options)]
    lib.lp_batch_create.restype = ctypes.c_int
    lib.lp_batch_solve.argtypes = [vp, P(lp_batch_result)]
    lib.lp_batch_solve.restype = ctypes.c_int
    lib.lp_batch_get.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.lp_batch_get.restype = ctypes.c_int
    lib.lp_batch_get_trace.argtypes = [vp, i32, vp, vp, i32, P(i32)]
    lib.lp_batch_get_trace.restype = ctypes.c_int
    lib.lp_batch_tune.argtypes = [vp, vp, i32]
    lib.lp_batch_tune.restype = ctypes.c_int
    lib.lp_batch_set_tuning.argtypes = [vp, vp]
    lib.lp_batch_set_tuning.restype = ctypes.c_int
    lib.lp_batch_destroy.argtypes = [vp]
    lib.lp_batch_destroy.restype = None
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int, where: str):
    if rc != LP_OK:
        raise LPError(rc, where)


def default_options(**overrides) -> lp_options:
    o = lp_options()
    _lib.lp_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _device_inputs_ready():
    """The library reads device inputs on the handle's own stream, which does
    not wait for work that torch (or another stream) still has queued on the
    tensors: finish every stream of the device before passing their pointers."""
    import torch
    torch.cuda.synchronize()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class Result:
    status: int
    iterations: int
    reinversions: int
    degenerate: int
    tabu_pushes: int
    bland_fallbacks: int
    aspirations: int
    objective: float
    seconds: float
    reinvert_seconds: float
    bytes_moved: float
    price_seconds: float = 0.0
    update_seconds: float = 0.0
    price_bytes: float = 0.0
    update_bytes: float = 0.0
    price_launches: int = 0
    update_launches: int = 0
    kernel_launches: int = 0
    warm_repairs: int = 0
    warm_fallback: int = 0
    screen_passes: int = 0
    full_passes: int = 0
    reinvert_gj_seconds: float = 0.0
    reinvert_assemble_seconds: float = 0.0
    chain_seconds: float = 0.0
    chain_bytes: float = 0.0
    chain_launches: int = 0
    persistent: int = 0
    phase1_iterations: int = 0
    phase1_exchanged: int = 0
    refined_reinversions: int = 0
    refine_residual_max: float = 0.0
    engine_reason: int = 0
    tc_reinversions: int = 0
    ooc_blocks: int = 0
    ooc_block_rows: int = 0
    ooc_bytes: float = 0.0

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


class LP:
    """One LP ``max c^T x, A x <= b, x >= 0`` resident on the current GPU.

    A, b, c may be numpy arrays (host) or torch CUDA tensors (device); A is
    m x n row-major, float64.
    """

    def __init__(self, A, b, c, **options):
        self._h = ctypes.c_void_p()
        on_dev = hasattr(A, "is_cuda") and A.is_cuda
        if on_dev:
            import torch
            A = A.to(torch.float64).contiguous()
            b = b.to(torch.float64).contiguous()
            c = c.to(torch.float64).contiguous()
            m, n = A.shape
            _device_inputs_ready()
        else:
            A = np.ascontiguousarray(A, dtype=np.float64)
            b = np.ascontiguousarray(b, dtype=np.float64)
            c = np.ascontiguousarray(c, dtype=np.float64)
            m, n = A.shape
        if b.shape[0] != m or c.shape[0] != n:
            raise ValueError("shape mismatch")
        self.m, self.n = int(m), int(n)
        self.options = default_options(**options)
        _check(_lib.lp_create(ctypes.byref(self._h), self.m, self.n, _ptr(A), _ptr(b), _ptr(c),
                              1 if on_dev else 0, ctypes.byref(self.options)), "lp_create")

    def close(self):
        if self._h:
            _lib.lp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self) -> Result:
        r = lp_result()
        _check(_lib.lp_solve(self._h, ctypes.byref(r)), "lp_solve")
        return Result(r.status, r.iterations, r.reinversions, r.degenerate, r.tabu_pushes,
                      r.bland_fallbacks, r.aspirations, r.objective, r.seconds,
                      r.reinvert_seconds, r.bytes_moved, r.price_seconds, r.update_seconds,
                      r.price_bytes, r.update_bytes, r.price_launches, r.update_launches,
                      r.kernel_launches, r.warm_repairs, r.warm_fallback, r.screen_passes,
                      r.full_passes, r.reinvert_gj_seconds, r.reinvert_assemble_seconds,
                      r.chain_seconds, r.chain_bytes, r.chain_launches, r.persistent,
                      r.phase1_iterations, r.phase1_exchanged, r.refined_reinversions,
                      r.refine_residual_max, r.engine_reason, r.tc_reinversions, r.ooc_blocks,
                      r.ooc_block_rows, r.ooc_bytes)

    def reset(self):
        _check(_lib.lp_reset(self._h), "lp_reset")

    def update_problem(self, A, b, c):
        on_dev = hasattr(A, "is_cuda") and A.is_cuda
        if on_dev:
            _device_inputs_ready()
        else:
            A = np.ascontiguousarray(A, dtype=np.float64)
            b = np.ascontiguousarray(b, dtype=np.float64)
            c = np.ascontiguousarray(c, dtype=np.float64)
        _check(_lib.lp_update_problem(self._h, _ptr(A), _ptr(b), _ptr(c), 1 if on_dev else 0),
               "lp_update_problem")

    def set_priority(self, vars_in_order):
        v = np.ascontiguousarray(vars_in_order, dtype=np.int32)
        _check(_lib.lp_set_priority(self._h, _ptr(v) if len(v) else None, len(v)), "lp_set_priority")

    def set_basis(self, basis):
        bb = np.ascontiguousarray(basis, dtype=np.int32)
        if bb.shape != (self.m,):
            raise ValueError("basis must have m entries")
        _check(_lib.lp_set_basis(self._h, _ptr(bb)), "lp_set_basis")

    def set_basis_repair(self, basis, max_repairs: int):
        bb = np.ascontiguousarray(basis, dtype=np.int32)
        if bb.shape != (self.m,):
            raise ValueError("basis must have m entries")
        _check(_lib.lp_set_basis_repair(self._h, _ptr(bb), int(max_repairs)), "lp_set_basis_repair")

    def set_crash(self, vars_in_order):
        v = np.ascontiguousarray(vars_in_order, dtype=np.int32)
        _check(_lib.lp_set_crash(self._h, _ptr(v) if len(v) else None, len(v)), "lp_set_crash")

    def solution(self):
        x = np.zeros(self.n)
        y = np.zeros(self.m)
        z = ctypes.c_double()
        _check(_lib.lp_get_solution(self._h, _ptr(x), _ptr(y), ctypes.byref(z)), "lp_get_solution")
        return x, y, z.value

    def basis(self):
        bb = np.zeros(self.m, np.int32)
        _check(_lib.lp_get_basis(self._h, _ptr(bb)), "lp_get_basis")
        return bb

    def state(self):
        binv = np.zeros((self.m, self.m))
        bbar = np.zeros(self.m)
        _check(_lib.lp_get_state(self._h, _ptr(binv), _ptr(bbar)), "lp_get_state")
        return binv, bbar

    def trace(self):
        cap = int(self.options.trace_cap)
        q = np.zeros(cap, np.int32)
        r = np.zeros(cap, np.int32)
        th = np.zeros(cap)
        dq = np.zeros(cap)
        fl = np.zeros(cap, np.int32)
        cnt = ctypes.c_int32()
        _check(_lib.lp_get_trace(self._h, _ptr(q), _ptr(r), _ptr(th), _ptr(dq), _ptr(fl), cap,
                                 ctypes.byref(cnt)), "lp_get_trace")
        k = cnt.value
        return dict(q=q[:k], r=r[:k], theta=th[:k], dq=dq[:k], flags=fl[:k])


def selftest_barrier_timeout(blocks: int = 4, stream=None) -> int:
    """lp_selftest_barrier_timeout: return code of a grid barrier that cannot
    complete (LP_ERR_TIMEOUT when its bounded wait works)."""
    st = None if stream is None else ctypes.c_void_p(stream)
    return _lib.lp_selftest_barrier_timeout(int(blocks), st)


LP_PRICE_STATIC_MAX_M = 12288


def price_static(m: int, n: int, A_colmajor, lda: int, c, y, pos, tol_d: float, q_out, dq_out,
                 stream=None) -> int:
    """lp_price_static: allocation-free PRICE + Dantzig CHUZC on caller-owned
    device tensors (torch CUDA tensors); returns the C return code."""
    st = None if stream is None else ctypes.c_void_p(stream)
    return _lib.lp_price_static(int(m), int(n), _ptr(A_colmajor), int(lda), _ptr(c), _ptr(y), _ptr(pos),
                                float(tol_d), _ptr(q_out), _ptr(dq_out), st)


def tc_gemm(A, B, D, bf16: bool, stream=None) -> int:
    """lp_tc_gemm: D = A B^T on the tensor cores for torch CUDA tensors (A:
    M x K and B: N x K, 16-bit, row strides multiples of 8 elements; D: M x N
    float32); returns the C return code.  Only the first K columns of A and B
    are read (their strides may be larger)."""
    st = None if stream is None else ctypes.c_void_p(stream)
    M, K = int(A.shape[0]), int(A.shape[1])
    N = int(B.shape[0])
    return _lib.lp_tc_gemm(M, N, K, _ptr(A), int(A.stride(0)), _ptr(B), int(B.stride(0)), _ptr(D),
                           int(D.stride(0)), 1 if bf16 else 0, st)


LP_BATCH_MAX_M = 256
LP_BATCH_MAX_N = 512


class Batch:
    """Many independent small LPs solved in persistent launches (lp_batch_*).

    ``problems`` is a list of (A, b, c) numpy triples (A row-major m x n);
    they are packed one after another as the C ABI expects.
    """

    def __init__(self, problems, **options):
        self._h = ctypes.c_void_p()
        ms = np.array([p[0].shape[0] for p in problems], np.int32)
        ns = np.array([p[0].shape[1] for p in problems], np.int32)
        A = np.concatenate([np.ascontiguousarray(p[0], np.float64).ravel() for p in problems])
        b = np.concatenate([np.ascontiguousarray(p[1], np.float64) for p in problems])
        c = np.concatenate([np.ascontiguousarray(p[2], np.float64) for p in problems])
        self.count = len(problems)
        self.ms, self.ns = ms, ns
        opts = default_options(price_mode=1, topk=8)
        for k, v in options.items():
            setattr(opts, k, v)
        self.options = opts
        _check(_lib.lp_batch_create(ctypes.byref(self._h), self.count, _ptr(ms), _ptr(ns), _ptr(A),
                                    _ptr(b), _ptr(c), 0, ctypes.byref(opts)), "lp_batch_create")

    def close(self):
        if self._h:
            _lib.lp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self):
        r = lp_batch_result()
        _check(_lib.lp_batch_solve(self._h, ctypes.byref(r)), "lp_batch_solve")
        return dict(solved=r.solved, unbounded=r.unbounded, iter_limit=r.iter_limit, failed=r.failed,
                    iterations=r.iterations, seconds=r.seconds, fp64_flops=r.fp64_flops)

    def results(self):
        st = np.zeros(self.count, np.int32)
        it = np.zeros(self.count, np.int32)
        obj = np.zeros(self.count)
        x = np.zeros(int(self.ns.sum()))
        y = np.zeros(int(self.ms.sum()))
        _check(_lib.lp_batch_get(self._h, _ptr(st), _ptr(it), _ptr(obj), _ptr(x), _ptr(y)), "lp_batch_get")
        xs = np.split(x, np.cumsum(self.ns)[:-1])
        ys = np.split(y, np.cumsum(self.ms)[:-1])
        return st, it, obj, xs, ys

    def trace(self, k):
        cap = int(self.options.trace_cap)
        q = np.zeros(cap, np.int32)
        r = np.zeros(cap, np.int32)
        cnt = ctypes.c_int32()
        _check(_lib.lp_batch_get_trace(self._h, int(k), _ptr(q), _ptr(r), cap, ctypes.byref(cnt)),
               "lp_batch_get_trace")
        return dict(q=q[:cnt.value], r=r[:cnt.value])

    def tune(self, trials: int = 1):
        table = np.zeros(8, np.int32)
        _check(_lib.lp_batch_tune(self._h, _ptr(table), int(trials)), "lp_batch_tune")
        return table

    def set_tuning(self, table):
        t = np.ascontiguousarray(table, np.int32)
        _check(_lib.lp_batch_set_tuning(self._h, _ptr(t)), "lp_batch_set_tuning")


def save_tuning(path: str, table) -> None:
    """Caches an autotuner table as JSON: bucket -> (threads, B^-1 in shared memory)."""
    import json
    t = [int(v) for v in table]
    json.dump({"buckets_m": [64, 128, 192, 256],
               "threads": t[0::2], "binv_in_shared_memory": t[1::2]}, open(path, "w"), indent=1)


def load_tuning(path: str):
    import json
    d = json.load(open(path))
    out = []
    for t, s in zip(d["threads"], d["binv_in_shared_memory"]):
        out += [t, s]
    return np.array(out, np.int32)


class MLP:
    """The warm start's network (lp_mlp_*): in -> hidden -> hidden -> out.

    X and T are torch CUDA float32 tensors; parameters move as numpy float32.
    """

    def __init__(self, in_dim: int, hidden: int, out_dim: int, max_batch: int, stream=None):
        self._h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(stream)
        _check(_lib.lp_mlp_create(ctypes.byref(self._h), in_dim, hidden, out_dim, max_batch, st), "lp_mlp_create")
        self.in_dim, self.hidden, self.out_dim, self.max_batch = in_dim, hidden, out_dim, max_batch
        self.num_params = int(_lib.lp_mlp_num_params(self._h))

    def shapes(self):
        i, h, o = self.in_dim, self.hidden, self.out_dim
        return [(i, h), (h,), (h, h), (h,), (h, o), (o,)]

    def close(self):
        if self._h:
            _lib.lp_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        assert f.size == self.num_params
        _check(_lib.lp_mlp_set_params(self._h, _ptr(f)), "lp_mlp_set_params")

    def get_params(self):
        f = np.zeros(self.num_params, np.float32)
        _check(_lib.lp_mlp_get_params(self._h, _ptr(f)), "lp_mlp_get_params")
        return f

    def forward(self, X, logits):
        _check(_lib.lp_mlp_forward(self._h, _ptr(X), int(X.shape[0]), _ptr(logits)), "lp_mlp_forward")

    def gradients(self, X, T):
        g = np.zeros(self.num_params, np.float32)
        loss = np.zeros(1, np.float32)
        _check(_lib.lp_mlp_gradients(self._h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(g), _ptr(loss)),
               "lp_mlp_gradients")
        return g, float(loss[0])

    def train_step(self, X, T, lr: float) -> float:
        loss = np.zeros(1, np.float32)
        _check(_lib.lp_mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr), _ptr(loss)),
               "lp_mlp_train_step")
        return float(loss[0])


def family_perturb(A0, b0, c0, key: int, sigma: float, A, b, c, stream=None):
    """lp_family_perturb on torch CUDA float64 tensors (A0, A: m x n)."""
    m, n = A0.shape
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(_lib.lp_family_perturb(int(m), int(n), _ptr(A0), _ptr(b0), _ptr(c0), ctypes.c_uint64(key),
                                  float(sigma), _ptr(A), _ptr(b), _ptr(c), st), "lp_family_perturb")


def family_features(A0, b0, c0, A, b, c, sigma: float, out, stream=None):
    """lp_family_features into a torch CUDA float32 tensor of 2(m+n) values."""
    m, n = A0.shape
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(_lib.lp_family_features(int(m), int(n), _ptr(A0), _ptr(b0), _ptr(c0), _ptr(A), _ptr(b), _ptr(c),
                                   float(sigma), _ptr(out), st), "lp_family_features")


def family_propose(scores, m: int, n: int, basis, work, threshold: float = 0.0, stream=None):
    """lp_family_propose: scores (torch CUDA float32, n+m) -> basis (int32, m)
    and work (int32, m+1: the proposed structurals, their count in work[m])."""
    st = None if stream is None else ctypes.c_void_p(stream)
    _check(_lib.lp_family_propose(int(m), int(n), _ptr(scores), float(threshold), _ptr(basis), _ptr(work), st),
           "lp_family_propose")
