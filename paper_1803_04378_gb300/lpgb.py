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

LP_RUNNING, LP_OPTIMAL, LP_UNBOUNDED, LP_ITER_LIMIT = 0, 1, 2, 3
STATUS_NAMES = {0: "running", 1: "optimal", 2: "unbounded", 3: "iter_limit"}
LP_TF_DEGENERATE, LP_TF_TABU_PUSH, LP_TF_ASPIRATION, LP_TF_BLAND, LP_TF_TIE_SET = 1, 2, 4, 8, 64


class lp_options(ctypes.Structure):
    _fields_ = [("reinvert_every", ctypes.c_int32), ("tabu_tenure", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("bland_after", ctypes.c_int32),
                ("price_mode", ctypes.c_int32), ("topk", ctypes.c_int32),
                ("trace_cap", ctypes.c_int32), ("graph_iters", ctypes.c_int32),
                ("kernel_timing", ctypes.c_int32), ("reserved_", ctypes.c_int32),
                ("tol_d", ctypes.c_double), ("tol_piv", ctypes.c_double),
                ("tol_tie", ctypes.c_double), ("cuda_stream", ctypes.c_void_p)]


class lp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("reinversions", ctypes.c_int32), ("degenerate", ctypes.c_int32),
                ("tabu_pushes", ctypes.c_int32), ("bland_fallbacks", ctypes.c_int32),
                ("aspirations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("objective", ctypes.c_double), ("seconds", ctypes.c_double),
                ("reinvert_seconds", ctypes.c_double), ("bytes_moved", ctypes.c_double),
                ("price_seconds", ctypes.c_double), ("update_seconds", ctypes.c_double),
                ("price_bytes", ctypes.c_double), ("update_bytes", ctypes.c_double),
                ("price_launches", ctypes.c_int32), ("update_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64)]


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
                      r.kernel_launches)

    def reset(self):
        _check(_lib.lp_reset(self._h), "lp_reset")

    def set_basis(self, basis):
        bb = np.ascontiguousarray(basis, dtype=np.int32)
        if bb.shape != (self.m,):
            raise ValueError("basis must have m entries")
        _check(_lib.lp_set_basis(self._h, _ptr(bb)), "lp_set_basis")

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


LP_PRICE_STATIC_MAX_M = 12288


def price_static(m: int, n: int, A_colmajor, lda: int, c, y, pos, tol_d: float, q_out, dq_out,
                 stream=None) -> int:
    """lp_price_static: allocation-free PRICE + Dantzig CHUZC on caller-owned
    device tensors (torch CUDA tensors); returns the C return code."""
    st = None if stream is None else ctypes.c_void_p(stream)
    return _lib.lp_price_static(int(m), int(n), _ptr(A_colmajor), int(lda), _ptr(c), _ptr(y), _ptr(pos),
                                float(tol_d), _ptr(q_out), _ptr(dq_out), st)
