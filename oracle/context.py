"""Multi-core FP64 power iteration, for context timing only (not an oracle).

Built from ppr_context.c with OpenMP when gcc supports it; the benchmark times
it beside the single-threaded oracle, and a CPU test checks it against the
oracle's PowItr.  Test and benchmark infrastructure: the CUDA library never
imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppr_context.c")
_LIB = os.path.join(_HERE, "libcontext.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:2] + ["-fopenmp"] + base[2:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)  # no OpenMP: one thread
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.ctx_graph_new.restype = P
            lib.ctx_graph_new.argtypes = [ctypes.c_int64, P, P]
            lib.ctx_graph_free.argtypes = [P]
            lib.ctx_graph_free.restype = None
            lib.ctx_powitr.argtypes = [P, ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int64, P, P]
            lib.ctx_powitr.restype = ctypes.c_int
            lib.ctx_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


class ContextGraph:
    """The transposed graph for the multi-core power iteration."""

    def __init__(self, row_ptr, col_idx):
        self.rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.n = len(self.rp) - 1
        self.handle = _load().ctx_graph_new(self.n, self.rp.ctypes.data, self.ci.ctypes.data)
        if not self.handle:
            raise MemoryError("context graph")

    def powitr(self, s: int, alpha: float = 0.2, lam: float = 1e-8, max_iter: int = 10_000):
        pi = np.zeros(self.n)
        it = ctypes.c_int64()
        rc = _load().ctx_powitr(self.handle, alpha, int(s), lam, max_iter, pi.ctypes.data, ctypes.byref(it))
        if rc != 0:
            raise RuntimeError(f"ctx_powitr returned {rc}")
        return pi, it.value

    def close(self):
        if self.handle:
            _load().ctx_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def threads() -> int:
    return int(_load().ctx_threads())
