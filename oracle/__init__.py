"""FP64 CPU oracle (test infrastructure only).

Plain, single-threaded C (ppr_oracle.c) with a thin ctypes wrapper.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg use this package;
the CUDA library never imports or links it, and it imports nothing from the
CUDA library.  Each function names the passage of arXiv 2101.03652 it follows.

ORACLE_LIBRARY, when set, names a build to load instead of liboracle.so: the
test that plants mistakes in copies of ppr_oracle.c uses it to check that the
pins catch each one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "ppr_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_GRAPH, ERR_OOM, ERR_NOT_CONVERGED = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    pass


class Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int64),
        ("pushes", ctypes.c_int64),
        ("edge_pushes", ctypes.c_int64),
        ("edge_pushes_at_lambda", ctypes.c_int64),
        ("fifo_pushes", ctypes.c_int64),
        ("scans", ctypes.c_int64),
        ("walks", ctypes.c_int64),
        ("walk_steps", ctypes.c_int64),
        ("r_sum", ctypes.c_double),
        ("W", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIBRARY") or build())
            P = ctypes.c_void_p
            I64, I32, U32, U64, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            S = ctypes.POINTER(Stats)
            sig = {
                "orc_validate": [I64, P, P],
                "orc_powitr": [I64, P, P, D, I32, D, I64, P, P, S],
                "orc_fifo_fwdpush": [I64, P, P, D, I32, D, D, P, P, S],
                "orc_fifo_refine": [I64, P, P, D, D, P, P, S],
                "orc_powerpush": [I64, P, P, D, I32, D, ctypes.c_int, D, P, P, S],
                "orc_dense_solve": [I64, P, P, D, I32, P],
                "orc_push_sequence": [I64, P, P, D, I32, P, I64, P, P],
                "orc_residual": [I64, P, P, D, I32, P, P],
                "orc_walks": [I64, P, P, D, P, D, U64, U32, I64, P, P, S],
                "orc_speedppr": [I64, P, P, D, I32, D, D, U64, U32, P, P, P, S],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_build_walk_index.argtypes = [I64, P, P, D, U64, I64, P]
            lib.orc_build_walk_index.restype = ctypes.c_int
            lib.orc_index_walks.argtypes = [I64, P, P, P, D, P, P, S]
            lib.orc_index_walks.restype = ctypes.c_int
            lib.orc_gaussian_rows.argtypes = [I64, I64, ctypes.c_int, U64, P]
            lib.orc_gaussian_rows.restype = None
            lib.orc_speedppr_W.argtypes = [I64, D, D]
            lib.orc_speedppr_W.restype = D
            _lib = lib
    return _lib


def _rc(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with status {rc}")


@dataclass
class Graph:
    """CSR graph held by the oracle side (int64 row_ptr, int32 col_idx)."""
    row_ptr: np.ndarray
    col_idx: np.ndarray

    def __post_init__(self):
        self.row_ptr = np.ascontiguousarray(self.row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(self.col_idx, dtype=np.int32)

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def args(self):
        return self.n, self.row_ptr.ctypes.data, self.col_idx.ctypes.data


def validate(g: Graph) -> int:
    return _load().orc_validate(*g.args())


def push_sequence(g: Graph, s: int, order, alpha: float = 0.2):
    """Algorithm 1 with the pushes done in the given order; returns (pi, r)."""
    o = np.ascontiguousarray(order, dtype=np.int32)
    pi = np.zeros(g.n)
    r = np.zeros(g.n)
    _rc(_load().orc_push_sequence(*g.args(), alpha, s, o.ctypes.data, len(o), pi.ctypes.data, r.ctypes.data),
        "push_sequence")
    return pi, r


def powitr(g: Graph, s: int, alpha: float = 0.2, lam: float = 1e-8, max_iter: int = 100000):
    """Power Iteration (Sec. 3.1 Eqs. 3-5); returns (pi, r, stats)."""
    pi = np.zeros(g.n)
    r = np.zeros(g.n)
    st = Stats()
    _rc(_load().orc_powitr(*g.args(), alpha, s, lam, max_iter, pi.ctypes.data, r.ctypes.data, ctypes.byref(st)),
        "powitr")
    return pi, r, st.as_dict()


def fifo_fwdpush(g: Graph, s: int, alpha: float = 0.2, rmax: float | None = None, lam: float = 1e-8):
    """Algorithm 2 with r_max (default lambda / m); returns (pi, r, stats)."""
    if rmax is None:
        rmax = lam / g.m
    pi = np.zeros(g.n)
    r = np.zeros(g.n)
    st = Stats()
    _rc(_load().orc_fifo_fwdpush(*g.args(), alpha, s, rmax, lam, pi.ctypes.data, r.ctypes.data,
                                 ctypes.byref(st)), "fifo_fwdpush")
    return pi, r, st.as_dict()


def fifo_refine(g: Graph, pi: np.ndarray, r: np.ndarray, alpha: float, rmax: float):
    """Algorithm 2's queue loop from the state (pi, r); updates copies and returns them."""
    pi = np.ascontiguousarray(pi, dtype=np.float64).copy()
    r = np.ascontiguousarray(r, dtype=np.float64).copy()
    st = Stats()
    _rc(_load().orc_fifo_refine(*g.args(), alpha, rmax, pi.ctypes.data, r.ctypes.data, ctypes.byref(st)),
        "fifo_refine")
    return pi, r, st.as_dict()


def powerpush(g: Graph, s: int, alpha: float = 0.2, lam: float = 1e-8, epoch_num: int = 8,
              scan_threshold: float | None = None):
    """Algorithm 3 (scan_threshold defaults to n/4); returns (pi, r, stats)."""
    if scan_threshold is None:
        scan_threshold = g.n / 4.0
    pi = np.zeros(g.n)
    r = np.zeros(g.n)
    st = Stats()
    _rc(_load().orc_powerpush(*g.args(), alpha, s, lam, epoch_num, scan_threshold, pi.ctypes.data,
                              r.ctypes.data, ctypes.byref(st)), "powerpush")
    return pi, r, st.as_dict()


def dense_solve(g: Graph, s: int, alpha: float = 0.2) -> np.ndarray:
    """Eq. 1 solved directly (Gaussian elimination, partial pivoting)."""
    pi = np.zeros(g.n)
    _rc(_load().orc_dense_solve(*g.args(), alpha, s, pi.ctypes.data), "dense_solve")
    return pi


def residual(g: Graph, s: int, x: np.ndarray, alpha: float = 0.2) -> np.ndarray:
    """r = (alpha e_s + (1-alpha) x P - x) / alpha, the push residual of estimate x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros(g.n)
    _rc(_load().orc_residual(*g.args(), alpha, s, x.ctypes.data, r.ctypes.data), "residual")
    return r


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def speedppr_W(n: int, eps: float, mu: float) -> float:
    """Eq. 8 (natural log)."""
    return _load().orc_speedppr_W(n, eps, mu)


def walks(g: Graph, r: np.ndarray, W: float, seed: int, source_index: int, alpha: float = 0.2,
          max_steps: int = 1 << 16):
    """SpeedPPR walk phase from residue r; returns (counts uint32, est float64, stats)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    counts = np.zeros(g.n, dtype=np.uint32)
    est = np.zeros(g.n)
    st = Stats()
    _rc(_load().orc_walks(*g.args(), alpha, r.ctypes.data, W, seed, source_index, max_steps,
                          counts.ctypes.data, est.ctypes.data, ctypes.byref(st)), "walks")
    return counts, est, st.as_dict()


def speedppr(g: Graph, s: int, eps: float = 0.5, mu: float | None = None, seed: int = 0x5EED,
             source_index: int = 0, alpha: float = 0.2):
    """Algorithm 4 end to end; returns (pi, r_before_walks, counts, stats)."""
    if mu is None:
        mu = 1.0 / g.n
    pi = np.zeros(g.n)
    r = np.zeros(g.n)
    counts = np.zeros(g.n, dtype=np.uint32)
    st = Stats()
    _rc(_load().orc_speedppr(*g.args(), alpha, s, eps, mu, seed, source_index, pi.ctypes.data, r.ctypes.data,
                             counts.ctypes.data, ctypes.byref(st)), "speedppr")
    return pi, r, counts, st.as_dict()


def gaussian_rows(u0: int, count: int, F: int, seed: int) -> np.ndarray:
    """Rows u0..u0+count-1 of the warm start's fixed Gaussian feature matrix."""
    out = np.zeros((count, F))
    _load().orc_gaussian_rows(u0, count, F, seed, out.ctypes.data)
    return out


def build_walk_index(g: Graph, seed: int, alpha: float = 0.2, max_steps: int = 1 << 16) -> np.ndarray:
    """SpeedPPR-Index: endpoint of the walk stored for every edge slot (m entries)."""
    idx = np.zeros(max(g.m, 1), dtype=np.int32)
    _rc(_load().orc_build_walk_index(*g.args(), alpha, seed, max_steps, idx.ctypes.data), "build_walk_index")
    return idx[:g.m]


def index_walks(g: Graph, index: np.ndarray, r: np.ndarray, W: float):
    """Walk phase of Algorithm 4 read from the index; returns (counts, est, stats)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    idx = np.ascontiguousarray(index, dtype=np.int32)
    counts = np.zeros(g.n, dtype=np.uint32)
    est = np.zeros(g.n)
    st = Stats()
    _rc(_load().orc_index_walks(g.n, g.row_ptr.ctypes.data, idx.ctypes.data, r.ctypes.data, W, counts.ctypes.data,
                                est.ctypes.data, ctypes.byref(st)), "index_walks")
    return counts, est, st.as_dict()
