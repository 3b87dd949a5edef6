"""Seeded synthetic inputs: directed power-law graphs (CSR) and source lists.

This module builds the inputs that both the FP64 oracle and the CUDA library
consume.  It contains no Personalized PageRank arithmetic.  The graphs stand
in for the SNAP datasets of the paper's experiments (Sec. 8, Table 2), which
are directed power-law graphs; every sink is given one uniform random
out-edge so that the no-dead-end assumption of Sec. 2 holds.

Workload recipes (sizes follow the configurations the library is measured on):

* ``chung_lu(10_000, 100_000, 2.2, seed=1)``: small directed Chung-Lu graph.
* ``rmat(20, 16)``, ``rmat(22, 16)``, ``rmat(25, 32)``: R-MAT with
  (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), ids randomly relabelled.
* ``sources(n, k, seed)``: k uniform random source ids.
* ``bfs_subgraph(...)``: the first nodes reached by BFS, induced edges.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libppr_inputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            pp64 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))
            pp32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
            lib.pg_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_int, i64p, pp64, pp32]
            lib.pg_rmat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i64p, pp64, pp32]
            lib.pg_sources.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            lib.pg_bfs_subgraph.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int64, ctypes.c_uint64, i64p, i64p, pp64, pp32]
            lib.pg_free.argtypes = [ctypes.c_void_p]
            for f in (lib.pg_chung_lu, lib.pg_rmat, lib.pg_sources, lib.pg_bfs_subgraph):
                f.restype = ctypes.c_int
            lib.pg_free.restype = None
            _lib = lib
    return _lib


def _take(lib, rp_ptr, ci_ptr, n: int, m: int):
    rp = np.ctypeslib.as_array(rp_ptr, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(ci_ptr, shape=(max(m, 1),))[:m].copy()
    lib.pg_free(ctypes.cast(rp_ptr, ctypes.c_void_p))
    lib.pg_free(ctypes.cast(ci_ptr, ctypes.c_void_p))
    return rp, ci


def _check(rc: int, what: str):
    if rc == -1:
        raise MemoryError(f"{what}: out of host memory")
    if rc != 0:
        raise ValueError(f"{what}: invalid arguments (rc={rc})")


def chung_lu(n: int, m_draws: int, gamma: float = 2.2, seed: int = 1, threads: int = 0):
    """Directed Chung-Lu graph; returns (row_ptr int64[n+1], col_idx int32[m])."""
    lib = _load()
    m = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    _check(lib.pg_chung_lu(n, m_draws, gamma, seed, threads, ctypes.byref(m), ctypes.byref(rp), ctypes.byref(ci)),
           "chung_lu")
    return _take(lib, rp, ci, n, m.value)


def rmat(scale: int, edge_factor: float = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, threads: int = 0):
    """R-MAT graph with n = 2**scale; returns (row_ptr int64[n+1], col_idx int32[m])."""
    lib = _load()
    m = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    _check(lib.pg_rmat(scale, edge_factor, a, b, c, seed, threads, ctypes.byref(m), ctypes.byref(rp),
                       ctypes.byref(ci)), "rmat")
    return _take(lib, rp, ci, 1 << scale, m.value)


def sources(n: int, k: int, seed: int) -> np.ndarray:
    """k uniform random source ids in [0, n) as int32."""
    out = np.empty(k, dtype=np.int32)
    _check(_load().pg_sources(n, k, seed, out.ctypes.data), "sources")
    return out


def bfs_subgraph(row_ptr: np.ndarray, col_idx: np.ndarray, root: int, count: int, seed: int = 1):
    """Induced subgraph on the first `count` BFS-visited nodes, relabelled in visit order."""
    lib = _load()
    rp_in = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci_in = np.ascontiguousarray(col_idx, dtype=np.int32)
    nn = ctypes.c_int64()
    m = ctypes.c_int64()
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    _check(lib.pg_bfs_subgraph(len(rp_in) - 1, rp_in.ctypes.data, ci_in.ctypes.data, root, count, seed,
                               ctypes.byref(nn), ctypes.byref(m), ctypes.byref(rp), ctypes.byref(ci)),
           "bfs_subgraph")
    return _take(lib, rp, ci, nn.value, m.value)


def from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """CSR from an explicit (src, dst) list (small hand-written graphs); rows sorted."""
    edges = sorted(set((int(a), int(b)) for a, b in edges))
    rp = np.zeros(n + 1, dtype=np.int64)
    for a, _ in edges:
        rp[a + 1] += 1
    rp = np.cumsum(rp).astype(np.int64)
    ci = np.array([b for _, b in edges], dtype=np.int32)
    return rp, ci


def fig1_graph() -> tuple[np.ndarray, np.ndarray]:
    """The 5-node example graph of Fig. 1 (v1..v5 read as ids 0..4), read off its
    printed transition matrix P: row v lists the columns where P[v] > 0."""
    out = {0: [1, 2], 1: [0, 2, 3, 4], 2: [1, 3], 3: [0, 1, 2], 4: [1, 2]}
    return from_edges(5, [(v, u) for v, us in out.items() for u in us])
