"""ctypes binding of the C ABI declared in include/ppr.h.

Argument marshalling only: every step of a query runs in the CUDA library.
There is no CPU fallback; if the library cannot be loaded or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

PPR_OK, PPR_ERR_ARG, PPR_ERR_GRAPH, PPR_ERR_OOM = 0, -1, -2, -3
PPR_ERR_NOT_CONVERGED, PPR_ERR_CUDA, PPR_ERR_ADMIT = -4, -5, -6
PPR_HP, PPR_APPROX = 0, 1
PPR_FLAG_PARTIAL = 1
PPR_FLAG_SYNC = 2
PPR_FLAG_INDEX = 4
PPR_FLAG_FIXED_PASSES = 8
PPR_FLAG_NO_ACTIVE = 16
PPR_FLAG_FP32_ONLY = 32
PPR_FLAG_TMA_GATHER = 64
PPR_INJECT_FREE_BYTES = 1
PPR_INJECT_ALLOC_FAIL = 2

STATUS_NAMES = {0: "PPR_OK", -1: "PPR_ERR_ARG", -2: "PPR_ERR_GRAPH", -3: "PPR_ERR_OOM",
                -4: "PPR_ERR_NOT_CONVERGED", -5: "PPR_ERR_CUDA", -6: "PPR_ERR_ADMIT"}


class PPRError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ppr_query_opts(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("k_tile", ctypes.c_int32),
        ("epoch_num", ctypes.c_int32),
        ("switch_edges", ctypes.c_int64),
        ("max_sweeps", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("warm_start", ctypes.c_void_p),
    ]


class ppr_stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int32),
        ("levels", ctypes.c_int32),
        ("edges_pushed", ctypes.c_int64),
        ("edges_swept", ctypes.c_int64),
        ("walks", ctypes.c_int64),
        ("walk_steps", ctypes.c_int64),
        ("initial_l1_residual", ctypes.c_double),
        ("final_l1_residual", ctypes.c_double),
        ("mass_deficit", ctypes.c_double),
        ("ms_push", ctypes.c_double),
        ("ms_sweep", ctypes.c_double),
        ("ms_walk", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("sweep_launches", ctypes.c_int64),
        ("W", ctypes.c_double),
        ("fp32_passes", ctypes.c_int32),
        ("refine_cycles", ctypes.c_int32),
        ("ms_fp32", ctypes.c_double),
        ("bf16_passes", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("ms_bf16", ctypes.c_double),
        ("relax", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ppr_model_opts(ctypes.Structure):
    _fields_ = [
        ("feat_dim", ctypes.c_int32),
        ("hidden", ctypes.c_int32),
        ("rank", ctypes.c_int32),
        ("correction_passes", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("lr", ctypes.c_float),
        ("epochs", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("lambda_", ctypes.c_double),
    ]


# every symbol include/ppr.h declares, with its ctypes signature
_P = ctypes.c_void_p
SIGNATURES = {
    "ppr_default_opts": (None, [ctypes.POINTER(ppr_query_opts)]),
    "ppr_graph_load": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, ctypes.POINTER(_P)]),
    "ppr_sssp_query": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int, ctypes.POINTER(ppr_query_opts),
                                      _P, _P, _P, _P, _P]),
    "ppr_free": (None, [_P]),
    "ppr_sssp_query_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P, _P,
                                              _P]),
    "ppr_last_error": (ctypes.c_char_p, []),
    "ppr_graph_n": (ctypes.c_int64, [_P]),
    "ppr_graph_m": (ctypes.c_int64, [_P]),
    "ppr_query_state_bytes": (ctypes.c_int64, [_P, ctypes.c_int32, ctypes.c_int32]),
    "ppr_workspace_bytes": (ctypes.c_int64, [_P]),
    "ppr_inject": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "ppr_selftest_fixconv": (ctypes.c_int, [ctypes.c_int64, ctypes.c_uint64, _P, _P]),
    "ppr_index_build": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, _P]),
    "ppr_index_get": (ctypes.c_int, [_P, _P]),
    "ppr_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(ppr_query_opts), _P,
                                    ctypes.POINTER(ppr_query_opts), ctypes.POINTER(ctypes.c_double), _P]),
    "ppr_model_default_opts": (None, [ctypes.POINTER(ppr_model_opts)]),
    "ppr_model_create": (ctypes.c_int, [_P, ctypes.POINTER(ppr_model_opts), ctypes.POINTER(_P)]),
    "ppr_model_train": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                                       _P, _P]),
    "ppr_model_train_step": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, ctypes.c_float, _P, _P]),
    "ppr_model_estimate": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "ppr_model_param_count": (ctypes.c_int64, [_P]),
    "ppr_model_get_params": (ctypes.c_int, [_P, _P, _P]),
    "ppr_model_set_params": (ctypes.c_int, [_P, _P]),
    "ppr_model_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "ppr_model_load": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(_P)]),
    "ppr_model_free": (None, [_P]),
}

_lock = threading.Lock()
_lib = None


def load_library(build: bool = True):
    """Load libppr_gb300.so (building it first if sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise ImportError(f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def ppr_last_error() -> str:
    return load_library().ppr_last_error().decode()


def _check(status: int):
    if status != PPR_OK:
        raise PPRError(status, ppr_last_error())


def ppr_default_opts(**kw) -> ppr_query_opts:
    o = ppr_query_opts()
    load_library().ppr_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, "lambda_" if k == "lam" else k, v)
    return o


def _ptr(x):
    """(address, is_device) of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _buf(x, k: int, n: int, kind: str, name: str):
    """Address of a k x n row-major buffer (numpy array or torch tensor, host
    or device) that the library reads or writes through a raw pointer, checked
    first: element type (kind "f64" = float64, "u32" = 32-bit counts),
    contiguity, and room for k x n elements with rows of n."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if kind == "f64":
            ok = x.dtype == np.float64
        else:
            ok = x.dtype in (np.int32, np.uint32)
        contiguous, size, shape, addr = x.flags["C_CONTIGUOUS"], x.size, x.shape, x.ctypes.data
    else:
        import torch
        if kind == "f64":
            ok = x.dtype == torch.float64
        else:
            ok = x.dtype in (torch.int32, getattr(torch, "uint32", torch.int32))
        contiguous, size, shape, addr = x.is_contiguous(), x.numel(), tuple(x.shape), x.data_ptr()
    if not ok:
        raise TypeError(f"{name}: needs {'float64' if kind == 'f64' else 'int32 or uint32'} elements, got {x.dtype}")
    if not contiguous:
        raise ValueError(f"{name}: must be contiguous (row-major)")
    if size < k * n or (len(shape) >= 2 and shape[-1] != n):
        raise ValueError(f"{name}: needs shape ({k}, {n}), got {tuple(shape)}")
    return addr


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def ppr_graph_load(row_ptr: np.ndarray, col_idx: np.ndarray, stream=None) -> int:
    """Upload a CSR graph; returns the opaque graph handle (an int)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load_library().ppr_graph_load(rp.ctypes.data, ci.ctypes.data, len(rp) - 1, len(ci), _stream(stream),
                                         ctypes.byref(h)))
    return h.value


def ppr_sssp_query(graph: int, src, mode: int, opts: ppr_query_opts, out_pi, out_r=None, out_walk_counts=None,
                   stats: bool = True, stream=None):
    """Run k queries; out_* are torch tensors (CUDA or CPU) or numpy arrays of shape (k, n)."""
    s = np.ascontiguousarray(src, dtype=np.int32)
    k, n = len(s), load_library().ppr_graph_n(graph)
    st = (ppr_stats * len(s))() if stats else None
    _check(load_library().ppr_sssp_query(graph, s.ctypes.data, len(s), mode, ctypes.byref(opts),
                                         _buf(out_pi, k, n, "f64", "out_pi"), _buf(out_r, k, n, "f64", "out_r"),
                                         _buf(out_walk_counts, k, n, "u32", "out_walk_counts"), st,
                                         _stream(stream)))
    return [x.as_dict() for x in st] if stats else None


def ppr_sssp_query_noalloc(graph: int, src, out_pi, alpha: float = 0.2, lam: float = 1e-8, stream=None):
    """High-precision queries through the entry point that allocates nothing
    (scratch compiled into the library); out_pi must be a (k, n) float64 CUDA
    tensor.  Returns the passes run per source."""
    s = np.ascontiguousarray(src, dtype=np.int32)
    sweeps = np.zeros(len(s), dtype=np.int32)
    out = _buf(out_pi, len(s), load_library().ppr_graph_n(graph), "f64", "out_pi")
    _check(load_library().ppr_sssp_query_noalloc(graph, s.ctypes.data, len(s), alpha, lam, out,
                                                 sweeps.ctypes.data, _stream(stream)))
    return sweeps


def ppr_inject(hook: int, value: int):
    """Test hook for the error paths (see include/ppr.h): PPR_INJECT_FREE_BYTES
    caps the free device bytes admission sees (value < 0: off);
    PPR_INJECT_ALLOC_FAIL makes the value-th workspace allocation fail (0: off)."""
    _check(load_library().ppr_inject(hook, value))


def ppr_selftest_fixconv(count: int = 1 << 24, seed: int = 0x5EED, stream=None) -> list:
    """Mismatch counts of the device's fixed-point <-> FP32/FP64 conversions
    against CUDA's intrinsics (see include/ppr.h); all zero when they agree."""
    out = np.zeros(7, dtype=np.int64)
    _check(load_library().ppr_selftest_fixconv(count, seed, out.ctypes.data, _stream(stream)))
    return out.tolist()


def ppr_free(graph: int):
    if graph:
        load_library().ppr_free(graph)


class Graph:
    """Owner of a device graph: ``Graph(row_ptr, col_idx).query(src, ...)``."""

    def __init__(self, row_ptr, col_idx, stream=None):
        self.n = len(row_ptr) - 1
        self.m = len(col_idx)
        self.handle = ppr_graph_load(row_ptr, col_idx, stream)

    def close(self):
        if self.handle:
            ppr_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, src, stream=None, **opts):
        """Time tile widths and switch thresholds on src; returns (k_tile,
        switch_edges, ms) of the fastest, which later auto calls use."""
        import torch
        s = np.ascontiguousarray(src, dtype=np.int32)
        out = torch.empty((len(s), self.n), dtype=torch.float64, device="cuda")
        base = ppr_default_opts(**opts)
        best = ppr_query_opts()
        ms = ctypes.c_double()
        _check(load_library().ppr_autotune(self.handle, s.ctypes.data, len(s), ctypes.byref(base), _ptr(out),
                                           ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
        return best.k_tile, best.switch_edges, ms.value

    def build_index(self, seed: int = 0x5EED, alpha: float = 0.2, stream=None):
        """SpeedPPR-Index: d_v stored walks per node (m endpoints) on the device."""
        _check(load_library().ppr_index_build(self.handle, seed, alpha, _stream(stream)))

    def get_index(self) -> np.ndarray:
        out = np.zeros(max(self.m, 1), dtype=np.int32)
        _check(load_library().ppr_index_get(self.handle, out.ctypes.data))
        return out[:self.m]

    def state_bytes(self, k: int, k_tile: int = 0) -> int:
        """Device workspace of a high-precision query of k sources."""
        return load_library().ppr_query_state_bytes(self.handle, k, k_tile)

    def workspace_bytes(self) -> int:
        """Device bytes the graph's query workspace holds now."""
        return load_library().ppr_workspace_bytes(self.handle)

    def query(self, src, mode: int = PPR_HP, out_pi=None, out_r=None, out_walk_counts=None, stream=None,
              warm_start=None, **opts):
        """Returns (pi, stats); pi is a (k, n) float64 CUDA tensor unless out_pi is given.
        warm_start: a Model of this graph (HP only)."""
        import torch
        k = len(src)
        if out_pi is None:
            out_pi = torch.empty((k, self.n), dtype=torch.float64, device="cuda")
        o = ppr_default_opts(**opts)
        if warm_start is not None:
            o.warm_start = warm_start.handle
        stats = ppr_sssp_query(self.handle, src, mode, o, out_pi, out_r, out_walk_counts, True, stream)
        return out_pi, stats


def ppr_model_default_opts(**kw) -> ppr_model_opts:
    o = ppr_model_opts()
    load_library().ppr_model_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, "lambda_" if k == "lam" else k, v)
    return o


class Model:
    """Learned warm start of a Graph (see include/ppr.h)."""

    def __init__(self, graph: Graph, handle=None, **opts):
        self.graph = graph
        if handle is None:
            h = ctypes.c_void_p()
            o = ppr_model_default_opts(**opts)
            _check(load_library().ppr_model_create(graph.handle, ctypes.byref(o), ctypes.byref(h)))
            handle = h.value
        self.handle = handle

    @classmethod
    def load(cls, graph: Graph, path: str) -> "Model":
        h = ctypes.c_void_p()
        _check(load_library().ppr_model_load(graph.handle, path.encode(), ctypes.byref(h)))
        return cls(graph, handle=h.value)

    def save(self, path: str):
        _check(load_library().ppr_model_save(self.handle, path.encode()))

    def close(self):
        if self.handle:
            load_library().ppr_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, src, epochs: int, lr: float = 1e-3, shuffle_seed: int = 0, stream=None):
        s = np.ascontiguousarray(src, dtype=np.int32)
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(load_library().ppr_model_train(self.handle, s.ctypes.data, len(s), epochs, lr, shuffle_seed,
                                              losses.ctypes.data, _stream(stream)))
        return losses[:epochs]

    def train_step(self, src, labels, lr: float = 0.0, stream=None) -> float:
        s = np.ascontiguousarray(src, dtype=np.int32)
        loss = ctypes.c_double()
        _check(load_library().ppr_model_train_step(self.handle, s.ctypes.data, len(s),
                                                   _buf(labels, len(s), self.graph.n, "f64", "labels"), lr,
                                                   ctypes.byref(loss), _stream(stream)))
        return loss.value

    def estimate(self, src, out=None, stream=None):
        s = np.ascontiguousarray(src, dtype=np.int32)
        if out is None:
            out = np.zeros((len(s), self.graph.n))
        _check(load_library().ppr_model_estimate(self.handle, s.ctypes.data, len(s),
                                                 _buf(out, len(s), self.graph.n, "f64", "out"), _stream(stream)))
        return out

    def param_count(self) -> int:
        return load_library().ppr_model_param_count(self.handle)

    def get_params(self, grads: bool = False):
        cnt = self.param_count()
        p = np.zeros(cnt, dtype=np.float32)
        g = np.zeros(cnt, dtype=np.float32) if grads else None
        _check(load_library().ppr_model_get_params(self.handle, p.ctypes.data, g.ctypes.data if grads else None))
        return (p, g) if grads else p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert len(p) == self.param_count()
        _check(load_library().ppr_model_set_params(self.handle, p.ctypes.data))
