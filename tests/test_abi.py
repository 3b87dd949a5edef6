"""The C ABI library builds, loads and exports every declared symbol (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2101_03652_gb300 as P
from paper_2101_03652_gb300 import binding
import ppr_inputs as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(ppr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = P.load_library()
    names = declared_functions()
    assert "ppr_graph_load" in names and "ppr_sssp_query" in names and "ppr_free" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, f"binding lacks {name}"


def test_default_opts_and_struct_layout():
    o = P.ppr_default_opts()
    assert o.alpha == 0.2 and o.lambda_ == 1e-8 and o.eps == 0.5 and o.seed == 0x5EED
    assert o.k_tile == 0 and o.epoch_num == 0 and o.switch_edges == -1 and o.max_sweeps == 0
    # layout fixed by include/ppr.h (x86-64 and aarch64 LP64 agree)
    assert ctypes.sizeof(binding.ppr_query_opts) == 72
    assert ctypes.sizeof(binding.ppr_stats) == 160


@pytest.mark.parametrize("case", ["sink", "self_loop", "unsorted", "out_of_range", "bad_rowptr"])
def test_graph_contract_violations_rejected_before_device(case):
    rp, ci = gen.fig1_graph()
    rp = rp.copy()
    ci = ci.copy()
    if case == "sink":       # node 0 loses its out-edges
        rp = np.array([0, 0, 4, 6, 9, 11], dtype=np.int64)
        ci = ci[2:]
    elif case == "self_loop":
        ci[0] = 0
    elif case == "unsorted":
        ci[0], ci[1] = ci[1], ci[0]
    elif case == "out_of_range":
        ci[-1] = 5
    elif case == "bad_rowptr":
        rp[-1] += 1
    with pytest.raises(P.PPRError) as e:
        P.ppr_graph_load(rp, ci)
    assert e.value.status == binding.PPR_ERR_GRAPH


def test_null_and_empty_arguments():
    lib = P.load_library()
    h = ctypes.c_void_p()
    assert lib.ppr_graph_load(None, None, 5, 13, None, ctypes.byref(h)) == binding.PPR_ERR_ARG
    assert lib.ppr_sssp_query(None, None, 0, 0, None, None, None, None, None, None) == binding.PPR_ERR_ARG
    lib.ppr_free(None)  # NULL-safe
    assert lib.ppr_graph_n(None) == 0


def test_no_cpu_fallback_without_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rp, ci = gen.fig1_graph()
    with pytest.raises(P.PPRError) as e:
        P.ppr_graph_load(rp, ci)
    assert e.value.status == binding.PPR_ERR_CUDA


def test_binding_constants_match_the_header():
    """Flags, statuses and modes in the binding are the header's values."""
    text = open(os.path.join(ROOT, "include", "ppr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(PPR_FLAG_[A-Z0-9_]+)\s+(\d+)", text)}
    hooks = {k: int(v) for k, v in re.findall(r"#define\s+(PPR_INJECT_[A-Z0-9_]+)\s+(\d+)", text)}
    assert len(hooks) == 2
    for name, value in hooks.items():
        assert getattr(binding, name) == value, name
    enums = {k: int(v) for k, v in re.findall(r"\b(PPR_(?:OK|ERR_[A-Z_]+|HP|APPROX))\s*=\s*(-?\d+)", text)}
    assert len(defines) >= 6 and len(enums) >= 9
    for name, value in {**defines, **enums}.items():
        assert getattr(binding, name) == value, name
    flags = list(defines.values())
    assert len(set(flags)) == len(flags) and all(f & (f - 1) == 0 for f in flags)  # distinct single bits


def test_stats_layout_matches_the_header():
    """ppr_stats: the binding's fields, in order, are the header's."""
    text = open(os.path.join(ROOT, "include", "ppr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\} ppr_stats;", text, flags=re.S).group(1)
    fields = re.findall(r"\b(?:int32_t|int64_t|double)\s+([A-Za-z_0-9]+)\s*;", body)
    assert [f for f, _ in binding.ppr_stats._fields_] == fields


@pytest.mark.parametrize("n,m", [(5, 1 << 31), (1 << 31, 1 << 31), (5, 4)])
def test_size_limits_rejected_before_reading(n, m):
    """n <= m < 2^31 (int32 ids and edge offsets); the sizes are checked before
    either array is read, so small arrays with out-of-range sizes are safe."""
    lib = P.load_library()
    rp, ci = gen.fig1_graph()
    h = ctypes.c_void_p()
    st = lib.ppr_graph_load(rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_int64(n), ctypes.c_int64(m), None, ctypes.byref(h))
    assert st == binding.PPR_ERR_GRAPH and not h.value
    assert b"2^31" in lib.ppr_last_error()


def test_buffers_are_checked_before_the_library_writes_through_them():
    """Output and label buffers reach the library as raw pointers; the binding
    checks element type, contiguity and size first, so a wrong buffer is a
    Python error instead of an out-of-bounds write on the device."""
    torch = pytest.importorskip("torch")
    k, n = 3, 7
    ok = np.zeros((k, n))
    assert binding._buf(ok, k, n, "f64", "out_pi") == ok.ctypes.data
    assert binding._buf(None, k, n, "f64", "out_r") is None
    assert binding._buf(np.zeros((k, n), dtype=np.uint32), k, n, "u32", "c") is not None
    assert binding._buf(torch.zeros((k, n), dtype=torch.int32), k, n, "u32", "c") is not None
    assert binding._buf(torch.zeros((k + 2, n), dtype=torch.float64), k, n, "f64", "out_pi") is not None
    with pytest.raises(TypeError):
        binding._buf(np.zeros((k, n), dtype=np.float32), k, n, "f64", "out_pi")
    with pytest.raises(TypeError):
        binding._buf(torch.zeros((k, n), dtype=torch.float32), k, n, "f64", "out_pi")
    with pytest.raises(TypeError):
        binding._buf(np.zeros((k, n)), k, n, "u32", "out_walk_counts")
    with pytest.raises(ValueError):
        binding._buf(np.zeros((k - 1, n)), k, n, "f64", "out_pi")          # too few rows
    with pytest.raises(ValueError):
        binding._buf(np.zeros((k, n + 1)), k, n, "f64", "out_pi")          # rows of the wrong length
    with pytest.raises(ValueError):
        binding._buf(np.zeros((n, k)).T, k, n, "f64", "out_pi")            # column-major
    with pytest.raises(ValueError):
        binding._buf(torch.zeros((k, 2 * n), dtype=torch.float64)[:, ::2], k, n, "f64", "out_pi")


class _RecordingLib:
    """Stands in for the CUDA library: records what the binding passes."""

    def __init__(self, n):
        self.n, self.calls = n, []

    def ppr_graph_n(self, g):
        return self.n

    def ppr_sssp_query(self, g, src, k, mode, opts, pi, r, counts, stats, stream):
        self.calls.append(("query", k, pi, r, counts))
        return binding.PPR_OK

    def ppr_sssp_query_noalloc(self, g, src, k, alpha, lam, pi, sweeps, stream):
        self.calls.append(("noalloc", k, pi))
        return binding.PPR_OK

    def ppr_model_train_step(self, m, src, k, labels, lr, loss, stream):
        self.calls.append(("train_step", k, labels))
        return binding.PPR_OK

    def ppr_model_estimate(self, m, src, k, out, stream):
        self.calls.append(("estimate", k, out))
        return binding.PPR_OK

    def ppr_model_free(self, m):
        pass


def test_query_marshalling_checks_buffers_against_the_graph(monkeypatch):
    k, n = 4, 9
    fake = _RecordingLib(n)
    monkeypatch.setattr(binding, "load_library", lambda build=True: fake)
    pi, r = np.zeros((k, n)), np.zeros((k, n))
    counts = np.zeros((k, n), dtype=np.uint32)
    st = binding.ppr_sssp_query(0x1000, np.arange(k), binding.PPR_APPROX, binding.ppr_query_opts(), pi, r, counts)
    assert len(st) == k
    assert fake.calls == [("query", k, pi.ctypes.data, r.ctypes.data, counts.ctypes.data)]
    binding.ppr_sssp_query_noalloc(0x1000, np.arange(k), pi)
    assert fake.calls[-1] == ("noalloc", k, pi.ctypes.data)
    with pytest.raises(ValueError):      # rows sized for another graph: rejected before the call
        binding.ppr_sssp_query(0x1000, np.arange(k), binding.PPR_HP, binding.ppr_query_opts(), np.zeros((k, n - 1)))
    with pytest.raises(TypeError):
        binding.ppr_sssp_query(0x1000, np.arange(k), binding.PPR_APPROX, binding.ppr_query_opts(), pi,
                               out_walk_counts=np.zeros((k, n)))
    assert len(fake.calls) == 2


def test_model_marshalling_checks_labels_and_outputs(monkeypatch):
    k, n = 2, 5
    fake = _RecordingLib(n)
    monkeypatch.setattr(binding, "load_library", lambda build=True: fake)

    class _G:
        pass
    g = _G()
    g.n = n
    m = binding.Model(g, handle=0x2000)
    labels = np.ones((k, n))
    m.train_step([0, 1], labels, lr=1e-3)
    assert fake.calls[-1] == ("train_step", k, labels.ctypes.data)
    x = m.estimate([0, 1])
    assert x.shape == (k, n) and fake.calls[-1] == ("estimate", k, x.ctypes.data)
    with pytest.raises(TypeError):
        m.train_step([0, 1], labels.astype(np.float32))
    with pytest.raises(ValueError):
        m.estimate([0, 1, 2], out=np.zeros((2, n)))
    assert len(fake.calls) == 2
    m.handle = None


def test_injection_hooks_and_workspace_query_without_device():
    """The error-path hooks are plain host state: set and cleared without a
    device; an unknown hook is an argument error; a NULL graph holds no
    workspace."""
    lib = P.load_library()
    assert lib.ppr_inject(binding.PPR_INJECT_FREE_BYTES, 1 << 20) == binding.PPR_OK
    assert lib.ppr_inject(binding.PPR_INJECT_FREE_BYTES, -1) == binding.PPR_OK
    assert lib.ppr_inject(binding.PPR_INJECT_ALLOC_FAIL, 3) == binding.PPR_OK
    assert lib.ppr_inject(binding.PPR_INJECT_ALLOC_FAIL, 0) == binding.PPR_OK
    assert lib.ppr_inject(99, 0) == binding.PPR_ERR_ARG
    assert b"unknown injection hook" in lib.ppr_last_error()
    assert lib.ppr_workspace_bytes(None) == -1


def test_conversion_selftest_rejects_bad_arguments_without_device():
    lib = P.load_library()
    out = np.zeros(7, dtype=np.int64)
    assert lib.ppr_selftest_fixconv(-1, 0, out.ctypes.data, None) == binding.PPR_ERR_ARG
    assert lib.ppr_selftest_fixconv(16, 0, None, None) == binding.PPR_ERR_ARG
    assert b"conversion self-test" in lib.ppr_last_error()
