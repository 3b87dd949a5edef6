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
    assert ctypes.sizeof(binding.ppr_stats) == 152


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
