"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle: a dropped term, a wrong
sign, index or operand, a swapped constant.  It then checks that the pin suite
(test_oracle_pins.py, test_oracle_warm.py) fails.  C mistakes are compiled
into a separate library that the pins load through ORACLE_LIBRARY, in a child
process.  Python mistakes (the warm-start oracle) replace one function for
the duration of the test.  Nothing here touches the CUDA library.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy.special import erf

import test_oracle_pins as pins
import test_oracle_warm as warm_pins
from oracle import warm as Wm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "ppr_oracle.c")
PIN_FILES = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_warm.py")]

# (name, text of the oracle, the same text with the mistake)
C_MUTANTS = [
    ("push_drops_damping",
     "  double share = (1.0 - alpha) * rv / (double)d;\n  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) r[ci[e]] += share;",
     "  double share = rv / (double)d;\n  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) r[ci[e]] += share;"),
    ("powitr_reserve_drops_alpha", "      pi[v] += alpha * r[v];", "      pi[v] += r[v];"),
    ("powitr_scatters_to_own_node", "nxt[ci[e]] += share;", "nxt[v] += share;"),
    ("fifo_active_test_uses_pusher_degree", "if (r[u] > (double)du * rmax && !Q->in[u])",
     "if (r[u] > (double)d * rmax && !Q->in[u])"),
    ("fifo_reserve_takes_whole_residue",
     "    pi[v] += alpha * rv;\n    double share = (1.0 - alpha) * rv / (double)d;\n    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {\n      int32_t u = ci[e];\n      r[u] += share;\n      int64_t du",
     "    pi[v] += rv;\n    double share = (1.0 - alpha) * rv / (double)d;\n    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {\n      int32_t u = ci[e];\n      r[u] += share;\n      int64_t du"),
    ("powerpush_queue_scatter_sign", "      r[u] += share;\n      if (!Q.in[u]", "      r[u] -= share;\n      if (!Q.in[u]"),
    ("powerpush_epochs_stop_early", "pow(lambda, (double)i / (double)epoch_num)",
     "pow(lambda, (double)(i - 1) / (double)epoch_num)"),
    ("dense_solve_transposed", "M[(int64_t)ci[e] * n + v] -= (1.0 - alpha) * p;",
     "M[v * n + (int64_t)ci[e]] -= (1.0 - alpha) * p;"),
    ("dense_solve_rhs_drops_alpha", "  b[s] = alpha;", "  b[s] = 1.0;"),
    ("residual_sign", "(b + (1.0 - alpha) * xp[u] - x[u]) / alpha", "(b - (1.0 - alpha) * xp[u] - x[u]) / alpha"),
    ("philox_output_words_swapped", "c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;", "c0 = n0; c1 = lo0; c2 = n2; c3 = lo1;"),
    ("philox_key_schedule", "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;"),
    ("W_base_2_logarithm", "log((double)n) / (eps * eps * mu)", "log2((double)n) / (eps * eps * mu)"),
    ("walk_stop_test_inverted", "if (stopw < stop_below) break;", "if (stopw >= stop_below) break;"),
    ("walk_moves_with_stop_word", "(((uint64_t)movew * (uint64_t)d) >> 32)", "(((uint64_t)stopw * (uint64_t)d) >> 32)"),
    ("walk_estimate_drops_residue", "double inc = r[v] / (double)Wv;\n    for (uint64_t k",
     "double inc = 1.0 / (double)Wv;\n    for (uint64_t k"),
    ("index_walk_count_floor", "int64_t Wv = (int64_t)ceil(r[v] * W);", "int64_t Wv = (int64_t)floor(r[v] * W);"),
    ("index_build_stop_inverted", "if (words[2 * (t & 1)] < stop_below) break;",
     "if (words[2 * (t & 1)] >= stop_below) break;"),
    ("gaussian_box_muller_radius", "sqrt(-2.0 * log(u1))", "sqrt(-log(u1))"),
]


@pytest.mark.parametrize("name,orig,bad", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_pins_catch_planted_c_mistake(tmp_path, name, orig, bad):
    src = open(ORACLE_C).read()
    assert src.count(orig) == 1, f"{name}: the text to mutate must occur exactly once"
    mutant = tmp_path / "ppr_oracle.c"
    mutant.write_text(src.replace(orig, bad))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                           "-o", str(lib), str(mutant), "-lm"])
    env = dict(os.environ, ORACLE_LIBRARY=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    # exit status 1: the pins ran and at least one failed (not a crash or a collection error)
    assert r.returncode == 1, f"{name} survived the pins:\n{r.stdout[-2000:]}"


def _wrong_gelu_grad(x):          # drops the x phi(x) term
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0)))


def _tanh_gelu(x):                # the tanh approximation instead of the erf form
    return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)))


def _transposed_transition(g, x):  # P x instead of x P
    d = np.diff(g.row_ptr)
    src = np.repeat(np.arange(g.n), d)
    return np.bincount(src, weights=x[g.col_idx], minlength=g.n) / d


def _sketch_drops_alive_mass(g, s, alpha=0.2):
    e = np.zeros(g.n)
    e[s] = 1.0
    p1 = Wm.transition_apply(g, e)
    p2 = Wm.transition_apply(g, p1)
    return alpha * e + alpha * (1 - alpha) * p1 + alpha * (1 - alpha) ** 2 * p2


def _bf16_truncate(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return (b & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)


_gaussian_rows = Wm.gaussian_rows


def _features_off_by_one(S, F, seed):
    rows = np.nonzero(np.any(S != 0, axis=1))[0]
    f = np.zeros((S.shape[1], F))
    for u in rows:
        f += np.outer(S[u], _gaussian_rows(int(u) + 1, 1, F, seed)[0])
    return f


def _basis_without_relu(S, U, h, rnd=None):
    r = rnd or (lambda x: x)
    Z = S + r(U) @ r(h).T
    sig = Z.sum(axis=0)
    X = np.where(sig > 0, Z / np.where(sig > 0, sig, 1.0), S)
    return X, (Z, sig)


_backward = Wm.backward


def _backward_wrong_dU(params, S, f, pi, rnd=None):
    L, g = _backward(params, S, f, pi, rnd)
    g[6] = -g[6]
    return L, g


def _adam_without_bias_correction(p, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    return p - lr * m / (np.sqrt(v) + eps), m, v


def _adam_decays_swapped(p, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    return _adam_step(p, m, v, g, lr, t, b1=b2, b2=b1, eps=eps)


def _adam_without_root(p, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    return p - lr * (m / (1.0 - b1 ** t)) / (v / (1.0 - b2 ** t) + eps), m, v


_adam_step = Wm.adam_step

PY_MUTANTS = [
    ("gelu_grad_drops_term", "gelu_grad", _wrong_gelu_grad),
    ("gelu_tanh_form", "gelu", _tanh_gelu),
    ("transition_transposed", "transition_apply", _transposed_transition),
    ("sketch_drops_alive_mass", "sketch", _sketch_drops_alive_mass),
    ("bf16_truncates", "bf16", _bf16_truncate),
    ("features_row_off_by_one", "features", _features_off_by_one),
    ("basis_without_relu", "basis_forward", _basis_without_relu),
    ("backward_dU_sign", "backward", _backward_wrong_dU),
    ("adam_without_bias_correction", "adam_step", _adam_without_bias_correction),
    ("adam_decays_swapped", "adam_step", _adam_decays_swapped),
    ("adam_without_root", "adam_step", _adam_without_root),
]


def _warm_pin_functions():
    return [getattr(warm_pins, n) for n in dir(warm_pins) if n.startswith("test_")]


@pytest.mark.parametrize("name,attr,fn", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_planted_python_mistake(monkeypatch, name, attr, fn):
    monkeypatch.setattr(Wm, attr, fn)
    caught = 0
    for pin in _warm_pin_functions():
        try:
            pin()
        except AssertionError:
            caught += 1
        except pytest.skip.Exception:
            pass
    assert caught >= 1, f"{name} survived the pins"


def test_unmodified_oracle_passes_the_pins_it_is_mutated_against():
    """The same in-process pin calls pass on the oracle as written."""
    for pin in _warm_pin_functions():
        try:
            pin()
        except pytest.skip.Exception:
            pass
    assert pins.ALPHA == warm_pins.ALPHA == 0.2
