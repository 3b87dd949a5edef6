"""Pins for the FP64 oracle against values and facts fixed outside the oracle.

Each test names what it is pinned to: numbers printed in the paper's worked
examples (tests/golden), closed forms (Eq. 6), the dense linear system of
Eq. 1 solved by LAPACK, Lemma 1's matrix-power identity, the invariants of
Sec. 3.2 and the counter bounds of Lemmas 3-4, Philox known answers and an
independent Philox implementation, and SpeedPPR's probabilistic guarantee.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import ppr_inputs as gen
from conftest import read_golden

ALPHA = 0.2


def fig1():
    return O.Graph(*gen.fig1_graph())


def dense_P(g):
    n = g.n
    P = np.zeros((n, n))
    for v in range(n):
        a, b = g.row_ptr[v], g.row_ptr[v + 1]
        P[v, g.col_idx[a:b]] = 1.0 / (b - a)
    return P


def lapack_ppr(g, s, alpha=ALPHA):
    """Eq. 1 via numpy.linalg.solve (LAPACK gesv), independent of the oracle."""
    P = dense_P(g)
    e = np.zeros(g.n)
    e[s] = alpha
    return np.linalg.solve(np.eye(g.n) - (1 - alpha) * P.T, e)


@pytest.fixture(scope="module")
def cl_small():
    return O.Graph(*gen.chung_lu(2000, 20000, 2.2, seed=7))


@pytest.fixture(scope="module")
def sub200():
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    return O.Graph(*gen.bfs_subgraph(rp, ci, 0, 200, seed=1))


# ----------------------------------------------------------------- Fig. 1-3
def test_fig1_transition_matrix():
    rows = read_golden("fig1_transition_matrix.txt")
    printed = np.array([[float(Fraction(x)) for x in row] for row in rows])
    assert np.array_equal(dense_P(fig1()), printed)


def test_fig2_fwdpush_running_example():
    g = fig1()
    gold = {(r[0], r[1]): np.array([float(x) for x in r[2:]]) for r in read_golden("fig2_fwdpush_example.txt")}
    for order, tag in (([0], "after_v1"), ([0, 2], "after_v3"), ([0, 2, 1], "final")):
        pi, r = O.push_sequence(g, 0, order, ALPHA)
        np.testing.assert_allclose(pi, gold[(tag, "reserve")], atol=1e-15)
        np.testing.assert_allclose(r, gold[(tag, "residue")], atol=1e-15)
    # "no node is active" at the end (r_max = 0.099)
    d = np.diff(g.row_ptr)
    assert np.all(r <= d * 0.099)


def test_fifo_fwdpush_fig1_by_hand():
    g = fig1()
    gold = {r[1]: np.array([float(x) for x in r[2:]]) for r in read_golden("fifo_fwdpush_fig1.txt")}
    pi, r, st = O.fifo_fwdpush(g, 0, ALPHA, rmax=0.099, lam=1e-8)
    np.testing.assert_allclose(pi, gold["reserve"], atol=1e-15)
    np.testing.assert_allclose(r, gold["residue"], atol=1e-15)
    assert st["pushes"] == 3


def test_fig3_simfwdpush_running_example():
    g = fig1()
    gold = {r[0]: np.array([float(x) for x in r[1:]]) for r in read_golden("fig3_simfwdpush_example.txt")}
    # PowItr stops once ||r||_1 <= lambda: lambda between 0.8^2 and 0.8 stops after two iterations
    _, r1, st1 = O.powitr(g, 0, ALPHA, lam=0.81)
    _, r2, st2 = O.powitr(g, 0, ALPHA, lam=0.65)
    assert st1["iterations"] == 1 and st2["iterations"] == 2
    np.testing.assert_allclose(r1, gold["r1"], atol=1e-15)
    np.testing.assert_allclose(r2, gold["r2"], atol=1e-15)


# ---------------------------------------------------------- closed forms
def test_powitr_83_iterations_closed_form(cl_small):
    """Eq. 6: the l1 error after j iterations is exactly (1-alpha)^j, so
    lambda = 1e-8, alpha = 0.2 needs ceil(ln 1e-8 / ln 0.8) = 83 iterations."""
    for s in (0, 5, 1234):
        pi, r, st = O.powitr(cl_small, s, ALPHA, 1e-8)
        assert st["iterations"] == 83
        assert abs(st["r_sum"] - 0.8 ** 83) <= 1e-12 * 0.8 ** 83
        assert abs(pi.sum() - (1 - 0.8 ** 83)) < 1e-13


def test_lemma1_matrix_power(cl_small):
    """Lemma 1 / Eq. 3: r^(j) = (1-alpha)^j e_s P^j, with P^j from numpy."""
    g = O.Graph(*gen.chung_lu(300, 3000, 2.2, seed=3))
    P = dense_P(g)
    s = 7
    e = np.zeros(g.n)
    e[s] = 1.0
    for j in (1, 2, 5, 9):
        _, r, st = O.powitr(g, s, ALPHA, lam=0.8 ** j * (1 + 1e-9))
        assert st["iterations"] == j
        expect = (0.8 ** j) * (e @ np.linalg.matrix_power(P, j))
        np.testing.assert_allclose(r, expect, atol=1e-15)


# ------------------------------------------------------------ dense solve
def test_dense_solve_matches_lapack(sub200):
    for s in (0, 17, 199):
        np.testing.assert_allclose(O.dense_solve(sub200, s, ALPHA), lapack_ppr(sub200, s), atol=1e-14)


def test_methods_within_lambda_of_exact(sub200):
    lam = 1e-8
    for s in (0, 3, 150):
        exact = lapack_ppr(sub200, s)
        for name, (pi, r, st) in {
            "powitr": O.powitr(sub200, s, ALPHA, lam),
            "fifo": O.fifo_fwdpush(sub200, s, ALPHA, lam=lam),
            "powerpush": O.powerpush(sub200, s, ALPHA, lam),
        }.items():
            err = np.abs(pi - exact).sum()
            assert err <= lam, (name, err)
            # Sec. 3.2 error identity: ||pi - pi_hat||_1 = sum r for r >= 0
            assert abs(err - r.sum()) <= 1e-13, name
            assert np.all(pi <= exact + 1e-15), name  # underestimate


def test_paper_dataset_rule_lambda(sub200):
    """lambda = min(1/m, 1e-8) (Sec. 2); on a tiny graph 1/m dominates."""
    lam = min(1.0 / sub200.m, 1e-8)
    pi, _, _ = O.powerpush(sub200, 0, ALPHA, lam)
    assert np.abs(pi - lapack_ppr(sub200, 0)).sum() <= lam


# -------------------------------------------------------------- invariants
def test_mass_invariant_and_termination(cl_small):
    lam = 1e-8
    m = cl_small.m
    d = np.diff(cl_small.row_ptr)
    for s in (1, 99):
        pi, r, st = O.fifo_fwdpush(cl_small, s, ALPHA, lam=lam)
        assert abs(pi.sum() + r.sum() - 1.0) <= 1e-12
        assert np.all(r >= 0)
        assert np.all(r <= d * (lam / m))          # Algorithm 2 terminates with no active node
        assert r.sum() <= lam                        # Sec. 3.2: sum r <= m r_max
        pi2, r2, st2 = O.powerpush(cl_small, s, ALPHA, lam)
        assert abs(pi2.sum() + r2.sum() - 1.0) <= 1e-12
        assert r2.sum() <= lam and np.all(r2 >= 0)


def test_theorem1_edge_push_counters(cl_small):
    """Lemma 3: edge pushes until r_sum <= lambda (at an iteration end) are at
    most (m/alpha) ln(1/lambda) + m.  Lemma 4: afterwards at most m/alpha more.
    Both need r_max < 1/(2m)."""
    m = cl_small.m
    for lam in (1e-4, 1e-8, 1e-10):
        rmax = lam / m
        assert rmax < 1 / (2 * m)
        _, _, st = O.fifo_fwdpush(cl_small, 3, ALPHA, rmax=rmax, lam=lam)
        t_lam = st["edge_pushes_at_lambda"]
        assert t_lam > 0
        assert t_lam <= (m / ALPHA) * math.log(1 / lam) + m
        assert st["edge_pushes"] - t_lam <= m / ALPHA


def test_push_methods_agree(cl_small):
    lam = 1e-8
    for s in (2, 500):
        a, _, _ = O.powitr(cl_small, s, ALPHA, lam)
        b, _, _ = O.fifo_fwdpush(cl_small, s, ALPHA, lam=lam)
        c, _, stc = O.powerpush(cl_small, s, ALPHA, lam)
        assert np.abs(a - b).sum() <= 2 * lam
        assert np.abs(a - c).sum() <= 2 * lam
        assert np.abs(b - c).sum() <= 2 * lam
        assert stc["scans"] > 0 or stc["fifo_pushes"] > 0


def test_powerpush_switches_to_scans(cl_small):
    """With scan_threshold small the queue phase ends early and epochs run."""
    pi, r, st = O.powerpush(cl_small, 4, ALPHA, 1e-8, scan_threshold=10)
    assert st["scans"] > 0 and st["fifo_pushes"] < st["pushes"]
    assert r.sum() <= 1e-8
    ref, _, _ = O.powitr(cl_small, 4, ALPHA, 1e-10)
    assert np.abs(pi - ref).sum() <= 2e-8


def test_residual_identity():
    """pi - x = r Pi with Pi = alpha (I - (1-alpha) P)^-1 (the push invariant
    of Sec. 3.2), checked with a numpy inverse on a small graph."""
    g = O.Graph(*gen.chung_lu(150, 1500, 2.2, seed=11))
    P = dense_P(g)
    Pi = ALPHA * np.linalg.inv(np.eye(g.n) - (1 - ALPHA) * P)
    rng = np.random.default_rng(0)
    s = 5
    x = rng.random(g.n)
    x /= x.sum()
    r = O.residual(g, s, x, ALPHA)
    exact = lapack_ppr(g, s)
    np.testing.assert_allclose(exact - x, r @ Pi, atol=1e-13)
    assert abs(r.sum() - (1 - x.sum())) < 1e-13           # mass: sum r = 1 - sum x
    np.testing.assert_allclose(O.residual(g, s, np.zeros(g.n), ALPHA), np.eye(g.n)[s], atol=0)
    assert np.abs(O.residual(g, s, exact, ALPHA)).sum() < 1e-12


def test_certificate_of_one_exact_pass():
    """The stopping rule of every high-precision mode: for any estimate x and
    x' = alpha e_s + (1-alpha) x P (one exact synchronous pass),
    ||pi - x'||_1 <= (1-alpha) ||x' - x||_1 / alpha, and the pass contracts the
    error by (1-alpha).  Checked against LAPACK on estimates of every kind the
    library meets: positive, signed, under or over mass, near the answer."""
    g = O.Graph(*gen.chung_lu(150, 1500, 2.2, seed=12))
    P = dense_P(g)
    s = 9
    exact = lapack_ppr(g, s)
    e_s = np.eye(g.n)[s]
    rng = np.random.default_rng(5)
    starts = [np.zeros(g.n), rng.random(g.n) / g.n, rng.normal(0, 1e-3, g.n),
              exact + rng.normal(0, 1e-9, g.n), 2.0 * exact, np.abs(rng.standard_cauchy(g.n))]
    for x in starts:
        x1 = ALPHA * e_s + (1 - ALPHA) * x @ P
        err1 = np.abs(exact - x1).sum()
        assert err1 <= (1 - ALPHA) * np.abs(x1 - x).sum() / ALPHA * (1 + 1e-12) + 1e-15
        assert err1 <= (1 - ALPHA) * np.abs(exact - x).sum() * (1 + 1e-12) + 1e-15


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        out = O.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_matches_independent_implementation():
    """Triton's Philox (its own source, run by its CPU interpreter) as a second
    implementation of the same published generator."""
    triton = pytest.importorskip("triton")
    import os
    import subprocess
    import sys
    code = r'''
import os
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(c0, c1, c2, c3, out, K0: tl.constexpr, K1: tl.constexpr, N: tl.constexpr):
    i = tl.arange(0, N)
    a = tl.load(c0 + i); b = tl.load(c1 + i); c = tl.load(c2 + i); d = tl.load(c3 + i)
    k0 = tl.full([N], K0, tl.uint32); k1 = tl.full([N], K1, tl.uint32)
    r0, r1, r2, r3 = tl.random.philox_impl(a, b, c, d, k0, k1, 10)
    tl.store(out + i * 4 + 0, r0); tl.store(out + i * 4 + 1, r1)
    tl.store(out + i * 4 + 2, r2); tl.store(out + i * 4 + 3, r3)
N = 8
rng = np.random.default_rng(5)
ctr = rng.integers(0, 2**32, size=(4, N), dtype=np.uint64).astype(np.uint32)
ts = [torch.from_numpy(ctr[j].view(np.int32).copy()).view(torch.uint32) for j in range(4)]
out = torch.zeros(N * 4, dtype=torch.uint32)
k[(1,)](*ts, out, 0x1234567, 0x89ABCDE, N)
np.save(os.environ["PHILOX_OUT"], np.stack([ctr.T.reshape(-1), out.view(torch.int32).numpy().view(np.uint32)]))
'''
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "o.npy")
        env = dict(os.environ, PHILOX_OUT=path, TRITON_INTERPRET="1")
        res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        if res.returncode != 0:
            pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
        ctr, out = np.load(path)
    ctr = ctr.reshape(-1, 4)
    out = out.reshape(-1, 4)
    for c, o in zip(ctr, out):
        assert list(O.philox4x32_10(c, [0x1234567, 0x89ABCDE])) == list(o)


def test_philox_words_are_uniform():
    """Chi-square of Philox-4x32-10 output over consecutive counters, as the
    walks use it (counter = walk id, step block): the top 4 bits of each of
    the four words, and the stop test's rate against floor(alpha 2^32)."""
    from scipy.stats import chi2
    words = np.array([O.philox4x32_10([w, 0, t, 3], [0x5EED, 0]) for w in range(2500) for t in range(4)],
                     dtype=np.uint64)
    for j in range(4):
        hist = np.bincount((words[:, j] >> 28).astype(np.int64), minlength=16)
        expect = len(words) / 16
        assert chi2.sf(((hist - expect) ** 2 / expect).sum(), 15) > 1e-6, j
    stop = (words[:, [0, 2]] < np.uint64(int(ALPHA * 2**32))).mean()
    assert abs(stop - ALPHA) < 5 * math.sqrt(ALPHA * (1 - ALPHA) / (2 * len(words)))


# --------------------------------------------------------------- SpeedPPR
def test_walk_endpoints_follow_ppr():
    """An alpha-walk from v stops at u with probability pi(v, u) (Sec. 2).
    One unit of residue at v with W walks: counts/W ~ pi_v (chi-square)."""
    g = O.Graph(*gen.fig1_graph())
    v = 2
    W = 200_000
    r = np.zeros(g.n)
    r[v] = 1.0
    counts, est, st = O.walks(g, r, W, seed=42, source_index=3, alpha=ALPHA)
    assert counts.sum() == W and st["walks"] == W
    exact = lapack_ppr(g, v)
    chi2 = ((counts - W * exact) ** 2 / (W * exact)).sum()
    assert chi2 < 20.5  # 4 d.o.f., p ~ 4e-4
    np.testing.assert_allclose(est, counts / W, rtol=1e-12)
    # mean walk length 1/alpha - 1 moves
    assert abs(st["walk_steps"] / W - (1 / ALPHA - 1)) < 0.05


def test_walk_count_rule_and_refinement(cl_small):
    """Algorithm 4: after refinement no node is active w.r.t. 1/W, so
    W_v = ceil(r(v) W) <= d_v and the total number of walks is at most m."""
    g = cl_small
    eps = 0.5
    pi, r, counts, st = O.speedppr(g, 11, eps=eps, seed=7)
    W = st["W"]
    d = np.diff(g.row_ptr)
    assert np.all(r <= d / W * (1 + 1e-12))
    Wv = np.ceil(r[r > 0] * W)
    assert Wv.sum() == st["walks"] <= g.m
    assert counts.sum() == st["walks"]
    assert abs(pi.sum() - 1.0) < 1e-9  # walks carry the whole residual mass


def test_speedppr_relative_error_guarantee():
    """Approx-SSPPR (Sec. 2): |pi_hat - pi| <= eps pi for every pi >= mu = 1/n,
    with failure probability at most 1/n; checked on three sources."""
    g = O.Graph(*gen.chung_lu(3000, 30000, 2.2, seed=5))
    eps = 0.5
    for k, s in enumerate((0, 10, 2000)):
        pi, _, _, st = O.speedppr(g, s, eps=eps, seed=1000 + k, source_index=k)
        exact, _, _ = O.powitr(g, s, ALPHA, 1e-13)
        big = exact >= 1.0 / g.n
        bad = np.abs(pi[big] - exact[big]) > eps * exact[big]
        assert bad.sum() == 0


def test_W_equation8_values():
    """Eq. 8 with the natural log; scale check against the value computed by
    hand for n = 2^22, eps = 0.5, mu = 1/n: 2 (7/3) ln(2^22) 2^22 / 0.25."""
    n = 1 << 22
    W = O.speedppr_W(n, 0.5, 1.0 / n)
    assert abs(W - 1.19391e9) / 1.19391e9 < 1e-4


def test_walk_index_endpoints_follow_ppr():
    """Index walks are alpha-walks: the d_v stored endpoints of the nodes of a
    small graph, pooled over many seeds, follow pi_v (chi-square)."""
    g = O.Graph(*gen.fig1_graph())
    v = 1  # d_v = 4
    counts = np.zeros(g.n)
    for seed in range(20000):
        idx = O.build_walk_index(g, seed)
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            counts[idx[e]] += 1
    total = counts.sum()
    exact = lapack_ppr(g, v)
    chi2 = ((counts - total * exact) ** 2 / (total * exact)).sum()
    assert chi2 < 20.5


def test_index_query_reads_first_walks():
    """With W_v <= d_v the index query uses v's first W_v stored walks."""
    g = O.Graph(*gen.chung_lu(500, 5000, 2.2, seed=2))
    idx = O.build_walk_index(g, 9)
    rng = np.random.default_rng(1)
    d = np.diff(g.row_ptr)
    W = 1000.0
    r = rng.random(g.n) * d / W            # no node active w.r.t. 1/W
    r[rng.random(g.n) < 0.3] = 0.0
    counts, est, st = O.index_walks(g, idx, r, W)
    expect = np.zeros(g.n)
    for v in np.nonzero(r > 0)[0]:
        Wv = int(np.ceil(r[v] * W))
        assert Wv <= d[v]
        for u in idx[g.row_ptr[v]:g.row_ptr[v] + Wv]:
            expect[u] += 1
    assert np.array_equal(counts, expect.astype(np.uint32))
    assert abs(est.sum() - r.sum()) < 1e-12
