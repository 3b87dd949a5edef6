"""Approximate queries (SpeedPPR, Algorithm 4) on the GPU against the oracle.

Walk endpoint counts are compared bit for bit with the oracle's replay of the
walk phase from the residue the GPU launched its walks from (same W, seed and
source index).  The end state of the push phase must leave no active node
w.r.t. 1/W, and the estimates must meet the Approx-SSPPR guarantee of Sec. 2
against an exact vector.
"""
import numpy as np
import pytest

import oracle as O
import ppr_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHA = 0.2
SEED = 0x5EED


@pytest.fixture(scope="module")
def P():
    import paper_2101_03652_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.load_library()
    return P


def run_approx(P, rp, ci, src, eps=0.5, **kw):
    n = len(rp) - 1
    g = P.Graph(rp, ci)
    k = len(src)
    out_r = torch.empty((k, n), dtype=torch.float64, device="cuda")
    counts = torch.empty((k, n), dtype=torch.int32, device="cuda")
    pi, st = g.query(np.asarray(src, dtype=np.int32), P.PPR_APPROX, out_r=out_r, out_walk_counts=counts, eps=eps,
                     seed=SEED, **kw)
    torch.cuda.synchronize()
    res = (pi.cpu().numpy(), out_r.cpu().numpy(), counts.cpu().numpy().view(np.uint32), st)
    g.close()
    return res


@pytest.mark.parametrize("k_tile", [1, 2, 4, 8, 16, 32])
def test_walk_counts_bit_exact(P, k_tile):
    rp, ci = gen.chung_lu(3000, 30000, 2.2, seed=5)
    og = O.Graph(rp, ci)
    src = gen.sources(3000, 5, seed=9)
    pi, r, counts, st = run_approx(P, rp, ci, src, k_tile=k_tile)
    d = np.diff(rp)
    for i, s in enumerate(src):
        W = st[i]["W"]
        assert W == O.speedppr_W(3000, 0.5, 1 / 3000)
        assert np.all(r[i] >= 0)
        assert np.all(r[i] <= d / W * (1 + 1e-6))          # no active node w.r.t. 1/W
        oc, oest, ost = O.walks(og, r[i], W, SEED, i, ALPHA)
        assert np.array_equal(counts[i], oc)                # bit-exact endpoint counts
        assert st[i]["walks"] == ost["walks"] and st[i]["walk_steps"] == ost["walk_steps"]
        assert st[i]["walks"] <= og.m + og.n
        reserve = pi[i] - oest                              # pi_hat = reserve + walk estimates
        assert reserve.min() >= -1e-12
        assert abs(pi[i].sum() - 1.0) < 1e-5                # walks carry the remaining mass


def test_relative_error_guarantee(P):
    rp, ci = gen.chung_lu(3000, 30000, 2.2, seed=5)
    og = O.Graph(rp, ci)
    src = gen.sources(3000, 4, seed=10)
    eps = 0.5
    pi, _, _, st = run_approx(P, rp, ci, src, eps=eps)
    for i, s in enumerate(src):
        exact, _, _ = O.powitr(og, int(s), ALPHA, 1e-13)
        big = exact >= 1.0 / og.n
        bad = np.abs(pi[i][big] - exact[big]) > eps * exact[big]
        assert bad.sum() == 0


def test_fig1_graph_approx(P):
    rp, ci = gen.fig1_graph()
    og = O.Graph(rp, ci)
    pi, r, counts, st = run_approx(P, rp, ci, [0, 3], eps=0.1)
    for i, s in enumerate([0, 3]):
        exact = O.dense_solve(og, s, ALPHA)
        assert np.all(np.abs(pi[i] - exact) <= 0.1 * exact)
        oc, _, _ = O.walks(og, r[i], st[i]["W"], SEED, i, ALPHA)
        assert np.array_equal(counts[i], oc)


def test_rmat22_configuration_sampled(P):
    """R-MAT scale 22 with the approximate workload's 256 sources (sixteen
    16-column tiles in one call): walk budget and mass checked for every
    source, the no-active end state and bit-exact walk counts (oracle replay)
    for four sources spread over the tiles, including the last one."""
    rp, ci = gen.rmat(22, 16, seed=1)
    og = O.Graph(rp, ci)
    n = og.n
    src = gen.sources(n, 256, seed=3)
    g = P.Graph(rp, ci)
    k = len(src)
    out_r = torch.empty((k, n), dtype=torch.float64, device="cuda")
    counts = torch.empty((k, n), dtype=torch.int32, device="cuda")
    pi, st = g.query(np.asarray(src, dtype=np.int32), P.PPR_APPROX, out_r=out_r, out_walk_counts=counts, eps=0.5,
                     seed=SEED, k_tile=16)
    torch.cuda.synchronize()
    mass = pi.sum(dim=1).cpu().numpy()
    assert np.all(np.abs(mass - 1.0) < 1e-4)
    d = np.diff(rp)
    for i in range(k):
        assert st[i]["walks"] <= og.m + og.n
        assert st[i]["W"] == O.speedppr_W(n, 0.5, 1.0 / n)
    for i in (0, 77, 170, 255):
        r = out_r[i].cpu().numpy()
        c = counts[i].cpu().numpy().view(np.uint32)
        assert np.all(r >= 0) and np.all(r <= d / st[i]["W"] * (1 + 1e-6))
        oc, _, _ = O.walks(og, r, st[i]["W"], SEED, i, ALPHA)
        assert np.array_equal(c, oc), i
    g.close()


def test_eps_sweep_accuracy(P):
    """The accuracy study over eps on a small graph: the relative-error
    guarantee holds at every eps (entries with pi >= 1/n, against an exact
    vector), with walks and with the index, and the l1 error falls as eps
    does."""
    rp, ci = gen.chung_lu(3000, 30000, 2.2, seed=5)
    og = O.Graph(rp, ci)
    n = og.n
    src = gen.sources(n, 4, seed=11)
    exact = np.stack([O.powitr(og, int(s), ALPHA, 1e-13)[0] for s in src])
    g = P.Graph(rp, ci)
    g.build_index(0x1DE5, ALPHA)
    l1 = {}
    for eps in (0.1, 0.3, 0.5):
        for flags in (0, P.PPR_FLAG_INDEX):
            pi, _ = g.query(np.asarray(src, dtype=np.int32), P.PPR_APPROX, eps=eps, seed=SEED, flags=flags)
            pi = pi.cpu().numpy()
            big = exact >= 1.0 / n
            assert np.all(np.abs(pi - exact)[big] <= eps * exact[big]), (eps, flags)
            l1[(eps, flags)] = np.abs(pi - exact).sum(axis=1).mean()
    g.close()
    for flags in (0, P.PPR_FLAG_INDEX):
        assert l1[(0.1, flags)] < l1[(0.5, flags)]
