"""SpeedPPR-Index (Sec. 6.2) on the GPU against the oracle.

* the stored walk of every edge slot ends where the oracle's does (bit-exact
  endpoints; both draw the same Philox-4x32-10 words per slot);
* an indexed query reads the first W_v = min(ceil(r(v) W), d_v) stored walks
  of each node: endpoint counts equal the oracle's replay from the residue the
  GPU left, and the estimates meet the Approx-SSPPR guarantee.
"""
import numpy as np
import pytest

import oracle as O
import ppr_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHA = 0.2
SEED = 0x1DE5


@pytest.fixture(scope="module")
def P():
    import paper_2101_03652_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.load_library()
    return P


@pytest.fixture(scope="module")
def chung_lu():
    return gen.chung_lu(3000, 30000, 2.2, seed=5)


def indexed_query(P, g, n, src, eps, k_tile=0):
    k = len(src)
    out_r = torch.empty((k, n), dtype=torch.float64, device="cuda")
    counts = torch.empty((k, n), dtype=torch.int32, device="cuda")
    pi, st = g.query(np.asarray(src, dtype=np.int32), P.PPR_APPROX, out_r=out_r, out_walk_counts=counts, eps=eps,
                     flags=P.PPR_FLAG_INDEX, k_tile=k_tile)
    torch.cuda.synchronize()
    return pi.cpu().numpy(), out_r.cpu().numpy(), counts.cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("graph", ["fig1", "chung_lu"])
def test_index_endpoints_bit_exact(P, chung_lu, graph):
    rp, ci = gen.fig1_graph() if graph == "fig1" else chung_lu
    g = P.Graph(rp, ci)
    g.build_index(SEED, ALPHA)
    idx = g.get_index()
    ref = O.build_walk_index(O.Graph(rp, ci), SEED, ALPHA)
    assert idx.shape == ref.shape
    assert np.array_equal(idx, ref)
    g.close()


@pytest.mark.parametrize("k_tile", [1, 8, 16, 32])
def test_index_query_counts_bit_exact(P, chung_lu, k_tile):
    rp, ci = chung_lu
    og = O.Graph(rp, ci)
    g = P.Graph(rp, ci)
    g.build_index(SEED, ALPHA)
    idx = O.build_walk_index(og, SEED, ALPHA)
    src = gen.sources(og.n, 6, seed=9)
    pi, r, counts, st = indexed_query(P, g, og.n, src, eps=0.5, k_tile=k_tile)
    d = np.diff(rp)
    for i in range(len(src)):
        W = st[i]["W"]
        assert np.all(r[i] <= d / W * (1 + 1e-6))
        oc, oest, ost = O.index_walks(og, idx, r[i], W)
        assert np.array_equal(counts[i], oc)
        assert st[i]["walks"] == ost["walks"] <= og.m
        assert abs(pi[i].sum() - 1.0) < 1e-4
    g.close()


def test_index_query_guarantee(P, chung_lu):
    rp, ci = chung_lu
    og = O.Graph(rp, ci)
    g = P.Graph(rp, ci)
    g.build_index(SEED, ALPHA)
    src = gen.sources(og.n, 4, seed=10)
    eps = 0.5
    pi, _, _, _ = indexed_query(P, g, og.n, src, eps=eps)
    for i, s in enumerate(src):
        exact, _, _ = O.powitr(og, int(s), ALPHA, 1e-13)
        big = exact >= 1.0 / og.n
        assert np.all(np.abs(pi[i][big] - exact[big]) <= eps * exact[big])
    g.close()


def test_index_heavy_nodes(P):
    """A star whose centre needs more than 32 index walks (the block-per-node
    branch): counts still equal the oracle's."""
    n = 400
    rows = [list(range(1, n))] + [[0] for _ in range(1, n)]
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(x) for x in rows])
    ci = np.concatenate([np.asarray(x, dtype=np.int32) for x in rows])
    og = O.Graph(rp, ci)
    g = P.Graph(rp, ci)
    g.build_index(SEED, ALPHA)
    idx = g.get_index()
    assert np.array_equal(idx, O.build_walk_index(og, SEED, ALPHA))
    pi, r, counts, st = indexed_query(P, g, n, [0, 5], eps=0.05)
    for i in range(2):
        oc, _, ost = O.index_walks(og, idx, r[i], st[i]["W"])
        assert np.array_equal(counts[i], oc)
        assert st[i]["walks"] == ost["walks"]
    assert int(np.ceil(r[0][0] * st[0]["W"])) > 32 or int(np.ceil(r[1][0] * st[1]["W"])) > 32
    g.close()


def test_index_errors(P, chung_lu):
    rp, ci = chung_lu
    g = P.Graph(rp, ci)
    with pytest.raises(P.PPRError):
        indexed_query(P, g, len(rp) - 1, [0], eps=0.5)        # no index yet
    with pytest.raises(P.PPRError):
        g.get_index()
    g.build_index(SEED, 0.3)
    with pytest.raises(P.PPRError):
        indexed_query(P, g, len(rp) - 1, [0], eps=0.5)        # index built for another alpha
    g.build_index(SEED, ALPHA)
    indexed_query(P, g, len(rp) - 1, [0], eps=0.5)
    g.close()
