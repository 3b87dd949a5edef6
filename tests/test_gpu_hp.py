"""High-precision queries on the GPU (C ABI) against the FP64 oracle.

Bar: l1 distance to the oracle <= 2 lambda per source (both are within
lambda of the exact vector), certified bound <= lambda, exact agreement with
PowItr when every pass pushes every node (Lemma 1), and the mass identity
sum(pi_hat) = 1 - ||r||_1 for zero starts.
"""
import numpy as np
import pytest

import oracle as O
import ppr_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM = 1e-8
ALPHA = 0.2


@pytest.fixture(scope="module")
def P():
    import paper_2101_03652_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.load_library()
    return P


@pytest.fixture(scope="module")
def c0():
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    return rp, ci, gen.sources(10_000, 10, seed=1)


@pytest.fixture(scope="module")
def c0_ref(c0):
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    return {int(s): O.powerpush(og, int(s), ALPHA, LAM)[0] for s in src}


def run(P, rp, ci, src, **kw):
    g = P.Graph(rp, ci)
    out_r = kw.pop("out_r", None)
    pi, st = g.query(np.asarray(src), P.PPR_HP, out_r=out_r, lam=kw.pop("lam", LAM), **kw)
    torch.cuda.synchronize()
    res = pi.cpu().numpy()
    g.close()
    return res, st


def check_bound_and_mass(st, lam=LAM):
    # 1 - sum(pi_hat) = sum(pi - pi_hat), so |deficit| <= ||pi - pi_hat||_1 <= bound;
    # a refined answer may sit slightly above pi, so the deficit can be negative
    for s in st:
        assert s["final_l1_residual"] <= lam
        assert abs(s["mass_deficit"]) <= s["final_l1_residual"] + 1e-15


@pytest.mark.parametrize("k_tile", [1, 2, 4, 8, 16, 32, 64])
def test_c0_chung_lu_against_powerpush(P, c0, c0_ref, k_tile):
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src, k_tile=k_tile)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    assert all(x["sweeps"] == st[0]["sweeps"] for x in st[: min(k_tile, len(st))])


def test_lemma1_sweeps_equal_powitr(P, c0):
    """With no queue phase and synchronous passes every pass is one SimFwdPush
    iteration: 83 passes for lambda = 1e-8, alpha = 0.2, equal to PowItr up to
    summation order."""
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    pi, st = run(P, rp, ci, src[:3], k_tile=4, switch_edges=0, flags=2)  # PPR_FLAG_SYNC
    for i, s in enumerate(src[:3]):
        ref, _, ost = O.powitr(og, int(s), ALPHA, LAM)
        assert ost["iterations"] == 83 and st[i]["sweeps"] == 83
        assert np.abs(pi[i] - ref).sum() <= 1e-13
    check_bound_and_mass(st)


def test_subgraph200_against_dense_solve(P, c0):
    rp, ci, _ = c0
    srp, sci = gen.bfs_subgraph(rp, ci, 0, 200, seed=1)
    og = O.Graph(srp, sci)
    src = np.arange(0, 200, 13, dtype=np.int32)
    pi, st = run(P, srp, sci, src)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - O.dense_solve(og, int(s), ALPHA)).sum() <= LAM
    check_bound_and_mass(st)


def test_fig1_and_two_node_graphs(P):
    rp, ci = gen.fig1_graph()
    og = O.Graph(rp, ci)
    src = np.array([0, 1, 2, 3, 4, 0], dtype=np.int32)
    pi, st = run(P, rp, ci, src)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - O.dense_solve(og, int(s), ALPHA)).sum() <= LAM
    rp2, ci2 = gen.from_edges(2, [(0, 1), (1, 0)])
    pi2, _ = run(P, rp2, ci2, [1])
    # pi(1,1) = alpha / (1 - (1-alpha)^2), pi(1,0) = (1-alpha) pi(1,1)
    p11 = ALPHA / (1 - (1 - ALPHA) ** 2)
    assert np.abs(pi2[0] - np.array([(1 - ALPHA) * p11, p11])).sum() <= LAM


def test_duplicates_and_ragged_tile(P, c0, c0_ref):
    rp, ci, src = c0
    dup = np.array([src[0], src[1], src[0], src[2], src[0]], dtype=np.int32)
    pi, st = run(P, rp, ci, dup, k_tile=4)
    for i, s in enumerate(dup):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM


def test_queue_phase_alone_and_loose_lambda(P, c0):
    """A loose lambda is reached inside the queue phase (no sweep)."""
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    lam = 1e-2
    pi, st = run(P, rp, ci, src[:4], lam=lam, switch_edges=10**12)
    for i, s in enumerate(src[:4]):
        assert st[i]["sweeps"] == 0
        ref, _, _ = O.powitr(og, int(s), ALPHA, 1e-12)
        assert np.abs(pi[i] - ref).sum() <= lam
    check_bound_and_mass(st, lam)


def test_returned_residual_matches_definition(P, c0):
    """out_r = (alpha e_s + (1-alpha) pi_hat P - pi_hat) / alpha of the returned
    pi_hat, recomputed by the oracle; its l1 norm is within the certified bound."""
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    k = 3
    out_r = torch.empty((k, len(rp) - 1), dtype=torch.float64, device="cuda")
    pi, st = run(P, rp, ci, src[:k], out_r=out_r)
    r = out_r.cpu().numpy()
    d_in = np.bincount(ci, minlength=len(rp) - 1)
    for i, s in enumerate(src[:k]):
        ref = O.residual(og, int(s), pi[i], ALPHA)
        # the oracle evaluates (alpha e_s + (1-alpha) x P - x) / alpha in FP64: up to
        # d_in + 2 terms no larger than max x, each rounded at 2^-53
        fp64 = (d_in.max() + 2) * 2.0**-53 * pi[i].max() / ALPHA
        assert np.abs(r[i] - ref).max() <= fp64 + 1e-9 * np.abs(ref).max()
        assert np.abs(r[i]).sum() <= st[i]["final_l1_residual"]
        assert abs(r[i].sum() - st[i]["mass_deficit"]) <= 1e-12


def test_host_output_buffers(P, c0, c0_ref):
    rp, ci, src = c0
    g = P.Graph(rp, ci)
    out = np.zeros((3, len(rp) - 1))
    out_r = np.zeros((3, len(rp) - 1))
    _, st = g.query(src[:3], P.PPR_HP, out_pi=out, out_r=out_r, lam=LAM)
    g.close()
    for i, s in enumerate(src[:3]):
        assert np.abs(out[i] - c0_ref[int(s)]).sum() <= 2 * LAM
        assert np.abs(out_r[i]).sum() <= st[i]["final_l1_residual"]


def test_argument_errors(P, c0):
    rp, ci, src = c0
    g = P.Graph(rp, ci)
    for bad in ([-1], [10_000]):
        with pytest.raises(P.PPRError):
            g.query(bad, P.PPR_HP)
    for mode in (P.PPR_HP, P.PPR_APPROX):  # an empty source list is an argument error
        with pytest.raises(P.PPRError):
            g.query(np.zeros(0, dtype=np.int32), mode)
    for kw in ({"lam": 0.0}, {"alpha": 1.0}, {"alpha": 0.0}, {"k_tile": 3}, {"max_sweeps": 5}):
        with pytest.raises(P.PPRError):
            g.query(src[:2], P.PPR_HP, **kw)
    g.close()


@pytest.fixture(scope="module")
def rmat20():
    rp, ci = gen.rmat(20, 16, seed=1)
    return rp, ci, gen.sources(len(rp) - 1, 64, seed=2)


def check_residual_all(og, ci, src, pi, st, lam=LAM):
    """Every returned pi_hat checked without the GPU's own bound: the oracle
    evaluates its push residual r = (alpha e_s + (1-alpha) pi_hat P - pi_hat) /
    alpha in FP64, and ||pi - pi_hat||_1 <= ||r||_1 (Sec. 3.2) must hold within
    lambda up to the FP64 evaluation error."""
    n = og.n
    d_in_max = int(np.bincount(ci, minlength=n).max())
    for i, s in enumerate(src):
        x = pi[i]
        assert x.min() >= 0
        r = O.residual(og, int(s), x, ALPHA)
        # node u sums d_in(u) shares plus a few rounded steps, each error at
        # most 2^-53 of the magnitudes summed (2 sum x + alpha in all)
        slack = (d_in_max + 5) * 2.0**-53 * (2 * x.sum() + ALPHA) / ALPHA
        assert slack < lam / 10
        assert np.abs(r).sum() <= min(st[i]["final_l1_residual"], lam) + slack, i


def test_rmat20_bench_configuration(P, rmat20):
    """The benchmark's launch: 64 sources in one 64-column tile with the
    autotuned switch threshold.  Two sampled sources are checked against the
    oracle's Algorithm 3 in full, and every source by the oracle's FP64 push
    residual of the returned answer, besides the certified bound and the mass
    identity."""
    rp, ci, src = rmat20
    g = P.Graph(rp, ci)
    kt, sw, _ = g.autotune(src, lam=LAM)
    g.close()
    assert kt in (1, 2, 4, 8, 16, 32, 64) and sw >= 0
    pi, st = run(P, rp, ci, src, k_tile=kt, switch_edges=sw)
    check_bound_and_mass(st)
    og = O.Graph(rp, ci)
    for i in (0, 37):
        ref, _, _ = O.powerpush(og, int(src[i]), ALPHA, LAM)
        assert np.abs(pi[i] - ref).sum() <= 2 * LAM
    check_residual_all(og, ci, src, pi, st)


def test_tma_gather_pass_against_oracle(P, c0, c0_ref, rmat20):
    """PPR_FLAG_TMA_GATHER: the FP32 passes of 64-source tiles gather the heavy
    rows by TMA; answers within 2 lambda of the oracle (the small graph in
    full, R-MAT scale 20 by two full solves and every source's residual)."""
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src, k_tile=64, flags=P.PPR_FLAG_TMA_GATHER)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    rp, ci, src = rmat20
    pi, st = run(P, rp, ci, src, k_tile=64, flags=P.PPR_FLAG_TMA_GATHER)
    check_bound_and_mass(st)
    assert all(s["fp32_passes"] > 0 for s in st)
    og = O.Graph(rp, ci)
    for i in (5, 50):
        ref, _, _ = O.powerpush(og, int(src[i]), ALPHA, LAM)
        assert np.abs(pi[i] - ref).sum() <= 2 * LAM
    check_residual_all(og, ci, src, pi, st)


@pytest.mark.parametrize("k_tile", [1, 8])
def test_algorithm3_epochs_against_oracle(P, c0, c0_ref, k_tile):
    """epoch_num = 8: Algorithm 3's thresholded epochs (r'_max = lambda^(i/8)/m)."""
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src, k_tile=k_tile, epoch_num=8)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    pi_all, st_all = run(P, rp, ci, src, k_tile=k_tile)
    # thresholded synchronous passes converge more slowly per pass than pushing every node
    assert st[0]["sweeps"] >= st_all[0]["sweeps"]


def test_algorithm3_epochs_from_zero_start(P, c0, c0_ref):
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src[:4], epoch_num=4, switch_edges=0)
    for i, s in enumerate(src[:4]):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)


def test_autotune_picks_a_setting_that_stays_exact(P, c0, c0_ref):
    rp, ci, src = c0
    g = P.Graph(rp, ci)
    kt, sw, ms = g.autotune(src, lam=LAM)
    assert kt in (1, 2, 4, 8, 16) and sw >= 0 and ms > 0
    pi, st = g.query(src, P.PPR_HP, lam=LAM)  # k_tile = 0 and switch_edges = -1 now use the tuned values
    torch.cuda.synchronize()
    pi = pi.cpu().numpy()
    for i, s in enumerate(src):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    # the tuned over-relaxation factor (or 1 once a stalled batch turned it off)
    assert any(abs(st[0]["relax"] - w) < 1e-6 for w in (1.0, 1.05, 1.1, 1.15)), st[0]["relax"]
    g.close()


def test_asynchronous_passes_need_fewer_than_powitr(P, c0, c0_ref):
    """Default in-place passes (asynchronous updates) certify the same bound
    with fewer passes than the synchronous ones."""
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src, switch_edges=0, flags=P.PPR_FLAG_FIXED_PASSES)
    pi_s, st_s = run(P, rp, ci, src, switch_edges=0, flags=P.PPR_FLAG_SYNC)
    for i, s in enumerate(src):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    assert st[0]["sweeps"] < st_s[0]["sweeps"] == 83


@pytest.mark.parametrize("k_tile,switch", [(1, -1), (8, 0), (16, -1), (64, -1)])
def test_fp32_refinement_is_certified(P, c0, c0_ref, k_tile, switch):
    """Default dense phase (FP32 correction passes folded into the Q1.63
    estimate, stop certified by an exact pass) against the oracle and against
    the all-Q1.63 passes: both within 2 lambda of the oracle, bound certified."""
    rp, ci, src = c0
    pi, st = run(P, rp, ci, src, k_tile=k_tile, switch_edges=switch)
    pi_32, st_32 = run(P, rp, ci, src, k_tile=k_tile, switch_edges=switch, flags=P.PPR_FLAG_FP32_ONLY)
    pi_f, st_f = run(P, rp, ci, src, k_tile=k_tile, switch_edges=switch, flags=P.PPR_FLAG_FIXED_PASSES)
    for i, s in enumerate(src):
        for est in (pi, pi_32, pi_f):
            assert np.abs(est[i] - c0_ref[int(s)]).sum() <= 2 * LAM
    check_bound_and_mass(st)
    check_bound_and_mass(st_32)
    assert np.all(pi >= 0) and np.all(pi_32 >= 0)
    assert st_32[0]["bf16_passes"] == 0
    print(f"k_tile {k_tile}: passes bf16+fp32 {st[0]['bf16_passes']}+{st[0]['fp32_passes']}, "
          f"fp32 only {st_32[0]['fp32_passes']}, fixed {st_f[0]['sweeps']}")


def test_fp32_refinement_residual_output(P, c0, c0_ref):
    """out_r of a refined answer: the residual of the returned estimate."""
    rp, ci, src = c0
    g = P.Graph(rp, ci)
    n = len(rp) - 1
    out = np.zeros((3, n))
    out_r = np.zeros((3, n))
    _, st = g.query(src[:3], P.PPR_HP, out_pi=out, out_r=out_r, lam=LAM, k_tile=4)
    g.close()
    og = O.Graph(rp, ci)
    for i, s in enumerate(src[:3]):
        assert np.abs(out[i] - c0_ref[int(s)]).sum() <= 2 * LAM
        # the residual of the returned estimate, recomputed by the oracle's definition
        ref_r = O.residual(og, int(s), out[i], ALPHA)
        assert np.abs(out_r[i] - ref_r).sum() <= 1e-12 + 1e-6 * np.abs(ref_r).sum()
        assert np.abs(out_r[i]).sum() <= st[i]["final_l1_residual"]


def _no_active_query(P, rp, ci, src, **kw):
    n = len(rp) - 1
    g = P.Graph(rp, ci)
    out_r = torch.empty((len(src), n), dtype=torch.float64, device="cuda")
    pi, st = g.query(src, P.PPR_HP, out_r=out_r, lam=LAM, epoch_num=8, flags=P.PPR_FLAG_NO_ACTIVE, **kw)
    torch.cuda.synchronize()
    res = pi.cpu().numpy(), out_r.cpu().numpy(), st
    g.close()
    return res


def test_no_active_end_state(P, c0, c0_ref):
    """PPR_FLAG_NO_ACTIVE with epochs: the Remark after Algorithm 3 -- the
    returned residue has no active node w.r.t. lambda/m, the answer is still
    within 2 lambda of the oracle and the residue sum certifies it."""
    rp, ci, src = c0
    m = len(ci)
    d = np.diff(rp)
    pi, r, st = _no_active_query(P, rp, ci, src[:4])
    for i, s in enumerate(src[:4]):
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
        assert r[i].min() >= 0.0
        assert np.all(r[i] <= d * (LAM / m))          # no active node
        assert r[i].sum() <= st[i]["final_l1_residual"] + 1e-15
    with pytest.raises(P.PPRError):                   # needs the residue form
        g = P.Graph(rp, ci)
        try:
            g.query(src[:1], P.PPR_HP, lam=LAM, flags=P.PPR_FLAG_NO_ACTIVE)
        finally:
            g.close()


def test_fifo_only_gpu_mode(P, c0, c0_ref):
    """A switch threshold no level reaches keeps the whole query in the queue
    phase: FIFO-FwdPush (Algorithm 2) by levels, run to no active node.  Edge
    pushes are compared with the sequential oracle's (same level structure,
    different order inside a level)."""
    rp, ci, src = c0
    m = len(ci)
    d = np.diff(rp)
    og = O.Graph(rp, ci)
    pi, r, st = _no_active_query(P, rp, ci, src[:3], switch_edges=1 << 62, k_tile=1)
    for i, s in enumerate(src[:3]):
        assert st[i]["sweeps"] == 0 and st[i]["levels"] > 0
        assert np.abs(pi[i] - c0_ref[int(s)]).sum() <= 2 * LAM
        assert np.all(r[i] <= d * (LAM / m))
        _, _, ost = O.fifo_fwdpush(og, int(s), ALPHA, lam=LAM)
        ratio = st[i]["edges_pushed"] / ost["edge_pushes"]
        assert 0.5 <= ratio <= 2.0, ratio


@pytest.mark.parametrize("lam", [5e-2, 1e-3])
def test_bf16_stage_is_certified(P, c0, lam):
    """A loose lambda puts the whole first cycle above the BF16 floor, so the
    BF16 correction passes run; the answer is certified and within 2 lambda
    of the exact vector either way."""
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    pi, st = run(P, rp, ci, src[:4], k_tile=4, lam=lam)
    for i, s in enumerate(src[:4]):
        assert st[i]["final_l1_residual"] <= lam
        exact = O.dense_solve(og, int(s), ALPHA) if og.n <= 200 else O.powitr(og, int(s), ALPHA, 1e-12)[0]
        assert np.abs(pi[i] - exact).sum() <= 2 * lam
    if lam >= 1e-2:
        assert st[0]["bf16_passes"] > 0


@pytest.mark.parametrize("graph", ["bipartite", "even_cycle"])
def test_relaxation_fallback_on_bipartite_graphs(P, graph):
    """Bipartite graphs give (1-alpha) P the eigenvalue -(1-alpha), the mode
    that over-relaxed passes amplify: the stalled batch must turn relaxation
    off and the answer must still be certified and match the exact vector."""
    if graph == "bipartite":
        a, b = 40, 60
        edges = [(i, a + j) for i in range(a) for j in range(b)] + [(a + j, i) for j in range(b) for i in range(a)]
        n = a + b
    else:
        n = 1000
        edges = [(i, (i + 1) % n) for i in range(n)] + [(i, (i - 1) % n) for i in range(n)]
    rp, ci = gen.from_edges(n, edges)
    og = O.Graph(rp, ci)
    src = np.array([0, 7, n - 1], dtype=np.int32)
    for kw in ({}, {"switch_edges": 0}):
        pi, st = run(P, rp, ci, src, k_tile=4, **kw)
        check_bound_and_mass(st)
        for i, s in enumerate(src):
            exact = O.dense_solve(og, int(s), ALPHA) if n <= 200 else O.powitr(og, int(s), ALPHA, 1e-13)[0]
            assert np.abs(pi[i] - exact).sum() <= 2 * LAM, (graph, kw, i)


def test_rmat22_hp_bench_configuration(P):
    """R-MAT scale 22, 64 sources in one 64-column tile (the 64-source HP
    workload of the bench line's rmat22_k64 record): every source certified
    and checked by the oracle's FP64 push residual of the returned answer,
    one sampled source against the oracle's Algorithm 3 in full."""
    rp, ci = gen.rmat(22, 16, seed=1)
    src = gen.sources(len(rp) - 1, 64, seed=2)
    pi, st = run(P, rp, ci, src, k_tile=64)
    check_bound_and_mass(st)
    og = O.Graph(rp, ci)
    ref, _, _ = O.powerpush(og, int(src[0]), ALPHA, LAM)
    assert np.abs(pi[0] - ref).sum() <= 2 * LAM
    check_residual_all(og, ci, src, pi, st)


def test_pinned_host_outputs_written_directly(P, c0, c0_ref):
    """Page-locked host outputs are written by the kernels through their mapped
    address (no staging); results equal those written to device buffers."""
    rp, ci, src = c0
    n = len(rp) - 1
    g = P.Graph(rp, ci)
    k = 4
    host_pi = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
    host_r = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
    _, st = g.query(src[:k], P.PPR_HP, out_pi=host_pi, out_r=host_r, lam=LAM, k_tile=4, flags=P.PPR_FLAG_SYNC)
    dev_pi, st_d = g.query(src[:k], P.PPR_HP, lam=LAM, k_tile=4, flags=P.PPR_FLAG_SYNC)
    torch.cuda.synchronize()
    assert np.array_equal(host_pi.numpy(), dev_pi.cpu().numpy())  # synchronous passes are deterministic
    for i, s in enumerate(src[:k]):
        assert np.abs(host_pi[i].numpy() - c0_ref[int(s)]).sum() <= 2 * LAM
        assert np.abs(host_r[i].numpy()).sum() <= st[i]["final_l1_residual"]
    apx_pi = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
    apx_c = torch.empty((k, n), dtype=torch.int32, pin_memory=True)
    apx_r = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
    _, st_a = g.query(src[:k], P.PPR_APPROX, out_pi=apx_pi, out_r=apx_r, out_walk_counts=apx_c, eps=0.5, k_tile=4,
                      seed=0x5EED)
    torch.cuda.synchronize()
    g.close()
    og = O.Graph(rp, ci)
    for i in range(k):
        # the counts written to host memory replay bit for bit from the residue written beside them
        oc, _, _ = O.walks(og, apx_r[i].numpy(), st_a[i]["W"], 0x5EED, i, ALPHA)
        assert np.array_equal(apx_c[i].numpy().view(np.uint32), oc)
        assert abs(apx_pi[i].numpy().sum() - 1.0) < 1e-4


def test_fixed_point_conversions_match_cuda(P):
    """The kernels convert between Q1.63 and FP32/FP64 with integer
    instructions; on 16.7 M generated inputs per conversion (every leading-zero
    count, exact FP32 and FP64 ties, both signs) they agree bit for bit with
    CUDA's conversion intrinsics (round to nearest even, or toward zero for
    the truncating ones)."""
    from paper_2101_03652_gb300 import binding
    for seed in (0x5EED, 7):
        assert binding.ppr_selftest_fixconv(1 << 24, seed) == [0] * 7
    assert binding.ppr_selftest_fixconv(0) == [0] * 7


def _random_tiny_graph(n, p, seed):
    """Erdos-Renyi G(n, p) digraph, no self-loops, every sink given one random
    out-edge (the library's graph contract)."""
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    for v in range(n):
        if not a[v].any():
            a[v, (v + 1 + rng.integers(n - 1)) % n] = True
    edges = [(int(u), int(v)) for u, v in zip(*np.nonzero(a))]
    return gen.from_edges(n, edges)


@pytest.mark.parametrize("n,p,seed", [(2, 0.5, 1), (5, 0.3, 2), (17, 0.1, 3), (33, 0.05, 4), (64, 0.02, 5),
                                      (64, 0.5, 6)])
def test_random_tiny_graphs_every_mode(P, n, p, seed):
    """Random graphs with n <= 64, every node as a source (one tile), every HP
    mode, against a brute-force dense solve of Eq. 1."""
    rp, ci = _random_tiny_graph(n, p, seed)
    og = O.Graph(rp, ci)
    exact = np.stack([O.dense_solve(og, s, ALPHA) for s in range(n)])
    src = np.arange(n, dtype=np.int32)
    modes = [{}, {"flags": P.PPR_FLAG_FIXED_PASSES}, {"flags": P.PPR_FLAG_SYNC}, {"switch_edges": 0},
             {"epoch_num": 8, "flags": P.PPR_FLAG_NO_ACTIVE}, {"flags": P.PPR_FLAG_FP32_ONLY}]
    for kw in modes:
        pi, st = run(P, rp, ci, src, **kw)
        check_bound_and_mass(st)
        err = np.abs(pi - exact).sum(axis=1)
        assert np.all(err <= LAM + 1e-12), (kw, err.max())


@pytest.mark.parametrize("n,p,seed", [(17, 0.1, 3), (64, 0.02, 5)])
def test_random_tiny_graphs_walk_counts(P, n, p, seed):
    """SpeedPPR on random tiny graphs: walk counts bit-exact against the
    oracle's replay from the residue the walks started from."""
    rp, ci = _random_tiny_graph(n, p, seed)
    og = O.Graph(rp, ci)
    g = P.Graph(rp, ci)
    src = np.arange(min(n, 16), dtype=np.int32)
    out_r = torch.empty((len(src), n), dtype=torch.float64, device="cuda")
    counts = torch.empty((len(src), n), dtype=torch.int32, device="cuda")
    _, st = g.query(src, P.PPR_APPROX, out_r=out_r, out_walk_counts=counts, eps=0.5, seed=0x5EED)
    torch.cuda.synchronize()
    r, c = out_r.cpu().numpy(), counts.cpu().numpy().view(np.uint32)
    g.close()
    for i in range(len(src)):
        oc, _, _ = O.walks(og, r[i], st[i]["W"], 0x5EED, i, ALPHA)
        assert np.array_equal(c[i], oc)


def test_many_sources_two_tiles(P, c0):
    """100 sources (duplicates included) in 64-column tiles: two tiles, the
    second ragged; every answer against the oracle."""
    rp, ci, _ = c0
    og = O.Graph(rp, ci)
    src = gen.sources(len(rp) - 1, 96, seed=12)
    src = np.concatenate([src, src[:4]]).astype(np.int32)
    pi, st = run(P, rp, ci, src)
    check_bound_and_mass(st)
    refs = {}
    for i, s in enumerate(src):
        if int(s) not in refs:
            refs[int(s)] = O.powerpush(og, int(s), ALPHA, LAM)[0]
        assert np.abs(pi[i] - refs[int(s)]).sum() <= 2 * LAM, i
    assert np.abs(pi[96:] - pi[:4]).sum(axis=1).max() <= 2 * LAM  # duplicates agree


def test_rmat25_serving_configuration(P):
    """R-MAT scale 25, edge factor 32 (n = 33.6 M, m = 1.06 G): one batch of 32
    sources as the serving workload launches it.  No full oracle solve fits
    this size, so every source is checked by its certified bound and the mass
    identity, and two sampled sources by the push residual of the returned
    pi_hat evaluated by the oracle in FP64: ||pi - pi_hat||_1 <= ||r||_1."""
    rp, ci = gen.rmat(25, 32, seed=1)
    n = len(rp) - 1
    src = gen.sources(n, 32, seed=6)
    g = P.Graph(rp, ci)
    pi_d, st = g.query(src, P.PPR_HP, lam=LAM)
    torch.cuda.synchronize()
    check_bound_and_mass(st)
    og = O.Graph(rp, ci)
    d_in_max = int(np.bincount(ci, minlength=n).max())
    for i in (0, 17):
        x = pi_d[i].cpu().numpy()
        assert x.min() >= 0
        r = O.residual(og, int(src[i]), x, ALPHA)
        # FP64 evaluation: node u sums d_in(u) shares plus a few rounded steps,
        # each error at most 2^-53 of the magnitudes summed (2 sum x + alpha in all)
        slack = (d_in_max + 5) * 2.0**-53 * (2 * x.sum() + ALPHA) / ALPHA
        assert slack < LAM / 10
        assert np.abs(r).sum() <= st[i]["final_l1_residual"] + slack <= LAM + slack
        assert abs(r.sum() - st[i]["mass_deficit"]) <= 1e-12 + slack
    g.close()
