"""The entry point that allocates nothing (ppr_sssp_query_noalloc).

Callers that cannot allocate device memory (a plug-in living on its host's
memory budget, a process whose memory sits in a caching pool) use this call;
its scratch is an array compiled into the library and shared by all calls.
The test runs calls in a row through the C ABI -- each call starts from the
previous call's leftovers in that shared array -- with source counts that
select every tile width of the call (1, 2, 4 and 8 sources per pass), and
compares each answer with ppr_sssp_query's and with the FP64 oracle's
PowerPush (Algorithm 3) within the high-precision bar of the other tests
(l1 <= 2 lambda per source).  It also checks the size limit and the
rejection of an alpha too small for lambda.  The file is named to run last.
"""
import numpy as np
import pytest

import oracle as O
import ppr_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM = 1e-8


@pytest.fixture(scope="module")
def P():
    import paper_2101_03652_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.load_library()
    return P


def test_noalloc_matches_query_on_two_calls(P):
    from paper_2101_03652_gb300 import binding
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    n = len(rp) - 1
    g = P.Graph(rp, ci)
    og = O.Graph(rp, ci)
    # k = 5, 11, 1, 3: tiles of 4 and 8 sources, then of 1 and 2
    calls = [gen.sources(n, 5, seed=31), gen.sources(n, 11, seed=32), gen.sources(n, 1, seed=33),
             gen.sources(n, 3, seed=34)]
    for call, src in enumerate(calls):
        out = torch.full((len(src), n), -1.0, dtype=torch.float64, device="cuda")
        sweeps = binding.ppr_sssp_query_noalloc(g.handle, src, out, alpha=0.2, lam=LAM)
        ref, _ = g.query(src, P.PPR_HP, lam=LAM)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        for i, s in enumerate(src):
            assert np.abs(a[i] - b[i]).sum() <= 2 * LAM, (call, i)
            orc = O.powerpush(og, int(s), 0.2, LAM)[0]
            assert np.abs(a[i] - orc).sum() <= 2 * LAM, (call, i)
        assert np.all(sweeps == 83)  # zero start, every node pushed each pass (Eq. 6)
    g.close()


def test_noalloc_rejects_alpha_too_small_for_lambda(P):
    from paper_2101_03652_gb300 import binding
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    g = P.Graph(rp, ci)
    out = torch.empty((1, len(rp) - 1), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PPRError) as e:
        binding.ppr_sssp_query_noalloc(g.handle, [0], out, alpha=1e-9, lam=1e-15)
    assert e.value.status == binding.PPR_ERR_ARG
    assert "too small" in str(e.value)
    g.close()


def test_noalloc_rejects_graph_beyond_scratch(P):
    from paper_2101_03652_gb300 import binding
    rp, ci = gen.rmat(20, 16, seed=1)
    g = P.Graph(rp, ci)
    out = torch.empty((1, len(rp) - 1), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PPRError) as e:
        binding.ppr_sssp_query_noalloc(g.handle, [0], out)
    assert e.value.status == binding.PPR_ERR_ARG
    assert "too large" in str(e.value)
    g.close()
