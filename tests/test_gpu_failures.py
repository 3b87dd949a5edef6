"""Error paths of the library, driven from the host (no GPU fault involved).

* Admission: a batch whose workspace does not fit in the free device memory
  the host reads is refused with PPR_ERR_ADMIT before any launch.  The free
  memory is capped through the library's injection hook.
* Allocation failure: an injected workspace allocation failure returns
  PPR_ERR_OOM, and the graph answers the next call correctly.
* ppr_query_state_bytes equals the workspace a query on a fresh graph really
  allocates (ppr_workspace_bytes).
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


@pytest.fixture
def hooks(P):
    from paper_2101_03652_gb300 import binding
    yield binding
    binding.ppr_inject(binding.PPR_INJECT_FREE_BYTES, -1)
    binding.ppr_inject(binding.PPR_INJECT_ALLOC_FAIL, 0)


def test_admission_refused_before_any_launch(P, c0, hooks):
    rp, ci, src = c0
    n = len(rp) - 1
    g = P.Graph(rp, ci)
    need = g.state_bytes(len(src), 16)
    out = torch.full((len(src), n), -7.0, dtype=torch.float64, device="cuda")
    hooks.ppr_inject(hooks.PPR_INJECT_FREE_BYTES, need - 1)
    with pytest.raises(P.PPRError) as e:
        g.query(src, P.PPR_HP, out_pi=out, lam=LAM, k_tile=16)
    assert e.value.status == hooks.PPR_ERR_ADMIT
    assert "admission refused" in str(e.value)
    torch.cuda.synchronize()
    assert bool((out == -7.0).all())          # nothing written
    assert g.workspace_bytes() == 0           # nothing allocated
    # exactly the state's size is admitted
    hooks.ppr_inject(hooks.PPR_INJECT_FREE_BYTES, need)
    pi, st = g.query(src, P.PPR_HP, out_pi=out, lam=LAM, k_tile=16)
    torch.cuda.synchronize()
    assert all(s["final_l1_residual"] <= LAM for s in st)
    # the workspace now held counts as available for the next batch of that size
    hooks.ppr_inject(hooks.PPR_INJECT_FREE_BYTES, 0)
    g.query(src, P.PPR_HP, out_pi=out, lam=LAM, k_tile=16)
    # but not for a larger one
    with pytest.raises(P.PPRError) as e:
        g.query(src, P.PPR_HP, out_pi=out, lam=LAM, k_tile=32)
    assert e.value.status == hooks.PPR_ERR_ADMIT
    g.close()


def test_injected_allocation_failure_is_oom_and_recoverable(P, c0, hooks):
    """A fresh graph's first query allocates its workspace buffer by buffer;
    the failure is injected at the first, third and seventh of them."""
    rp, ci, src = c0
    og = O.Graph(rp, ci)
    for nth in (1, 3, 7):
        g = P.Graph(rp, ci)
        hooks.ppr_inject(hooks.PPR_INJECT_ALLOC_FAIL, nth)
        with pytest.raises(P.PPRError) as e:
            g.query(src[:4], P.PPR_HP, lam=LAM, k_tile=4)
        assert e.value.status == hooks.PPR_ERR_OOM
        assert "injected allocation failure" in str(e.value)
        hooks.ppr_inject(hooks.PPR_INJECT_ALLOC_FAIL, 0)
        pi, st = g.query(src[:4], P.PPR_HP, lam=LAM, k_tile=4)
        torch.cuda.synchronize()
        pi = pi.cpu().numpy()
        for i in (0, 3):
            ref = O.powerpush(og, int(src[i]), ALPHA, LAM)[0]
            assert np.abs(pi[i] - ref).sum() <= 2 * LAM
        g.close()


@pytest.mark.parametrize("k,k_tile", [(64, 64), (10, 8), (3, 0), (1, 1)])
def test_state_bytes_equal_the_allocated_workspace(P, c0, k, k_tile):
    rp, ci, _ = c0
    n = len(rp) - 1
    src = gen.sources(n, k, seed=41)
    g = P.Graph(rp, ci)
    expect = g.state_bytes(k, k_tile)
    assert g.workspace_bytes() == 0
    _, st = g.query(src, P.PPR_HP, lam=LAM, alpha=ALPHA, k_tile=k_tile)
    torch.cuda.synchronize()
    assert all(s["final_l1_residual"] <= LAM for s in st)
    assert g.workspace_bytes() == expect
    g.close()
