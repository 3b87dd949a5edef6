"""Learned warm start on the GPU against the FP64 oracle of the model.

* forward: the model's estimate equals the oracle's (which applies BF16
  rounding where the GPU feeds BF16 GEMMs) within FP32-accumulation error;
* backward: gradients of the l1 loss match the oracle's analytic gradients
  (relative l2 error <= 2e-2 per parameter block, BF16 operands);
* training lowers the loss; a warm-started HP query stays within 2 lambda of
  the oracle and its certified bound stays <= lambda;
* checkpoints round-trip.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from oracle import warm as Wm
import ppr_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHA = 0.2
LAM = 1e-8
SEED = 0x5EED


@pytest.fixture(scope="module")
def P():
    import paper_2101_03652_gb300 as P
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    P.load_library()
    return P


@pytest.fixture(scope="module")
def setup(P):
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    g = P.Graph(rp, ci)
    og = O.Graph(rp, ci)
    yield rp, ci, g, og
    g.close()


def randomize(model, n, rng, u_scale=2e-6):
    p = model.get_params()
    F, H, R = 128, 512, 64
    parts = Wm.unflatten(p, n)
    parts[1] = rng.normal(0, 0.1, H)
    parts[3] = rng.normal(0, 0.1, H)
    parts[5] = rng.normal(0, 0.1, R)
    parts[6] = rng.normal(0, u_scale, (n, R))
    flat = np.concatenate([x.reshape(-1) for x in parts]).astype(np.float32)
    model.set_params(flat)
    return Wm.unflatten(flat.astype(np.float64), n)


def test_forward_matches_oracle(P, setup):
    rp, ci, g, og = setup
    rng = np.random.default_rng(1)
    m = P.Model(g, seed=SEED)
    params = randomize(m, og.n, rng)
    src = gen.sources(og.n, 5, seed=21)
    X_gpu = m.estimate(src)
    X_orc = Wm.warm_estimate(og, src, params, 128, SEED, ALPHA, rnd=Wm.bf16).T
    for i in range(len(src)):
        err = np.abs(X_gpu[i] - X_orc[i]).sum()
        assert err <= 5e-3, (i, err)
        assert abs(X_gpu[i].sum() - 1.0) < 1e-4 and X_gpu[i].min() >= 0
    m.close()


def test_untrained_model_returns_sketch(P, setup):
    rp, ci, g, og = setup
    m = P.Model(g, seed=SEED)
    src = gen.sources(og.n, 3, seed=22)
    X = m.estimate(src)
    for i, s in enumerate(src):
        assert np.abs(X[i] - Wm.sketch(og, int(s), ALPHA)).sum() <= 1e-5
    m.close()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_gradients_match_oracle(P, setup):
    rp, ci, g, og = setup
    rng = np.random.default_rng(2)
    m = P.Model(g, seed=SEED)
    params = randomize(m, og.n, rng)
    src = gen.sources(og.n, 16, seed=23)
    labels = np.stack([O.powerpush(og, int(s), ALPHA, 1e-10)[0] for s in src])  # oracle labels, k x n
    loss_gpu = m.train_step(src, labels, lr=0.0)
    _, grads = m.get_params(grads=True)
    S = Wm.sketches(og, src, ALPHA)
    f = Wm.features(S, 128, SEED)
    L, og_grads = Wm.backward(params, S, f, labels.T, rnd=Wm.bf16)
    assert abs(loss_gpu - L) <= 1e-3 * L
    gparts = Wm.unflatten(grads.astype(np.float64), og.n)
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "U"]
    for name, a, b in zip(names, gparts, og_grads):
        assert rel_l2(a, b) <= 2e-2, (name, rel_l2(a, b))
    m.close()


def test_against_the_model_with_bf16_weights_only(P, setup):
    """The model as specified keeps BF16 weights and FP32 accumulation; the
    GPU also rounds activations to BF16 where they feed a GEMM.  Against the
    FP64 model with only its weights rounded (W1, W2, W3, U), no activation
    rounding: the estimate within l1 5e-3 per source (the bar of the rounded
    comparison; activation rounding itself moves it by about 3e-5 here) and
    every gradient block within relative l2 5e-2, about 25 BF16 unit
    roundoffs (2^-9): four rounding points (f, h1, h2, h) and the l1
    subgradient's sign flips near X = pi move the blocks by 1-4 %."""
    rp, ci, g, og = setup
    rng = np.random.default_rng(5)
    m = P.Model(g, seed=SEED)
    params = randomize(m, og.n, rng)
    wonly = [Wm.bf16(p) if i in (0, 2, 4, 6) else p for i, p in enumerate(params)]
    src = gen.sources(og.n, 5, seed=21)
    X_gpu = m.estimate(src)
    X_ref = Wm.warm_estimate(og, src, wonly, 128, SEED, ALPHA, rnd=None).T
    for i in range(len(src)):
        assert np.abs(X_gpu[i] - X_ref[i]).sum() <= 5e-3, i
    src = gen.sources(og.n, 16, seed=23)
    labels = np.stack([O.powerpush(og, int(s), ALPHA, 1e-10)[0] for s in src])
    loss_gpu = m.train_step(src, labels, lr=0.0)
    _, grads = m.get_params(grads=True)
    S = Wm.sketches(og, src, ALPHA)
    f = Wm.features(S, 128, SEED)
    L, ref_grads = Wm.backward(wonly, S, f, labels.T, rnd=None)
    assert abs(loss_gpu - L) <= 1e-3 * L
    gparts = Wm.unflatten(grads.astype(np.float64), og.n)
    for name, a, b in zip(["W1", "b1", "W2", "b2", "W3", "b3", "U"], gparts, ref_grads):
        assert rel_l2(a, b) <= 5e-2, (name, rel_l2(a, b))
    m.close()


def test_adam_step_matches_oracle(P, setup):
    """One training step of a fresh model (Adam step 1, zero moments): the
    parameters move as the oracle's Adam step predicts from the gradients the
    step computed.  The kernel works in FP32, with the decay rates rounded to
    FP32 (up to 5e-5 relative in a bias correction); the steps are compared
    within 1e-4 of lr, plus the rounding of the FP32 parameter."""
    rp, ci, g, og = setup
    rng = np.random.default_rng(4)
    m = P.Model(g, seed=SEED)
    randomize(m, og.n, rng)
    p0 = m.get_params().astype(np.float64)
    src = gen.sources(og.n, 8, seed=25)
    labels = np.stack([O.powerpush(og, int(s), ALPHA, 1e-10)[0] for s in src])
    lr = 1e-3
    m.train_step(src, labels, lr=lr)
    p1, grads = m.get_params(grads=True)
    zero = np.zeros_like(p0)
    ref, _, _ = Wm.adam_step(p0, zero, zero, grads.astype(np.float64), lr=lr, t=1)
    assert np.abs(p1 - p0).max() > 0.5 * lr       # the step was taken
    np.testing.assert_allclose(p1, ref, rtol=2.0**-23, atol=1e-4 * lr)
    m.close()


def test_training_reduces_loss_and_warm_query_is_exact(P, setup):
    rp, ci, g, og = setup
    n = og.n
    train = gen.sources(n, 512, seed=4)
    held = gen.sources(n, 16, seed=5)
    m = P.Model(g, seed=SEED)
    losses = m.train(train, epochs=15, lr=2e-3, shuffle_seed=7)
    assert losses[-1] < 0.8 * losses[0], losses
    # warm-started HP queries: same guarantee as the zero start
    pi, st = g.query(held, P.PPR_HP, lam=LAM, warm_start=m)
    pi0, st0 = g.query(held, P.PPR_HP, lam=LAM)
    torch.cuda.synchronize()
    pi = pi.cpu().numpy()
    for i, s in enumerate(held[:6]):
        ref, _, _ = O.powerpush(og, int(s), ALPHA, LAM)
        assert np.abs(pi[i] - ref).sum() <= 2 * LAM
    for s_ in st:
        assert s_["final_l1_residual"] <= LAM
        assert abs(s_["mass_deficit"]) <= s_["final_l1_residual"] + 1e-15
    # the residual norm the warm start hands to the solver, against the zero start's 1
    r0 = np.array([s_["initial_l1_residual"] for s_ in st])
    assert np.all(np.isfinite(r0))
    m.close()


def test_checkpoint_round_trip(P, setup):
    rp, ci, g, og = setup
    rng = np.random.default_rng(3)
    m = P.Model(g, seed=SEED)
    randomize(m, og.n, rng)
    src = gen.sources(og.n, 4, seed=24)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "model.bin")
        m.save(path)
        m2 = P.Model.load(g, path)
        assert np.array_equal(m.get_params(), m2.get_params())
        # the sketch and projection add with FP32 atomics in no fixed order, so two
        # evaluations of one model agree to FP32 rounding, not bit for bit
        np.testing.assert_allclose(m.estimate(src), m2.estimate(src), rtol=1e-5, atol=1e-9)
        m2.close()
        with pytest.raises(P.PPRError) as e:      # not a checkpoint
            P.Model.load(g, os.path.join(td, "missing.bin"))
        assert e.value.status == P.binding.PPR_ERR_ARG
    if os.path.exists("/dev/full"):               # a write that fails: ENOSPC
        with pytest.raises(P.PPRError) as e:
            m.save("/dev/full")
        assert e.value.status == P.binding.PPR_ERR_ARG
    m.close()


def test_correction_model_gain_on_rmat20(P):
    """The learned correction of the remaining mass (correction_passes = 8) on the
    R-MAT scale-20 graph: the answers keep the guarantee and the solver needs
    fewer passes than from the zero start: after two epochs on 512 sources
    about 26 against 37.  The pass counts of in-place passes vary by a few
    from call to call, so the bar is a fifth fewer."""
    rp, ci = gen.rmat(20, 16, seed=1)
    g = P.Graph(rp, ci)
    n = len(rp) - 1
    train = gen.sources(n, 512, seed=4)
    held = gen.sources(n, 64, seed=5)
    m = P.Model(g, seed=SEED, correction_passes=8)
    losses = m.train(train, epochs=2, lr=2e-3, shuffle_seed=1)
    print(f"correction model losses {losses}")
    # FP32 atomics in the sketch and the projection make the trajectory vary
    # from run to run (0.0015 - 0.025 observed after two epochs)
    assert losses[-1] < 0.05
    pi_w, st_w = g.query(held, P.PPR_HP, lam=LAM, warm_start=m)
    pi_0, st_0 = g.query(held, P.PPR_HP, lam=LAM)
    torch.cuda.synchronize()
    a, b = pi_w.cpu().numpy(), pi_0.cpu().numpy()
    for i in range(len(held)):
        assert np.abs(a[i] - b[i]).sum() <= 2 * LAM
        assert st_w[i]["final_l1_residual"] <= LAM
    og = O.Graph(rp, ci)
    ref, _, _ = O.powerpush(og, int(held[0]), ALPHA, LAM)
    assert np.abs(a[0] - ref).sum() <= 2 * LAM
    sw_w = np.mean([s["sweeps"] for s in st_w])
    sw_0 = np.mean([s["sweeps"] for s in st_0])
    print(f"passes: warm {sw_w:.1f} vs zero start {sw_0:.1f}")
    assert sw_w < 0.8 * sw_0
    m.close()
    g.close()
