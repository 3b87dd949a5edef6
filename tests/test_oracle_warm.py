"""Pins for the warm-start oracle: finite differences pin the analytic
backward, the sketch is pinned by its definition through PowItr (Eq. 3, 5)
and by its mass, the Gaussian rows by their moments."""
import numpy as np
import pytest

import oracle as O
from oracle import warm as Wm
import ppr_inputs as gen

ALPHA = 0.2


def small_graph():
    return O.Graph(*gen.chung_lu(50, 400, 2.2, seed=4))


def test_sketch_is_two_iterations_plus_alive_mass():
    g = small_graph()
    s = 3
    S = Wm.sketch(g, s, ALPHA)
    # PowItr after 2 iterations: reserve pi^(2) and alive mass gamma^(2) (lam between 0.8^2 and 0.8)
    pi2, r2, st = O.powitr(g, s, ALPHA, lam=0.65)
    assert st["iterations"] == 2
    np.testing.assert_allclose(S, pi2 + r2, atol=1e-15)
    assert abs(S.sum() - 1.0) < 1e-14


def test_gaussian_rows_moments_and_determinism():
    G = O.gaussian_rows(0, 4000, 128, seed=11)
    assert abs(G.mean()) < 0.01 and abs(G.std() - 1.0) < 0.01
    np.testing.assert_array_equal(G[100:105], O.gaussian_rows(100, 5, 128, seed=11))
    assert not np.array_equal(G[:5], O.gaussian_rows(0, 5, 128, seed=12))
    # fourth moment of a standard normal is 3
    assert abs((G ** 4).mean() - 3.0) < 0.1


def random_params(rng, n, F, H, R, scale=0.3):
    return [rng.normal(0, scale, (F, H)), rng.normal(0, 0.1, H), rng.normal(0, scale, (H, H)),
            rng.normal(0, 0.1, H), rng.normal(0, scale, (H, R)), rng.normal(0, 0.1, R),
            rng.normal(0, 0.02, (n, R))]


def test_backward_matches_finite_differences():
    g = small_graph()
    rng = np.random.default_rng(0)
    F, H, R = 8, 16, 4
    src = [1, 7, 20]
    S = Wm.sketches(g, src, ALPHA)
    f = Wm.features(S, F, seed=3)
    pi = np.stack([O.dense_solve(g, s, ALPHA) for s in src], axis=1)
    params = random_params(rng, g.n, F, H, R)
    L, grads = Wm.backward(params, S, f, pi)

    def loss_at(p):
        X, *_ = Wm.forward(p, S, f)
        return Wm.loss(X, pi)

    assert abs(loss_at(params) - L) < 1e-14
    h = 1e-6
    for pi_idx in range(7):
        P = params[pi_idx]
        flat_idx = rng.choice(P.size, size=min(6, P.size), replace=False)
        for fi in flat_idx:
            idx = np.unravel_index(fi, P.shape)
            plus = [p.copy() for p in params]
            minus = [p.copy() for p in params]
            plus[pi_idx][idx] += h
            minus[pi_idx][idx] -= h
            num = (loss_at(plus) - loss_at(minus)) / (2 * h)
            ana = grads[pi_idx][idx]
            assert abs(num - ana) <= 1e-6 + 1e-4 * abs(num), (pi_idx, idx, num, ana)


def test_zero_basis_returns_sketch():
    """With U = 0 the estimate is the normalised sketch, which is S itself."""
    g = small_graph()
    S = Wm.sketches(g, [2, 5], ALPHA)
    h = np.ones((2, 4))
    X, _ = Wm.basis_forward(S, np.zeros((g.n, 4)), h)
    np.testing.assert_allclose(X, S, atol=1e-15)


def test_gelu_at_standard_normal_table_values():
    """GELU(x) = x Phi(x) (erf form); Phi(1) and Phi(2) from a standard normal
    table, and the derivative Phi(x) + x phi(x) at 0 and 1 (phi(1) = 0.2419707245)."""
    x = np.array([0.0, 1.0, -1.0, 2.0])
    np.testing.assert_allclose(Wm.gelu(x), [0.0, 0.8413447461, -0.1586552539, 2 * 0.9772498681], atol=1e-9)
    np.testing.assert_allclose(Wm.gelu_grad(np.array([0.0, 1.0])), [0.5, 0.8413447461 + 0.2419707245], atol=1e-9)


def test_bf16_rounding_matches_torch():
    """Round to nearest, ties to even: torch's float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-6, 1000)]).astype(np.float32)
    # exact halfway cases around 1 and 2^-100 (both even and odd lower neighbours)
    hi = np.concatenate([0x3F80 + np.arange(64), 0x0D80 + np.arange(64)]).astype(np.uint32)
    ties = (hi << 16 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(Wm.bf16(x), ref)


def test_features_equal_dense_product():
    """f = S^T G, brute force with every row of G drawn (the oracle skips the
    rows where S is zero)."""
    g = small_graph()
    S = Wm.sketches(g, [0, 9, 31], ALPHA)
    G = O.gaussian_rows(0, g.n, 16, seed=5)
    np.testing.assert_allclose(Wm.features(S, 16, seed=5), S.T @ G, rtol=1e-12, atol=1e-14)


def test_adam_step_closed_forms():
    """Adam (Kingma & Ba, 2015): with bias correction the first step has size lr
    in every coordinate whatever the gradient's scale, a constant gradient keeps
    that size at every step, and a zero gradient moves nothing.  Gradients +1
    then -1 give, by hand from the algorithm, -lr then +lr/19: in all
    -(18/19) lr."""
    g = np.array([3.0, -1e-3, 250.0, 0.0])
    z = np.zeros(4)
    p1, m1, v1 = Wm.adam_step(z, z, z, g, lr=1e-2, t=1)
    np.testing.assert_allclose(p1, -1e-2 * np.sign(g), rtol=1e-5)
    p, m, v = z, z, z
    for t in range(1, 51):
        p, m, v = Wm.adam_step(p, m, v, g, lr=1e-2, t=t)
    np.testing.assert_allclose(p, -0.5 * np.sign(g), rtol=1e-5)
    one = np.ones(1)
    p, m, v = Wm.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), one, lr=1.0, t=1)
    p, m, v = Wm.adam_step(p, m, v, -one, lr=1.0, t=2)
    np.testing.assert_allclose(p, -18.0 / 19.0, rtol=1e-6)
