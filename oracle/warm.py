"""FP64 oracle of the learned warm start (test infrastructure only).

The warm start maps a cheap sketch of the source to an initial estimate x,
whose push residual r = (alpha e_s + (1-alpha) x P - x) / alpha is then pushed
to lambda like any other residual (so the answer's guarantee does not depend
on the model).  The paper has no learned component; the model here is:

* sketch  S = alpha e_s + alpha (1-alpha) e_s P + (1-alpha)^2 e_s P^2: the
  reserve after two Power Iterations (Eq. 5) plus the alive mass left at the
  second step (Eq. 3), so sum(S) = 1;
* features f = S G with G a fixed n x F standard-normal matrix
  (``oracle.gaussian_rows``);
* MLP  a1 = f W1 + b1, h1 = gelu(a1); a2 = h1 W2 + b2, h2 = gelu(a2);
  h = h2 W3 + b3  (gelu(x) = x Phi(x), the erf form);
* basis  Z = S + U h (U is n x R), Y = max(0, Z), X = Y / sum(Y), with X = S
  when sum(Y) = 0;
* loss   mean over the batch of ||X - pi||_1.

Layouts: S, Z, X, pi are n x B (one column per source); f is B x F; weights
are (in x out).  Everything is float64; the GPU's BF16 weights are passed in
already rounded.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import Graph, gaussian_rows

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def transition_apply(g: Graph, x: np.ndarray) -> np.ndarray:
    """x P for a vector x over nodes (P_v = A_v / d_v, Sec. 2)."""
    d = np.diff(g.row_ptr)
    src = np.repeat(np.arange(g.n), d)
    out = np.zeros(g.n)
    np.add.at(out, g.col_idx, (x / d)[src])
    return out


def sketch(g: Graph, s: int, alpha: float = 0.2) -> np.ndarray:
    e = np.zeros(g.n)
    e[s] = 1.0
    p1 = transition_apply(g, e)
    p2 = transition_apply(g, p1)
    return alpha * e + alpha * (1 - alpha) * p1 + (1 - alpha) ** 2 * p2


def sketches(g: Graph, src, alpha: float = 0.2) -> np.ndarray:
    return np.stack([sketch(g, int(s), alpha) for s in src], axis=1)  # n x B


def features(S: np.ndarray, F: int, seed: int) -> np.ndarray:
    """f = S^T G over the nonzero rows of S (B x F)."""
    rows = np.nonzero(np.any(S != 0, axis=1))[0]
    f = np.zeros((S.shape[1], F))
    for u in rows:
        f += np.outer(S[u], gaussian_rows(int(u), 1, F, seed)[0])
    return f


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32, back to float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(f, W1, b1, W2, b2, W3, b3, rnd=None):
    """rnd(x) rounds a tensor where the GPU feeds it to a BF16 GEMM (identity by default)."""
    r = rnd or (lambda x: x)
    f = r(f)
    a1 = f @ W1 + b1
    h1 = r(gelu(a1))
    a2 = h1 @ W2 + b2
    h2 = r(gelu(a2))
    h = h2 @ W3 + b3
    return h, (f, a1, h1, a2, h2)


def basis_forward(S, U, h, rnd=None):
    r = rnd or (lambda x: x)
    Z = S + r(U) @ r(h).T
    Y = np.maximum(Z, 0.0)
    sig = Y.sum(axis=0)
    X = np.where(sig > 0, Y / np.where(sig > 0, sig, 1.0), S)
    return X, (Z, sig)


def loss(X, pi):
    return np.abs(X - pi).sum() / X.shape[1]


def forward(params, S, f, rnd=None):
    W1, b1, W2, b2, W3, b3, U = params
    r = rnd or (lambda x: x)
    h, mcache = mlp_forward(f, r(W1), b1, r(W2), b2, r(W3), b3, rnd)
    X, bcache = basis_forward(S, U, h, rnd)
    return X, h, mcache, bcache


def backward(params, S, f, pi, rnd=None):
    """Loss and gradients (subgradient sign(X - pi) of the l1 loss).  With rnd,
    the forward pass rounds where the GPU does and the backward pass uses the
    rounded tensors; gradients themselves stay float64."""
    r = rnd or (lambda x: x)
    W1, b1, W2, b2, W3, b3, U = [r(p) if i in (0, 2, 4, 6) else p for i, p in enumerate(params)]
    X, h, (f_, a1, h1, a2, h2), (Z, sig) = forward([W1, b1, W2, b2, W3, b3, U], S, f, rnd)
    B = X.shape[1]
    L = loss(X, pi)
    dX = np.sign(X - pi) / B
    t = (dX * X).sum(axis=0)
    live = sig > 0
    dY = np.where(live, (dX - t) / np.where(live, sig, 1.0), 0.0)
    dZ = dY * (Z > 0)
    dU = dZ @ h
    dh = dZ.T @ U
    dW3 = h2.T @ dh
    db3 = dh.sum(axis=0)
    da2 = (dh @ W3.T) * gelu_grad(a2)
    dW2 = h1.T @ da2
    db2 = da2.sum(axis=0)
    da1 = (da2 @ W2.T) * gelu_grad(a1)
    dW1 = f_.T @ da1
    db1 = da1.sum(axis=0)
    return L, [dW1, db1, dW2, db2, dW3, db3, dU]


def adam_step(p, m, v, g, lr: float, t: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015, Algorithm 1) at step t >= 1:
    exponential moving averages of the gradient and of its square, each
    divided by one minus its decay rate to the power t (bias correction), and
    a step of lr times the corrected mean over the root of the corrected
    second moment plus eps.  Returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def warm_estimate(g: Graph, src, params, F: int, seed: int, alpha: float = 0.2, rnd=None) -> np.ndarray:
    """X for a batch of sources (n x B)."""
    S = sketches(g, src, alpha)
    f = features(S, F, seed)
    X, *_ = forward(params, S, f, rnd)
    return X


def unflatten(flat, n: int, F: int = 128, H: int = 512, R: int = 64):
    """Split the library's flat parameter order W1, b1, W2, b2, W3, b3, U."""
    flat = np.asarray(flat, dtype=np.float64)
    shapes = [(F, H), (H,), (H, H), (H,), (H, R), (R,), (n, R)]
    out, o = [], 0
    for sh in shapes:
        cnt = int(np.prod(sh))
        out.append(flat[o:o + cnt].reshape(sh))
        o += cnt
    assert o == len(flat)
    return out
