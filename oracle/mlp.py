"""ORACLE for the learned router -- test infrastructure only (only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline leg may import it).

The paper has no learned component.  The router is an addition to the method:
an 8 -> 64 -> 64 -> 3 perceptron (ReLU after the two hidden layers) that
predicts, for one oriented edge, the standardised log cost of each of three
intersection variants.  Its features are defined on the oriented graph of
Sec. 3.2 (rank space, u < v):

    f0 log1p deg+(u)     f1 log1p deg+(v)     f2 log1p |{w in N+(u): w > v}|
    f3 log1p deg-(u)     f4 log1p deg-(v)     f5 log1p deg(u)
    f6 log1p deg(v)      f7 (v - u) / n

Two numeric modes:
  exact=True   float64 throughout (pins the backward pass by finite
               differences and closed forms)
  exact=False  the kernels' numerics: inputs, parameters and hidden
               activations rounded to bfloat16 (round to nearest even), every
               dot product and bias add accumulated in high precision, the
               output left unrounded.
Loss: L = sum over batch and outputs of (y - t)^2 / B.
"""
from __future__ import annotations

import numpy as np

SIZES = ((64, 8), (64,), (64, 64), (64,), (3, 64), (3,))  # W1 b1 W2 b2 W3 b3
NUM_PARAMS = sum(int(np.prod(s)) for s in SIZES)  # 4931


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(theta):
    out, k = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], np.float64).reshape(s))
        k += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in params])


def init(seed: int):
    """He-style initialisation (the trainer's starting point)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2 / 8), (64, 8))
    W2 = rng.normal(0, np.sqrt(2 / 64), (64, 64))
    W3 = rng.normal(0, np.sqrt(1 / 64), (3, 64))
    return [W1, np.zeros(64), W2, np.zeros(64), W3, np.zeros(3)]


def forward(params, X, exact=False):
    W1, b1, W2, b2, W3, b3 = params
    r = (lambda a: a) if exact else bf16
    X, W1, b1, W2, b2, W3, b3 = (r(a) for a in (X, W1, b1, W2, b2, W3, b3))
    z1 = X @ W1.T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + b2
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ W3.T + b3
    return y, (X, W1, W2, W3, z1, h1, z2, h2)


def loss(params, X, T, exact=False):
    y, _ = forward(params, X, exact)
    return float(((y - T) ** 2).sum() / X.shape[0])


def backward(params, X, T, exact=False):
    """Gradients of L in the order W1, b1, W2, b2, W3, b3 (activations and
    weights as the forward pass used them)."""
    y, (Xr, W1, W2, W3, z1, h1, z2, h2) = forward(params, X, exact)
    B = X.shape[0]
    dy = 2.0 * (y - T) / B
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dh2 = (dy @ W3) * (z2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    dW1 = dh1.T @ Xr
    db1 = dh1.sum(0)
    return [dW1, db1, dW2, db2, dW3, db3]


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of the float64 master copy."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(off, adj, deg):
    """Per oriented edge (CSR order of the rank-space out-lists off/adj) the
    eight router features; deg = undirected degree per rank."""
    n = len(off) - 1
    outd = np.diff(off).astype(np.float64)
    ind = deg.astype(np.float64) - outd
    u = np.repeat(np.arange(n), np.diff(off))
    v = adj.astype(np.int64)
    pos = np.arange(len(adj)) - off[u]
    suf = outd[u] - pos - 1
    f = np.stack([np.log1p(outd[u]), np.log1p(outd[v]), np.log1p(suf), np.log1p(ind[u]),
                  np.log1p(ind[v]), np.log1p(deg[u].astype(np.float64)),
                  np.log1p(deg[v].astype(np.float64)), (v - u) / max(n, 1)], axis=1)
    return f
