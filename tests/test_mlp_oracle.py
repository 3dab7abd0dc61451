"""Pins for the router network's oracle (oracle/mlp.py): finite differences,
closed forms and the bfloat16 rounding rule -- nothing checked against itself."""
import numpy as np
import pytest

from oracle import mlp


def rand_params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return [rng.normal(0, scale, s) for s in mlp.SIZES]


def test_param_count():
    assert mlp.NUM_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 4931


def test_bf16_rounding_rule():
    # 8 significant bits: ties go to the even neighbour
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (odd neighbour 1+2^-7 loses)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7     # above the midpoint
    assert mlp.bf16(-2.5) == -2.5
    assert mlp.bf16(3.14159265) == 3.140625
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)
    assert np.array_equal(mlp.bf16(r), r)                      # idempotent


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    params = rand_params(seed)
    X = rng.normal(size=(7, 8))
    T = rng.normal(size=(7, 3))
    grads = mlp.backward(params, X, T, exact=True)
    eps = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            orig = flat[idx]
            flat[idx] = orig + eps
            lp = mlp.loss(params, X, T, exact=True)
            flat[idx] = orig - eps
            lm = mlp.loss(params, X, T, exact=True)
            flat[idx] = orig
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g.ravel()[idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, g.ravel()[idx])


def test_zero_weights_output_is_bias():
    params = [np.zeros(s) for s in mlp.SIZES]
    params[5] = np.array([0.5, -1.25, 2.0])
    X = np.random.default_rng(1).normal(size=(5, 8))
    y, _ = mlp.forward(params, X)
    assert np.array_equal(y, np.tile(params[5], (5, 1)))
    T = np.zeros((5, 3))
    g = mlp.backward(params, X, T, exact=True)
    assert np.allclose(g[5], 2 * params[5])        # dL/db3 = 2 * mean (y - t) * B / B
    for k in range(5):
        assert not np.any(g[k])                      # dead ReLUs, zero weights


def test_linear_regime_composes_matrices():
    rng = np.random.default_rng(3)
    params = rand_params(3, 0.1)
    params[1] = np.full(64, 100.0)   # every hidden unit active: the net is affine
    params[3] = np.full(64, 1.0e5)
    X = rng.normal(size=(9, 8))
    W1, b1, W2, b2, W3, b3 = params
    assert np.all((X @ W1.T + b1) > 0) and np.all(((X @ W1.T + b1) @ W2.T + b2) > 0)
    want = ((X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    y, _ = mlp.forward(params, X, exact=True)
    assert np.allclose(y, want, rtol=1e-10, atol=1e-6)


def test_bf16_mode_is_close_to_exact():
    rng = np.random.default_rng(4)
    params = rand_params(4, 0.3)
    X = rng.normal(size=(64, 8))
    ye, _ = mlp.forward(params, X, exact=True)
    yb, _ = mlp.forward(params, X, exact=False)
    assert np.allclose(yb, ye, rtol=0.05, atol=0.05)
    assert not np.array_equal(yb, ye)


def test_adam_first_step_moves_by_lr_times_sign():
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    t2, m, v = mlp.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step is lr * g / (|g| + eps)
    assert np.allclose(t2[:2], theta[:2] - 0.01 * np.sign(g[:2]), atol=1e-7)
    assert t2[2] == theta[2]


def test_features_closed_form_on_a_path():
    # path 0-1-2 (degrees 1,2,1); DESC eta ranks: 1 -> 0, 0 -> 1, 2 -> 2
    off = np.array([0, 2, 2, 2])       # rank 0 points to ranks 1 and 2
    adj = np.array([1, 2])
    deg = np.array([2, 1, 1])
    f = mlp.features(off, adj, deg)
    assert f.shape == (2, 8)
    assert np.allclose(f[0], [np.log1p(2), 0, np.log1p(1), 0, np.log1p(1), np.log1p(2), np.log1p(1), 1 / 3])
    assert np.allclose(f[1], [np.log1p(2), 0, 0, 0, np.log1p(1), np.log1p(2), np.log1p(1), 2 / 3])
