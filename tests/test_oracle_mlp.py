"""Pins of the oracle's cost-model network: central finite differences for the
backward pass, the affine closed form when every ReLU is active, and the
published first-step property of Adam."""
import numpy as np
import pytest

from oracle import mlp


def rand_params(F, H, V, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(0, scale, s) for k, s in mlp.shapes(F, H, V).items()}


def test_backward_matches_finite_differences():
    F, H, V, M = 5, 7, 3, 11
    p = rand_params(F, H, V, 0)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(M, F))
    T = rng.normal(size=(M, V))
    mask = (rng.random((M, V)) < 0.8).astype(np.float64)
    Y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, Y, T, mask)
    h = 1e-6
    for name in mlp.PARAM_NAMES:
        it = np.nditer(p[name], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[name][idx]
            p[name][idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)[0], T, mask)
            p[name][idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)[0], T, mask)
            p[name][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_forward_affine_closed_form():
    """With positive weights, biases and inputs every ReLU is active and the
    network is the affine map X (W3 W2 W1)^T + (W3 (W2 b1 + b2) + b3)."""
    F, H, V = 4, 6, 2
    rng = np.random.default_rng(2)
    p = {k: np.abs(rng.normal(0, 0.5, s)) + 0.01 for k, s in mlp.shapes(F, H, V).items()}
    X = np.abs(rng.normal(size=(9, F)))
    M = p["W3"] @ p["W2"] @ p["W1"]
    c = p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"]
    Y, _ = mlp.forward(p, X)
    assert np.allclose(Y, X @ M.T + c, rtol=1e-13, atol=0)


def test_loss_and_output_bias_gradient():
    F, H, V, M = 3, 4, 2, 5
    p = rand_params(F, H, V, 3)
    rng = np.random.default_rng(3)
    X, T = rng.normal(size=(M, F)), rng.normal(size=(M, V))
    mask = np.ones((M, V))
    mask[0, 1] = 0
    Y, cache = mlp.forward(p, X)
    assert mlp.loss(Y, T, mask) == pytest.approx(((Y - T) ** 2 * mask).sum() / 9)
    g = mlp.backward(p, cache, Y, T, mask)
    assert np.allclose(g["b3"], (2 * mask * (Y - T)).sum(axis=0) / 9)


def test_adam_first_step_is_lr_times_sign():
    """Adam's bias correction makes the first step lr * g/(|g| + eps) ~ lr*sign(g)."""
    p = {k: np.zeros(2) for k in mlp.PARAM_NAMES}
    g = {k: np.array([0.3, -2.0]) for k in mlp.PARAM_NAMES}
    st = {}
    mlp.adam_step(p, g, st, 1, lr=0.01)
    for k in mlp.PARAM_NAMES:
        assert np.allclose(p[k], [-0.01, 0.01], rtol=1e-6)
    # a zero gradient afterwards keeps moving with the first moment only
    z = {k: np.zeros(2) for k in mlp.PARAM_NAMES}
    before = {k: v.copy() for k, v in p.items()}
    mlp.adam_step(p, z, st, 2, lr=0.01)
    m_hat = 0.9 * 0.1 * np.array([0.3, -2.0]) / (1 - 0.81)
    v_hat = 0.999 * 0.001 * np.array([0.09, 4.0]) / (1 - 0.999 ** 2)
    for k in mlp.PARAM_NAMES:
        assert np.allclose(p[k] - before[k], -0.01 * m_hat / (np.sqrt(v_hat) + 1e-8), rtol=1e-12)


def test_adam_steps_two_and_three_hand_computed():
    """Adam (Kingma and Ba) on one parameter, worked by hand in exact fractions
    with beta1 = 1/2, beta2 = 3/4, lr = 1/10, eps = 0 and gradients 2, -2, 2:

      t=1: m = 1,    v = 1,     m^ = 1/(1/2) = 2,       v^ = 1/(1/4) = 4,        p = 0 - (1/10)(2/2)       = -1/10
      t=2: m = -1/2, v = 7/4,   m^ = (-1/2)/(3/4) = -2/3, v^ = (7/4)/(7/16) = 4,  p = -1/10 + (1/10)(1/3)  = -1/15
      t=3: m = 3/4,  v = 37/16, m^ = (3/4)/(7/8) = 6/7,   v^ = (37/16)/(37/64) = 4, p = -1/15 - (1/10)(3/7) = -23/210

    A first moment or second moment not carried from one step to the next, or
    a bias correction with the wrong power of beta, changes steps 2 and 3."""
    p = {k: np.zeros(1) for k in mlp.PARAM_NAMES}
    st = {}
    expected = [-1 / 10, -1 / 15, -23 / 210]
    for t, (gv, want) in enumerate(zip((2.0, -2.0, 2.0), expected), start=1):
        g = {k: np.array([gv]) for k in mlp.PARAM_NAMES}
        mlp.adam_step(p, g, st, t, lr=0.1, beta1=0.5, beta2=0.75, eps=0.0)
        for k in mlp.PARAM_NAMES:
            assert p[k][0] == pytest.approx(want, rel=1e-15, abs=1e-17), (t, k)
    assert st["m_W1"][0] == pytest.approx(0.75, rel=1e-15) and st["v_W1"][0] == pytest.approx(37 / 16, rel=1e-15)
