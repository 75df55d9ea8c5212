"""Pins of the proposal network's CPU oracle: gradient against central finite
differences, the purely linear regime against a closed form, and the top-k rule
against sorting."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    x = rng.standard_normal((7, mlp.F))
    t = rng.standard_normal(7)
    _, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.N_PARAMS, size=200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS); e[i] = h
        num = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_linear_regime_closed_form():
    # all pre-activations positive: y = ((x W1 + b1) W2 + b2) w3 + b3
    rng = np.random.default_rng(2)
    q = {"W1": np.abs(rng.standard_normal((12, 64))), "b1": np.ones(64), "W2": np.abs(rng.standard_normal((64, 64))),
         "b2": np.ones(64), "w3": rng.standard_normal(64), "b3": np.array([0.5])}
    p = np.concatenate([q[name].ravel() for name, _ in mlp.SIZES])
    x = np.abs(rng.standard_normal((5, 12)))
    y = ((x @ q["W1"] + q["b1"]) @ q["W2"] + q["b2"]) @ q["w3"] + 0.5
    assert np.allclose(mlp.forward(p, x), y, rtol=1e-12, atol=1e-12)
    # and the gradient of the output layer is the mean of 2 (y - t) h2
    t = rng.standard_normal(5)
    _, g = mlp.loss_and_grad(p, x, t)
    h2 = (x @ q["W1"] + q["b1"]) @ q["W2"] + q["b2"]
    w3_off = 12 * 64 + 64 + 64 * 64 + 64
    assert np.allclose(g[w3_off:w3_off + 64], h2.T @ (2 * (y - t) / 5), rtol=1e-10)


def test_zero_weights_output_is_bias():
    p = np.zeros(mlp.N_PARAMS); p[-1] = 3.25
    assert np.all(mlp.forward(p, np.ones((4, 12))) == 3.25)


def test_topk_rule():
    s = np.array([0.5, 2.0, 2.0, -1.0, 2.0, 0.5])
    assert list(mlp.topk(s, 2)) == [1, 2]
    assert list(mlp.topk(s, 4)) == [0, 1, 2, 4]
    rng = np.random.default_rng(3)
    s = rng.integers(0, 5, size=300).astype(float)
    k = 77
    sel = mlp.topk(s, k)
    thr = np.sort(s)[::-1][k - 1]
    assert np.all(s[sel] >= thr) and np.sum(s > thr) <= k and len(sel) == k
