"""Pins of the FP64 MLP oracle (CPU only): central finite differences of the
loss against the analytic gradients, a linear-network closed form, and the
first Adam steps against their closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    layers = (6, 16, 12, 8, 1)
    params = mlp.init_params(3, layers)
    for W, b in params:
        b += rng.normal(0, 0.3, b.shape)     # move pre-activations off the ReLU kink
    X = rng.normal(0, 1, (40, 6))
    t = rng.normal(0, 1, 40)
    loss, grads = mlp.mse_loss_and_grad(params, X, t)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            idx = list(zip(*[rng.integers(0, s, 6) for s in arr.shape]))
            for ix in idx:
                old = arr[ix]
                arr[ix] = old + h
                lp, _ = mlp.mse_loss_and_grad(params, X, t)
                arr[ix] = old - h
                lm, _ = mlp.mse_loss_and_grad(params, X, t)
                arr[ix] = old
                assert g[ix] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_linear_network_matches_closed_form():
    # a single linear layer: y = X w + b, MSE gradient = 2/n X^T (y - t)
    rng = np.random.default_rng(2)
    params = mlp.init_params(0, (6, 1))
    X = rng.normal(0, 1, (25, 6))
    t = rng.normal(0, 1, 25)
    loss, grads = mlp.mse_loss_and_grad(params, X, t)
    y = X @ params[0][0][0] + params[0][1][0]
    np.testing.assert_allclose(grads[0][0][0], 2.0 / 25 * X.T @ (y - t), rtol=1e-12)
    np.testing.assert_allclose(grads[0][1][0], 2.0 / 25 * np.sum(y - t), rtol=1e-12)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)


def test_adam_first_steps_closed_form():
    # with a constant gradient g, bias correction makes every step -lr * sign(g)
    # (up to eps): m_hat = g and v_hat = g^2 after any number of steps
    params = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    g = [[np.array([[0.3, -0.7]]), np.array([2.0])]]
    state = {}
    for k in range(3):
        mlp.adam_step(params, g, state, lr=0.01, eps=0.0)
    np.testing.assert_allclose(params[0][0], [[1.0 - 0.03, -2.0 + 0.03]], rtol=1e-12)
    np.testing.assert_allclose(params[0][1], [0.5 - 0.03], rtol=1e-12)


def test_relu_network_is_piecewise_linear():
    # scaling all inputs and the first-layer biases by c > 0 scales the output's
    # affine part consistently: f(cX; W1, c b1, ...) with linear later layers
    rng = np.random.default_rng(4)
    params = mlp.init_params(5, (6, 10, 1))
    X = rng.normal(0, 1, (7, 6))
    y1, _ = mlp.forward(params, X)
    params2 = [[params[0][0], params[0][1] * 3.0], [params[1][0], params[1][1] * 3.0]]
    y3, _ = mlp.forward(params2, 3.0 * X)
    np.testing.assert_allclose(y3, 3.0 * y1, rtol=1e-12)


def test_feature_encoding_special_angles():
    # theta = 0: flight direction +x, lateral axis +y, so u_a(p) = y and p.omega = x;
    # theta = pi/2: omega = +y, t = -x, so u_a(p) = -x and p.omega = y
    x, y, u, e, att, lf, lt = 30.0, -20.0, 5.0, 150.0, 0.75, 3.0, 4.5
    f0 = mlp.features(x, y, 0.0, u, e, att, lf, lt)
    np.testing.assert_allclose(f0, [(u - y) / 50.0, x / 100.0, y / 100.0, -1.0, (e - 137.5) / 37.5, -0.5,
                                    1.0, 2.0], rtol=1e-12, atol=1e-15)
    f1 = mlp.features(x, y, np.pi / 2, u, e, att, lf, lt)
    np.testing.assert_allclose(f1, [(u + x) / 50.0, y / 100.0, -x / 100.0, -0.5, (e - 137.5) / 37.5, -0.5,
                                    1.0, 2.0], rtol=1e-12, atol=1e-15)
    # an event on the pixel's projection has zero offset at any angle
    th = np.linspace(0.0, 2 * np.pi, 7)
    ua = -x * np.sin(th) + y * np.cos(th)
    np.testing.assert_allclose(mlp.features(x, y, th, ua, e, att, lf, lt)[:, 0], 0.0, atol=1e-14)
