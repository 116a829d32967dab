"""FP64 reference of the scatter surrogate's multilayer perceptron.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The surrogate replaces
the sum over scatter pixels of the path model (paper Eq. 2 restricted to the
first-order paths of Section 2.2) by a learned function of eight inputs:

    pixel x, pixel y, detector angle, event position u, event energy E,
    attenuation from the pixel to the detector along the detector direction,
    attenuation along the event's detector line from the pixel's depth on,
    attenuation along that whole line,

encoded in the detector frame of the angle (``features`` below): the event's
offset from the pixel's projection u - u_a(p), the pixel's coordinate along
the flight direction p . omega_a, its projection u_a(p) = p . t_a, the
angle, the energy and the three attenuations, each mapped to O(1) by a fixed
affine scaling.  The offset puts the quantity the scatter term varies
fastest with on one axis; the two line attenuations describe the object
along the line on which the event's scatter points lie (the callers take
them from ``Problem.line_attenuation``).
Architecture: 8 -> 256 -> 256 -> 256 -> 256 -> 1, ReLU after every hidden
layer, linear output; the output is the standardised natural log of the
scatter part of p_jn.  Parameters: W_l (out x in, row-major), b_l (out).
Training: mean squared error, Adam (Kingma & Ba 2015: bias-corrected first
and second moments).

Everything here is plain numpy in float64, one line per formula.
"""
from __future__ import annotations

import numpy as np

LAYERS = (8, 256, 256, 256, 256, 1)

def features(x_mm, y_mm, theta, u_mm, e_kev, atten, line_from, line_total):
    """Scaled network inputs (..., 8) of pixel centres (x, y), angles theta
    (flight direction omega = (cos, sin), lateral axis t = (-sin, cos)),
    event positions u, energies E, pixel-to-detector attenuation, and the
    attenuation along the event's detector line from the pixel's depth on
    and along the whole line."""
    x, y, th = (np.asarray(v, dtype=np.float64) for v in (x_mm, y_mm, theta))
    u_a = -x * np.sin(th) + y * np.cos(th)
    s_a = x * np.cos(th) + y * np.sin(th)
    u, e, att, lf, lt = (np.asarray(v, dtype=np.float64) for v in (u_mm, e_kev, atten, line_from, line_total))
    return np.stack(np.broadcast_arrays((u - u_a) / 50.0, s_a / 100.0, u_a / 100.0, (th - np.pi) / np.pi,
                                        (e - 137.5) / 37.5, (att - 1.5) / 1.5, (lf - 1.5) / 1.5,
                                        (lt - 1.5) / 1.5), axis=-1)


def init_params(seed=0, layers=LAYERS):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(layers[:-1], layers[1:]):
        W = rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)
        params.append([W, np.zeros(fan_out)])
    return params


def forward(params, X):
    """Returns the output (n,) and the per-layer cache (inputs, pre-activations)."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for k, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = np.maximum(z, 0.0) if k < len(params) - 1 else z
    return h[:, 0], cache


def backward(params, cache, dy):
    """Gradients of sum(dy * y) with respect to every W and b."""
    g = np.asarray(dy, dtype=np.float64)[:, None]
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        if k < len(params) - 1:
            g = g * (z > 0.0)
        W, _ = params[k]
        grads[k] = [g.T @ h, g.sum(axis=0)]
        g = g @ W
    return grads


def mse_loss_and_grad(params, X, t):
    """Mean squared error and its gradients."""
    y, cache = forward(params, X)
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    grads = backward(params, cache, 2.0 * r / len(r))
    return loss, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state = {'t': step, 'm': [...], 'v': [...]}."""
    if not state:
        state.update(t=0, m=[[np.zeros_like(p) for p in layer] for layer in params],
                     v=[[np.zeros_like(p) for p in layer] for layer in params])
    state["t"] += 1
    t = state["t"]
    for l, layer in enumerate(params):
        for i, p in enumerate(layer):
            g = grads[l][i]
            state["m"][l][i] = beta1 * state["m"][l][i] + (1 - beta1) * g
            state["v"][l][i] = beta2 * state["v"][l][i] + (1 - beta2) * g * g
            mhat = state["m"][l][i] / (1 - beta1 ** t)
            vhat = state["v"][l][i] / (1 - beta2 ** t)
            layer[i] = p - lr * mhat / (np.sqrt(vhat) + eps)
    return params
