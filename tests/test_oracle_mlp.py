"""Pins of the FP64 surrogate-network reference (CPU only).

- Analytic gradients against central finite differences of the loss.
- SiLU and its derivative at closed-form points.
- Adam's first step is -lr * g / (|g| + eps) (bias corrections cancel), and Adam
  minimises a quadratic bowl.
- Parameter count of the 5 -> 256 -> 256 -> 256 -> 1 network.
- Input scaling maps the parameter box onto [-1, 1].
"""
import math

import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.n_params() == 133_377


def test_silu_closed_forms():
    assert mlp.silu(np.array(0.0)) == 0.0
    assert abs(mlp.silu(np.array(1.0)) - 1.0 / (1.0 + math.exp(-1.0))) < 1e-16
    assert mlp.silu_grad(np.array(0.0)) == 0.5
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.silu_grad(z))) < 1e-9


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    layers = (5, 16, 16, 16, 1)
    params = mlp.init_params(rng, layers)
    X = rng.uniform(-1, 1, (12, 5))
    y = rng.normal(size=12)
    grads = mlp.backward(params, X, y)
    h = 1e-6
    for li, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            lp = mlp.loss(params, X, y)
            flat[k] = old - h
            lm = mlp.loss(params, X, y)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g.reshape(-1)[k]) < 1e-7 * max(1.0, abs(fd)), (li, k)


def test_gradient_shapes_and_full_size_network():
    rng = np.random.default_rng(1)
    params = mlp.init_params(rng)
    X = rng.uniform(-1, 1, (4, 5))
    grads = mlp.backward(params, X, np.zeros(4))
    assert [g.shape for g in grads] == [p.shape for p in params]


def test_adam_first_step_and_convergence():
    g = np.array([0.3, -2.0, 1e-3])
    p = [np.zeros(3)]
    newp, m, v = mlp.adam_step(p, [g], [np.zeros(3)], [np.zeros(3)], 1, lr=0.01)
    assert np.allclose(newp[0], -0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # quadratic bowl 0.5 * |A w - c|^2
    rng = np.random.default_rng(2)
    A = rng.normal(size=(6, 3))
    c = rng.normal(size=6)
    w_star = np.linalg.lstsq(A, c, rcond=None)[0]
    w = [np.zeros(3)]
    m, v = [np.zeros(3)], [np.zeros(3)]
    for t in range(1, 4001):
        grad = A.T @ (A @ w[0] - c)
        w, m, v = mlp.adam_step(w, [grad], m, v, t, lr=0.01)
    assert np.max(np.abs(w[0] - w_star)) < 1e-4


def test_input_scaling_maps_box_to_unit_cube():
    lo = mlp.scale_inputs(0.0, 1.0, 0.0, 0.5, 1e-4)
    hi = mlp.scale_inputs(8.0, 10.0, 1.0, 2.0, 1e-1)
    assert np.allclose(lo, -1.0) and np.allclose(hi, 1.0)
