"""FP64 reference of the surrogate network (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this network maps the parameters of Eq. 1
(a, omega, f, gamma, log10 D) to the ensemble mean velocity <<v>> of Sec. 5
(asymptotic velocity, the time-averaged observable).  Architecture: 5 -> 256 ->
256 -> 256 -> 1, SiLU after each hidden layer, linear output, mean-squared-error
loss, Adam (Kingma & Ba 2015, Algorithm 1) on the weights.

Parameters are a list [W1, b1, W2, b2, W3, b3, W4, b4] with W_l of shape
(out, in), row-major, so that a layer computes y = x @ W_l.T + b_l.
Every array here is float64; nothing is fused or reordered.
"""
import numpy as np

LAYERS = (5, 256, 256, 256, 1)

# Parameter box of the surrogate and the affine map of each input onto [-1, 1].
BOX = {
    "a": (0.0, 8.0),
    "omega": (1.0, 10.0),
    "f": (0.0, 1.0),
    "gamma": (0.5, 2.0),
    "log10D": (-4.0, -1.0),
}


def scale_inputs(a, omega, f, gamma, D):
    """Map raw parameters to the network's input features in [-1, 1]."""
    cols = [a, omega, f, gamma, np.log10(D)]
    out = []
    for c, (lo, hi) in zip(cols, BOX.values()):
        out.append(2.0 * (np.asarray(c, dtype=np.float64) - lo) / (hi - lo) - 1.0)
    return np.stack(out, axis=-1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(rng, layers=LAYERS):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    params = []
    for fin, fout in zip(layers[:-1], layers[1:]):
        bound = 1.0 / np.sqrt(fin)
        params.append(rng.uniform(-bound, bound, size=(fout, fin)))
        params.append(rng.uniform(-bound, bound, size=(fout,)))
    return params


def forward(params, X):
    """Returns (output of shape (B,), cache of pre-activations and activations)."""
    h = np.asarray(X, dtype=np.float64)
    acts = [h]
    pres = []
    nl = len(params) // 2
    for l in range(nl):
        W, b = params[2 * l], params[2 * l + 1]
        z = h @ W.T + b
        pres.append(z)
        h = silu(z) if l < nl - 1 else z
        acts.append(h)
    return h[:, 0], (pres, acts)


def loss(params, X, y):
    """Mean-squared error: mean over the batch of (net(x) - y)^2."""
    out, _ = forward(params, X)
    return np.mean((out - y) ** 2)


def backward(params, X, y):
    """Gradient of loss() with respect to every parameter (same order)."""
    out, (pres, acts) = forward(params, X)
    B = out.shape[0]
    g = (2.0 / B) * (out - y)[:, None]          # dL/d(output pre-activation)
    nl = len(params) // 2
    grads = [None] * len(params)
    for l in range(nl - 1, -1, -1):
        W = params[2 * l]
        grads[2 * l] = g.T @ acts[l]
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            g = (g @ W) * silu_grad(pres[l - 1])
    return grads


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); t counts from 1.
    Returns new (params, m, v)."""
    newp, newm, newv = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = beta1 * mi + (1.0 - beta1) * g
        vi = beta2 * vi + (1.0 - beta2) * g * g
        mhat = mi / (1.0 - beta1 ** t)
        vhat = vi / (1.0 - beta2 ** t)
        newp.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        newm.append(mi)
        newv.append(vi)
    return newp, newm, newv


def n_params(layers=LAYERS):
    return sum(fin * fout + fout for fin, fout in zip(layers[:-1], layers[1:]))
