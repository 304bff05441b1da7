"""MLP oracle for the learned mode switch -- TEST INFRASTRUCTURE ONLY.

Plain float64 numpy restatement of the 8-16-16-1 network (tanh hidden units,
logistic output) and of the gradient of its weighted logistic loss, written
from the chain rule. Parameters are one flat vector in the order
W1[16][8], b1[16], W2[16][16], b2[16], w3[16], b3 (433 values).

Pinned in tests/test_oracle_mlp.py by central finite differences of the loss
(an independent check of every partial derivative) and by closed forms at
zero weights.
"""
import numpy as np

IN, H = 8, 16
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == NPARAMS
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = w[k : k + size].reshape(shape)
        k += size
    return out


def forward(w, x):
    """Logits z[i] and hidden activations for samples x[i] (n x 8)."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    z = h2 @ p["w3"] + p["b3"][0]
    return z, h1, h2


def prob(w, x):
    z, _, _ = forward(w, x)
    return 1.0 / (1.0 + np.exp(-z))


def loss(w, x, y, wt):
    """sum_i wt_i * (softplus(z_i) - y_i z_i) / sum_i wt_i."""
    z, _, _ = forward(w, x)
    wt = np.asarray(wt, dtype=np.float64)
    sp = np.logaddexp(0.0, z)
    return float(np.sum(wt * (sp - np.asarray(y, dtype=np.float64) * z)) / np.sum(wt))


def grad(w, x, y, wt):
    """Gradient of `loss` with respect to the flat parameter vector."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    wt = np.asarray(wt, dtype=np.float64)
    z, h1, h2 = forward(w, x)
    dz = wt * (1.0 / (1.0 + np.exp(-z)) - y) / np.sum(wt)  # dL/dz per sample
    g = {}
    g["w3"] = dz @ h2
    g["b3"] = np.array([dz.sum()])
    d2 = np.outer(dz, p["w3"]) * (1.0 - h2 ** 2)           # dL/d(pre-activation 2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (1.0 - h1 ** 2)                   # dL/d(pre-activation 1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return np.concatenate([g[name].ravel() for name, _ in SHAPES])


def adam_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015), t counted from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
