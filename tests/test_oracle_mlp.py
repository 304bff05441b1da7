"""Pins for the MLP oracle (CPU): central finite differences of the loss
check every partial derivative of `grad`; closed forms at zero weights check
the forward pass and the loss."""
import numpy as np

from oracle import mlp


def sample(seed, n=40):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.4, mlp.NPARAMS)
    x = rng.uniform(0, 1, (n, mlp.IN))
    y = (rng.uniform(size=n) < 0.5).astype(np.float64)
    wt = rng.uniform(0.1, 2.0, n)
    return w, x, y, wt


def test_gradient_matches_finite_differences():
    for seed in (1, 2, 3):
        w, x, y, wt = sample(seed)
        g = mlp.grad(w, x, y, wt)
        h = 1e-6
        num = np.empty_like(w)
        for k in range(w.size):
            e = np.zeros_like(w)
            e[k] = h
            num[k] = (mlp.loss(w + e, x, y, wt) - mlp.loss(w - e, x, y, wt)) / (2 * h)
        assert np.max(np.abs(g - num)) < 1e-7 * max(1.0, np.max(np.abs(num))) + 1e-9


def test_zero_weights_closed_form():
    # all weights zero: z = 0, p = 1/2, loss = log 2 whatever the labels
    w = np.zeros(mlp.NPARAMS)
    _, x, y, wt = sample(4)
    assert np.allclose(mlp.prob(w, x), 0.5)
    assert abs(mlp.loss(w, x, y, wt) - np.log(2.0)) < 1e-12
    # dL/db3 = sum wt (1/2 - y) / sum wt; every other gradient is zero
    g = mlp.grad(w, x, y, wt)
    assert abs(g[-1] - np.sum(wt * (0.5 - y)) / np.sum(wt)) < 1e-12
    assert np.all(g[:-1] == 0)


def test_output_bias_only_network():
    # only b3 set: z = b3 for every sample
    w = np.zeros(mlp.NPARAMS)
    w[-1] = 1.3
    _, x, y, wt = sample(5)
    assert np.allclose(mlp.prob(w, x), 1 / (1 + np.exp(-1.3)))


def test_adam_first_step_is_sign_times_lr():
    # with bias correction the first Adam step moves every parameter with a
    # non-zero gradient by lr * g / (|g| + eps) ~ lr * sign(g)
    rng = np.random.default_rng(6)
    w = rng.normal(size=10)
    g = rng.normal(size=10)
    w1, _, _ = mlp.adam_step(w, np.zeros(10), np.zeros(10), g, 1, lr=0.01)
    assert np.allclose(w - w1, 0.01 * np.sign(g), rtol=1e-6)
