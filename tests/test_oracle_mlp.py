"""Pins of the surrogate network's oracle (oracle/mlp.py).

References: central finite differences of the loss (every tensor of the
network), the closed-form derivative of the Gaussian negative log-likelihood
with respect to the outputs and its minimiser, and the closed form of the
first Adam step.  A planted mistake (a dropped SiLU derivative factor, a
transposed weight, a sign slip in the likelihood) fails one of them."""
import numpy as np
import pytest

import synth
from oracle import mlp


def _data(n=40, seed=1):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 6)), rng.standard_normal(n) * 0.7


def test_parameter_count_and_layout():
    assert mlp.n_params() == 6 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 2 + 2 == 34178
    th = synth.mlp_init(3).astype(float)
    ls = mlp.unpack(th)
    assert [W.shape for W, _ in ls] == [(128, 6), (128, 128), (128, 128), (2, 128)]
    assert np.all(ls[0][1] == 0) and ls[0][0][0, 0] == th[0] and ls[0][0][0, 1] == th[1]


def test_gradient_matches_central_differences():
    """Back-propagation against (L(th + h e_i) - L(th - h e_i)) / 2h for
    parameters in every weight matrix and bias vector."""
    X, y = _data()
    rng = np.random.default_rng(2)
    th = synth.mlp_init(4).astype(float)
    th[mlp.n_params() - 2:] = [0.1, -0.3]         # non-trivial output biases
    th += 0.01 * rng.standard_normal(th.shape)     # non-zero hidden biases too
    _, g = mlp.grad(th, X, y)
    offs = np.cumsum([0] + [o * i + o for i, o in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], 12) for k in range(4)] + [np.arange(offs[4] - 4, offs[4])])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (mlp.nll(th + e, X, y) - mlp.nll(th - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), i


def test_output_gradient_closed_form_and_minimiser():
    """With the output weights zero the network outputs its biases (mu0, s0);
    then dL/dmu0 = -mean(y - mu0) e^-s0 and dL/ds0 = (1 - mean((y - mu0)^2) e^-s0)/2,
    which vanish at mu0 = mean(y), s0 = log mean((y - mean y)^2)."""
    X, y = _data(64, 5)
    th = synth.mlp_init(6).astype(float)
    n = mlp.n_params()
    th[n - 2 - 256:n - 2] = 0.0
    mu0, s0 = 0.3, -0.4
    th[n - 2:] = [mu0, s0]
    _, g = mlp.grad(th, X, y)
    assert g[n - 2] == pytest.approx(-np.mean(y - mu0) * np.exp(-s0), rel=1e-12)
    assert g[n - 1] == pytest.approx(0.5 * (1 - np.mean((y - mu0) ** 2) * np.exp(-s0)), rel=1e-12)
    th[n - 2:] = [np.mean(y), np.log(np.mean((y - np.mean(y)) ** 2))]
    _, g = mlp.grad(th, X, y)
    assert abs(g[n - 2]) < 1e-14 and abs(g[n - 1]) < 1e-14


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(7)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    z = np.zeros(50)
    th1, m, v = mlp.adam(th, g, z, z, 1, lr=1e-3, eps=1e-8)
    assert np.allclose(th1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features():
    q = np.array([[0.3, 0.0, 0.4], [0.0, -1.0, 0.0]])
    X = mlp.features(q, [1.0, 2.0], [np.e ** 10, 1.0], qmax=2.0, wmax=4.0)
    assert np.allclose(X, [[0.25, 0.6, 0.0, 0.8, 0.25, 1.0], [0.5, 0.0, -1.0, 0.0, 0.5, 0.0]])
