"""FP64 oracle of the learned local-field correction (a surrogate that the
paper does not have): a multilayer perceptron that maps
(|q|, q direction, w, L_noLFE) to the log-ratio log(L_LFE / L_noLFE) of the
loss-function heads and its log-variance, so that L_LFE can be estimated from
the cheap L_noLFE (Eq. (eps_noLFE), one diagonal element of chi0) where the
network is confident, with the Dyson route (Eq. (eps_LFE)) as fallback.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: 6 -> 128 -> 128 -> 128 -> 2, SiLU(z) = z / (1 + e^-z) after each
hidden layer, outputs (mu, s) with s = log sigma^2.  Loss per sample: the
Gaussian negative log-likelihood without its constant,
    l = (s + (y - mu)^2 e^-s) / 2,
averaged over the batch.  Optimiser: Adam (Kingma and Ba, 2015) with bias
correction.  Parameter vector layout (shared with the GPU kernels because it
is an interface): for each layer W [out][in] row-major, then b [out].

Parity: gradients pinned by central finite differences of the loss; the
output-layer gradient by the closed-form derivative of l; the Adam step by
its closed form at t = 1 (update = -lr g / (|g| + eps)).
"""
from __future__ import annotations

import numpy as np

LAYERS = (6, 128, 128, 128, 2)


def n_params(layers=LAYERS) -> int:
    return sum(o * i + o for i, o in zip(layers[:-1], layers[1:]))


def unpack(theta, layers=LAYERS):
    """[(W [out][in], b [out])] views into theta."""
    out, p = [], 0
    for i, o in zip(layers[:-1], layers[1:]):
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X):
    """Outputs [n][2] = (mu, s) and the pre-activations of every layer."""
    a = np.asarray(X, float)
    zs, acts = [], [a]
    layers = unpack(np.asarray(theta, float))
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = silu(z) if li < len(layers) - 1 else z
        acts.append(a)
    return a, (zs, acts)


def nll(theta, X, y):
    out, _ = forward(theta, X)
    mu, s = out[:, 0], out[:, 1]
    r = np.asarray(y, float) - mu
    return float(np.mean(0.5 * (s + r * r * np.exp(-s))))


def grad(theta, X, y):
    """(loss, d loss / d theta) by back-propagation."""
    theta = np.asarray(theta, float)
    out, (zs, acts) = forward(theta, X)
    n = out.shape[0]
    mu, s = out[:, 0], out[:, 1]
    r = np.asarray(y, float) - mu
    e = np.exp(-s)
    loss = float(np.mean(0.5 * (s + r * r * e)))
    d = np.stack([-r * e, 0.5 * (1.0 - r * r * e)], axis=1) / n     # d loss / d (mu, s)
    layers = unpack(theta)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * dsilu(zs[li - 1])
    g = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, g


def adam(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(qvec, w, L_nolfe, qmax, wmax):
    """Inputs of the network: (|q|/qmax, q/|q|, w/wmax, ln(L_noLFE)/10)."""
    qvec = np.atleast_2d(np.asarray(qvec, float))
    qn = np.linalg.norm(qvec, axis=1)
    X = np.empty((qvec.shape[0], 6))
    X[:, 0] = qn / qmax
    X[:, 1:4] = qvec / qn[:, None]
    X[:, 4] = np.asarray(w, float) / wmax
    X[:, 5] = np.log(np.asarray(L_nolfe, float)) / 10.0
    return X
