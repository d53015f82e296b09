"""Surrogate network kernels (forward, backward, Adam) against the oracle.

The oracle runs in FP64 on the values the kernels compute with (BF16 weight
matrices widened to FP32, FP32 biases), so the comparison measures the
kernels' FP32 arithmetic only.  Tolerances: gradients 1e-4 of each tensor's
largest entry (FP32 sums of up to 128 x 200 terms), loss and outputs 1e-5
relative, one Adam step 1e-6 absolute where the gradient is not negligible."""
import numpy as np
import pytest

import synth
from oracle import mlp
from paper_2603_12326_gb300 import qcx
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 6)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + 0.3 * X[:, 4] - 0.2 * X[:, 5] ** 2).astype(np.float32)
    return X, y


def _tensors(v):
    offs = np.cumsum([0] + [o * i + o for i, o in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])])
    out = []
    for k in range(4):
        i, o = mlp.LAYERS[k], mlp.LAYERS[k + 1]
        out.append(v[offs[k]:offs[k] + o * i])
        out.append(v[offs[k] + o * i:offs[k + 1]])
    return out


def test_gradient_and_loss_match_oracle(ctx):
    th0 = synth.mlp_init(11)
    th0[-2:] = [0.2, -0.5]
    ctx.mlp_set_params(th0)
    master, comp = ctx.mlp_get_params()
    assert np.array_equal(master, th0)
    X, y = _data(203, 1)                      # 203: a ragged last tile of 11 samples
    loss, g = ctx.mlp_grad(X, y)
    lo, go = mlp.grad(comp.astype(float), X.astype(float), y.astype(float))
    assert loss == pytest.approx(lo, rel=1e-5)
    for a, b in zip(_tensors(g), _tensors(go)):
        assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b)) + 1e-12


def test_predict_matches_oracle_forward(ctx):
    ctx.mlp_set_params(synth.mlp_init(12))
    _, comp = ctx.mlp_get_params()
    X, _ = _data(1000, 2)
    mu, lv = ctx.mlp_predict(X)
    out, _ = mlp.forward(comp.astype(float), X.astype(float))
    assert np.max(np.abs(mu - out[:, 0])) <= 1e-5 * np.max(np.abs(out[:, 0]))
    assert np.max(np.abs(lv - out[:, 1])) <= 1e-5 * np.max(np.abs(out[:, 1]))


def test_one_adam_step_matches_oracle(ctx):
    th0 = synth.mlp_init(13)
    ctx.mlp_set_params(th0)
    _, comp = ctx.mlp_get_params()
    X, y = _data(256, 3)
    curve = ctx.mlp_train(X, y, qcx.mlp_opts(epochs=1, batch=256, lr=1e-3))
    th1, _ = ctx.mlp_get_params()
    lo, go = mlp.grad(comp.astype(float), X.astype(float), y.astype(float))
    assert curve[0] == pytest.approx(lo, rel=1e-5)
    want, _, _ = mlp.adam(th0.astype(float), go, np.zeros_like(go), np.zeros_like(go), 1, lr=1e-3)
    big = np.abs(go) > 1e-4 * np.max(np.abs(go))
    assert np.max(np.abs(th1[big] - want[big])) < 1e-6
    # where the gradient is negligible the step is still bounded by lr (plus FP32 rounding of |theta| ~ 1.3)
    assert np.max(np.abs(th1 - th0)) <= 1e-3 + 2.5e-7


def test_training_lowers_the_loss_and_is_deterministic(ctx):
    X, y = _data(4096, 4)
    res = []
    for _ in range(2):
        ctx.mlp_set_params(synth.mlp_init(14))
        curve = ctx.mlp_train(X, y, qcx.mlp_opts(epochs=40, batch=256, lr=2e-3, seed=9))
        res.append((curve, ctx.mlp_get_params()[0]))
    curve = res[0][0]
    print("loss per epoch:", np.round(curve[[0, 9, 19, 39]], 4))
    assert curve[-1] < curve[0] - 1.0
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][0], res[1][0])
    # the trained network predicts the smooth target on fresh inputs
    Xt, yt = _data(2000, 5)
    mu, lv = ctx.mlp_predict(Xt)
    assert np.sqrt(np.mean((mu - yt) ** 2)) < 0.35 * np.std(yt)     # predicting the mean gives 1.0
