"""The learned local-field correction on its own workload: 110 q of the
mid-size workload (200 w each), heads from the mixed Dyson route; the network
is trained on 100 q and evaluated on 10 held-out q.

What it gains over the method without it: the no-LFE method takes
L_LFE = L_noLFE (log ratio 0); the trained network must predict the held-out
log ratios better than that.  The surrogate route must give exactly the Dyson
heads wherever it falls back, L_noLFE e^mu where it accepts, and an L_noLFE
equal to the Dyson route's eps_00 value."""
import numpy as np
import pytest

import synth
from paper_2603_12326_gb300 import QCX_MIXED, qcx, states, surrogate
from tests.gpu_util import context

pytestmark = pytest.mark.gpu
NTRAIN = 100


@pytest.fixture(scope="module")
def setup():
    ctx = context()
    p = synth.make_surrogate_set()
    L1, L2 = surrogate.head_table(ctx, p, range(p.nq))
    unit = 2.0 * np.pi / p.cell.a
    qmax, wmax = 4.0 * unit, float(p.w[-1])
    tr = list(range(NTRAIN))
    te = list(range(NTRAIN, p.nq))
    X, y, _ = surrogate.dataset(ctx, p, tr, L1[:NTRAIN], L2[:NTRAIN], qmax, wmax)
    Xt, yt, rc = surrogate.dataset(ctx, p, te, L1[NTRAIN:], L2[NTRAIN:], qmax, wmax)
    ctx.mlp_set_params(synth.mlp_init(2024))
    curve = ctx.mlp_train(X, y, qcx.mlp_opts(epochs=200, batch=256, lr=1e-3, seed=5))
    yield ctx, p, L1, L2, (X, y), (Xt, yt, rc), curve, qmax, wmax
    ctx.close()


def test_network_gains_over_no_lfe_on_held_out_q(setup):
    ctx, p, L1, L2, (X, y), (Xt, yt, _), curve, *_ = setup
    assert len(y) > 15000 and len(yt) > 1500
    mu, lv = ctx.mlp_predict(Xt)
    mae_net = float(np.mean(np.abs(mu - yt)))
    mae_nolfe = float(np.mean(np.abs(yt)))                 # L_LFE = L_noLFE
    mae_const = float(np.mean(np.abs(yt - np.median(y))))  # best constant from training data
    inside = float(np.mean(np.abs(mu - yt) < 2.0 * np.exp(0.5 * lv)))
    print(f"held-out |log ratio| error: network {mae_net:.4f}, no-LFE {mae_nolfe:.4f}, constant {mae_const:.4f}; "
          f"within 2 sigma {inside:.2f}; loss {curve[0]:.3f} -> {curve[-1]:.3f}")
    assert curve[-1] < curve[0]
    assert mae_net < mae_nolfe
    assert inside > 0.5


def test_surrogate_route_and_fallback(setup):
    ctx, p, L1, L2, _, (Xt, yt, rc), _, qmax, wmax = setup
    te = list(range(NTRAIN, p.nq))
    states.load_problem(ctx, p, te)
    opts = qcx.SurrogateOpts(qmax, wmax, 1e-2, 0.05, 1e-2, 7)
    La, Lb, src, chk = ctx.surrogate_heads(range(len(te)), p.G_int, p.w[1:], p.eta, opts, QCX_MIXED)
    Ld, Ln = L1[NTRAIN:, 1:], L2[NTRAIN:, 1:]
    print(f"accepted {np.mean(src == 0):.3f}, spot-checked {np.sum(src == 2)}, largest miss {chk:.2e}")
    fb = src != 0
    assert np.max(np.abs(La[fb] - Ld[fb]) / np.abs(Ld[fb])) < 1e-12      # the Dyson heads themselves
    # the cheap head (FP64, one G) against the mixed Dyson route's eps_00 value
    m = Ln > 1e-3 * Ln.max(axis=1, keepdims=True)
    assert np.max(np.abs(Lb[m] - Ln[m]) / Ln[m]) < 1e-4
    acc = src == 0
    if np.any(acc):
        qv = np.repeat(p.qpts[te], len(p.w) - 1, axis=0)
        X, _ = ctx.surrogate_features(qv, np.tile(p.w[1:], len(te)), Lb.reshape(-1), qmax, wmax)
        mu, _ = ctx.mlp_predict(X)
        assert np.allclose(La[acc], (Lb * np.exp(mu.reshape(Lb.shape)))[acc], rtol=1e-6)
