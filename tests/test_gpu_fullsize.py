"""Parity at the benchmark's full size: the first q of the mid workload
(512 k, N_b = 96, N_t = 65 536, N_G = 181, 200 w) through the mixed path in the
launch configuration bench.py times (one chi0 launch over all 200 w), and
through the FP64 path; the oracle recomputes four of the frequencies in full
(every G and G').  Tolerances as in the other parity tests: chi0 5e-5 and the
loss functions 1e-4 (per spectrum where L > 1e-3 of its maximum over the
sampled frequencies) for the mixed path, 1e-10 for the FP64 path."""
import numpy as np
import pytest

import synth
from oracle import rpa, spectral
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED
from tests.gpu_util import context, rel, rel_spectrum, set_oracle_states

pytestmark = pytest.mark.gpu
SAMPLE_W = [40, 80, 120, 160]


@pytest.fixture(scope="module")
def mid():
    p = synth.make_mid(nq=1)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq, w=p.w[SAMPLE_W])
    return p, Ck, Ckq, o


def _masked(a, b, frac=1e-3):
    top = np.max(np.abs(b), axis=0, keepdims=True)
    m = np.abs(b) > frac * top
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def test_mid_workload_full_size_mixed(mid):
    p, Ck, Ckq, o = mid
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, QCX_MIXED)
    chi = ctx.chi0(0, p.w, p.eta, QCX_MIXED, want=True)          # all 200 w in one launch
    ctx.invert_eps(0, QCX_MIXED, want=False)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    e_chi = rel(chi[SAMPLE_W], o["chi0"])
    e1 = _masked(L1[SAMPLE_W], o["L_lfe"])
    e2 = _masked(L2[SAMPLE_W], o["L_nolfe"])
    print(f"mid full size, mixed: chi0 {e_chi:.2e}, L_LFE {e1:.2e}, L_noLFE {e2:.2e}")
    assert e_chi < 5e-5 and e1 < 1e-4 and e2 < 1e-4
    assert np.all(np.isfinite(L1)) and np.all(L1[1:] > -1e-8)     # the whole table: finite, no negative loss


def test_mid_workload_full_size_fp64(mid):
    p, Ck, Ckq, o = mid
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, QCX_FP64)
    chi = ctx.chi0(0, p.w[SAMPLE_W], p.eta, QCX_FP64, want=True)
    ctx.invert_eps(0, QCX_FP64, want=False)
    L1, L2 = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    assert rel(chi, o["chi0"]) < 1e-10
    assert rel(L1, o["L_lfe"]) < 1e-10 and rel(L2, o["L_nolfe"]) < 1e-10


def test_mid_workload_every_q_mixed_vs_fp64_gpu():
    """All 50 q of the benchmark workload: the mixed path's loss tables (all
    200 w in one launch per q, as the benchmark runs them) against the FP64 GPU
    path (itself held to 1e-10 of the oracle) at eight frequencies per q.
    Bar: 1e-4 relative per spectrum (fixed q and G) where L exceeds 1e-3 of the
    spectrum's maximum over the 200 frequencies."""
    from paper_2603_12326_gb300 import states
    p = synth.make_mid()
    ctx = context()
    states.load_problem(ctx, p)
    sample = np.linspace(1, len(p.w) - 1, 8).astype(int)
    worst = {"L_lfe": 0.0, "L_nolfe": 0.0}
    for iq in range(p.nq):
        ctx.pair_density(iq, p.G_int, QCX_MIXED)
        ctx.chi0(iq, p.w, p.eta, QCX_MIXED)
        ctx.invert_eps(iq, QCX_MIXED, want=False)
        m1, m2 = ctx.loss_function(iq, QCX_MIXED)
        ctx.pair_density(iq, p.G_int, QCX_FP64)
        ctx.chi0(iq, p.w[sample], p.eta, QCX_FP64)
        ctx.invert_eps(iq, QCX_FP64, want=False)
        d1, d2 = ctx.loss_function(iq, QCX_FP64)
        for key, m, d in (("L_lfe", m1, d1), ("L_nolfe", m2, d2)):
            top = np.max(np.abs(m), axis=0, keepdims=True)
            mask = np.abs(d) > 1e-3 * top
            worst[key] = max(worst[key], float(np.max(np.abs(m[sample][mask] - d[mask]) / np.abs(d[mask]))))
    ctx.close()
    print("mid workload, 50 q x 8 w, mixed vs FP64 GPU:", {k: f"{v:.2e}" for k, v in worst.items()})
    assert worst["L_lfe"] < 1e-4 and worst["L_nolfe"] < 1e-4


def test_mid_workload_spectral_route(mid):
    """The spectral route at the benchmark's size: q = 0 of the mid workload,
    all 200 w, grid step eta/20 (about 8000 grid points, one chunk).  FP64
    against the oracle's spectral route on a sampled 12 x 12 block of (G, G')
    (the weights of a block need only its columns of rho) at 1e-10; the mixed
    route against the FP64 route at the mixed bars (chi0 5e-5, loss 1e-4 per
    spectrum where L > 1e-3 of its maximum)."""
    p, Ck, Ckq, o = mid
    step = p.eta / 20
    dE = o["dE"]
    E0 = step * np.floor(dE.min() / step) - step
    nbin = int(np.floor((dE.max() - E0) / step)) + 3
    ng = p.G_int.shape[0]
    cols = np.unique(np.linspace(0, ng - 1, 12).astype(int))
    S_sub = spectral.spectral_weights(o["rho"][:, cols], dE, E0, step, nbin, p.nk, p.cell.volume)
    chi_sub = spectral.chi0_from_spectral(S_sub, E0, step, p.w, p.eta)
    ctx = context()
    set_oracle_states(ctx, p, [0], Ck, [Ckq])
    assert ctx.spectral_grid(0, step) == (E0, nbin)
    ctx.pair_density(0, p.G_int, QCX_FP64)
    chi64, _ = ctx.chi0_spectral(0, p.w, p.eta, E0, step, nbin, QCX_FP64, want=True)
    ctx.invert_eps(0, QCX_FP64, want=False)
    L64 = ctx.loss_function(0, QCX_FP64)
    ctx.pair_density(0, p.G_int, QCX_MIXED)
    chim, _ = ctx.chi0_spectral(0, p.w, p.eta, E0, step, nbin, QCX_MIXED, want=True)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    Lm = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    e64 = rel(chi64[:, cols][:, :, cols], chi_sub)
    em = rel(chim, chi64), rel_spectrum(Lm[0], L64[0]), rel_spectrum(Lm[1], L64[1])
    dd = rel_spectrum(L64[0][SAMPLE_W], o["L_lfe"])
    print(f"mid spectral route ({nbin} points): FP64 vs oracle {e64:.2e}; mixed vs FP64 chi0 {em[0]:.2e}, "
          f"L_LFE {em[1]:.2e}, L_noLFE {em[2]:.2e}; L_LFE vs the direct sum {dd:.2e}")
    assert e64 < 1e-10
    assert em[0] < 5e-5 and em[1] < 1e-4 and em[2] < 1e-4
