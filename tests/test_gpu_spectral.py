"""The spectral route to chi0 on the GPU (Eq. (eRPA_spectral) with the
principal part from the Kramers-Kronig relations, Section II.D) against the
oracle of the same route (hat weights on a uniform energy grid, the retarded
broadening of the direct sum in the transform), and against the direct sum of
Eq. (RPA) where the two coincide (every transition energy on the grid).

Bars: FP64 1e-10 relative to the largest value (the FP64 bar of the other
parity tests); the mixed route (FP32 pair densities, weights and contraction)
chi0 5e-5 and the loss functions 1e-4 per spectrum where L > 1e-3 of the
spectrum's maximum, the bars of the mixed direct path."""
import numpy as np
import pytest

import synth
from oracle import rpa, spectral
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx
from tests.gpu_util import context, rel, rel_spectrum, set_oracle_states

pytestmark = pytest.mark.gpu


def _grid(dE, step):
    """The grid rule of qcx_spectral_grid, written out for the oracle's energies."""
    E0 = step * np.floor(dE.min() / step) - step
    return E0, int(np.floor((dE.max() - E0) / step)) + 3


@pytest.fixture(scope="module")
def small():
    p = synth.make_small(nq=2, nw=24)
    iq = 1
    Ck, Ckq = rpa.states(p, iq)
    o = rpa.solve_q(p, iq, Ck, Ckq)
    step = p.eta / 4
    E0, nbin = _grid(o["dE"], step)
    S = spectral.spectral_weights(o["rho"], o["dE"], E0, step, nbin, p.nk, p.cell.volume)
    chi = spectral.chi0_from_spectral(S, E0, step, p.w, p.eta)
    eps = rpa.dielectric_matrix(chi, o["vs"])
    L1, L2, _, _ = rpa.loss_functions(eps)
    return p, iq, Ck, Ckq, dict(step=step, E0=E0, nbin=nbin, S=S, chi=chi, L_lfe=L1, L_nolfe=L2)


def _ctx(p, iq, Ck, Ckq, prec):
    ctx = context()
    set_oracle_states(ctx, p, [iq], Ck, [Ckq])
    ctx.pair_density(0, p.G_int, prec)
    return ctx


def test_grid_rule_matches_the_oracles_energies(small):
    p, iq, Ck, Ckq, o = small
    ctx = _ctx(p, iq, Ck, Ckq, QCX_FP64)
    E0, nbin = ctx.spectral_grid(0, o["step"])
    ctx.close()
    assert E0 == o["E0"] and nbin == o["nbin"]


@pytest.mark.parametrize("chunk", [0, 32])
def test_fp64_spectral_route_matches_oracle(small, chunk):
    """Weights, chi0 and both loss functions; chunk 32 splits the grid into
    several chunks (added in FP64), which changes nothing beyond rounding."""
    p, iq, Ck, Ckq, o = small
    ctx = _ctx(p, iq, Ck, Ckq, QCX_FP64)
    ctx.set_spectral_chunk(chunk)
    chi, S = ctx.chi0_spectral(0, p.w, p.eta, o["E0"], o["step"], o["nbin"], QCX_FP64, want=True, want_S=True)
    ctx.invert_eps(0, QCX_FP64, want=False)
    L1, L2 = ctx.loss_function(0, QCX_FP64)
    ctx.close()
    assert o["nbin"] > 32 * 4                      # several chunks at chunk = 32
    assert rel(S, o["S"]) < 1e-10
    assert rel(chi, o["chi"]) < 1e-10
    assert rel(L1, o["L_lfe"]) < 1e-10 and rel(L2, o["L_nolfe"]) < 1e-10
    top = np.max(np.abs(S))
    for b in (0, o["nbin"] // 2, o["nbin"] - 1):   # every weight matrix is Hermitian
        assert np.max(np.abs(S[b] - S[b].conj().T)) <= 1e-13 * top


@pytest.mark.parametrize("engine", ["tensor", "cuda_cores"])
@pytest.mark.parametrize("chunk", [0, 64])
def test_mixed_spectral_route_at_the_mixed_bar(small, engine, chunk):
    """Both engines of the mixed contraction (tcgen05 split BF16, CUDA-core FP32),
    in one chunk and in chunks of 64 grid points."""
    p, iq, Ck, Ckq, o = small
    ctx = _ctx(p, iq, Ck, Ckq, QCX_MIXED)
    ctx.set_spectral_engine(engine == "cuda_cores")
    ctx.set_spectral_chunk(chunk)
    chi, _ = ctx.chi0_spectral(0, p.w, p.eta, o["E0"], o["step"], o["nbin"], QCX_MIXED, want=True)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    ctx.close()
    e = rel(chi, o["chi"]), rel_spectrum(L1, o["L_lfe"]), rel_spectrum(L2, o["L_nolfe"])
    print(f"mixed spectral route ({engine}, chunk {chunk}) vs oracle: chi0 %.2e, L_LFE %.2e, L_noLFE %.2e" % e)
    assert e[0] < 5e-5 and e[1] < 1e-4 and e[2] < 1e-4


def test_on_grid_energies_give_the_direct_sum():
    """Band energies rounded to multiples of step = 2^-8 Hartree put every
    dE_t exactly on a grid point (x = 0), where the route is the direct sum of
    Eq. (RPA) term by term: the GPU's spectral chi0 equals the oracle's direct
    chi0 with those energies (and the GPU's direct chi0)."""
    p = synth.make_small(nq=1, nw=16)
    step = 2.0 ** -8
    p.Ek = np.round(p.Ek / step) * step
    p.Ekq = np.round(p.Ekq / step) * step
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    E0, nbin = _grid(o["dE"], step)
    ctx = _ctx(p, 0, Ck, Ckq, QCX_FP64)
    direct = ctx.chi0(0, p.w, p.eta, QCX_FP64, want=True)
    chi, _ = ctx.chi0_spectral(0, p.w, p.eta, E0, step, nbin, QCX_FP64, want=True)
    ctx.close()
    assert rel(chi, o["chi0"]) < 1e-10
    assert rel(chi, direct) < 1e-10


def test_bad_grids_and_order_are_reported(small):
    p, iq, Ck, Ckq, o = small
    ctx = context()
    set_oracle_states(ctx, p, [iq], Ck, [Ckq])
    with pytest.raises(qcx.QcxError) as e:             # no pair densities yet
        ctx.chi0_spectral(0, p.w, p.eta, o["E0"], o["step"], o["nbin"], QCX_FP64)
    assert e.value.status == 7
    ctx.pair_density(0, p.G_int, QCX_FP64)
    for E0, nbin in ((o["E0"] + 10 * o["step"], o["nbin"]),     # lowest transitions below the grid
                     (o["E0"], o["nbin"] - 3),                     # highest above it
                     (o["E0"], 1)):
        with pytest.raises(qcx.QcxError) as e:
            ctx.chi0_spectral(0, p.w, p.eta, E0, o["step"], nbin, QCX_FP64)
        assert e.value.status == 1
    # the context stays usable
    chi, _ = ctx.chi0_spectral(0, p.w, p.eta, o["E0"], o["step"], o["nbin"], QCX_FP64, want=True)
    ctx.close()
    assert rel(chi, o["chi"]) < 1e-10
