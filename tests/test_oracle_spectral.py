"""Pins of the spectral-route oracle (oracle/spectral.py), CPU only.

The route bins each transition's conj(rho) rho once per q on an energy grid
with hat weights and recovers chi0(w) with the retarded kernel.  Pinned by:
exact agreement with the direct sum (Eq. (RPA)) when every transition energy
lies on the grid; exact conservation of the zeroth and first energy moments of
every delta by the hat weights (so the first-moment sum of the spectral
weights equals that of the transitions); second-order convergence to the
direct sum as the grid is refined; and the N_G = 1 single-oscillator case."""
import numpy as np
import pytest

import synth
from oracle import rpa, spectral


@pytest.fixture(scope="module")
def tiny():
    p = synth.make_tiny(seed=11, shells_per_atom=2, n_k=2, nv=2, nc=3, ng=7, nq=1, nw=9)
    Ck, Ckq = rpa.states(p, 0)
    o = rpa.solve_q(p, 0, Ck, Ckq)
    return p, o


def _direct(p, o, dE, w):
    return rpa.chi0(o["rho"], rpa.transition_weights(dE, w, p.eta), p.nk, p.cell.volume)


def test_exact_when_transitions_lie_on_the_grid(tiny):
    p, o = tiny
    step = 0.01
    dE = np.round(o["dE"] / step) * step              # move every transition onto the grid
    E0 = np.floor(dE.min() / step) * step - 2 * step
    nbin = int(round((dE.max() - E0) / step)) + 3
    S = spectral.spectral_weights(o["rho"], dE, E0, step, nbin, p.nk, p.cell.volume)
    got = spectral.chi0_from_spectral(S, E0, step, p.w, p.eta)
    want = _direct(p, o, dE, p.w)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_hat_weights_keep_zeroth_and_first_moments(tiny):
    p, o = tiny
    step = 0.037
    E0 = o["dE"].min() - 1.3 * step
    nbin = int((o["dE"].max() - E0) / step) + 3
    S = spectral.spectral_weights(o["rho"], o["dE"], E0, step, nbin, p.nk, p.cell.volume)
    E = E0 + step * np.arange(nbin)
    pref = 2.0 / (p.nk * p.cell.volume)
    rho = o["rho"]
    m0 = pref * rho.conj().T @ rho
    m1 = pref * (rho.conj().T * o["dE"][None, :]) @ rho
    assert np.allclose(S.sum(axis=0), m0, rtol=1e-12, atol=1e-14 * np.abs(m0).max())
    assert np.allclose(np.einsum("b,bgh->gh", E, S), m1, rtol=1e-12, atol=1e-14 * np.abs(m1).max())
    # every weight is a non-negative combination: the diagonal spectral weights are >= 0
    assert np.all(np.einsum("bgg->bg", S).real >= -1e-18) and np.abs(np.einsum("bgg->bg", S).imag).max() < 1e-15


def test_second_order_convergence_to_the_direct_sum(tiny):
    p, o = tiny
    w = p.w[1:]
    want = _direct(p, o, o["dE"], w)
    errs = []
    for step in (0.002, 0.001, 0.0005):            # step <= eta / 9, the asymptotic regime
        E0 = o["dE"].min() - 1.5 * step
        nbin = int((o["dE"].max() - E0) / step) + 3
        S = spectral.spectral_weights(o["rho"], o["dE"], E0, step, nbin, p.nk, p.cell.volume)
        got = spectral.chi0_from_spectral(S, E0, step, w, p.eta)
        errs.append(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    print("relative errors", errs, "ratios", r1, r2)
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0        # halving the step divides the error by ~4


def test_single_oscillator():
    """One transition of weight |rho|^2 = 1 at dE between grid points: chi0 is the
    two-pole interpolation, and at eta -> large the hat-split kernel equals the
    exact one to second order in the offset."""
    rho = np.array([[1.0 + 0.0j]])
    dE = np.array([0.3 + 0.25 * 0.1])
    S = spectral.spectral_weights(rho, dE, 0.0, 0.1, 6, 1, 1.0)
    assert np.allclose(S[:, 0, 0], [0, 0, 0, 1.5, 0.5, 0])        # pref 2, weights 0.75 / 0.25
    w = np.array([0.05, 0.7])
    got = spectral.chi0_from_spectral(S, 0.0, 0.1, w, 1.0)[:, 0, 0]
    K = lambda E: 1 / (w - E + 1j) - 1 / (w + E + 1j)
    assert np.allclose(got, 2 * (0.75 * K(0.3) + 0.25 * K(0.4)), rtol=1e-14)
    assert np.allclose(got, 2 * K(dE[0]), rtol=5e-3)
    with pytest.raises(ValueError):
        spectral.hat_weights(np.array([0.55]), 0.0, 0.1, 6)         # beyond the last interval
