"""The rate end on the GPU against the oracle: the composite dielectric
function binned in three-dimensional momentum space (Eq. (e_comp) and the
binning of Section III, with and without filling of empty bins), the isotropic
loss under each screening choice (Eqs. (ELF_screening), (MTF), (Lindhard)), and
the general rate with a velocity flux, vector and scalar mediators, its recoil
spectrum and the reach (Eqs. (general_rate), (H), (cross_section_iso), (v_min),
(excitation_rate)).  FP64 throughout: 1e-12 relative to the largest value
(counts exact), the FP64 bar of the other parity tests with room for the
different summation orders, except under Lindhard screening, whose bound per
point scales with the cancellation in the Lindhard sum (its condition number
reaches about 6e5 on these shells); the mixed path's tables at the mixed bar,
1e-4."""
import numpy as np
import pytest

import synth
from oracle import bins3d, rate as orate, rpa, screening
from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx
from tests.gpu_util import context, rel, set_oracle_states

pytestmark = pytest.mark.gpu
NSHELL, DQ, NTH, NPH = 24, 0.1, 3, 4          # coarse angular cells so that bins fill


@pytest.fixture(scope="module")
def small3():
    p = synth.make_small(nq=4, nw=20)
    iqs = [0, 1, 2, 3]
    refs = []
    for iq in iqs:
        Ck, Ckq = rpa.states(p, iq)
        refs.append((Ck, Ckq, rpa.solve_q(p, iq, Ck, Ckq)))
    return p, iqs, refs


def _oracle_tables(p, iqs, refs, q_lfe):
    kv = [p.qpts[iq][None, :] + p.G_int @ p.cell.recip for iq in iqs]
    ev = [bins3d.composite_eps(k, r[2]["eps_inv_diag"], r[2]["eps_diag"], q_lfe) for k, r in zip(kv, refs)]
    return kv, ev


def test_bin_eps3d_matches_oracle(small3):
    p, iqs, refs = small3
    ctx = context()
    set_oracle_states(ctx, p, iqs, refs[0][0], [r[1] for r in refs])
    for j in range(len(iqs)):
        ctx.pair_density(j, p.G_int, QCX_FP64)
        ctx.chi0(j, p.w, p.eta, QCX_FP64)
        ctx.invert_eps(j, QCX_FP64, want=False)
    for q_lfe in (0.0, 1.1, 10.0):
        kv, ev = _oracle_tables(p, iqs, refs, q_lfe)
        oe, oc = bins3d.bin_eps(kv, ev, DQ, NSHELL, NTH, NPH)
        for fill in (False, True):
            ge, gc = ctx.bin_eps3d(list(range(len(iqs))), q_lfe, NSHELL, DQ, NTH, NPH, len(p.w), fill=fill)
            we, wc = bins3d.fill_empty(oe, oc, DQ) if fill else (oe, oc)
            assert np.array_equal(gc, wc), (q_lfe, fill)
            assert rel(ge, we) < 1e-12, (q_lfe, fill)
            if fill:
                assert np.any(wc == -1)           # the case exercises the filling
    with pytest.raises(qcx.QcxError) as e:
        ctx.bin_eps3d([0, 7], 1.0, NSHELL, DQ, NTH, NPH, len(p.w))
    assert e.value.status in (1, 7)
    ctx.close()


def _lindhard_condition(wev, qs, ne, fp):
    """Condition number of the Lindhard evaluation at each (shell centre, w):
    the sum 1/2 + F_+ + F_- of Eq. (Lindhard) cancels to a small fraction of its
    terms when |Q_pm| is large, so its rounding error is about the unit roundoff
    times (1/2 + |F_+| + |F_-|)/|1/2 + F_+ + F_-|, carried into eps_L by the factor
    |eps_L - 1|/|eps_L|.  Bounds rounding only; the values come from the oracle."""
    qf, vf, wp = screening.electron_gas(ne)
    out = np.zeros((len(qs), len(wev)))
    for i, q in enumerate(qs):
        for j, w in enumerate(wev):
            a, b = q / (2.0 * qf), (w + 1j * fp * wp) / (q * vf)
            t = [qf / (4.0 * q) * (1.0 - Q * Q) * np.log((Q + 1.0) / (Q - 1.0)) for Q in (a + b, a - b)]
            s = 0.5 + t[0] + t[1]
            em1 = 3.0 * wp * wp / (q * q * vf * vf) * s
            out[i, j] = (0.5 + abs(t[0]) + abs(t[1])) / abs(s) * abs(em1) / abs(1.0 + em1)
    return out


def test_isotropic_loss_under_each_screening(small3):
    p, iqs, refs = small3
    kv, ev = _oracle_tables(p, iqs, refs, 1.1)
    e, c = bins3d.fill_empty(*bins3d.bin_eps(kv, ev, DQ, NSHELL, NTH, NPH), DQ)
    ctx = context()
    ne = 8.0 / p.cell.volume                                   # 8 valence electrons per cell (bohr^-3)
    qs = (np.arange(NSHELL) + 0.5) * DQ * orate.AME_EV          # shell centres (eV)
    wev = p.w * orate.HARTREE_EV
    ne_ev3 = ne * orate.AME_EV ** 3
    cases = {
        qcx.SCREEN_SELF: None,
        qcx.SCREEN_NONE: np.ones((NSHELL, len(p.w))),
        qcx.SCREEN_MTF: np.array([[screening.eps_mtf(w, q, 11.3, 1.563, 16.6, 4130.0) for w in wev] for q in qs]),
        qcx.SCREEN_LINDHARD: np.array([[screening.eps_lindhard(w, q, ne_ev3, 0.1) for w in wev] for q in qs]),
    }
    for model, scr in cases.items():
        want, nc = bins3d.isotropic_loss(e, c, scr)
        got, gnc = ctx.loss_isotropic(e, c, p.w, DQ, qcx.screening(model, ne_bohr3=ne, fp=0.1))
        assert np.array_equal(gnc, nc)
        if model == qcx.SCREEN_LINDHARD:
            # per point: the Lindhard sum cancels, so rounding scales with its condition number
            kap = _lindhard_condition(wev, qs, ne_ev3, 0.1)
            bound = 1e-12 * np.max(np.abs(want)) + 32 * 2.2e-16 * kap * np.abs(want)
            assert np.all(np.abs(got - want) <= bound), model
        else:
            assert rel(got, want) < 1e-12, model
    with pytest.raises(qcx.QcxError):
        ctx.loss_isotropic(e, c, p.w, DQ, qcx.screening(qcx.SCREEN_LINDHARD, ne_bohr3=ne, fp=0.0))
    ctx.close()


@pytest.mark.parametrize("m_med,kind,m_chi", [(-1.0, 0, 1e9), (0.0, 1, 1e9), (10.0e3, 0, 3e6), (0.0, 0, 1e6)])
def test_general_rate_matches_oracle(m_med, kind, m_chi):
    c = orate.C_KM_S
    hp = orate.HaloParams()
    v0, vesc, vE = hp.v0_kms / c, hp.vesc_kms / c, hp.vE_kms / c
    rng = np.random.default_rng(3)
    q = np.linspace(0.05, 4.0, 60)
    w = np.linspace(0.0, 60.0, 31) / orate.HARTREE_EV
    L = rng.uniform(0.0, 1.0, (len(q), len(w)))
    v = np.linspace(1e-6, 0.05, 2001) if m_chi < 1e7 else np.linspace(1e-6, (vesc + vE) * 1.001, 2001)
    flux = rng.uniform(0.5, 1.5, len(v)) * 1e6
    rp = orate.RelParams(m_chi_eV=m_chi, m_med_eV=m_med, mediator=kind)
    want = orate.dR_dw_general(q, w, L, v, flux, rp)
    wantQ = orate.recoil_spectrum(w, want, orate.HaloParams(), 12)
    ctx = context()
    got, gQ, reach = ctx.rate_general(q, w, L, v, flux, qcx.rate_params(m_chi_eV=m_chi, m_med_eV=m_med, mediator=kind,
                                                                        exposure_kg_yr=2.0),
                                      nQ=12, want_reach=True)
    ctx.close()
    assert np.max(want) > 0
    assert rel(got, want) < 1e-12 and rel(gQ, wantQ) < 1e-12
    wr = orate.reach(wantQ, 1e-39, 2.0)
    fin = np.isfinite(wr)
    assert np.array_equal(np.isfinite(reach), fin)
    assert np.allclose(reach[fin], wr[fin], rtol=1e-12, atol=0)


def test_mixed_path_isotropic_loss_at_the_mixed_bar(small3):
    """The mixed path's composite tables (binned and filled on the GPU) give
    the oracle's isotropic loss within 1e-4 where it exceeds 1e-3 of its
    maximum (per shell)."""
    p, iqs, refs = small3
    ctx = context()
    set_oracle_states(ctx, p, iqs, refs[0][0], [r[1] for r in refs])
    for j in range(len(iqs)):
        ctx.pair_density(j, p.G_int, QCX_MIXED)
        ctx.chi0(j, p.w, p.eta, QCX_MIXED)
        ctx.invert_eps(j, QCX_MIXED, want=False)
    ge, gc = ctx.bin_eps3d(list(range(len(iqs))), 1.1, NSHELL, DQ, NTH, NPH, len(p.w), fill=True)
    got, _ = ctx.loss_isotropic(ge, gc, p.w, DQ, qcx.screening(qcx.SCREEN_SELF))
    ctx.close()
    kv, ev = _oracle_tables(p, iqs, refs, 1.1)
    want, _ = bins3d.isotropic_loss(*bins3d.fill_empty(*bins3d.bin_eps(kv, ev, DQ, NSHELL, NTH, NPH), DQ))
    worst = 0.0
    for s in range(NSHELL):
        top = np.max(np.abs(want[s]))
        if top <= 0:
            continue
        m = np.abs(want[s]) > 1e-3 * top
        worst = max(worst, float(np.max(np.abs(got[s][m] - want[s][m]) / np.abs(want[s][m]))))
    print(f"mixed isotropic loss vs oracle: {worst:.2e}")
    assert worst < 1e-4
