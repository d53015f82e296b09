"""Pins of the oracle's rate-end extensions (CPU only): the model dielectric
functions and the screened loss (Eqs. (MTF), (Lindhard), (ELF_screening)), the
general rate with a velocity flux and vector or scalar mediators (Eqs.
(general_rate), (H), (cross_section_iso), (v_min)), the reach, and the
composite function binned in three-dimensional momentum space (Eq. (e_comp)
and the binning it describes).  Each pin is a limit, an identity, a sum rule or
a value worked out by hand."""
import numpy as np
import pytest

from oracle import bins3d, rate, screening

SI_MTF = dict(eps0=11.3, tau=1.563, wp=16.6, qtf=4130.0)          # the paper's Si parameters (eV)


def _ne_for(wp):
    """Electron density (eV^3) of a gas with plasma energy wp."""
    return wp * wp * screening.ME_EV / (4.0 * np.pi * screening.ALPHA)


# ------------------------------------------------------------------- screening
def test_mtf_static_limit_plasmon_pole_and_free_electron_limit():
    # static, long-wavelength limit: the dielectric constant eps0
    assert screening.eps_mtf(0.0, 0.0, **SI_MTF) == pytest.approx(11.3, rel=1e-14)
    # at q = 0 the bracket vanishes at w = w_p / sqrt(eps0 - 1): eps changes sign through a pole
    wpole = 16.6 / np.sqrt(10.3)
    lo, hi = screening.eps_mtf(wpole * (1 - 1e-6), 0.0, **SI_MTF), screening.eps_mtf(wpole * (1 + 1e-6), 0.0, **SI_MTF)
    assert lo > 1e5 and hi < -1e5
    # large q: the q^4 term dominates, eps - 1 -> 4 m_e^2 w_p^2 / q^4
    q = 2e6
    got = (screening.eps_mtf(0.0, q, **SI_MTF) - 1.0) * q ** 4 / (4 * screening.ME_EV ** 2 * 16.6 ** 2)
    assert got == pytest.approx(1.0, rel=2e-3)


def test_lindhard_thomas_fermi_and_high_frequency_limits():
    ne = _ne_for(16.6)
    qf, vf, wp = screening.electron_gas(ne)
    assert wp == pytest.approx(16.6, rel=1e-12)
    # static, q -> 0: Thomas-Fermi screening eps = 1 + k_TF^2/q^2, k_TF^2 = 3 w_p^2 / v_F^2
    q = 1e-3 * qf
    e = screening.eps_lindhard(0.0, q, ne, 1e-9)
    assert e.real == pytest.approx(1.0 + 3 * wp * wp / (vf * vf * q * q), rel=1e-5)
    assert abs(e.imag) < 1e-6 * e.real
    # w >> q v_F: a free electron gas, eps -> 1 - w_p^2/w^2
    q = 0.05 * qf
    for w in (40.0, 80.0):
        e = screening.eps_lindhard(w, q, ne, 1e-9)
        assert e.real == pytest.approx(1.0 - wp * wp / (w * w), rel=2e-3)
    # at q = 2 q_F the logarithm's weight vanishes: eps is finite, 1 + (3/8) w_p^2/(q_F^2 v_F^2)
    e = screening.eps_lindhard(0.0, 2 * qf * (1 + 1e-9), ne, 1e-9)
    assert e.real == pytest.approx(1.0 + 0.375 * wp * wp / (qf * qf * vf * vf), rel=1e-6)


def test_lindhard_f_sum_rule():
    """int_0^inf w Im eps(w, q) dw = (pi/2) w_p^2 at any q (weak damping)."""
    ne = _ne_for(16.6)
    qf, vf, wp = screening.electron_gas(ne)
    q = 0.6 * qf
    wmax = q * vf + q * q / (2 * screening.ME_EV)
    w = np.linspace(0.0, 1.6 * wmax, 40001)
    im = np.array([screening.eps_lindhard(x, q, ne, 1e-5).imag for x in w])
    assert np.trapezoid(w * im, w) == pytest.approx(0.5 * np.pi * wp * wp, rel=3e-3)


def test_screened_loss_identities():
    eps = np.array([1.5 + 0.7j, 3.0 + 0.1j, -0.4 + 2.0j])
    assert np.allclose(screening.screened_loss(eps, eps), (-1.0 / eps).imag, rtol=1e-15)
    assert np.allclose(screening.screened_loss(eps, np.ones(3)), eps.imag, rtol=1e-15)


# ------------------------------------------------------------------ rate end
def _shm():
    p = rate.HaloParams()
    c = rate.C_KM_S
    return p, p.v0_kms / c, p.vesc_kms / c, p.vE_kms / c


def test_speed_distribution_normalised_and_consistent_with_eta():
    p, v0, vesc, vE = _shm()
    v = np.linspace(1e-7, (vesc + vE) * 1.001, 40001)
    f = rate.shm_speed_distribution(v, v0, vesc, vE)
    assert np.trapezoid(f, v) == pytest.approx(1.0, abs=1e-8)
    for vmin in (3e-4, 1e-3, 2e-3):
        got = np.trapezoid(np.where(v >= vmin, f / v, 0.0), v)
        assert got == pytest.approx(rate.eta_shm(vmin, v0, vesc, vE), rel=2e-4)


def test_mediator_functions_by_hand():
    # m = 1, E = 2, E' = 1.5, q = 0.5:  H_V = 3.5^2 - 0.25 = 12,  H_phi = 4 - 0.25 + 0.25 = 4
    assert rate.h_mediator(2.0, 1.5, 0.5, 1.0, 0) == pytest.approx(12.0, rel=1e-15)
    assert rate.h_mediator(2.0, 1.5, 0.5, 1.0, 1) == pytest.approx(4.0, rel=1e-15)
    assert rate.mediator_factor(10.0, 3e4, -1.0) == 1.0
    assert rate.mediator_factor(0.0, rate.AME_EV, 0.0) == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("m_med,kind", [(-1.0, 0), (-1.0, 1), (0.0, 0), (0.0, 1)])
def test_general_rate_reduces_to_the_halo_rate(m_med, kind):
    """With the halo flux n_chi v f(v) and a GeV particle (v ~ 1e-3: H -> 4 m^2,
    E E' -> m^2, w << q) the general rate is the nonrelativistic one, within
    the v-grid's resolution of the step Theta(v - v_min)."""
    p, v0, vesc, vE = _shm()
    q = np.linspace(0.2, 3.0, 15)
    w = np.array([0.2, 0.3, 0.45, 0.6, 1.6])
    L = np.random.default_rng(1).uniform(0.1, 1.0, (len(q), len(w)))
    v = np.linspace(1e-7, (vesc + vE) * 1.001, 40001)
    flux = p.rho_chi_GeV_cm3 * 1e9 / p.m_chi_eV * (v * rate.C_KM_S * 1e5) * rate.shm_speed_distribution(v, v0, vesc, vE)
    g = rate.dR_dw_general(q, w, L, v, flux, rate.RelParams(m_chi_eV=p.m_chi_eV, m_med_eV=m_med, mediator=kind))
    nr = rate.dR_dw(q, w, L, rate.HaloParams(m_med_eV=m_med))
    m = nr > 1e-3 * nr.max()
    assert m.sum() >= 3
    assert np.allclose(g[m], nr[m], rtol=2e-4, atol=0)
    assert np.all(g[~m] <= 1e-3 * nr.max())


def test_general_rate_is_closed_beyond_the_kinetic_energy():
    """A 1 MeV particle at v = 0.01 carries 50 eV of kinetic energy: no rate at
    w = 60 eV, whatever the flux."""
    q = np.linspace(0.5, 3.0, 6)
    w = np.array([10.0, 60.0]) / rate.HARTREE_EV
    L = np.ones((6, 2))
    v = np.array([0.0099, 0.01, 0.0101])
    g = rate.dR_dw_general(q, w, L, v, np.ones(3), rate.RelParams(m_chi_eV=1e6))
    assert g[1] == 0.0 and g[0] > 0.0


def test_reach_by_hand():
    got = rate.reach([4.0, 3.0, 2.0, 1.0, 0.0], 1e-39, 2.0)
    want = [2.3e-39 / 20, 2.3e-39 / 12, 2.3e-39 / 6, 2.3e-39 / 2, np.inf]
    assert np.allclose(got[:4], want[:4], rtol=1e-15) and np.isinf(got[4])


# --------------------------------------------------------------- 3-D binning
def test_bin_index_by_hand():
    nth, nph = 9, 16
    assert bins3d.bin_index([0.0, 0.0, 0.55], 0.1, 20, nth, nph) == (5, 0, 0)
    assert bins3d.bin_index([0.0, 0.0, -0.55], 0.1, 20, nth, nph) == (5, 8, 0)        # theta = pi: last cell
    assert bins3d.bin_index([0.0, 0.31, 0.0], 0.1, 20, nth, nph) == (3, 4, 4)         # theta = pi/2, phi = pi/2
    assert bins3d.bin_index([0.0, -0.31, 0.0], 0.1, 20, nth, nph) == (3, 4, 12)       # phi = 3 pi/2
    assert bins3d.bin_index([0.2, -1e-9, 0.0], 0.1, 20, nth, nph) == (2, 4, 15)       # phi just below 2 pi
    assert bins3d.bin_index([-0.2, -1e-9, 0.0], 0.1, 20, nth, nph) == (2, 4, 8)       # phi just above pi
    assert bins3d.bin_index([0.0, 0.0, 0.0], 0.1, 20, nth, nph) is None
    assert bins3d.bin_index([0.0, 0.0, 2.05], 0.1, 20, nth, nph) is None             # past the last shell


def test_composite_binning_fill_and_isotropic_loss_by_hand():
    k = np.array([[0.0, 0.0, 0.15], [0.0, 0.0, 0.16], [0.0, 0.0, 0.45], [0.0, 0.0, 0.17]])
    dinv = np.array([[0.5 - 0.25j, 1.0 + 0.0j, 0.25 + 0.0j, 0.4 - 0.2j]])     # 1/dinv: 1.6+0.8j, 1, 4, 2+1j
    ed = np.array([[9.0 + 1j, 9.0 + 1j, 2.0 + 2.0j, 9.0 + 1j]])
    e = bins3d.composite_eps(k, dinv, ed, q_lfe=0.3)
    assert np.allclose(e[0], [1.6 + 0.8j, 1.0, 2.0 + 2.0j, 2.0 + 1.0j])
    eps, cnt = bins3d.bin_eps([k], [e], 0.1, 6, 2, 2)
    assert cnt[1, 0, 0] == 3 and cnt[4, 0, 0] == 1 and cnt.sum() == 4
    assert np.allclose(eps[1, 0, 0, 0], (1.6 + 0.8j + 1.0 + 2.0 + 1.0j) / 3)            # the mean, not the sum
    f, fc = bins3d.fill_empty(eps, cnt, 0.1)
    # shells 2 and 3 lie between filled shells 1 and 4: 2/3 and 1/3 of the way
    m1, m4 = eps[1, 0, 0, 0], eps[4, 0, 0, 0]
    assert np.allclose(f[2, 0, 0, 0], (2 * m1 + m4) / 3) and np.allclose(f[3, 0, 0, 0], (m1 + 2 * m4) / 3)
    assert fc[2, 0, 0] == -1 and fc[0, 0, 0] == 0 and fc[5, 0, 0] == 0                  # outside: still empty
    L, nc = bins3d.isotropic_loss(f, fc)
    assert nc[1] == 1 and nc[0] == 0 and L[0, 0] == 0.0
    assert L[4, 0] == pytest.approx((-1.0 / (2.0 + 2.0j)).imag, rel=1e-15)
    # two cells in one shell: the mean of their losses; with eps_scr = 1: the mean of Im eps
    two = np.zeros((1, 1, 2, 1), complex)
    two[0, 0, :, 0] = [1.0 + 1.0j, 2.0 + 1.0j]
    L2, _ = bins3d.isotropic_loss(two, np.ones((1, 1, 2)))
    assert L2[0, 0] == pytest.approx(0.5 * (0.5 + 0.2), rel=1e-15)
    L3, _ = bins3d.isotropic_loss(two, np.ones((1, 1, 2)), eps_scr=np.ones((1, 1)))
    assert L3[0, 0] == pytest.approx(1.0, rel=1e-15)


def test_synthetic_halo_flux_is_the_oracle_halo_flux():
    """The benchmark's flux input (synth.halo_flux) is n_chi v f(v) with the
    oracle's speed distribution."""
    import synth
    p, v0, vesc, vE = _shm()
    v = np.linspace(1e-6, 3e-3, 501)
    want = p.rho_chi_GeV_cm3 * 1e9 / p.m_chi_eV * v * rate.C_KM_S * 1e5 * rate.shm_speed_distribution(v, v0, vesc, vE)
    assert np.allclose(synth.halo_flux(v), want, rtol=1e-13, atol=0)
