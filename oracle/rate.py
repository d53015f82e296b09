"""FP64 oracle: dark-matter--electron scattering rate and recoil spectrum.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Nonrelativistic halo rate (Eqs. (general_rate) and (cross_section) with
Eq. (dynamic_structure_factor), final form at the end of Appendix A):

  dR/dw = (rho_chi/m_chi) (1/rho_T) sigma_e / (8 pi^2 alpha mu^2)
          int dq q^3 |F_DM(q)|^2 Im[-1/eps(w,q)] eta(v_min(q,w)),
  v_min = q/(2 m_chi) + w/q  (Eq. (v_min), gamma = 1),
  eta(v_min) = int_{|v|>v_min} d^3v f_chi(v)/|v|,

with the standard truncated Maxwellian halo (Section II; escape speed, Earth
speed and local density from the footnote to Section IV.B; v0 is not printed
in the paper and is a stated assumption, 238 km/s).  The recoil spectrum is
Eq. (excitation_rate) with the step ionisation model
Q(w) = 1 + floor((w - w_gap)/w_pp) of the caption of the code-comparison
figure (Section IV.D), reparametrised for the synthetic cell.

Everything is evaluated in natural units (eV, c = hbar = 1) and returned in
events / (kg yr eV) and events / (kg yr).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from math import erf, exp, sqrt, pi, floor

# CODATA 2018 and standard conversions
ALPHA = 1.0 / 137.035999084
ME_EV = 510998.95000
HBARC_EV_CM = 1.973269804e-5          # hbar c in eV cm
HBAR_EV_S = 6.582119569e-16           # hbar in eV s
C_KM_S = 299792.458
EV_PER_KG = 5.609588603804452e35      # c^2 = 1
EV_PER_GRAM = EV_PER_KG * 1e-3
YEAR_S = 365.25 * 24 * 3600.0
HARTREE_EV = 27.211386245988
AME_EV = ALPHA * ME_EV                # 1 bohr^-1 = alpha m_e c


@dataclass
class HaloParams:
    m_chi_eV: float = 1e9
    sigma_e_cm2: float = 1e-39
    rho_chi_GeV_cm3: float = 0.3
    v0_kms: float = 238.0
    vesc_kms: float = 544.0
    vE_kms: float = 250.2
    rho_T_g_cm3: float = 2.329
    m_med_eV: float = -1.0            # < 0: heavy mediator (F = 1); 0: light (F = (alpha m_e)^2/q^2)
    w_gap_eV: float = 1.1
    w_pp_eV: float = 3.75


def eta_shm(vmin, v0, vesc, vE):
    """eta(v_min) = int_{|v|>v_min} f(v)/|v| d^3v for the truncated Maxwellian
    f ~ exp(-|v+v_E|^2/v0^2) Theta(v_esc - |v+v_E|) (velocities in units of c)."""
    x, y, z = vmin / v0, vE / v0, vesc / v0
    nesc = erf(z) - 2.0 / sqrt(pi) * z * exp(-z * z)
    pref = 1.0 / (2.0 * nesc * v0 * y)
    if x < z - y:
        return pref * (erf(x + y) - erf(x - y) - 4.0 / sqrt(pi) * y * exp(-z * z))
    if x < z + y:
        return pref * (erf(z) - erf(x - y) - 2.0 / sqrt(pi) * (z + y - x) * exp(-z * z))
    return 0.0


def form_factor_sq(q_eV, m_med_eV):
    """|F_DM(q)|^2, Eq. (F_DM): ((alpha m_e)^2 + m^2)/(q^2 + m^2); m < 0 means the heavy limit F = 1."""
    if m_med_eV < 0:
        return 1.0
    f = (AME_EV ** 2 + m_med_eV ** 2) / (q_eV ** 2 + m_med_eV ** 2)
    return f * f


def rate_prefactor(p: HaloParams):
    """(rho_chi/m_chi)(1/rho_T) sigma_e/(8 pi^2 alpha mu^2) in natural units (eV^-4 ... see module doc)."""
    n_chi = p.rho_chi_GeV_cm3 * 1e9 / p.m_chi_eV * HBARC_EV_CM ** 3          # eV^3
    rho_T = p.rho_T_g_cm3 * EV_PER_GRAM * HBARC_EV_CM ** 3                   # eV^4
    sigma = p.sigma_e_cm2 / HBARC_EV_CM ** 2                                  # eV^-2
    mu = p.m_chi_eV * ME_EV / (p.m_chi_eV + ME_EV)
    return n_chi / rho_T * sigma / (8.0 * pi * pi * ALPHA * mu * mu)


def natural_to_kg_yr(x):
    """events/(eV_mass * eV^-1_time) -> events/(kg yr)."""
    return x * EV_PER_KG * (YEAR_S / HBAR_EV_S)


def dR_dw(qbin_bohr, w_ha, L, p: HaloParams):
    """dR/dw [events/(kg yr eV)] on the omega grid.

    qbin_bohr: [nq] ascending |q| (bohr^-1); w_ha: [nw] (Hartree);
    L: [nq][nw] loss function Im[-1/eps].  The q integral is the composite
    trapezoid rule over the q grid (L = 0 outside it)."""
    q = np.asarray(qbin_bohr, float) * AME_EV
    w = np.asarray(w_ha, float) * HARTREE_EV
    v0, vesc, vE = p.v0_kms / C_KM_S, p.vesc_kms / C_KM_S, p.vE_kms / C_KM_S
    pref = rate_prefactor(p)
    out = np.zeros(w.shape[0])
    for iw, wv in enumerate(w):
        g = np.zeros(q.shape[0])
        for iq, qv in enumerate(q):
            vmin = qv / (2.0 * p.m_chi_eV) + wv / qv
            g[iq] = qv ** 3 * form_factor_sq(qv, p.m_med_eV) * L[iq][iw] * eta_shm(vmin, v0, vesc, vE)
        out[iw] = pref * np.trapezoid(g, q)
    return natural_to_kg_yr(out)


def ionisation_q(w_eV, w_gap, w_pp):
    """Step model Q(w) = 1 + floor((w - w_gap)/w_pp) for w >= w_gap, else 0."""
    if w_eV < w_gap:
        return 0
    return 1 + int(floor((w_eV - w_gap) / w_pp))


def recoil_spectrum(w_ha, dRdw, p: HaloParams, nQ):
    """Delta R_Q = sum_w dR/dw dw [Q(w) = Q], Q = 1..nQ (Eq. (excitation_rate))."""
    w = np.asarray(w_ha, float) * HARTREE_EV
    dw = w[1] - w[0]
    out = np.zeros(nQ)
    for iw, wv in enumerate(w):
        Qv = ionisation_q(wv, p.w_gap_eV, p.w_pp_eV)
        if 1 <= Qv <= nQ:
            out[Qv - 1] += dRdw[iw] * dw
    return out


def bin_loss(qmag_bohr, L, edges_bohr):
    """Average loss values into |q| bins: qmag [n], L [n][nw] -> [nbin][nw]
    (empty bins are 0), bin centres."""
    qmag = np.asarray(qmag_bohr, float)
    nb = len(edges_bohr) - 1
    out = np.zeros((nb, L.shape[1]))
    cnt = np.zeros(nb)
    idx = np.searchsorted(edges_bohr, qmag, side="right") - 1
    for i, b in enumerate(idx):
        if 0 <= b < nb:
            out[b] += L[i]
            cnt[b] += 1
    nz = cnt > 0
    out[nz] /= cnt[nz][:, None]
    return out, 0.5 * (np.asarray(edges_bohr[1:]) + np.asarray(edges_bohr[:-1])), cnt


# --------------------------------------------------------------------------
# General (relativistic) rate with a velocity flux and a vector or scalar
# mediator: Eqs. (general_rate), (H), (cross_section_iso) and (v_min).
# --------------------------------------------------------------------------
CM2_S_TO_EV3 = (HBARC_EV_CM ** 2) * HBAR_EV_S      # 1 / (cm^2 s) in eV^3


def shm_speed_distribution(v, v0, vesc, vE):
    """Normalised speed distribution f(v) (int f dv = 1, speeds in units of c) of
    the truncated Maxwellian f(v_vec) ~ exp(-|v_vec + v_E|^2/v0^2) Theta(vesc - |v_vec + v_E|):
    f(v) = v^2 int dOmega f(v_vec), the angular integral done in closed form
    (2 pi int_{-1}^{c_max} dc exp(-(v^2 + vE^2 + 2 v vE c)/v0^2), c_max the
    escape-speed cut)."""
    z = vesc / v0
    norm = pi ** 1.5 * v0 ** 3 * (erf(z) - 2.0 / sqrt(pi) * z * exp(-z * z))
    out = np.zeros(np.shape(v))
    for i, vi in enumerate(np.atleast_1d(v)):
        if vi <= 0.0:
            continue
        B = 2.0 * vi * vE / v0 ** 2
        cmax = min(1.0, (vesc ** 2 - vi ** 2 - vE ** 2) / (2.0 * vi * vE))
        if cmax < -1.0:
            continue
        A = (vi ** 2 + vE ** 2) / v0 ** 2
        out[i] = 2.0 * pi * vi * vi / (norm * B) * (exp(-(A - B)) - exp(-(A + B * cmax)))
    return out


def h_mediator(E, Ep, q, m_chi, kind):
    """H_A'(q) of Eq. (H): kind 0 vector, (E + E')^2 - q^2; kind 1 scalar, 4 m^2 - (E - E')^2 + q^2."""
    if kind == 0:
        return (E + Ep) ** 2 - q * q
    return 4.0 * m_chi * m_chi - (E - Ep) ** 2 + q * q


@dataclass
class RelParams:
    m_chi_eV: float = 1e9
    sigma_e_cm2: float = 1e-39
    m_med_eV: float = -1.0            # < 0: heavy mediator; 0: massless; > 0: that mass
    mediator: int = 0                 # 0 vector, 1 scalar
    rho_T_g_cm3: float = 2.329
    w_gap_eV: float = 1.1
    w_pp_eV: float = 3.75


def mediator_factor(w, q, m_med):
    """(m_A'^2 + (alpha m_e)^2)^2 / (w^2 - q^2 - m_A'^2)^2; 1 in the heavy limit (m_med < 0)."""
    if m_med < 0:
        return 1.0
    return (m_med ** 2 + AME_EV ** 2) ** 2 / (w * w - q * q - m_med ** 2) ** 2


def dR_dw_general(qbin_bohr, w_ha, L, v, dphidv, p: RelParams):
    """dR/dw [events/(kg yr eV)] = (1/rho_T) int dv dPhi/dv dsigma/dw per target
    mass, dsigma/dw of Eq. (cross_section_iso):
      sigma_e/(16 pi mu^2) 1/(E (E - w)) int dq q H(q) F_med(w, q) S(w, q) Theta(v - v_min)/v^2,
      S = q^2 L/(2 pi alpha),  E = gamma m_chi,  v_min = q/(2 gamma m_chi) + w/q (Eq. (v_min)).
    v[nv] (units of c), dphidv[nv] (1/(cm^2 s) per unit v): trapezoid in v; the
    q integral is the trapezoid over qbin (L = 0 outside).  Energy transfers
    with E - w <= m_chi are kinematically closed and contribute 0."""
    q = np.asarray(qbin_bohr, float) * AME_EV
    w = np.asarray(w_ha, float) * HARTREE_EV
    v = np.asarray(v, float)
    flux = np.asarray(dphidv, float) * CM2_S_TO_EV3
    m = p.m_chi_eV
    mu = m * ME_EV / (m + ME_EV)
    sigma = p.sigma_e_cm2 / HBARC_EV_CM ** 2
    rho_T = p.rho_T_g_cm3 * EV_PER_GRAM * HBARC_EV_CM ** 3
    out = np.zeros(w.shape[0])
    for iw, wv in enumerate(w):
        per_v = np.zeros(v.shape[0])
        for ivel, vv in enumerate(v):
            if vv <= 0.0 or vv >= 1.0:
                continue
            gam = 1.0 / sqrt(1.0 - vv * vv)
            E = gam * m
            Ep = E - wv
            if Ep <= m:
                continue
            vmin = q / (2.0 * gam * m) + wv / q
            S = q * q * np.asarray(L)[:, iw] / (2.0 * pi * ALPHA)
            g = q * h_mediator(E, Ep, q, m, p.mediator) * mediator_factor(wv, q, p.m_med_eV) * S / (vv * vv)
            g = np.where(vv >= vmin, g, 0.0)
            per_v[ivel] = sigma / (16.0 * pi * mu * mu) / (E * Ep) * np.trapezoid(g, q)
        out[iw] = np.trapezoid(flux * per_v, v) / rho_T
    return natural_to_kg_yr(out)


def reach(dRQ, sigma_ref_cm2, exposure_kg_yr, n_events=2.3):
    """Cross section at which n_events are expected for exposure_kg_yr above each
    ionisation threshold Q = 1..nQ (the rate is linear in sigma_e; zero
    background): n_events sigma_ref / (exposure sum_{Q' >= Q} dR_Q'(sigma_ref))."""
    tail = np.cumsum(np.asarray(dRQ, float)[::-1])[::-1]
    out = np.full(tail.shape, np.inf)
    nz = tail > 0
    out[nz] = n_events * sigma_ref_cm2 / (exposure_kg_yr * tail[nz])
    return out
